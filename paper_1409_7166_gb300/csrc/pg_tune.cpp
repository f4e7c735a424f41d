// pg_autotune: choose solver and launch options for one netlist by timed trials.
//
// The paper fixes neither the relaxation factor nor the parallel schedule
// (Section IV leaves omega and the sweep order open), and the best choice
// depends on the grid: its size and layer count decide whether the column-block
// inner solve pays for its ghost zones and which region shape (34 x 34 columns,
// or 34 x 66 at one block per SM) does, which colouring the point sweeps take
// (red-black, or four colours on a lattice), how far the FP32 inner solve should
// reduce the defect before the next FP64 residual pass, and whether omega a
// little above or below the automatic value (Young's, taken 1 % high) does
// better on this grid's transient.  Every candidate runs under the same certified stopping rule, so
// any candidate that converges meets the tolerance and the search only compares
// time.

#include <algorithm>
#include <cmath>
#include <vector>

#include "pg_grid.h"

namespace {

constexpr double kInnerReductions[] = {1e-3, 1e-2, 1e-1};
constexpr double kOmegaScales[] = {1.0, 1.01, 0.98};   // applied to omega - 1

}  // namespace

extern "C" pg_status pg_autotune(const pg_netlist* nl, const pg_options* base, double h, int32_t trial_steps,
                                 void* stream, pg_options* best, double* best_ms) {
    if (!nl || !best || trial_steps < 1 || !(h > 0.0) || !std::isfinite(h)) return PG_ERR_INVALID_ARG;
    pg_options b0;
    if (base) b0 = *base;
    else pg_default_options(&b0);
    const bool mixed = b0.precision == PG_PREC_MIXED;
    const bool lattice = mixed && (nl->n_lat > 0 || (nl->lat_nx > 0 && nl->lat_ny > 0 && nl->lat_nl > 0));
    std::vector<int32_t> ks = lattice ? std::vector<int32_t>{-1, 1, 2, 3} : std::vector<int32_t>{b0.lattice_sweeps};
    const bool lat_net = nl->n_lat > 0 || (nl->lat_nx > 0 && nl->lat_ny > 0 && nl->lat_nl > 0);
    // per inner-solve form, the layout candidates: region rows for the lattice solve,
    // colourings for the point sweeps (four colours only where the netlist is a lattice)
    auto layouts = [&](int32_t k) {
        std::vector<std::pair<int32_t, int32_t>> v;    // (tile_rows, colouring)
        if (lattice && k > 0) {
            v.push_back({34, b0.colouring});
            v.push_back({66, b0.colouring});
        } else {
            v.push_back({b0.tile_rows, PG_COLOUR_AUTO});
            if (lat_net) v.push_back({b0.tile_rows, PG_COLOUR_FOUR});
        }
        return v;
    };
    const std::vector<int32_t> bps = {0, 1};
    std::vector<double> reds;
    if (mixed) reds.assign(std::begin(kInnerReductions), std::end(kInnerReductions));
    else reds.push_back(b0.inner_reduction);

    double best_t = INFINITY;
    int32_t best_sweeps_step = 0;       // most sweeps a step of the winner needed
    pg_options win = b0;
    pg_status last = PG_OK;
    for (int32_t k : ks) {
      for (const auto& lay : layouts(k)) {
        for (int32_t bp : bps) {
            pg_options o = b0;
            o.lattice_sweeps = k;
            o.blocks_per_sm = bp;
            o.tile_rows = lay.first;
            o.colouring = lay.second;
            pg_grid* g = nullptr;
            pg_status s = pg_create_grid(nl, &o, &g);
            if (s) { last = s; continue; }
            if (stream) pg_set_stream(g, stream);
            pg_run_stats st;
            if ((s = pg_transient(g, h, 0, nullptr, &st))) {   // assemble h: omega, kappa, stopping rule
                last = s;
                pg_destroy(g);
                continue;
            }
            const double w0 = g->omega;
            const bool fixed_omega = b0.omega > 0.0 || !(w0 > 1.0);
            for (double red : reds) {
                for (double sc : kOmegaScales) {
                    if (fixed_omega && sc != 1.0) continue;
                    g->opt.inner_reduction = red;
                    g->omega = std::min(1.0 + (w0 - 1.0) * sc, 0.5 * (w0 + 2.0));   // stays below 2
                    double t = INFINITY;
                    int32_t msw = 0;
                    for (int rep = 0; rep < 2 && !s; ++rep) {   // first run warms caches and clocks
                        if ((s = pg_reset(g))) break;
                        if ((s = pg_transient(g, h, trial_steps, nullptr, &st))) break;
                        t = std::min(t, (double)st.device_ms);
                        msw = std::max(msw, st.max_sweeps_step);
                    }
                    if (s) {
                        last = s;
                        s = PG_OK;
                        continue;
                    }
                    if (t < best_t) {
                        best_t = t;
                        best_sweeps_step = msw;
                        win = o;
                        win.inner_reduction = red;
                        win.omega = sc == 1.0 ? b0.omega : g->omega;
                    }
                }
            }
            g->omega = w0;
            pg_destroy(g);
        }
      }
    }
    // damped Jacobi (undamped, omega = 1): allowed 4x the winner's sweeps per step, so a
    // candidate that cannot compete fails fast instead of running to the sweep cap
    if (std::isfinite(best_t) && b0.jacobi == 0) {
        pg_options o = b0;
        o.jacobi = 1;
        o.lattice_sweeps = -1;
        o.omega = 0.0;
        o.max_sweeps = std::max<int32_t>(16, 4 * best_sweeps_step);
        pg_grid* g = nullptr;
        pg_run_stats st;
        if (pg_create_grid(nl, &o, &g) == PG_OK) {
            if (stream) pg_set_stream(g, stream);
            double t = INFINITY;
            pg_status s = pg_transient(g, h, 0, nullptr, &st);
            for (int rep = 0; rep < 2 && !s; ++rep) {
                if ((s = pg_reset(g))) break;
                if ((s = pg_transient(g, h, trial_steps, nullptr, &st))) break;
                t = std::min(t, (double)st.device_ms);
            }
            if (!s && t < best_t) {
                best_t = t;
                win = o;
                win.max_sweeps = b0.max_sweeps;
            }
            pg_destroy(g);
        }
    }
    if (!std::isfinite(best_t)) return last ? last : PG_ERR_NOT_CONVERGED;
    *best = win;
    if (best_ms) *best_ms = best_t;
    return PG_OK;
}
