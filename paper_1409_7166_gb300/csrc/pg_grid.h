// Internal definition of the opaque pg_grid handle (shared by the C ABI
// translation units).
#pragma once

#include <memory>
#include <string>
#include <vector>

#include "pg_internal.h"

namespace pg {

// Copy of the caller's netlist (needed to derive the DC sub-problem).
struct NetCopy {
    int32_t n = 0, p = 0;
    std::vector<double> vdd;
    std::vector<int32_t> r_a, r_b, c_a, c_b, l_a, l_b, i_a, i_b;
    std::vector<double> r_g, c_val, l_val, i_t, i_v;
    std::vector<int64_t> i_ptr;
    int32_t nx = 0, ny = 0, nl = 0;
    std::vector<int32_t> lat_desc;

    void from(const pg_netlist* nl_) {
        n = nl_->n_nodes; p = nl_->n_sources;
        vdd.assign(nl_->vdd, nl_->vdd + p);
        auto cp = [](auto& dst, auto* src, int64_t m) { dst.assign(src, src + m); };
        cp(r_a, nl_->r_a, nl_->n_r); cp(r_b, nl_->r_b, nl_->n_r); cp(r_g, nl_->r_g, nl_->n_r);
        cp(c_a, nl_->c_a, nl_->n_c); cp(c_b, nl_->c_b, nl_->n_c); cp(c_val, nl_->c_val, nl_->n_c);
        cp(l_a, nl_->l_a, nl_->n_l); cp(l_b, nl_->l_b, nl_->n_l); cp(l_val, nl_->l_val, nl_->n_l);
        cp(i_a, nl_->i_a, nl_->n_i); cp(i_b, nl_->i_b, nl_->n_i);
        if (nl_->n_i) {
            cp(i_ptr, nl_->i_ptr, nl_->n_i + 1);
            cp(i_t, nl_->i_t, nl_->i_ptr[nl_->n_i]); cp(i_v, nl_->i_v, nl_->i_ptr[nl_->n_i]);
        } else {
            i_ptr.assign(1, 0);
        }
        nx = nl_->lat_nx; ny = nl_->lat_ny; nl = nl_->lat_nl;
        if (nl_->n_lat > 0 && nl_->lat_desc) lat_desc.assign(nl_->lat_desc, nl_->lat_desc + 4 * nl_->n_lat);
    }
    // The DC network at t = 0: capacitors open, inductors carrying i_l(0) = 0 (open).
    pg_netlist dc_view() const {
        pg_netlist d{};
        d.n_nodes = n; d.n_sources = p; d.vdd = vdd.data();
        d.n_r = (int64_t)r_g.size(); d.r_a = r_a.data(); d.r_b = r_b.data(); d.r_g = r_g.data();
        d.n_i = (int64_t)i_a.size(); d.i_a = i_a.data(); d.i_b = i_b.data();
        d.i_ptr = i_ptr.data(); d.i_t = i_t.data(); d.i_v = i_v.data();
        return d;
    }
};

inline double pwl_at(const NetCopy& nc, int64_t e, double t) {
    int64_t lo = nc.i_ptr[e], hi = nc.i_ptr[e + 1] - 1;
    if (t <= nc.i_t[lo]) return nc.i_v[lo];
    if (t > nc.i_t[hi]) return nc.i_v[hi];
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (t <= nc.i_t[mid]) hi = mid; else lo = mid;
    }
    return nc.i_v[lo] + (nc.i_v[hi] - nc.i_v[lo]) * ((t - nc.i_t[lo]) / (nc.i_t[hi] - nc.i_t[lo]));
}

}  // namespace pg

struct pg_grid {
    using Packed = pg::Packed;
    using NetCopy = pg::NetCopy;
    using DevGrid = pg::DevGrid;
    using DevState = pg::DevState;
    using DevCtl = pg::DevCtl;
    Packed P;
    NetCopy nc;
    pg_options opt{};
    int device = 0;
    cudaStream_t stream = nullptr;
    int n_sm = 0;
    int blocks = 1, threads = 256;
    size_t smem = 0;               // dynamic shared memory of the persistent launch
    bool mixed = false;
    int lat_k = 0;                 // lattice inner solve: block sweeps per device barrier (0 = off)
    std::vector<void*> allocs;
    DevGrid dg{};
    DevState ds{};
    DevCtl dc{};
    double* d_x = nullptr;        // scratch [n] for setup solves (caller numbering)
    double* d_rhs = nullptr;      // pg_solve's permuted right-hand side [n_pad], allocated on first use
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // per-h
    double h = -1.0;
    double omega = 0.0, rho = 0.0, kappa = 0.0, q = 0.0, step_tol = 0.0, target = 0.0;
    double kacc = 0.0;             // bound of sum_j ||(M^-1 C/h)^j||: per-step errors -> accumulated error
    double sor_omega = 0.0;        // omega of the setup solves (coloured SOR even when Jacobi runs the steps)
    // transient state
    bool has_state = false;
    int64_t step = 0;
    int vL = 0, vP = 1;
    bool have_prev = false;
    bool inc_ok = false;          // r64 and md hold the last step's final residual and M d (see run)
    int32_t last_outer = 0;       // outer passes of that step (a step after more than 4 starts in full)
    // largest certified error bound (V) of the state the series started from (the DC solve;
    // 0 for a state the caller set) and of every step since: the accumulated error of the
    // current state is at most kacc times this
    double series_bound = 0.0;
    bool dc_trivial = false;      // DC point is v = Vdd everywhere (see compute_dc_trivial)
    double dc_vdd = 0.0;
    std::unique_ptr<pg_grid> dcgrid;  // DC sub-problem, built on first use

    template <typename T>
    T* alloc(size_t count) {
        if (count == 0) count = 1;
        void* p = nullptr;
        if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) return nullptr;
        allocs.push_back(p);
        return static_cast<T*>(p);
    }
    ~pg_grid() {
        if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
        for (void* p : allocs) cudaFree(p);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

namespace pg {
// Per-call launch parameters filled from the grid's options and per-h constants.
RunParams base_params(const pg_grid* g);
// Section IV-B initial conditions: the levels v(0), v(h) and i_l(h) (host, caller numbering);
// DC solves on derived grids to `tol`, issued on `stream`.
pg_status paper_initial_levels(const NetCopy& nc, double h, double tol, void* stream, const double* vc0,
                               const double* il0, std::vector<double>& v0, std::vector<double>& v1,
                               std::vector<double>& il1);
// Record the detail message returned by pg_last_error().
void set_last_error(const std::string& msg);
// Run statistics of one launch in the public form (shared by every solve entry point):
// `st` the device statistics record, `ms` its event time, `prior` the largest per-step
// bound of the series before the launch.
pg_status fill_run_stats(pg_grid* g, const double* st, float ms, pg_run_stats* out, double prior);
// Look up, once per device and with that device current, the device address of the fixed
// scratch array of pg_solve_noalloc (pg_noalloc.cu).  The array's module is loaded, and its
// memory reserved, by this first lookup; pg_create_grid calls it so that the reservation
// happens at grid creation and never inside pg_solve_noalloc.  A failure is remembered and
// reported by pg_solve_noalloc; it does not fail the grid's creation.
void noalloc_bind_device(int device);
}  // namespace pg
