// The initial-condition procedure of Section IV-B, which supplies the two
// levels v(0), v(h) that the three-level form (Eq. 11) starts from:
//
//   1. DC at t = 0 with every capacitor a voltage source v_c(0) and every
//      inductor a current source i_l(0): v(0), the capacitor currents i_c(0),
//      the inductor voltages v_l(0);
//   2. v_c(h) = v_c(0) + h i_c(0) / C,  i_l(h) = i_l(0) + h v_l(0) / L;
//   3. DC at t = h with the capacitors at v_c(h) and the inductors carrying
//      i_l(h): v(h).
//
// Each DC analysis is solved by the library's own relaxation on a derived
// netlist: the nodes that carry a capacitor become sources at their fixed
// voltage, inductors and loads become constant current sources, and the rest
// of the grid keeps its resistors.  The bookkeeping around the two solves
// (the capacitor currents by Kirchhoff's current law, the forward updates) is
// O(elements) host arithmetic done once per call.

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "pg_grid.h"

namespace pg {
namespace {

struct Derived {
    std::vector<double> vdd;
    std::vector<int32_t> r_a, r_b, i_a, i_b;
    std::vector<double> r_g, i_t, i_v;
    std::vector<int64_t> i_ptr;
};

// DC solve with the nodes in `fixed` held at vfix, constant currents: loads at t,
// inductor currents il.  v receives every node's voltage (caller numbering).
pg_status dc_fixed(const NetCopy& nc, const std::vector<uint8_t>& fixed, const std::vector<double>& vfix,
                   double t, const std::vector<double>& il, double tol, void* stream, std::vector<double>& v) {
    const int n = nc.n, p = nc.p;
    std::vector<int32_t> map(n, -1), fix_src(n, -1);
    int nf = 0, nfix = 0;
    for (int i = 0; i < n; ++i) {
        if (fixed[i]) fix_src[i] = p + nfix++;
        else map[i] = nf++;
    }
    v.assign(n, 0.0);
    for (int i = 0; i < n; ++i)
        if (fixed[i]) v[i] = vfix[i];
    if (nf == 0) return PG_OK;
    auto T = [&](int32_t x) -> int32_t {
        if (x < 0) return x;
        return fixed[x] ? (int32_t)(-2 - fix_src[x]) : map[x];
    };
    Derived d;
    d.vdd = nc.vdd;
    for (int i = 0; i < n; ++i)
        if (fixed[i]) d.vdd.push_back(vfix[i]);
    for (size_t e = 0; e < nc.r_g.size(); ++e) {
        const int32_t a = T(nc.r_a[e]), b = T(nc.r_b[e]);
        if (a < 0 && b < 0) continue;               // no free node: no equation of this solve
        d.r_a.push_back(a); d.r_b.push_back(b); d.r_g.push_back(nc.r_g[e]);
    }
    d.i_ptr.push_back(0);
    auto current = [&](int32_t a0, int32_t b0, double I) {
        const int32_t a = T(a0), b = T(b0);
        if ((a < 0 && b < 0) || I == 0.0) return;
        d.i_a.push_back(a); d.i_b.push_back(b);
        d.i_t.push_back(0.0); d.i_v.push_back(I);
        d.i_ptr.push_back((int64_t)d.i_t.size());
    };
    for (size_t e = 0; e + 1 < nc.i_ptr.size(); ++e) current(nc.i_a[e], nc.i_b[e], pwl_at(nc, (int64_t)e, t));
    for (size_t e = 0; e < nc.l_val.size(); ++e) current(nc.l_a[e], nc.l_b[e], il[e]);

    pg_netlist nl{};
    nl.n_nodes = nf; nl.n_sources = (int32_t)d.vdd.size(); nl.vdd = d.vdd.data();
    nl.n_r = (int64_t)d.r_g.size(); nl.r_a = d.r_a.data(); nl.r_b = d.r_b.data(); nl.r_g = d.r_g.data();
    nl.n_i = (int64_t)d.i_a.size(); nl.i_a = d.i_a.data(); nl.i_b = d.i_b.data();
    nl.i_ptr = d.i_ptr.data(); nl.i_t = d.i_t.data(); nl.i_v = d.i_v.data();
    pg_options o;
    pg_default_options(&o);
    o.precision = PG_PREC_FP64;
    std::vector<double> vf(nf);
    pg_status s = PG_OK;
    // a target below what FP64 residuals can certify on this grid (kappa * 1e-13) is relaxed
    // tenfold until it is reachable
    for (int tries = 0; tries < 8; ++tries, tol *= 10.0) {
        o.tol = tol;
        pg_grid* dg = nullptr;
        if ((s = pg_create_grid(&nl, &o, &dg))) return s;
        if (stream) pg_set_stream(dg, stream);
        int64_t step = 0;
        if (!(s = pg_transient(dg, 1.0, 0, nullptr, nullptr)))   // the DC operating point of the derived grid
            s = pg_get_state(dg, vf.data(), nullptr, &step, 1);
        pg_destroy(dg);
        if (s != PG_ERR_INVALID_ARG) break;
    }
    if (s) return s;
    for (int i = 0; i < n; ++i)
        if (!fixed[i]) v[i] = vf[map[i]];
    return PG_OK;
}

double volt(const NetCopy& nc, const std::vector<double>& v, int32_t x) {
    return x >= 0 ? v[x] : (x == PG_GROUND ? 0.0 : nc.vdd[-2 - x]);
}

}  // namespace

pg_status paper_initial_levels(const NetCopy& nc, double h, double tol, void* stream, const double* vc0,
                               const double* il0, std::vector<double>& v0, std::vector<double>& v1,
                               std::vector<double>& il1) {
    const int n = nc.n;
    const size_t nl = nc.l_val.size(), ncap = nc.c_val.size();
    std::vector<double> il(nl, 0.0);
    if (il0) il.assign(il0, il0 + nl);
    std::vector<double> cn(n, 0.0), gsum(n, 0.0);
    std::vector<uint8_t> capped(n, 0);
    for (size_t e = 0; e < ncap; ++e) {
        const int32_t k = nc.c_a[e] >= 0 ? nc.c_a[e] : nc.c_b[e];
        cn[k] += nc.c_val[e];
        capped[k] = 1;
    }
    for (size_t e = 0; e < nc.r_g.size(); ++e) {
        if (nc.r_a[e] >= 0) gsum[nc.r_a[e]] += nc.r_g[e];
        if (nc.r_b[e] >= 0) gsum[nc.r_b[e]] += nc.r_g[e];
    }
    pg_status s;
    std::vector<double> vcap(n, 0.0), vcap1(n, 0.0);
    il1.assign(nl, 0.0);
    auto inductor_step = [&]() {
        for (size_t e = 0; e < nl; ++e)
            il1[e] = il[e] + h * (volt(nc, v0, nc.l_a[e]) - volt(nc, v0, nc.l_b[e])) / nc.l_val[e];
    };
    if (!vc0) {
        // v_c(0) = the DC operating point with the capacitors open.  Step 1 then returns
        // that point and no capacitor carries current (i_c(0) = 0 by construction), so
        // v_c(h) = v_c(0) and only the inductor currents move.
        if ((s = dc_fixed(nc, std::vector<uint8_t>(n, 0), vcap, 0.0, il, tol, stream, v0))) return s;
        for (int i = 0; i < n; ++i)
            if (capped[i]) vcap1[i] = v0[i];
        inductor_step();
        return dc_fixed(nc, capped, vcap1, h, il1, tol, stream, v1);
    }
    std::vector<uint8_t> seen(n, 0);
    for (size_t e = 0; e < ncap; ++e) {
        const int32_t k = nc.c_a[e] >= 0 ? nc.c_a[e] : nc.c_b[e];
        if (!std::isfinite(vc0[e])) { set_last_error("non-finite capacitor voltage"); return PG_ERR_INVALID_ARG; }
        if (seen[k] && vcap[k] != vc0[e]) {
            set_last_error("parallel capacitors on one node need one voltage");
            return PG_ERR_INVALID_ARG;
        }
        vcap[k] = vc0[e];
        seen[k] = 1;
    }
    // step 2 multiplies an error of v(0) near a capacitor node by up to 1 + h sum(g) / C,
    // so step 1 is solved that much tighter (down to what FP64 residuals can certify)
    double amp = 1.0;
    for (int i = 0; i < n; ++i)
        if (capped[i]) amp = std::max(amp, 1.0 + h * gsum[i] / cn[i]);
    if ((s = dc_fixed(nc, capped, vcap, 0.0, il, tol / amp, stream, v0))) return s;
    // capacitor currents by KCL: i_c = -(sum of the currents leaving the node through the other branches)
    std::vector<double> f(n, 0.0);
    for (size_t e = 0; e < nc.r_g.size(); ++e) {
        const int32_t a = nc.r_a[e], b = nc.r_b[e];
        const double cur = nc.r_g[e] * (volt(nc, v0, a) - volt(nc, v0, b));
        if (a >= 0) f[a] += cur;
        if (b >= 0) f[b] -= cur;
    }
    for (size_t e = 0; e + 1 < nc.i_ptr.size(); ++e) {
        const double I = pwl_at(nc, (int64_t)e, 0.0);
        if (nc.i_a[e] >= 0) f[nc.i_a[e]] += I;
        if (nc.i_b[e] >= 0) f[nc.i_b[e]] -= I;
    }
    for (size_t e = 0; e < nl; ++e) {
        if (nc.l_a[e] >= 0) f[nc.l_a[e]] += il[e];
        if (nc.l_b[e] >= 0) f[nc.l_b[e]] -= il[e];
    }
    // step 2
    for (int i = 0; i < n; ++i)
        if (capped[i]) vcap1[i] = vcap[i] + h * (-f[i]) / cn[i];
    inductor_step();
    // step 3
    return dc_fixed(nc, capped, vcap1, h, il1, tol, stream, v1);
}

}  // namespace pg
