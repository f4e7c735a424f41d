// The C ABI (include/pg.h): grid lifetime, per-h coefficient assembly
// (Eq. 14: diagonal sum g + h sum 1/L + C/h and off-diagonal g + h/L), the
// stopping-rule constants, DC initial conditions (Section IV-B) and the
// transient driver (Algorithm 1), which runs as one persistent launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "pg_grid.h"

using namespace pg;

namespace {

thread_local std::string g_last_error;

}  // namespace

void pg::set_last_error(const std::string& msg) { g_last_error = msg; }

namespace {

constexpr int kSetupSweeps = 200000;

// Device buffers owned by one call, freed when it returns.
struct DeviceScratch {
    std::vector<void*> p;
    ~DeviceScratch() { for (void* q : p) cudaFree(q); }
    template <typename T>
    T* get(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return nullptr;
        p.push_back(q);
        return static_cast<T*>(q);
    }
};

pg_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return PG_ERR_CUDA;
}
#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)

template <typename T>
pg_status upload(pg_grid* g, T* dst, const std::vector<T>& src) {
    if (src.empty()) return PG_OK;
    CK(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, g->stream));
    return PG_OK;
}

void compute_dc_trivial(pg_grid* g) {
    // v(0) = V everywhere solves the DC system exactly when every branch to a
    // fixed potential goes to a source of the same voltage V (none to ground)
    // and no load draws current at t = 0: then G (V 1) = -G_s v_d.
    const NetCopy& nc = g->nc;
    bool ok = nc.p > 0;
    double V = ok ? nc.vdd[0] : 0.0;
    for (int k = 0; k < nc.p && ok; ++k) ok = nc.vdd[k] == V;
    auto fixed_ok = [&](int32_t a, int32_t b) {
        if ((a >= 0) == (b >= 0)) return true;
        int32_t o = a >= 0 ? b : a;
        return o != PG_GROUND;
    };
    for (size_t e = 0; e < nc.r_g.size() && ok; ++e) ok = fixed_ok(nc.r_a[e], nc.r_b[e]);
    for (size_t e = 0; e < nc.l_val.size() && ok; ++e) ok = fixed_ok(nc.l_a[e], nc.l_b[e]);
    for (size_t e = 0; e + 1 < nc.i_ptr.size() && ok; ++e) ok = pwl_at(nc, (int64_t)e, 0.0) == 0.0;
    g->dc_trivial = ok;
    g->dc_vdd = V;
}

pg_status alloc_device(pg_grid* g) {
    const Packed& P = g->P;
    const int np = P.n_pad;
    DevGrid& d = g->dg;
    d.n_pad = np; d.ncol = P.ncol; d.n_slices = P.n_slices; d.n_real = P.n;
    d.natural = P.ncol == 1;
    for (int i = 0; i < P.n && d.natural; ++i) d.natural = P.orig[i] == i;
    std::vector<int32_t> cs(P.ncol + 1);
    for (int c = 0; c <= P.ncol; ++c) cs[c] = P.colour_start[c] / kSlice;
    int32_t* colour_slice = g->alloc<int32_t>(cs.size());
    int64_t* slice_off = g->alloc<int64_t>(P.slice_off.size());
    int32_t* slice_w = g->alloc<int32_t>(P.slice_w.size());
    int32_t* slice_doff = g->alloc<int32_t>(P.slice_doff.size());
    int32_t* dia_off = g->alloc<int32_t>(P.dia_off.size());
    int32_t* ell_col = g->alloc<int32_t>(P.n_ell);
    int32_t* orig = g->alloc<int32_t>(np);
    int32_t* ld_ptr = g->alloc<int32_t>(P.ld_ptr.size());
    int32_t* ld_idx = g->alloc<int32_t>(P.ld_idx.size());
    int64_t* pwl_ptr = g->alloc<int64_t>(P.pwl_ptr.size());
    double* pwl_t = g->alloc<double>(P.pwl_t.size());
    double* pwl_v = g->alloc<double>(P.pwl_v.size());
    double* pwl_s = g->alloc<double>(P.pwl_s.size());
    unsigned long long* pwl_tk = g->alloc<unsigned long long>(P.pwl_tk.size());
    int32_t* ind_a = g->alloc<int32_t>(P.n_l);
    int32_t* ind_b = g->alloc<int32_t>(P.n_l);
    double* ind_hl = g->alloc<double>(P.n_l);
    int32_t* ind_ptr = g->alloc<int32_t>(P.ind_ptr.size());
    int32_t* ind_idx = g->alloc<int32_t>(P.ind_idx.size());
    double* vdd = g->alloc<double>(P.vdd.size());
    double* w64 = g->alloc<double>(P.n_ell);
    double* D64 = g->alloc<double>(np);
    double* invD64 = g->alloc<double>(np);
    double* ch = g->alloc<double>(np);
    double* cinj = g->alloc<double>(np);
    float* w32 = g->mixed ? g->alloc<float>(P.n_ell) : nullptr;
    float* invD32 = g->mixed ? g->alloc<float>(np) : nullptr;
    float* w32lo = g->mixed ? g->alloc<float>(P.n_ell) : nullptr;
    float* D32 = g->mixed ? g->alloc<float>(np) : nullptr;
    float* D32lo = g->mixed ? g->alloc<float>(np) : nullptr;
    // lattice column-block inner solve: on by default for multi-layer lattices (the via
    // couplings go into the blocks) and for small single-layer ones (auto_lattice_k)
    const int lat_k = g->opt.jacobi ? 0
                    : g->opt.lattice_sweeps > 0 ? g->opt.lattice_sweeps
                    : (g->opt.lattice_sweeps == 0 ? auto_lattice_k(P.lat_maxnl, P.n) : 0);
    std::vector<int32_t> lat_tile0, lat_info;
    std::vector<int64_t> lat_col0;
    // (FP64 grids too, on natural-order packing, with 34-row regions; FP32 copies of the five
    // arrays serve the omega power iteration)
    if (P.lattice && lat_k > 0 && (g->mixed || d.natural)) {
        g->lat_k = lat_k;
        float* lw[5];
        for (auto& q : lw) if (!(q = g->alloc<float>(P.n))) return PG_ERR_OOM;
        d.lwE = lw[0]; d.lwN = lw[1]; d.lwU = lw[2]; d.lm = lw[3]; d.lip = lw[4];
        if (!g->mixed) {
            double* lw64[5];
            for (auto& q : lw64) if (!(q = g->alloc<double>(P.n))) return PG_ERR_OOM;
            d.lwE64 = lw64[0]; d.lwN64 = lw64[1]; d.lwU64 = lw64[2]; d.lm64 = lw64[3]; d.lip64 = lw64[4];
        }
        // tiles of T x TY interior columns per lattice, and columns per lattice
        const int rows = g->opt.tile_rows > 0 ? g->opt.tile_rows : kLatSide;
        const int nlat = (int)P.lats.size() / 4, T = lattice_tile_side(lat_k), TY = lattice_tile_rows(lat_k, rows);
        d.lat_rows = rows;
        d.lat_astride = P.lat_maxnl * rows * kLatW;
        lat_info = P.lats;
        lat_tile0.assign(nlat + 1, 0);
        lat_col0.assign(nlat + 1, 0);
        for (int L = 0; L < nlat; ++L) {
            const int nx = P.lats[4 * L + 1], ny = P.lats[4 * L + 2];
            lat_tile0[L + 1] = lat_tile0[L] + ((nx + T - 1) / T) * ((ny + TY - 1) / TY);
            lat_col0[L + 1] = lat_col0[L] + (int64_t)nx * ny;
        }
        int32_t* li = g->alloc<int32_t>(lat_info.size());
        int32_t* lt = g->alloc<int32_t>(lat_tile0.size());
        int64_t* lc = g->alloc<int64_t>(lat_col0.size());
        int32_t* nlatv = g->alloc<int32_t>(np);
        if (!li || !lt || !lc || !nlatv) return PG_ERR_OOM;
        d.n_lats = nlat; d.lat_info = li; d.lat_tile0 = lt; d.lat_tiles = lat_tile0[nlat];
        d.lat_col0 = lc; d.lat_cols = lat_col0[nlat]; d.node_lat = nlatv;
    }
    if (!colour_slice || !slice_off || !slice_w || !slice_doff || !dia_off || !ell_col || !orig || !ld_ptr ||
        !ld_idx || !pwl_ptr || !pwl_t || !pwl_v || !pwl_s || !pwl_tk || !ind_a || !ind_b || !ind_hl || !ind_ptr || !ind_idx || !vdd ||
        !w64 || !D64 || !invD64 || !ch || !cinj || (g->mixed && (!w32 || !invD32 || !w32lo || !D32 || !D32lo)))
        return PG_ERR_OOM;
    d.colour_slice = colour_slice; d.slice_off = slice_off; d.slice_w = slice_w; d.slice_doff = slice_doff;
    d.dia_off = dia_off; d.ell_col = ell_col; d.orig = orig; d.ld_ptr = ld_ptr; d.ld_idx = ld_idx;
    d.pwl_ptr = pwl_ptr; d.pwl_t = pwl_t; d.pwl_v = pwl_v; d.pwl_s = pwl_s; d.pwl_tk = pwl_tk; d.n_l = P.n_l; d.ind_a = ind_a; d.ind_b = ind_b;
    d.ind_hl = ind_hl; d.ind_ptr = ind_ptr; d.ind_idx = ind_idx; d.vdd = vdd;
    d.w64 = w64; d.D64 = D64; d.invD64 = invD64; d.ch = ch; d.cinj = cinj; d.w32 = w32; d.invD32 = invD32;
    d.w32lo = w32lo; d.D32 = D32; d.D32lo = D32lo;
    pg_status s;
    {
        // component of each permuted node (independent sub-circuits, Fig. 1)
        std::vector<int32_t> nc(np, -1);
        for (int i = 0; i < np; ++i)
            if (P.orig[i] >= 0) nc[i] = P.comp_of[P.orig[i]];
        int32_t* node_comp = g->alloc<int32_t>(np);
        if (!node_comp) return PG_ERR_OOM;
        if ((s = upload(g, node_comp, nc))) return s;
        d.n_comp = P.n_comp;
        d.node_comp = node_comp;
    }
    if (d.lwE &&
        ((s = upload(g, const_cast<int32_t*>(d.lat_info), lat_info)) ||
         (s = upload(g, const_cast<int32_t*>(d.lat_tile0), lat_tile0)) ||
         (s = upload(g, const_cast<int64_t*>(d.lat_col0), lat_col0)) ||
         (s = upload(g, const_cast<int32_t*>(d.node_lat), P.node_lat))))
        return s;
    if ((s = upload(g, colour_slice, cs)) || (s = upload(g, slice_off, P.slice_off)) ||
        (s = upload(g, slice_w, P.slice_w)) || (s = upload(g, slice_doff, P.slice_doff)) ||
        (s = upload(g, dia_off, P.dia_off)) || (s = upload(g, ell_col, P.ell_col)) || (s = upload(g, orig, P.orig)) ||
        (s = upload(g, ld_ptr, P.ld_ptr)) || (s = upload(g, ld_idx, P.ld_idx)) ||
        (s = upload(g, pwl_ptr, P.pwl_ptr)) || (s = upload(g, pwl_t, P.pwl_t)) || (s = upload(g, pwl_v, P.pwl_v)) ||
        (s = upload(g, pwl_s, P.pwl_s)) || (s = upload(g, pwl_tk, P.pwl_tk)) ||
        (s = upload(g, ind_a, P.ind_a)) || (s = upload(g, ind_b, P.ind_b)) || (s = upload(g, ind_ptr, P.ind_ptr)) ||
        (s = upload(g, ind_idx, P.ind_idx)) || (s = upload(g, vdd, P.vdd)))
        return s;

    DevState& st = g->ds;
    for (int k = 0; k < 3; ++k) {
        st.v[k] = g->alloc<double>(np);
        if (!st.v[k]) return PG_ERR_OOM;
        CK(cudaMemsetAsync(st.v[k], 0, np * sizeof(double), g->stream));
    }
    st.il = g->alloc<double>(P.n_l);
    st.md = g->alloc<double>(np);
    if (!st.md) return PG_ERR_OOM;
    d.n_src = (int32_t)(P.pwl_ptr.size() - 1);
    {
        // per-node load currents: a node with one load takes its source's value directly, a
        // node with several sums them (CSR order, deterministic)
        std::vector<int32_t> na(std::max(d.n_src, 1), kLoadNone), nb(std::max(d.n_src, 1), kLoadNone), multi;
        for (int i = 0; i < np; ++i) {
            const int cnt = P.ld_ptr[i + 1] - P.ld_ptr[i];
            if (cnt >= 2) multi.push_back(i);
            for (int q = P.ld_ptr[i]; q < P.ld_ptr[i + 1]; ++q) {
                const int sid = P.ld_idx[q];
                const int e = (sid > 0 ? sid : -sid) - 1;
                (sid > 0 ? na : nb)[e] = cnt == 1 ? i : kLoadMulti;
            }
        }
        int32_t* sa = g->alloc<int32_t>(na.size());
        int32_t* sb = g->alloc<int32_t>(nb.size());
        int32_t* mn = g->alloc<int32_t>(std::max<size_t>(multi.size(), 1));
        st.inode = g->alloc<double>(2 * (size_t)np);
        st.pwl_cur = g->alloc<int32_t>(std::max<size_t>(na.size(), 1));
        st.dinode = g->alloc<double>(np);
        if (!sa || !sb || !mn || !st.inode || !st.pwl_cur || !st.dinode) return PG_ERR_OOM;
        CK(cudaMemsetAsync(st.dinode, 0, (size_t)np * sizeof(double), g->stream));
        CK(cudaMemsetAsync(st.pwl_cur, 0, std::max<size_t>(na.size(), 1) * sizeof(int32_t), g->stream));
        if ((s = upload(g, sa, na)) || (s = upload(g, sb, nb)) || (s = upload(g, mn, multi))) return s;
        CK(cudaMemsetAsync(st.inode, 0, 2 * (size_t)np * sizeof(double), g->stream));
        d.src_na = sa; d.src_nb = sb; d.n_multi = (int32_t)multi.size(); d.multi_node = mn;
    }
    st.r64 = g->alloc<double>(np);
    if (!st.il || !st.r64) return PG_ERR_OOM;
    CK(cudaMemsetAsync(st.il, 0, std::max(1, P.n_l) * sizeof(double), g->stream));
    if (g->mixed) {
        st.r32 = g->alloc<float>(np);
        st.d32[0] = g->alloc<float>(np);
        st.d32[1] = g->alloc<float>(np);
        if (!st.r32 || !st.d32[0] || !st.d32[1]) return PG_ERR_OOM;
        // padding entries are never written by the lattice solve: they stay zero
        CK(cudaMemsetAsync(st.d32[0], 0, np * sizeof(float), g->stream));
        CK(cudaMemsetAsync(st.d32[1], 0, np * sizeof(float), g->stream));
        CK(cudaMemsetAsync(st.r32, 0, np * sizeof(float), g->stream));
    } else {
        st.d64[0] = g->alloc<double>(np);
        st.d64[1] = g->alloc<double>(np);
        if (!st.d64[0] || !st.d64[1]) return PG_ERR_OOM;
    }
    g->d_x = g->alloc<double>(P.n);
    if (!g->d_x) return PG_ERR_OOM;

    // launch shape: every warp gets the same number of slices per colour sweep
    g->smem = persistent_smem_bytes(g->mixed, d.lat_rows, d.lwE ? P.lat_maxnl : 0);   // FP64: 8-byte elements
    int bps = 0;
    CK(persistent_occupancy(g->mixed, d.lat_rows, g->threads, g->smem, &bps));
    if (g->opt.blocks_per_sm > 0) bps = std::min(bps, g->opt.blocks_per_sm);
    if (bps < 1) { g_last_error = "kernel does not fit on an SM"; return PG_ERR_CUDA; }
    const int wpb = g->threads / 32;
    const int max_warps = g->n_sm * bps * wpb;
    int smax = 1;
    for (int c = 0; c < P.ncol; ++c) smax = std::max(smax, cs[c + 1] - cs[c]);
    const int rounds = (smax + max_warps - 1) / max_warps;
    const int warps = (smax + rounds - 1) / rounds;
    g->blocks = std::max(1, std::min(g->n_sm * bps, (warps + wpb - 1) / wpb));

    DevCtl& c = g->dc;
    c.bar_count = g->alloc<unsigned>(1);
    c.bar_gen = g->alloc<unsigned>(1);
    c.err = g->alloc<int32_t>(1);
    c.red = g->alloc<unsigned long long>(kRedSlots);
    c.blk_min = g->alloc<unsigned long long>(2 * g->blocks);
    c.blk_arg = g->alloc<int32_t>(2 * g->blocks);
    c.stats = g->alloc<double>(kStatCount);
    if (!c.bar_count || !c.bar_gen || !c.err || !c.red || !c.blk_min || !c.blk_arg || !c.stats) return PG_ERR_OOM;
    if (d.lwE && !(c.lat_R = g->alloc<unsigned long long>(2 * (size_t)d.n_lats))) return PG_ERR_OOM;
    if (!(c.tile_ctr = g->alloc<unsigned>(1))) return PG_ERR_OOM;
    if (!(c.ld_flags = g->alloc<unsigned>(4))) return PG_ERR_OOM;
    CK(cudaMemsetAsync(c.bar_gen, 0, sizeof(unsigned), g->stream));
    CK(cudaEventCreate(&g->ev0));
    CK(cudaEventCreate(&g->ev1));
    CK(cudaStreamSynchronize(g->stream));
    return PG_OK;
}

// Per-h coefficients of Eq. 14 (node form of M = C/h + G + h L).
pg_status assemble_h(pg_grid* g, double h) {
    const Packed& P = g->P;
    const int np = P.n_pad;
    std::vector<double> D(np, 0.0), iD(np, 0.0), ch(np, 0.0), cinj(np, 0.0);
    for (int i = 0; i < np; ++i) {
        const int o = P.orig[i];
        if (o < 0) continue;
        double s = 0.0;
        for (int64_t a = P.adj_ptr[o]; a < P.adj_ptr[o + 1]; ++a) s += P.adj_g[a] + h * P.adj_il[a];
        const double d = s + P.g_gnd[o] + h * P.il_gnd[o] + P.cap[o] / h;
        D[i] = d; iD[i] = 1.0 / d; ch[i] = P.cap[o] / h; cinj[i] = P.inj_g[o] + h * P.inj_il[o];
    }
    std::vector<double> w(P.n_ell, 0.0);
    for (int64_t e = 0; e < P.n_ell; ++e) {
        const int64_t a = P.ell_adj[e];
        if (a >= 0) w[e] = P.adj_g[a] + h * P.adj_il[a];
    }
    std::vector<double> hl(P.n_l);
    for (int e = 0; e < P.n_l; ++e) hl[e] = h * P.ind_invL[e];
    pg_status s;
    if ((s = upload(g, const_cast<double*>(g->dg.D64), D)) || (s = upload(g, const_cast<double*>(g->dg.invD64), iD)) ||
        (s = upload(g, const_cast<double*>(g->dg.ch), ch)) || (s = upload(g, const_cast<double*>(g->dg.cinj), cinj)) ||
        (s = upload(g, const_cast<double*>(g->dg.w64), w)) || (s = upload(g, const_cast<double*>(g->dg.ind_hl), hl)))
        return s;
    if (g->dg.lwE) {
        // lattice form of the FP32 inner solve: each branch weight once, caller order
        std::vector<float> e(P.n, 0.f), nn(P.n, 0.f), u(P.n, 0.f), mm(P.n, 0.f), ip(P.n, 0.f);
        std::vector<double> u64(P.n, 0.0), e64(P.n, 0.0), n64(P.n, 0.0), m64(P.n, 0.0), ip64(P.n, 0.0);
        for (int o = 0; o < P.n; ++o) {
            for (int64_t a = P.adj_ptr[o]; a < P.adj_ptr[o + 1]; ++a) {
                const double w = P.adj_g[a] + h * P.adj_il[a];
                if (P.adj_dir[a] == 0) { e[o] = (float)w; e64[o] = w; }
                else if (P.adj_dir[a] == 1) { nn[o] = (float)w; n64[o] = w; }
                else if (P.adj_dir[a] == 2) { u[o] = (float)w; u64[o] = w; }
            }
        }
        // Thomas factors of each column's block (diagonal D_l, off-diagonal -u_l between l and l+1)
        for (size_t L = 0; L < P.lats.size() / 4; ++L) {
          const int64_t off = P.lats[4 * L], plane = (int64_t)P.lats[4 * L + 1] * P.lats[4 * L + 2];
          for (int64_t c = 0; c < plane; ++c) {
            double dp_prev = 0.0;
            for (int l = 0; l < P.lats[4 * L + 3]; ++l) {
                const int64_t o = off + c + l * plane;
                double dp = D[P.perm[o]];
                if (l > 0) {
                    const double m = u64[o - plane] / dp_prev;
                    dp -= m * u64[o - plane];
                    mm[o] = (float)m;
                    m64[o] = m;
                }
                ip[o] = (float)(1.0 / dp);
                ip64[o] = 1.0 / dp;
                dp_prev = dp;
            }
          }
        }
        if ((s = upload(g, const_cast<float*>(g->dg.lwE), e)) || (s = upload(g, const_cast<float*>(g->dg.lwN), nn)) ||
            (s = upload(g, const_cast<float*>(g->dg.lwU), u)) || (s = upload(g, const_cast<float*>(g->dg.lm), mm)) ||
            (s = upload(g, const_cast<float*>(g->dg.lip), ip)))
            return s;
        if (g->dg.lwE64 &&
            ((s = upload(g, const_cast<double*>(g->dg.lwE64), e64)) ||
             (s = upload(g, const_cast<double*>(g->dg.lwN64), n64)) ||
             (s = upload(g, const_cast<double*>(g->dg.lwU64), u64)) ||
             (s = upload(g, const_cast<double*>(g->dg.lm64), m64)) ||
             (s = upload(g, const_cast<double*>(g->dg.lip64), ip64))))
            return s;
    }
    if (g->mixed) {
        // FP32 pairs: hi = the rounded value, lo = the rounded remainder
        std::vector<float> w32(P.n_ell), wlo(P.n_ell), iD32(np), d32(np), dlo(np);
        for (int64_t e = 0; e < P.n_ell; ++e) {
            w32[e] = (float)w[e];
            wlo[e] = (float)(w[e] - (double)w32[e]);
        }
        for (int i = 0; i < np; ++i) {
            iD32[i] = (float)iD[i];
            d32[i] = (float)D[i];
            dlo[i] = (float)(D[i] - (double)d32[i]);
        }
        if ((s = upload(g, const_cast<float*>(g->dg.w32), w32)) || (s = upload(g, const_cast<float*>(g->dg.invD32), iD32)) ||
            (s = upload(g, const_cast<float*>(g->dg.w32lo), wlo)) || (s = upload(g, const_cast<float*>(g->dg.D32), d32)) ||
            (s = upload(g, const_cast<float*>(g->dg.D32lo), dlo)))
            return s;
    }
    CK(cudaStreamSynchronize(g->stream));
    return PG_OK;
}

}  // namespace

// warm_start = 2: extrapolation weight once the loads have been static for two intervals
// (full extrapolation there carries the previous steps' iteration errors forward, up to
// three times the per-step target)
constexpr double kThetaStatic = 0.5;

RunParams pg::base_params(const pg_grid* g) {
    RunParams rp{};
    rp.mixed = g->mixed;
    rp.h = g->h;
    rp.omega = g->omega;
    rp.kappa = g->kappa;
    rp.target = g->target;
    rp.inner_reduction = g->opt.inner_reduction;
    rp.max_sweeps = g->opt.max_sweeps;
    rp.max_outer = 50;
    rp.timeout_ns = (long long)(g->opt.barrier_timeout_s * 1e9);
    rp.debug_flags = g->opt.debug_flags;
    rp.cur = g->vL; rp.prev = g->vP;
    // automatic warm start: damped once the loads are quiet on RC grids, full extrapolation
    // on grids with inductors (their LC response keeps moving after the loads stop)
    const int ws = g->opt.warm_start < 0 ? (g->P.n_l == 0 ? 2 : 1) : g->opt.warm_start;
    rp.warm_extrap = ws != 0;
    rp.warm_theta_static = ws == 2 ? kThetaStatic : 1.0;
    rp.lat_k = g->dg.lwE ? g->lat_k : 0;
    rp.three_level = g->opt.form == PG_FORM_THREE_LEVEL;
    rp.jacobi = g->opt.jacobi;
    rp.inc_start = g->inc_ok && g->have_prev;
    rp.prev_outer = g->last_outer;
    return rp;
}

namespace {

// Clear the launch's control words (barrier, error flag, reduction slots); stream-ordered.
pg_status clear_ctl(pg_grid* g) {
    CK(cudaMemsetAsync(g->dc.bar_count, 0, sizeof(unsigned), g->stream));
    CK(cudaMemsetAsync(g->dc.bar_gen, 0, sizeof(unsigned), g->stream));
    CK(cudaMemsetAsync(g->dc.err, 0, sizeof(int32_t), g->stream));
    CK(cudaMemsetAsync(g->dc.red, 0, kRedSlots * sizeof(unsigned long long), g->stream));
    CK(cudaMemsetAsync(g->dc.tile_ctr, 0, sizeof(unsigned), g->stream));
    if (g->dc.lat_R)
        CK(cudaMemsetAsync(g->dc.lat_R, 0, 2 * (size_t)g->dg.n_lats * sizeof(unsigned long long), g->stream));
    return PG_OK;
}

// One persistent launch; reads back the status word and statistics.
pg_status run(pg_grid* g, const RunParams& rp, double* stats, float* ms) {
    pg_status s0 = clear_ctl(g);
    if (s0) return s0;
    CK(cudaEventRecord(g->ev0, g->stream));
    CK(launch_persistent(g->mixed, g->dg, g->ds, g->dc, rp, g->blocks, g->threads, g->smem, g->stream));
    CK(cudaEventRecord(g->ev1, g->stream));
    int32_t err = 0;
    CK(cudaMemcpyAsync(&err, g->dc.err, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaMemcpyAsync(stats, g->dc.stats, kStatCount * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (ms) CK(cudaEventElapsedTime(ms, g->ev0, g->ev1));
    // the final residual and M d of an explicit transient carry into the next launch
    g->inc_ok = err == 0 && rp.mode == kModeTransient && !rp.three_level && stats[kStatSteps] >= 1.0 &&
                stats[kStatSteps] == (double)rp.nsteps;
    if (g->inc_ok) g->last_outer = (int32_t)stats[kStatLastOuter];
    if (err == PG_ERR_TIMEOUT) { g_last_error = "device barrier timed out"; return PG_ERR_TIMEOUT; }
    if (err == PG_ERR_NOT_CONVERGED) { g_last_error = "relaxation did not converge"; return PG_ERR_NOT_CONVERGED; }
    if (err != 0) { g_last_error = "device error"; return PG_ERR_CUDA; }
    return PG_OK;
}

// Solve M x = rhs (rhs: device, permuted) from x = 0 to max|r|/D <= tgt; x (caller order) -> g->d_x.
pg_status solve_internal(pg_grid* g, const double* rhs_perm, double tgt, double* final_R) {
    RunParams rp = base_params(g);
    rp.max_sweeps = std::max(g->opt.max_sweeps, kSetupSweeps);   // setup solves ignore the per-step cap
    // the stopping-rule constants are properties of M, not of the iteration: setup solves
    // always take the coloured SOR (its red-black omega when Jacobi runs the steps)
    if (rp.jacobi) {
        rp.jacobi = 0;
        rp.omega = g->sor_omega;
    }
    rp.mode = kModeSolve;
    rp.nsteps = 1;
    rp.step0 = 0;
    rp.target = tgt;
    rp.have_prev = 0;
    rp.warm_extrap = 0;
    rp.solve_out = g->d_x;
    g->ds.rhs = rhs_perm;
    double stats[kStatCount];
    pg_status s = run(g, rp, stats, nullptr);
    g->ds.rhs = nullptr;
    if (final_R) *final_R = stats[kStatLastR];
    return s;
}

double host_max(pg_grid* g, const double* dptr, int n, pg_status* s) {
    std::vector<double> x(n);
    if (cudaMemcpy(x.data(), dptr, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) {
        *s = PG_ERR_CUDA;
        return 0.0;
    }
    double m = -INFINITY;
    for (double v : x) m = std::max(m, v);
    return m;
}

// Jacobi spectral radius by power iteration on (I + D^-1 W)/2 (Rayleigh quotient: a lower bound).
pg_status estimate_rho(pg_grid* g, double* rho) {
    const int np = g->P.n_pad, iters = 300;
    double *x = nullptr, *y = nullptr, *acc = nullptr;
    unsigned long long* mx = nullptr;
    struct Scratch {
        std::vector<void*> p;
        ~Scratch() { for (void* q : p) cudaFree(q); }
    } scratch;
    auto take = [&](void** q, size_t bytes) {
        if (cudaMalloc(q, bytes) != cudaSuccess) return false;
        scratch.p.push_back(*q);
        return true;
    };
    if (!take((void**)&x, np * sizeof(double)) || !take((void**)&y, np * sizeof(double)) ||
        !take((void**)&acc, 2 * iters * sizeof(double)) || !take((void**)&mx, iters * sizeof(unsigned long long)))
        return PG_ERR_OOM;
    std::vector<double> ones(np, 0.0);
    for (int i = 0; i < np; ++i) ones[i] = g->P.orig[i] >= 0 ? 1.0 : 0.0;
    pg_status s;
    if ((s = upload(g, x, ones))) return s;
    CK(cudaMemsetAsync(acc, 0, 2 * iters * sizeof(double), g->stream));
    CK(cudaMemsetAsync(mx, 0, iters * sizeof(unsigned long long), g->stream));
    const int blocks = std::max(1, std::min(g->n_sm * 4, (g->P.n_slices + 7) / 8));
    for (int k = 0; k < iters; ++k) {
        CK(launch_power_step(g->dg, x, y, k ? mx + (k - 1) : nullptr, acc + 2 * k, mx + k, blocks, g->stream));
        std::swap(x, y);
    }
    std::vector<double> a(2 * iters);
    CK(cudaMemcpyAsync(a.data(), acc, a.size() * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    const double num = a[2 * (iters - 1)], den = a[2 * (iters - 1) + 1];
    *rho = den > 0.0 ? std::min(std::max(num / den, 0.0), 1.0) : 0.0;
    return PG_OK;
}

pg_status create_impl(const pg_netlist* nl, const pg_options* opt, std::unique_ptr<pg_grid>& out);
pg_status prepare_h(pg_grid* g, double h);

// The resistive (DC) network of the grid: capacitors open, inductors open (i_l = 0).
pg_status ensure_dc_grid(pg_grid* g) {
    if (g->dcgrid) return PG_OK;
    pg_netlist d = g->nc.dc_view();
    pg_options o = g->opt;          // same precision as the grid (FP64 sweeps are slow on GB300)
    o.omega = 0.0;
    o.jacobi = 0;                   // the DC network is solved once: coloured SOR
    o.step_tol = 0.5 * g->opt.tol;
    d.lat_nx = g->nc.nx; d.lat_ny = g->nc.ny; d.lat_nl = g->nc.nl;
    d.n_lat = (int32_t)(g->nc.lat_desc.size() / 4);
    d.lat_desc = g->nc.lat_desc.empty() ? nullptr : g->nc.lat_desc.data();
    std::unique_ptr<pg_grid> sub;
    pg_status s = create_impl(&d, &o, sub);
    if (s == PG_ERR_FLOATING_NODE)
        g_last_error = "the resistive network needs every sub-circuit tied to a source or ground by a resistor: " +
                       g_last_error;
    if (s) return s;
    sub->stream = g->stream;
    g->dcgrid = std::move(sub);
    return PG_OK;
}

// kacc >= 1 + ||(G + G0)^-1 (C/h) 1||_inf from one relaxation solve on the DC network, with the
// remainder bounded by that network's own kappa.
pg_status accumulation_bound(pg_grid* g, double h, double* kacc) {
    pg_status s = ensure_dc_grid(g);
    if (s) return s;
    pg_grid* d = g->dcgrid.get();
    d->stream = g->stream;
    if ((s = prepare_h(d, 1.0))) return s;
    std::vector<double> rhs(d->P.n_pad, 0.0);
    for (int i = 0; i < d->P.n_pad; ++i)
        if (d->P.orig[i] >= 0) rhs[i] = g->P.cap[d->P.orig[i]] / h;
    double* rd = nullptr;
    CK(cudaMalloc(&rd, rhs.size() * sizeof(double)));
    if (cudaMemcpy(rd, rhs.data(), rhs.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(rd);
        return PG_ERR_CUDA;
    }
    double R = 0.0;
    s = solve_internal(d, rd, 1e-3 / d->kappa, &R);
    cudaFree(rd);
    if (s) return s;
    const double zmax = host_max(d, d->d_x, d->P.n, &s);
    if (s) return s;
    *kacc = 1.0 + zmax + d->kappa * R;
    return PG_OK;
}

// Spectral radius of the column-block Jacobi operator of a lattice grid (the inner solve's
// relaxation), by power iteration on (I + B^-1 W)/2; Rayleigh quotient, a lower bound.
pg_status estimate_rho_lattice(pg_grid* g, double* rho) {
    const int n = g->P.n, iters = 300;
    DeviceScratch sc;
    double* x = sc.get<double>(n);
    double* y = sc.get<double>(n);
    double* acc = sc.get<double>(2 * iters);
    unsigned long long* mx = sc.get<unsigned long long>(iters);
    if (!x || !y || !acc || !mx) return PG_ERR_OOM;
    std::vector<double> ones(n, 1.0);
    pg_status s;
    if ((s = upload(g, x, ones))) return s;
    CK(cudaMemsetAsync(acc, 0, 2 * iters * sizeof(double), g->stream));
    CK(cudaMemsetAsync(mx, 0, iters * sizeof(unsigned long long), g->stream));
    const int64_t cols = g->dg.lat_cols;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(g->n_sm * 4, (cols + 255) / 256));
    for (int k = 0; k < iters; ++k) {
        CK(launch_lattice_power(g->dg, x, y, k ? mx + (k - 1) : nullptr, acc + 2 * k, mx + k, blocks, g->stream));
        std::swap(x, y);
    }
    std::vector<double> a(2 * iters);
    CK(cudaMemcpyAsync(a.data(), acc, a.size() * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    const double num = a[2 * (iters - 1)], den = a[2 * (iters - 1) + 1];
    *rho = den > 0.0 ? std::min(std::max(num / den, 0.0), 1.0) : 0.0;
    return PG_OK;
}

// Automatic omega: Young's value with omega - 1 scaled by this factor (measured on every
// workload of the test suite: faster than Young's value itself, the best scale between
// 1.005 and 1.03).
constexpr double kOmegaOver = 1.01;

// Per-h setup: coefficients, omega, and the stopping-rule constants kappa, q.
pg_status prepare_h(pg_grid* g, double h) {
    if (g->h == h) return PG_OK;
    if (!(h > 0.0) || !std::isfinite(h)) { g_last_error = "h must be > 0"; return PG_ERR_INVALID_ARG; }
    // A state carried into a new system (another h, or new element values): its accumulated
    // error bound under the old system becomes the starting error of the new series.
    if (g->has_state && g->series_bound > 0.0)
        g->series_bound = std::isfinite(g->kacc) && g->kacc > 0.0 ? g->series_bound * g->kacc : INFINITY;
    pg_status s = assemble_h(g, h);
    if (s) return s;
    g->h = h;
    if (g->opt.omega > 0.0) {
        g->omega = g->opt.omega;
        g->rho = 0.0;
    } else if (g->opt.jacobi) {
        g->omega = 1.0;              // undamped Jacobi unless the caller damps it
        g->rho = 0.0;
    } else {
        if ((s = g->dg.lwE ? estimate_rho_lattice(g, &g->rho) : estimate_rho(g, &g->rho))) return s;
        const double r = std::min(g->rho, 1.0 - 1e-12);
        // red-black (2-cyclic, consistently ordered; the column blocks of the lattice solve
        // are too): Young's optimum, taken 1 % high in omega - 1.  The SOR radius falls
        // steeply up to the optimum and rises with slope 1 past it, so an omega from an
        // estimated rho errs upward.  Other colourings use Gauss-Seidel.
        // (the four-colour lattice order takes the red-black value too: a heuristic that
        // pg_autotune scales up and down)
        if (g->P.ncol == 2 || g->dg.lwE || (g->opt.colouring == PG_COLOUR_FOUR && g->P.lattice)) {
            const double young = 2.0 / (1.0 + std::sqrt(1.0 - r * r));
            g->omega = std::min(1.0 + kOmegaOver * (young - 1.0), 0.5 * (young + 2.0));
        } else {
            g->omega = 1.0;
        }
    }
    g->sor_omega = g->omega;
    if (g->opt.jacobi) {
        // the setup solves below run the coloured SOR: Young's omega for red-black grids
        double r = 0.0;
        if ((s = estimate_rho(g, &r))) return s;
        r = std::min(r, 1.0 - 1e-12);
        g->sor_omega = g->P.ncol == 2 ? 2.0 / (1.0 + std::sqrt(1.0 - r * r)) : 1.0;
        g->rho = r;
    }
    // kappa >= ||M^-1 D||_inf: solve M x = D 1 to max|r|/D <= 1e-3, then bound the remainder.
    g->kappa = 1.0;
    double R = 0.0;
    const double save_omega = g->omega;
    if ((s = solve_internal(g, g->dg.D64, 1e-3, &R))) { g->h = -1.0; return s; }
    double xm = host_max(g, g->d_x, g->P.n, &s);
    if (s) return s;
    g->kappa = xm / (1.0 - R);
    // q >= ||M^-1 C/h||_inf: solve M y = (C/h) 1 and bound the remainder with kappa.
    double cmax = 0.0;
    for (int i = 0; i < g->P.n; ++i) cmax = std::max(cmax, g->P.cap[i] / h);
    if (cmax > 0.0) {
        // a remainder of at most 1e-6 on q: max|r|/D <= 1e-6 / kappa
        if ((s = solve_internal(g, g->dg.ch, 1e-6 / g->kappa, &R))) { g->h = -1.0; return s; }
        const double ym = host_max(g, g->d_x, g->P.n, &s);
        if (s) return s;
        g->q = ym + g->kappa * R;
    } else {
        g->q = 0.0;
    }
    g->omega = save_omega;
    // Accumulation of per-step errors (RC).  With T = M^-1 C/h >= 0 the error of step s is
    // e_s = T e_{s-1} + eta_s, so |e_s| <= max_k |eta_k| * sum_j T^j 1 = max|eta| (I - T)^-1 1, and
    // (I - T)^-1 1 = 1 + (G + G0)^-1 (C/h) 1 because M = C/h + (G + G0).  kacc bounds its max with
    // one solve on the resistive (DC) network; it never exceeds 1 / (1 - q).
    g->kacc = INFINITY;
    if (g->P.n_l == 0) {
        if (cmax == 0.0) g->kacc = 1.0;
        else if ((s = accumulation_bound(g, h, &g->kacc))) { g->h = -1.0; return s; }
        if (g->q < 1.0) g->kacc = std::min(g->kacc, 1.0 / (1.0 - g->q));
    }
    const double tol = g->opt.tol;
    if (g->opt.step_tol > 0.0) g->step_tol = g->opt.step_tol;
    else if (std::isfinite(g->kacc)) g->step_tol = 0.9 * tol / g->kacc;
    else g->step_tol = 1e-4 * tol;
    const double slack = 1e-13;   // rounding allowance on max|r|/D (V)
    g->target = g->step_tol / g->kappa - slack;
    if (!(g->target > 0.0)) {
        g_last_error = "tolerance below the rounding floor (kappa " + std::to_string(g->kappa) + ", q " +
                       std::to_string(g->q) + ", step_tol " + std::to_string(g->step_tol) + ")";
        g->h = -1.0;
        return PG_ERR_INVALID_ARG;
    }
    return PG_OK;
}

pg_status set_state_host(pg_grid* g, const double* v, const double* il, int64_t step) {
    const Packed& P = g->P;
    g->inc_ok = false;
    std::vector<double> vp(P.n_pad, 0.0);
    for (int i = 0; i < P.n_pad; ++i)
        if (P.orig[i] >= 0) vp[i] = v[P.orig[i]];
    g->vL = 0; g->vP = 1;
    pg_status s;
    if ((s = upload(g, g->ds.v[0], vp))) return s;
    if (P.n_l) {
        if (il) CK(cudaMemcpyAsync(g->ds.il, il, P.n_l * sizeof(double), cudaMemcpyHostToDevice, g->stream));
        else CK(cudaMemsetAsync(g->ds.il, 0, P.n_l * sizeof(double), g->stream));
    }
    CK(cudaStreamSynchronize(g->stream));
    g->has_state = true;
    g->step = step;
    g->have_prev = false;
    return PG_OK;
}

// State from a device vector in caller numbering (src) or a constant (src == nullptr).
pg_status set_state_device(pg_grid* g, const double* src, double fill, const double* il, int64_t step) {
    g->inc_ok = false;
    g->series_bound = 0.0;
    g->vL = 0; g->vP = 1;
    CK(launch_permute_in(g->dg.orig, src, fill, g->ds.v[0], g->P.n_pad, g->n_sm, g->stream));
    if (g->P.n_l) {
        if (il) CK(cudaMemcpyAsync(g->ds.il, il, g->P.n_l * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        else CK(cudaMemsetAsync(g->ds.il, 0, g->P.n_l * sizeof(double), g->stream));
    }
    g->has_state = true;
    g->step = step;
    g->have_prev = false;
    return PG_OK;
}

// DC operating point at t = 0 (Section IV-B, first step): capacitors open, i_l(0) = 0.
pg_status dc_init(pg_grid* g) {
    if (g->dc_trivial) return set_state_device(g, nullptr, g->dc_vdd, nullptr, 0);
    pg_status s = ensure_dc_grid(g);
    if (s) return s;
    pg_grid* d = g->dcgrid.get();
    d->stream = g->stream;
    double vmean = 0.0;
    for (double x : g->nc.vdd) vmean += x;
    vmean = g->nc.vdd.empty() ? 0.0 : vmean / g->nc.vdd.size();
    // The DC network has no C and no L, so its coefficients do not depend on h (any h > 0
    // assembles them).  Its solve error enters the transient like one more step error, so it
    // gets the main grid's per-step target.
    if ((s = prepare_h(d, 1.0))) return s;
    const double target = (g->step_tol > 0.0 ? g->step_tol : 0.5 * g->opt.tol) / d->kappa - 1e-13;
    if ((s = set_state_device(d, nullptr, vmean, nullptr, -1))) return s;
    RunParams rp = base_params(d);
    rp.mode = kModeTransient;
    rp.nsteps = 1;
    rp.step0 = -1;   // one step landing on t = 0
    rp.have_prev = 0;
    rp.target = target;
    rp.solve_out = d->d_x;
    double stats[kStatCount];
    if ((s = run(d, rp, stats, nullptr))) return s;
    if ((s = set_state_device(g, d->d_x, 0.0, nullptr, 0))) return s;
    g->series_bound = d->kappa * (stats[kStatMaxBound] + 1e-13);
    return PG_OK;
}

pg_status create_impl(const pg_netlist* nl, const pg_options* opt, std::unique_ptr<pg_grid>& out) {
    std::unique_ptr<pg_grid> g(new pg_grid());
    pg_default_options(&g->opt);
    if (opt) g->opt = *opt;
    pg_options& o = g->opt;
    if (o.precision != PG_PREC_FP64 && o.precision != PG_PREC_MIXED) { g_last_error = "bad precision"; return PG_ERR_INVALID_ARG; }
    if (o.omega < 0.0 || o.omega >= 2.0 || !std::isfinite(o.omega)) {
        g_last_error = "omega must be in (0, 2) (Eq. 17), or 0 for automatic";
        return PG_ERR_INVALID_ARG;
    }
    if (o.tol <= 0.0) o.tol = 1e-6;
    if (o.max_sweeps <= 0) o.max_sweeps = 20000;
    // 0 = by grid class (what pg_autotune finds): batches of many lattices take more frequent
    // FP64 passes, whose per-lattice residuals let converged grids drop out of the inner solve
    if (o.inner_reduction <= 0.0) o.inner_reduction = nl && nl->n_lat > 8 ? 1e-1 : 1e-3;
    if (o.threads_per_block <= 0) o.threads_per_block = 256;
    if (o.threads_per_block != 256) { g_last_error = "threads_per_block must be 256"; return PG_ERR_INVALID_ARG; }
    if (o.barrier_timeout_s <= 0.0) o.barrier_timeout_s = 2.0;
    if (o.lattice_sweeps > 7) { g_last_error = "lattice_sweeps must be <= 7"; return PG_ERR_INVALID_ARG; }
    if (o.jacobi != 0 && o.jacobi != 1) { g_last_error = "jacobi must be 0 or 1"; return PG_ERR_INVALID_ARG; }
    if (o.warm_start < -1 || o.warm_start > 2) { g_last_error = "warm_start must be -1, 0, 1 or 2"; return PG_ERR_INVALID_ARG; }
    if (o.jacobi && o.omega > 1.0) { g_last_error = "damped Jacobi needs omega <= 1"; return PG_ERR_INVALID_ARG; }
    if (o.colouring < PG_COLOUR_AUTO || o.colouring > PG_COLOUR_FOUR) {
        g_last_error = "colouring must be PG_COLOUR_AUTO, PG_COLOUR_RED_BLACK or PG_COLOUR_FOUR";
        return PG_ERR_INVALID_ARG;
    }
    if (o.tile_rows != 0 && o.tile_rows != 34 && o.tile_rows != 66) {
        g_last_error = "tile_rows must be 0, 34 or 66";
        return PG_ERR_INVALID_ARG;
    }
    if (o.tile_rows == 66 && o.precision != PG_PREC_MIXED) {
        g_last_error = "tile_rows 66 needs mixed precision (the FP64 lattice solve takes 34-row regions)";
        return PG_ERR_INVALID_ARG;
    }
    if (o.form != PG_FORM_EXPLICIT && o.form != PG_FORM_THREE_LEVEL) {
        g_last_error = "form must be PG_FORM_EXPLICIT or PG_FORM_THREE_LEVEL";
        return PG_ERR_INVALID_ARG;
    }
    g->threads = o.threads_per_block;
    g->mixed = o.precision == PG_PREC_MIXED;
    std::string why;
    // automatic lattice solve: in FP64 only for netlists of at most 8 lattices (one FP64 region
    // fills an SM, and a batch of small grids runs faster on the point sweeps)
    int32_t lat_policy = o.jacobi ? INT32_MIN : o.lattice_sweeps;
    if (lat_policy == 0 && o.precision != PG_PREC_MIXED && nl && nl->n_lat > 8) lat_policy = -1;
    pg_status s = build_packed(nl, &g->P, &why, lat_policy, o.colouring);
    if (s) { g_last_error = why; return s; }
    g->nc.from(nl);
    compute_dc_trivial(g.get());
    CK(cudaGetDevice(&g->device));
    CK(cudaDeviceGetAttribute(&g->n_sm, cudaDevAttrMultiProcessorCount, g->device));
    int coop = 0;
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device));
    if (!coop) { g_last_error = "device lacks cooperative launch"; return PG_ERR_CUDA; }
    pg::noalloc_bind_device(g->device);
    if ((s = alloc_device(g.get()))) return s;
    out = std::move(g);
    return PG_OK;
}

// `prior`: the largest per-step bound of the series before this run (the start state's
// error and earlier runs continued by this one); the accumulated bound covers both.
pg_status fill_stats(pg_grid* g, const double* st, float ms, pg_run_stats* out, double prior) {
    return pg::fill_run_stats(g, st, ms, out, prior);
}

}  // namespace

pg_status pg::fill_run_stats(pg_grid* g, const double* st, float ms, pg_run_stats* out, double prior) {
    if (!out) return PG_OK;
    std::memset(out, 0, sizeof(*out));
    out->steps_done = (int64_t)st[kStatSteps];
    out->total_sweeps = (int64_t)st[kStatSweeps];
    out->max_sweeps_step = (int32_t)st[kStatMaxSweeps];
    out->total_outer = (int64_t)st[kStatOuter];
    out->max_outer_step = (int32_t)st[kStatMaxOuter];
    out->max_step_bound = g->kappa * (st[kStatMaxBound] + 1e-13);
    // the three-level form carries no i_l state: its step errors add up instead of decaying
    out->err_bound = std::isfinite(g->kacc) && g->opt.form == PG_FORM_EXPLICIT
                         ? std::max(out->max_step_bound, prior) * g->kacc : NAN;
    out->failed_step = (int64_t)st[kStatFailedStep];
    out->omega = g->omega;
    out->rho_jacobi = g->rho;
    out->kappa = g->kappa;
    out->q = g->q;
    out->step_tol = g->step_tol;
    out->device_ms = ms;
    out->kacc = g->kacc;
    out->lattice_sweeps = g->lat_k;
    for (int k = 0; k < 4; ++k) out->phase_ms[k] = st[kStatTimeA + k] * 1e-6;
    return PG_OK;
}

extern "C" {

void pg_default_options(pg_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = PG_PREC_FP64;
    o->omega = 0.0;
    o->tol = 1e-6;
    o->step_tol = 0.0;
    o->max_sweeps = 20000;
    o->warm_start = -1;
    o->inner_reduction = 0.0;
    o->threads_per_block = 256;
    o->blocks_per_sm = 0;
    o->barrier_timeout_s = 2.0;
    o->debug_flags = 0;
    o->form = PG_FORM_EXPLICIT;
}

const char* pg_status_str(pg_status s) {
    switch (s) {
        case PG_OK: return "PG_OK";
        case PG_ERR_INVALID_ARG: return "PG_ERR_INVALID_ARG";
        case PG_ERR_FLOATING_NODE: return "PG_ERR_FLOATING_NODE";
        case PG_ERR_OOM: return "PG_ERR_OOM";
        case PG_ERR_CUDA: return "PG_ERR_CUDA";
        case PG_ERR_NOT_CONVERGED: return "PG_ERR_NOT_CONVERGED";
        case PG_ERR_TIMEOUT: return "PG_ERR_TIMEOUT";
        case PG_ERR_UNSUPPORTED: return "PG_ERR_UNSUPPORTED";
    }
    return "PG_ERR_UNKNOWN";
}

// Human-readable detail of the last error on this thread (not part of the
// stable ABI contract; useful in bindings and logs).
const char* pg_last_error(void) { return g_last_error.c_str(); }

pg_status pg_create_grid(const pg_netlist* nl, const pg_options* opt, pg_grid** out) {
    if (!out) return PG_ERR_INVALID_ARG;
    *out = nullptr;
    std::unique_ptr<pg_grid> g;
    pg_status s;
    try {
        s = create_impl(nl, opt, g);
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return PG_ERR_OOM;
    }
    if (s) return s;
    *out = g.release();
    return PG_OK;
}

void pg_destroy(pg_grid* g) { delete g; }

pg_status pg_set_stream(pg_grid* g, void* stream) {
    if (!g) return PG_ERR_INVALID_ARG;
    g->stream = static_cast<cudaStream_t>(stream);
    if (g->dcgrid) g->dcgrid->stream = g->stream;
    return PG_OK;
}

pg_status pg_grid_info(const pg_grid* g, int32_t* n, int32_t* nl, int32_t* ncol, int32_t* npad) {
    if (!g) return PG_ERR_INVALID_ARG;
    if (n) *n = g->P.n;
    if (nl) *nl = g->P.n_l;
    if (ncol) *ncol = g->P.ncol;
    if (npad) *npad = g->P.n_pad;
    return PG_OK;
}

pg_status pg_initial_conditions(pg_grid* g, double h, const double* vc0, const double* il0, int32_t on_host) {
    if (!g) return PG_ERR_INVALID_ARG;
    g->inc_ok = false;              // the carried step-start data no longer match
    pg_status s = prepare_h(g, h);
    if (s) return s;
    const NetCopy& nc = g->nc;
    std::vector<double> hvc, hil;
    const double* pvc = vc0;
    const double* pil = il0;
    if (!on_host) {
        if (vc0) {
            hvc.resize(nc.c_val.size());
            CK(cudaMemcpy(hvc.data(), vc0, hvc.size() * sizeof(double), cudaMemcpyDeviceToHost));
            pvc = hvc.data();
        }
        if (il0) {
            hil.resize(nc.l_val.size());
            CK(cudaMemcpy(hil.data(), il0, hil.size() * sizeof(double), cudaMemcpyDeviceToHost));
            pil = hil.data();
        }
    }
    std::vector<double> v0, v1, il1;
    // each DC solve to the per-step target (a derived grid without capacitors has kacc = 1,
    // so its step target is half its tol)
    if ((s = pg::paper_initial_levels(nc, h, 2.0 * g->step_tol, g->stream, pvc, pil, v0, v1, il1))) return s;
    const Packed& P = g->P;
    std::vector<double> p0(P.n_pad, 0.0), p1(P.n_pad, 0.0);
    for (int i = 0; i < P.n_pad; ++i)
        if (P.orig[i] >= 0) { p0[i] = v0[P.orig[i]]; p1[i] = v1[P.orig[i]]; }
    g->vL = 0; g->vP = 1;
    if ((s = upload(g, g->ds.v[0], p1)) || (s = upload(g, g->ds.v[1], p0))) return s;
    if (P.n_l) CK(cudaMemcpyAsync(g->ds.il, il1.data(), P.n_l * sizeof(double), cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    g->has_state = true;
    g->step = 1;
    g->have_prev = true;
    return PG_OK;
}

pg_status pg_grid_components(const pg_grid* g, int32_t* n_comp, int32_t* comp_of) {
    if (!g) return PG_ERR_INVALID_ARG;
    if (n_comp) *n_comp = g->P.n_comp;
    if (comp_of) std::memcpy(comp_of, g->P.comp_of.data(), g->P.n * sizeof(int32_t));
    return PG_OK;
}

pg_status pg_set_state(pg_grid* g, const double* v, const double* il, int64_t step, int32_t on_host) {
    if (!g) return PG_ERR_INVALID_ARG;
    if (!v) {
        g->has_state = false;
        return PG_OK;
    }
    if (!on_host) return set_state_device(g, v, 0.0, il, step);
    return set_state_host(g, v, il, step);
}

pg_status pg_get_state(pg_grid* g, double* v, double* il, int64_t* step, int32_t on_host) {
    if (!g) return PG_ERR_INVALID_ARG;
    if (!g->has_state) { g_last_error = "no state"; return PG_ERR_INVALID_ARG; }
    const Packed& P = g->P;
    if (v) {
        std::vector<double> vp(P.n_pad), out(P.n);
        CK(cudaMemcpyAsync(vp.data(), g->ds.v[g->vL], P.n_pad * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        CK(cudaStreamSynchronize(g->stream));
        for (int i = 0; i < P.n_pad; ++i)
            if (P.orig[i] >= 0) out[P.orig[i]] = vp[i];
        if (on_host) std::memcpy(v, out.data(), P.n * sizeof(double));
        else CK(cudaMemcpy(v, out.data(), P.n * sizeof(double), cudaMemcpyHostToDevice));
    }
    if (il && P.n_l) {
        CK(cudaMemcpyAsync(il, g->ds.il, P.n_l * sizeof(double),
                           on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, g->stream));
        CK(cudaStreamSynchronize(g->stream));
    }
    if (step) *step = g->step;
    return PG_OK;
}

pg_status pg_reset(pg_grid* g) {
    if (!g) return PG_ERR_INVALID_ARG;
    g->inc_ok = false;              // the carried step-start data no longer match
    g->has_state = false;
    return PG_OK;
}

pg_status pg_update_sources(pg_grid* g, const double* i_t, const double* i_v, int32_t on_host) {
    if (!g) return PG_ERR_INVALID_ARG;
    g->inc_ok = false;              // the carried step-start data no longer match
    const size_t m = g->P.pwl_t.size();
    if (m == 0) return PG_OK;
    auto pull = [&](const double* src, std::vector<double>& dst) -> pg_status {
        if (on_host) std::memcpy(dst.data(), src, m * sizeof(double));
        else CK(cudaMemcpy(dst.data(), src, m * sizeof(double), cudaMemcpyDeviceToHost));
        return PG_OK;
    };
    std::vector<double> t = g->nc.i_t, v = g->nc.i_v;
    pg_status s;
    if (i_t && (s = pull(i_t, t))) return s;
    if (i_v && (s = pull(i_v, v))) return s;
    for (size_t e = 0; e + 1 < g->nc.i_ptr.size(); ++e)
        for (int64_t k = g->nc.i_ptr[e]; k < g->nc.i_ptr[e + 1]; ++k) {
            if (!std::isfinite(t[k]) || !std::isfinite(v[k])) { g_last_error = "non-finite PWL"; return PG_ERR_INVALID_ARG; }
            if (k > g->nc.i_ptr[e] && t[k] < t[k - 1]) { g_last_error = "PWL times must be non-decreasing"; return PG_ERR_INVALID_ARG; }
        }
    if (i_t) {
        CK(cudaMemcpyAsync(const_cast<double*>(g->dg.pwl_t), i_t, m * sizeof(double),
                           on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream));
        g->nc.i_t = t;
    }
    if (i_v) {
        CK(cudaMemcpyAsync(const_cast<double*>(g->dg.pwl_v), i_v, m * sizeof(double),
                           on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, g->stream));
        g->nc.i_v = v;
    }
    // the slopes and time keys follow the new breakpoints
    pwl_aux(g->P.pwl_ptr, t, v, &g->P.pwl_s, &g->P.pwl_tk);
    g->P.pwl_t = t;
    g->P.pwl_v = v;
    CK(cudaMemcpyAsync(const_cast<double*>(g->dg.pwl_s), g->P.pwl_s.data(), m * sizeof(double),
                       cudaMemcpyHostToDevice, g->stream));
    CK(cudaMemcpyAsync(const_cast<unsigned long long*>(g->dg.pwl_tk), g->P.pwl_tk.data(),
                       m * sizeof(unsigned long long), cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));        // the host vectors are the copies' sources
    compute_dc_trivial(g);
    g->dcgrid.reset();
    return PG_OK;
}

pg_status pg_update_values(pg_grid* g, const double* r_g, const double* c_val, const double* l_val, int32_t on_host) {
    if (!g) return PG_ERR_INVALID_ARG;
    g->inc_ok = false;              // the carried step-start data no longer match
    NetCopy& nc = g->nc;
    auto pull = [&](const double* src, std::vector<double>& dst) -> pg_status {
        if (!src || dst.empty()) return PG_OK;
        if (on_host) std::memcpy(dst.data(), src, dst.size() * sizeof(double));
        else CK(cudaMemcpy(dst.data(), src, dst.size() * sizeof(double), cudaMemcpyDeviceToHost));
        return PG_OK;
    };
    NetCopy trial = nc;
    pg_status s;
    if ((s = pull(r_g, trial.r_g)) || (s = pull(c_val, trial.c_val)) || (s = pull(l_val, trial.l_val))) return s;
    pg_netlist view{};
    view.n_nodes = trial.n; view.n_sources = trial.p; view.vdd = trial.vdd.data();
    view.n_r = (int64_t)trial.r_g.size(); view.r_a = trial.r_a.data(); view.r_b = trial.r_b.data(); view.r_g = trial.r_g.data();
    view.n_c = (int64_t)trial.c_val.size(); view.c_a = trial.c_a.data(); view.c_b = trial.c_b.data(); view.c_val = trial.c_val.data();
    view.n_l = (int64_t)trial.l_val.size(); view.l_a = trial.l_a.data(); view.l_b = trial.l_b.data(); view.l_val = trial.l_val.data();
    std::string why;
    // refill_values changes only the value arrays: keep those to restore on a refusal
    Packed& P = g->P;
    auto keep = std::make_tuple(P.adj_g, P.adj_il, P.g_gnd, P.il_gnd, P.cap, P.inj_g, P.inj_il, P.ind_invL);
    if ((s = refill_values(&view, &P, &why))) {
        std::tie(P.adj_g, P.adj_il, P.g_gnd, P.il_gnd, P.cap, P.inj_g, P.inj_il, P.ind_invL) = std::move(keep);
        g_last_error = why;
        return s;
    }
    nc = std::move(trial);
    g->h = -1.0;            // re-assemble the per-h coefficients on the next call
    // The resistive (DC) network has the same topology: refill its resistor values in place
    // (capacitors and inductors are not part of it); rebuild it only if that fails.
    if (g->dcgrid && r_g) {
        pg_netlist dv = nc.dc_view();
        std::string why2;
        if (refill_values(&dv, &g->dcgrid->P, &why2) == PG_OK) {
            g->dcgrid->nc.r_g = nc.r_g;
            g->dcgrid->h = -1.0;
            g->dcgrid->inc_ok = false;
        } else {
            g->dcgrid.reset();
        }
    }
    return PG_OK;
}

pg_status pg_transient(pg_grid* g, double h, int32_t nsteps, const pg_output* out, pg_run_stats* stats) {
    if (!g || nsteps < 0) return PG_ERR_INVALID_ARG;
    pg_status s = prepare_h(g, h);
    if (s) return s;
    if (!g->has_state && (s = dc_init(g))) return s;
    if (g->opt.form == PG_FORM_THREE_LEVEL && out && out->il_all) {
        g_last_error = "the three-level form keeps no inductor currents";
        return PG_ERR_INVALID_ARG;
    }
    if (nsteps == 0) {
        double z[kStatCount] = {0};
        z[kStatFailedStep] = -1;
        return fill_stats(g, z, 0.f, stats, g->series_bound);
    }
    RunParams rp = base_params(g);
    rp.mode = kModeTransient;
    rp.nsteps = nsteps;
    rp.step0 = g->step;
    rp.have_prev = g->have_prev;
    const Packed& P = g->P;
    // outputs: device pointers directly, or device staging for host pointers
    const bool host = out && out->on_host;
    std::vector<void*> tmp;
    auto stage = [&](void* user, size_t bytes) -> void* {
        if (!user) return nullptr;
        if (!host) return user;
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
        tmp.push_back(p);
        return p;
    };
    auto cleanup = [&]() { for (void* p : tmp) cudaFree(p); };
    int32_t* probes_perm = nullptr;
    if (out) {
        rp.v_all = (double*)stage(out->v_all, (size_t)nsteps * P.n * sizeof(double));
        rp.il_all = P.n_l ? (double*)stage(out->il_all, (size_t)nsteps * P.n_l * sizeof(double)) : nullptr;
        rp.vmin = (double*)stage(out->vmin, (size_t)nsteps * sizeof(double));
        rp.vmin_node = (int32_t*)stage(out->vmin_node, (size_t)nsteps * sizeof(int32_t));
        rp.comp_vmin = (double*)stage(out->comp_vmin, (size_t)nsteps * P.n_comp * sizeof(double));
        if (out->n_probes > 0 && out->probes && out->probe_v) {
            std::vector<int32_t> pr(out->n_probes);
            if (host) std::memcpy(pr.data(), out->probes, pr.size() * sizeof(int32_t));
            else if (cudaMemcpy(pr.data(), out->probes, pr.size() * sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
                cleanup();
                return PG_ERR_CUDA;
            }
            for (auto& x : pr) {
                if (x < 0 || x >= P.n) { cleanup(); g_last_error = "probe out of range"; return PG_ERR_INVALID_ARG; }
                x = P.perm[x];
            }
            if (cudaMalloc((void**)&probes_perm, pr.size() * sizeof(int32_t)) != cudaSuccess) { cleanup(); return PG_ERR_OOM; }
            tmp.push_back(probes_perm);
            if (cudaError_t e = cudaMemcpy(probes_perm, pr.data(), pr.size() * sizeof(int32_t),
                                           cudaMemcpyHostToDevice)) {
                cleanup();
                return cuda_fail(e, "probe upload");
            }
            rp.n_probes = out->n_probes;
            rp.probes_perm = probes_perm;
            rp.probe_v = (double*)stage(out->probe_v, (size_t)nsteps * out->n_probes * sizeof(double));
        }
        if ((out->v_all && !rp.v_all) || (out->vmin && !rp.vmin) || (out->comp_vmin && !rp.comp_vmin)) {
            cleanup();
            return PG_ERR_OOM;
        }
    }
    double st[kStatCount];
    float ms = 0.f;
    const double prior = g->series_bound;
    s = run(g, rp, st, &ms);
    // advance the state by the steps that completed
    const int64_t done = (int64_t)st[kStatSteps];
    if (done > 0) g->series_bound = std::max(prior, g->kappa * (st[kStatMaxBound] + 1e-13));
    for (int64_t k = 0; k < done; ++k) {
        const int vF = 3 - g->vL - g->vP;
        g->vP = g->vL;
        g->vL = vF;
    }
    g->step += done;
    if (done > 0) g->have_prev = true;
    cudaError_t copy_err = cudaSuccess;   // the first failed copy-back, reported if the run succeeded
    if (host && out) {
        auto back = [&](void* user, void* dev, size_t bytes) {
            if (!user || !dev || !bytes) return;
            const cudaError_t e = cudaMemcpy(user, dev, bytes, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess && copy_err == cudaSuccess) copy_err = e;
        };
        back(out->v_all, rp.v_all, (size_t)done * P.n * sizeof(double));
        back(out->il_all, rp.il_all, (size_t)done * P.n_l * sizeof(double));
        back(out->vmin, rp.vmin, (size_t)done * sizeof(double));
        back(out->vmin_node, rp.vmin_node, (size_t)done * sizeof(int32_t));
        back(out->probe_v, rp.probe_v, (size_t)done * rp.n_probes * sizeof(double));
        back(out->comp_vmin, rp.comp_vmin, (size_t)done * P.n_comp * sizeof(double));
    }
    cleanup();
    fill_stats(g, st, ms, stats, prior);
    if (s == PG_OK && copy_err != cudaSuccess) return cuda_fail(copy_err, "output copy to the host");
    return s;
}

pg_status pg_transient_async(pg_grid* g, double h, int32_t nsteps, const double* v0, const pg_output* out,
                             void* dstats) {
    if (!g || nsteps < 1) return PG_ERR_INVALID_ARG;
    const bool any_out = out && (out->v_all || out->il_all || out->vmin || out->vmin_node || out->comp_vmin);
    if (out && ((any_out && out->on_host) || out->n_probes > 0)) {
        g_last_error = "pg_transient_async takes device outputs and no probes";
        return PG_ERR_INVALID_ARG;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(g->stream, &cap));
    if (cap == cudaStreamCaptureStatusNone) {
        // outside a capture, refuse pointers the device cannot address
        const void* ptrs[] = {v0, out ? out->v_all : nullptr, out ? out->il_all : nullptr,
                              out ? out->vmin : nullptr, out ? out->vmin_node : nullptr,
                              out ? out->comp_vmin : nullptr, dstats};
        for (const void* p : ptrs) {
            if (!p) continue;
            cudaPointerAttributes a{};
            if (cudaPointerGetAttributes(&a, p) != cudaSuccess ||
                (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
                cudaGetLastError();
                g_last_error = "pg_transient_async: a buffer is not device memory";
                return PG_ERR_INVALID_ARG;
            }
        }
    }
    pg_status s;
    if (g->h != h) {
        if (cap != cudaStreamCaptureStatusNone) {
            g_last_error = "h is not assembled: call pg_transient(g, h, 0, ...) before capturing";
            return PG_ERR_INVALID_ARG;
        }
        if ((s = prepare_h(g, h))) return s;
    }
    const NetCopy& nc = g->nc;
    if (!v0) {
        bool one = nc.p > 0;
        for (int k = 1; k < nc.p && one; ++k) one = nc.vdd[k] == nc.vdd[0];
        if (!one) {
            g_last_error = "v0 = NULL needs a single supply level";
            return PG_ERR_INVALID_ARG;
        }
    }
    if ((s = set_state_device(g, v0, v0 ? 0.0 : nc.vdd[0], nullptr, 0))) return s;
    RunParams rp = base_params(g);
    rp.mode = kModeTransient;
    rp.nsteps = nsteps;
    rp.step0 = 0;
    rp.have_prev = 0;
    if (out) {
        rp.v_all = out->v_all;
        rp.il_all = g->P.n_l ? out->il_all : nullptr;
        rp.vmin = out->vmin;
        rp.vmin_node = out->vmin_node;
        rp.comp_vmin = out->comp_vmin;
    }
    g->has_state = false;          // the host does not follow the device state of this launch
    if ((s = clear_ctl(g))) return s;
    CK(launch_persistent(g->mixed, g->dg, g->ds, g->dc, rp, g->blocks, g->threads, g->smem, g->stream));
    if (dstats) {
        CK(cudaMemcpyAsync(dstats, g->dc.stats, kStatCount * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        CK(cudaMemcpyAsync(static_cast<char*>(dstats) + kStatCount * sizeof(double), g->dc.err, sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, g->stream));
    }
    return PG_OK;
}

pg_status pg_async_stats(pg_grid* g, const void* dstats, pg_run_stats* stats) {
    if (!g || !dstats) return PG_ERR_INVALID_ARG;
    static_assert(kStatCount * sizeof(double) + sizeof(int32_t) <= PG_ASYNC_STATS_BYTES, "stats record size");
    unsigned char rec[PG_ASYNC_STATS_BYTES];
    CK(cudaMemcpyAsync(rec, dstats, kStatCount * sizeof(double) + sizeof(int32_t), cudaMemcpyDeviceToHost,
                       g->stream));
    CK(cudaStreamSynchronize(g->stream));
    double st[kStatCount];
    int32_t err = 0;
    std::memcpy(st, rec, sizeof(st));
    std::memcpy(&err, rec + sizeof(st), sizeof(err));
    fill_stats(g, st, 0.f, stats, 0.0);   // the run started from the state it set itself
    if (err == PG_ERR_TIMEOUT) { g_last_error = "device barrier timed out"; return PG_ERR_TIMEOUT; }
    if (err == PG_ERR_NOT_CONVERGED) { g_last_error = "relaxation did not converge"; return PG_ERR_NOT_CONVERGED; }
    if (err != 0) { g_last_error = "device error"; return PG_ERR_CUDA; }
    return PG_OK;
}

pg_status pg_step(pg_grid* g, double h, double* v_out, pg_run_stats* stats) {
    pg_output o{};
    o.v_all = v_out;
    return pg_transient(g, h, 1, v_out ? &o : nullptr, stats);
}

pg_status pg_adjoint(pg_grid* g, double h, int32_t nsteps, const pg_objective* obj, int32_t ckpt_every,
                     double* J, double* dJ_dG, double* dJ_dC, double* dJ_dL, int32_t on_host, pg_run_stats* stats) {
    if (!g || nsteps < 1 || !obj || ckpt_every < 0) return PG_ERR_INVALID_ARG;
    if (obj->kind != PG_OBJ_SOFTPLUS_DROP) { g_last_error = "unknown objective"; return PG_ERR_INVALID_ARG; }
    if (g->opt.form != PG_FORM_EXPLICIT) { g_last_error = "the adjoint needs the explicit form"; return PG_ERR_UNSUPPORTED; }
    const int ck = ckpt_every > 0 ? ckpt_every : 50;
    pg_status s = prepare_h(g, h);
    if (s) return s;
    const Packed& P = g->P;
    const int np = P.n_pad;
    const int nseg = (nsteps + ck - 1) / ck;
    DeviceScratch sc;   // released on every exit path
    double* ck_v = sc.get<double>((size_t)nseg * np);
    double* ck_vp = sc.get<double>((size_t)nseg * np);
    double* part = sc.get<double>((size_t)nsteps * g->blocks);
    double* vseg = sc.get<double>((size_t)(ck + 1) * np);
    double* lam = sc.get<double>(np);
    double* lam_next = sc.get<double>(np);
    double* rhs = sc.get<double>(np);
    double* acc_slot = sc.get<double>(P.n_ell);
    double* acc_lv = sc.get<double>(np);
    double* acc_l = sc.get<double>(np);
    double* acc_dv = sc.get<double>(np);
    unsigned long long* scale = sc.get<unsigned long long>(1);
    const int nl = P.n_l;
    double* ck_il = nl ? sc.get<double>((size_t)nseg * nl) : nullptr;   // i_l at each segment start
    // the step-start residual and M d carried across launches, so that a replayed segment
    // repeats the forward pass exactly whatever the checkpoint spacing
    double* ck_r = sc.get<double>((size_t)nseg * np);
    double* ck_md = sc.get<double>((size_t)nseg * np);
    if (!ck_r || !ck_md) return PG_ERR_OOM;
    std::vector<char> ck_inc(nseg, 0);
    std::vector<int32_t> ck_outer(nseg, 0);
    double* mu_l = nl ? sc.get<double>(nl) : nullptr;                   // inductor multipliers
    double* acc_L = nl ? sc.get<double>(nl) : nullptr;
    if (!ck_v || !ck_vp || !part || !vseg || !lam || !lam_next || !rhs || !acc_slot || !acc_lv || !acc_l ||
        !acc_dv || !scale || (nl && (!ck_il || !mu_l || !acc_L)))
        return PG_ERR_OOM;
    std::vector<int> ck_have(nseg, 0);
    auto advance = [&](int64_t done) {
        for (int64_t k = 0; k < done; ++k) { const int vF = 3 - g->vL - g->vP; g->vP = g->vL; g->vL = vF; }
        g->step += done;
        if (done > 0) g->have_prev = true;
    };
    double st[kStatCount];
    float ms_total = 0.f, ms = 0.f;
    int64_t sweeps = 0, outer = 0;
    double worst = 0.0;
    auto account = [&]() {
        ms_total += ms; sweeps += (int64_t)st[kStatSweeps]; outer += (int64_t)st[kStatOuter];
        worst = std::max(worst, st[kStatMaxBound]);
    };

    // forward pass from the DC point, keeping (v_s, v_{s-1}) at every segment start
    g->has_state = false;
    if ((s = dc_init(g))) return s;
    const double dc_bound = g->series_bound;
    for (int k = 0; k < nseg; ++k) {
        const int s0 = k * ck, len = std::min(ck, nsteps - s0);
        CK(cudaMemcpyAsync(ck_v + (size_t)k * np, g->ds.v[g->vL], np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        CK(cudaMemcpyAsync(ck_vp + (size_t)k * np, g->ds.v[g->vP], np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        if (nl)
            CK(cudaMemcpyAsync(ck_il + (size_t)k * nl, g->ds.il, nl * sizeof(double), cudaMemcpyDeviceToDevice,
                               g->stream));
        ck_have[k] = g->have_prev;
        CK(cudaMemcpyAsync(ck_r + (size_t)k * np, g->ds.r64, np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        CK(cudaMemcpyAsync(ck_md + (size_t)k * np, g->ds.md, np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        ck_inc[k] = g->inc_ok;
        ck_outer[k] = g->last_outer;
        RunParams rp = base_params(g);
        rp.mode = kModeTransient;
        rp.nsteps = len;
        rp.step0 = g->step;
        rp.have_prev = g->have_prev;
        rp.obj_partials = part + (size_t)s0 * g->blocks;
        rp.obj_vref = obj->vref;
        rp.obj_margin = obj->margin;
        s = run(g, rp, st, &ms);
        account();
        advance((int64_t)st[kStatSteps]);
        if (s) { g->has_state = false; return s; }
    }
    {
        // J: fixed-order compensated sum of the per-step, per-block partial sums
        std::vector<double> hp((size_t)nsteps * g->blocks);
        CK(cudaMemcpy(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost));
        double sum = 0.0, comp = 0.0;
        for (double x : hp) {
            const double t = sum + x;
            comp += std::fabs(sum) >= std::fabs(x) ? (sum - t) + x : (x - t) + sum;
            sum = t;
        }
        if (J) *J = sum + comp;
    }

    // backward pass, segment by segment, recomputing each segment's states
    CK(cudaMemsetAsync(lam_next, 0, np * sizeof(double), g->stream));
    CK(cudaMemsetAsync(acc_slot, 0, std::max<int64_t>(P.n_ell, 1) * sizeof(double), g->stream));
    CK(cudaMemsetAsync(acc_lv, 0, np * sizeof(double), g->stream));
    CK(cudaMemsetAsync(acc_l, 0, np * sizeof(double), g->stream));
    CK(cudaMemsetAsync(acc_dv, 0, np * sizeof(double), g->stream));
    if (nl) {
        CK(cudaMemsetAsync(mu_l, 0, nl * sizeof(double), g->stream));
        CK(cudaMemsetAsync(acc_L, 0, nl * sizeof(double), g->stream));
    }
    const int kb = std::max(1, std::min(g->n_sm * 4, (P.n_slices + 7) / 8));
    for (int k = nseg - 1; k >= 0; --k) {
        const int s0 = k * ck, len = std::min(ck, nsteps - s0);
        g->vL = 0; g->vP = 1;
        CK(cudaMemcpyAsync(g->ds.v[0], ck_v + (size_t)k * np, np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        CK(cudaMemcpyAsync(g->ds.v[1], ck_vp + (size_t)k * np, np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        CK(cudaMemcpyAsync(vseg, ck_v + (size_t)k * np, np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        if (nl)
            CK(cudaMemcpyAsync(g->ds.il, ck_il + (size_t)k * nl, nl * sizeof(double), cudaMemcpyDeviceToDevice,
                               g->stream));
        g->have_prev = ck_have[k] != 0;
        g->step = s0;
        CK(cudaMemcpyAsync(g->ds.r64, ck_r + (size_t)k * np, np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        CK(cudaMemcpyAsync(g->ds.md, ck_md + (size_t)k * np, np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
        g->inc_ok = ck_inc[k] != 0;
        g->last_outer = ck_outer[k];
        RunParams rp = base_params(g);
        rp.mode = kModeTransient;
        rp.nsteps = len;
        rp.step0 = s0;
        rp.have_prev = g->have_prev;
        rp.v_perm_all = vseg + np;            // rows 1..len: v_{s0+1} .. v_{s0+len}
        if ((s = run(g, rp, st, &ms))) { g->has_state = false; return s; }
        account();
        for (int t = len; t >= 1; --t) {
            const double* v_s = vseg + (size_t)t * np;
            const double* v_p = vseg + (size_t)(t - 1) * np;
            CK(cudaMemsetAsync(scale, 0, sizeof(unsigned long long), g->stream));
            if (nl) CK(launch_adjoint_mu(g->dg, lam_next, mu_l, kb, g->stream));   // mu_s from lambda_(s+1)
            CK(launch_adjoint_rhs(g->dg, v_s, lam_next, mu_l, rhs, obj->vref, obj->margin, scale, kb, g->stream));
            RunParams sp = base_params(g);
            sp.mode = kModeSolve;
            sp.nsteps = 1;
            sp.step0 = 0;
            sp.have_prev = 0;
            sp.warm_extrap = 0;
            sp.x0 = lam_next;
            sp.target = 1e-9;                 // relative: max|r|/D <= 1e-9 max|rhs|/D
            sp.target_scale = scale;
            sp.max_sweeps = std::max(g->opt.max_sweeps, kSetupSweeps);
            g->ds.rhs = rhs;
            s = run(g, sp, st, &ms);
            g->ds.rhs = nullptr;
            if (s) { g->has_state = false; return s; }
            account();
            const int vF = 3 - g->vL - g->vP;
            CK(cudaMemcpyAsync(lam, g->ds.v[vF], np * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
            CK(launch_adjoint_grad(g->dg, lam, v_s, v_p, acc_slot, acc_lv, acc_l, acc_dv, kb, g->stream));
            if (nl) CK(launch_adjoint_lgrad(g->dg, lam, v_s, mu_l, acc_L, kb, g->stream));
            std::swap(lam, lam_next);
        }
    }
    g->has_state = false;

    // map the slot and node sums to element gradients (host)
    std::vector<double> h_slot(std::max<int64_t>(P.n_ell, 1)), h_lv(np), h_l(np), h_dv(np);
    CK(cudaMemcpy(h_slot.data(), acc_slot, h_slot.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(h_lv.data(), acc_lv, np * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(h_l.data(), acc_l, np * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(h_dv.data(), acc_dv, np * sizeof(double), cudaMemcpyDeviceToHost));
    const NetCopy& nc = g->nc;
    auto slot_of = [&](int32_t lo, int32_t hi) -> int64_t {
        const int sl = lo / kSlice, q = lo % kSlice;
        for (int k = 0; k < P.slice_w[sl]; ++k) {
            const int64_t e = P.slice_off[sl] + (int64_t)k * kSlice + q;
            if (P.ell_col[e] == hi && P.ell_adj[e] >= 0) return e;
        }
        return -1;
    };
    std::vector<double> gG(nc.r_g.size(), 0.0), gC(nc.c_val.size(), 0.0);
    for (size_t e = 0; e < nc.r_g.size(); ++e) {
        const int32_t a = nc.r_a[e], b = nc.r_b[e];
        if (a >= 0 && b >= 0) {
            const int32_t i = P.perm[a], j = P.perm[b];
            const int64_t sl = slot_of(std::min(i, j), std::max(i, j));
            gG[e] = sl >= 0 ? -h_slot[sl] : 0.0;
        } else if (a >= 0 || b >= 0) {
            const int32_t i = P.perm[a >= 0 ? a : b], o = a >= 0 ? b : a;
            const double V = o == PG_GROUND ? 0.0 : nc.vdd[-2 - o];
            gG[e] = -(h_lv[i] - V * h_l[i]);
        }
    }
    for (size_t e = 0; e < nc.c_val.size(); ++e) {
        const int32_t a = nc.c_a[e], b = nc.c_b[e];
        if (a >= 0 || b >= 0) gC[e] = -h_dv[P.perm[a >= 0 ? a : b]] / h;
    }
    // the DC point depends on the resistors unless it is the trivial v = Vdd
    if (!g->dc_trivial) {
        if ((s = ensure_dc_grid(g))) return s;
        pg_grid* d = g->dcgrid.get();
        d->stream = g->stream;
        if ((s = prepare_h(d, 1.0))) return s;
        // mu solves G mu = (C/h) lambda_1, in the DC network's own numbering
        std::vector<double> lam1(np), rd(d->P.n_pad, 0.0), v0p(np);
        CK(cudaMemcpy(lam1.data(), lam_next, np * sizeof(double), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(v0p.data(), ck_v, np * sizeof(double), cudaMemcpyDeviceToHost));
        for (int i = 0; i < d->P.n_pad; ++i) {
            const int o = d->P.orig[i];
            if (o >= 0) rd[i] = P.cap[o] / h * lam1[P.perm[o]];
        }
        double rmax = 0.0;
        for (int i = 0; i < d->P.n_pad; ++i)
            if (d->P.orig[i] >= 0) rmax = std::max(rmax, std::fabs(rd[i]) / 1.0);
        double* rdd = sc.get<double>(rd.size());
        if (!rdd) return PG_ERR_OOM;
        CK(cudaMemcpy(rdd, rd.data(), rd.size() * sizeof(double), cudaMemcpyHostToDevice));
        double R = 0.0;
        if (rmax > 0.0) {
            // relative residual 1e-9 of the scaled right-hand side
            double dmin = INFINITY;
            std::vector<double> Dh(d->P.n_pad);
            CK(cudaMemcpy(Dh.data(), d->dg.D64, Dh.size() * sizeof(double), cudaMemcpyDeviceToHost));
            double smax = 0.0;
            for (int i = 0; i < d->P.n_pad; ++i)
                if (d->P.orig[i] >= 0) { smax = std::max(smax, std::fabs(rd[i]) / Dh[i]); dmin = std::min(dmin, Dh[i]); }
            if ((s = solve_internal(d, rdd, 1e-9 * smax, &R))) return s;
            std::vector<double> mu(P.n);
            CK(cudaMemcpy(mu.data(), d->d_x, P.n * sizeof(double), cudaMemcpyDeviceToHost));
            std::vector<double> v0(P.n);
            for (int i = 0; i < np; ++i)
                if (P.orig[i] >= 0) v0[P.orig[i]] = v0p[i];
            auto tvv = [&](int32_t t) { return t >= 0 ? v0[t] : (t == PG_GROUND ? 0.0 : nc.vdd[-2 - t]); };
            auto tmu = [&](int32_t t) { return t >= 0 ? mu[t] : 0.0; };
            for (size_t e = 0; e < nc.r_g.size(); ++e)
                gG[e] -= (tmu(nc.r_a[e]) - tmu(nc.r_b[e])) * (tvv(nc.r_a[e]) - tvv(nc.r_b[e]));
        }
    }
    auto emit = [&](double* dst, const std::vector<double>& src) -> pg_status {
        if (!dst || src.empty()) return PG_OK;
        if (on_host) std::memcpy(dst, src.data(), src.size() * sizeof(double));
        else CK(cudaMemcpy(dst, src.data(), src.size() * sizeof(double), cudaMemcpyHostToDevice));
        return PG_OK;
    };
    std::vector<double> gL(nc.l_val.size(), 0.0);
    if (nl) {
        // dJ/dL_e = (h / L_e^2) sum_s u_(s,e) (A_l lambda_s - mu_s)_e
        std::vector<double> hL(nl);
        CK(cudaMemcpy(hL.data(), acc_L, nl * sizeof(double), cudaMemcpyDeviceToHost));
        for (int e = 0; e < nl; ++e) gL[e] = h / (nc.l_val[e] * nc.l_val[e]) * hL[e];
    }
    if ((s = emit(dJ_dG, gG)) || (s = emit(dJ_dC, gC)) || (s = emit(dJ_dL, gL))) return s;
    if (stats) {
        double z[kStatCount] = {0};
        z[kStatSteps] = nsteps;
        z[kStatSweeps] = (double)sweeps;
        z[kStatOuter] = (double)outer;
        z[kStatMaxBound] = worst;
        z[kStatFailedStep] = -1;
        fill_stats(g, z, ms_total, stats, dc_bound);
    }
    return PG_OK;
}

pg_status pg_solve(pg_grid* g, double h, const double* b, double* x, double tol, pg_run_stats* stats) {
    if (!g || !b || !x || !(tol > 0.0)) return PG_ERR_INVALID_ARG;
    pg_status s = prepare_h(g, h);
    if (s) return s;
    if (!g->d_rhs && !(g->d_rhs = g->alloc<double>(g->P.n_pad))) return PG_ERR_OOM;
    RunParams rp = base_params(g);
    rp.mode = kModeSolve;
    rp.nsteps = 1;
    rp.target = tol / g->kappa - 1e-13;
    rp.solve_out = x;
    if (!(rp.target > 0.0)) {
        g_last_error = "tol below the rounding floor (kappa * 1e-13)";
        return PG_ERR_INVALID_ARG;
    }
    CK(launch_permute_in(g->dg.orig, b, 0.0, g->d_rhs, g->P.n_pad, g->n_sm, g->stream));
    double st[kStatCount];
    float ms = 0.f;
    g->ds.rhs = g->d_rhs;
    s = run(g, rp, st, &ms);
    g->ds.rhs = nullptr;
    fill_stats(g, st, ms, stats, 0.0);
    return s;
}

}  // extern "C"
