// Many load scenarios of one grid in one persistent launch, sharing every
// coefficient of the system.  Grids built for the lattice inner solve relax the
// scenarios with its column-block tiles (four scenarios per shared-memory region);
// other grids with the coloured neighbour-list sweeps.
//
// Every scenario has the same nodal matrix M = C/h + G + G0 (Eq. 2) and its own
// right-hand side (its own load currents), so the relaxation of Eq. 16-17 runs
// on S right-hand sides at once.  Scenarios are interleaved in groups of four
// per node: node i of group q holds its four values in one 16-byte (FP32) or
// 32-byte (FP64) vector, so one weight load serves four scenarios and one
// neighbour gather brings the neighbour's four values.  The step is that of
// the single-scenario persistent kernel: right-hand side, extrapolated warm
// start and FP64 residual; coloured SOR sweeps on the correction (FP32 or FP64);
// FP64 defect-correction passes until the certified bound of the worst scenario
// meets the step target; outputs; the next step's load currents.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "pg_device.cuh"
#include "pg_grid.h"

namespace pg {

namespace {

constexpr int kGroup = 4;      // scenarios per interleaved vector

struct ScenState {
    int32_t n_groups, n_scen;
    double* v[3];              // [n_groups][n_pad][4] rotating voltage buffers
    double* r64;               // residual b - M v
    float* r32;                // its FP32 copy (mixed precision)
    void* d[2];                // corrections (float or double)
    double* inode[2];          // load current drawn from each node, slot S & 1
    const double* pwl_v;       // [n_scen][n_points] the scenarios' PWL breakpoint values
    unsigned long long* vmin_key;   // [nsteps][n_scen] order keys of the smallest voltage
};

struct ScenParams {
    int32_t nsteps;
    double h, omega, target, inner_reduction;
    int32_t max_sweeps, max_outer;
    long long timeout_ns;
    double* v_all;             // [nsteps][n_scen][n_real] or null
    int32_t lat_k;             // > 0: lattice inner solve, lat_k exact block sweeps per round
    int32_t lat_maxnl;         // layers held per region (the grid's largest lattice layer count)
};

// ---- lattice inner solve for scenario groups
//
// The column-block red-black SOR of the single-scenario lattice solve (k exact block
// sweeps per device barrier on 34 x 34-column regions with ghost zones of 2k columns;
// each (x, y) column's layers solved exactly with the precomputed Thomas factors), with a
// group's four scenarios in one region: their corrections and residuals as one float4
// per column and layer, the coefficients staged once for all four.
constexpr int kScW = 36;                       // shared-memory row stride (columns)
constexpr int kScPlane = kLatSide * kScW;      // one layer of one staged array

__host__ __device__ inline size_t scen_region_bytes(int maxnl) {
    return (size_t)maxnl * kScPlane * (2 * sizeof(float4) + 5 * sizeof(float));
}

template <int NL>
__device__ float scen_lattice_tile(const DevGrid& g, int off, int nx, int ny, int tile, int q, const float* dold,
                                   float* dnew, const float* r, float omega, int k, int maxnl, unsigned char* smem) {
    const int H = 2 * k, T = kLatSide - 2 * H;
    const int tiles_x = (nx + T - 1) / T;
    const int A = maxnl * kScPlane;                          // elements per staged array
    float4* sd = reinterpret_cast<float4*>(smem);
    float4* sr = sd + A;
    float* se = reinterpret_cast<float*>(sr + A);
    float* sn = se + A;
    float* su = se + 2 * A;
    float* sm = se + 3 * A;
    float* sp = se + 4 * A;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = lane & 15, rsub = lane >> 4;
    const long long plane = (long long)nx * ny;
    const long long gq = (long long)q * g.n_pad;            // the group's first node
    const int x0 = (tile % tiles_x) * T - H, y0 = (tile / tiles_x) * T - H;
    const int lead = x0 & 3;
    const int xa = x0 - lead;
    // corrections and residuals: one 16-byte copy per column and layer
    for (int qq = threadIdx.x; qq < kScPlane; qq += blockDim.x) {
        const int ry = qq / kScW, c = qq - ry * kScW;
        const int xx = xa + c, yy = y0 + ry;
        const bool in = yy >= 0 && yy < ny && xx >= 0 && xx < nx;
        const long long o = in ? off + (long long)yy * nx + xx : 0;
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            const long long e = in ? (gq + o + l * plane) * kGroup : 0;
            cp_async16(sd + l * kScPlane + qq, dold + e, in ? 16u : 0u);
            cp_async16(sr + l * kScPlane + qq, r + e, in ? 16u : 0u);
        }
    }
    // the coefficients, shared by the group: 16-byte pieces where the lattice allows them
    auto src_of = [&](int arr) -> const float* {
        return arr == 0 ? g.lwE : arr == 1 ? g.lwN : arr == 2 ? g.lwU : arr == 3 ? g.lm : g.lip;
    };
    if ((nx & 3) == 0 && (off & 3) == 0) {
        constexpr int kChunks = kScW / 4;
        constexpr int kPieces = kLatSide * kChunks;
        for (int qq = threadIdx.x; qq < kPieces * 5; qq += blockDim.x) {
            const int arr = qq / kPieces, pos = qq - arr * kPieces;
            const int ry = pos / kChunks, c4 = 4 * (pos - ry * kChunks);
            const int xx = xa + c4, yy = y0 + ry;
            const bool in = yy >= 0 && yy < ny && xx >= 0 && xx < nx;
            const long long o = in ? off + (long long)yy * nx + xx : 0;
            float* dst = se + arr * A + ry * kScW + c4;
#pragma unroll
            for (int l = 0; l < NL; ++l)
                cp_async16(dst + l * kScPlane, src_of(arr) + (in ? o + l * plane : 0), in ? 16u : 0u);
        }
    } else {
        for (int qq = threadIdx.x; qq < kScPlane; qq += blockDim.x) {
            const int ry = qq / kScW, c = qq - ry * kScW;
            const int xx = xa + c, yy = y0 + ry;
            const bool in = yy >= 0 && yy < ny && xx >= 0 && xx < nx;
            const long long o = in ? off + (long long)yy * nx + xx : 0;
#pragma unroll
            for (int arr = 0; arr < 5; ++arr)
#pragma unroll
                for (int l = 0; l < NL; ++l)
                    cp_async4(se + arr * A + l * kScPlane + qq, src_of(arr) + (in ? o + l * plane : 0), in ? 4u : 0u);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    float mon = 0.f;
    for (int hs = 0; hs < 2 * k; ++hs) {
        const bool last = hs >= 2 * k - 2;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int ry = 1 + 2 * (warp + 8 * j) + rsub, y = y0 + ry;
            const int cx = 1 + 2 * pair + ((hs + x0 + 1 + y) & 1);
            const int x = x0 + cx;
            const int edge = min(min(cx, ry), min(kLatSide - 1 - cx, kLatSide - 1 - ry));
            if (edge <= hs || x < 0 || x >= nx || y < 0 || y >= ny) continue;
            const int a0 = ry * kScW + cx + lead;
            float4 f[NL], xv[NL];
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const int a = a0 + l * kScPlane;
                const float we = se[a], ww = se[a - 1], wn = sn[a], ws = sn[a - kScW];
                const float4 rr = sr[a], de = sd[a + 1], dw = sd[a - 1], dn = sd[a + kScW], ds = sd[a - kScW];
                f[l].x = rr.x + we * de.x + ww * dw.x + wn * dn.x + ws * ds.x;
                f[l].y = rr.y + we * de.y + ww * dw.y + wn * dn.y + ws * ds.y;
                f[l].z = rr.z + we * de.z + ww * dw.z + wn * dn.z + ws * ds.z;
                f[l].w = rr.w + we * de.w + ww * dw.w + wn * dn.w + ws * ds.w;
            }
#pragma unroll
            for (int l = 1; l < NL; ++l) {
                const float m = sm[a0 + l * kScPlane];
                f[l].x = fmaf(m, f[l - 1].x, f[l].x); f[l].y = fmaf(m, f[l - 1].y, f[l].y);
                f[l].z = fmaf(m, f[l - 1].z, f[l].z); f[l].w = fmaf(m, f[l - 1].w, f[l].w);
            }
            {
                const float p = sp[a0 + (NL - 1) * kScPlane];
                xv[NL - 1] = make_float4(f[NL - 1].x * p, f[NL - 1].y * p, f[NL - 1].z * p, f[NL - 1].w * p);
            }
#pragma unroll
            for (int l = NL - 2; l >= 0; --l) {
                const float u = su[a0 + l * kScPlane], p = sp[a0 + l * kScPlane];
                xv[l] = make_float4(fmaf(u, xv[l + 1].x, f[l].x) * p, fmaf(u, xv[l + 1].y, f[l].y) * p,
                                    fmaf(u, xv[l + 1].z, f[l].z) * p, fmaf(u, xv[l + 1].w, f[l].w) * p);
            }
            const bool interior = edge >= H;
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const int a = a0 + l * kScPlane;
                const float4 dv = sd[a];
                const float4 up = make_float4(xv[l].x - dv.x, xv[l].y - dv.y, xv[l].z - dv.z, xv[l].w - dv.w);
                sd[a] = make_float4(fmaf(omega, up.x, dv.x), fmaf(omega, up.y, dv.y), fmaf(omega, up.z, dv.z),
                                    fmaf(omega, up.w, dv.w));
                if (last && interior)
                    mon = nanmaxf(nanmaxf(mon, nanmaxf(fabsf(up.x), fabsf(up.y))), nanmaxf(fabsf(up.z), fabsf(up.w)));
            }
        }
        __syncthreads();
    }
    for (int qq = threadIdx.x; qq < T * T; qq += blockDim.x) {
        const int iy = qq / T, ix = qq - iy * T;
        const int x = x0 + H + ix, y = y0 + H + iy;
        if (x >= nx || y >= ny) continue;
        const long long b = off + (long long)y * nx + x;
        const int a = (H + iy) * kScW + H + ix + lead;
#pragma unroll
        for (int l = 0; l < NL; ++l)
            *reinterpret_cast<float4*>(dnew + (gq + b + l * plane) * kGroup) = sd[l * kScPlane + a];
    }
    __syncthreads();   // the next tile overwrites the region
    return mon;
}

// One round over every (tile, scenario group) of every lattice; the max unrelaxed update
// of the last sweep over the tile interiors.
__device__ double scen_lattice_round(const DevGrid& g, const float* dold, float* dnew, const float* r, float omega,
                                     int k, int maxnl, int n_groups, unsigned char* smem) {
    float mon = 0.f;
    const long long tasks = (long long)g.lat_tiles * n_groups;
    for (long long task = blockIdx.x; task < tasks; task += gridDim.x) {
        const int t = (int)(task / n_groups), q = (int)(task - (long long)t * n_groups);
        int lo = 0, hi = g.n_lats;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(g.lat_tile0 + mid) <= t) lo = mid; else hi = mid;
        }
        const int off = __ldg(g.lat_info + 4 * lo), nx = __ldg(g.lat_info + 4 * lo + 1),
                  ny = __ldg(g.lat_info + 4 * lo + 2), nl = __ldg(g.lat_info + 4 * lo + 3);
        const int tile = t - __ldg(g.lat_tile0 + lo);
        float m;
        if (nl == 1) m = scen_lattice_tile<1>(g, off, nx, ny, tile, q, dold, dnew, r, omega, k, maxnl, smem);
        else if (nl == 2) m = scen_lattice_tile<2>(g, off, nx, ny, tile, q, dold, dnew, r, omega, k, maxnl, smem);
        else m = scen_lattice_tile<3>(g, off, nx, ny, tile, q, dold, dnew, r, omega, k, maxnl, smem);
        mon = nanmaxf(mon, m);
    }
    return (double)mon;
}

__device__ __forceinline__ long long vbase(const DevGrid& g, int q, int i) {
    return ((long long)q * g.n_pad + i) * kGroup;
}
__device__ __forceinline__ void ldv(const double* X, long long b, double (&x)[4]) {
    const double2 a = reinterpret_cast<const double2*>(X + b)[0], c = reinterpret_cast<const double2*>(X + b)[1];
    x[0] = a.x; x[1] = a.y; x[2] = c.x; x[3] = c.y;
}
__device__ __forceinline__ void ldv(const float* X, long long b, float (&x)[4]) {
    const float4 a = *reinterpret_cast<const float4*>(X + b);
    x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
}
__device__ __forceinline__ void stv(double* X, long long b, const double (&x)[4]) {
    reinterpret_cast<double2*>(X + b)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(X + b)[1] = make_double2(x[2], x[3]);
}
__device__ __forceinline__ void stv(float* X, long long b, const float (&x)[4]) {
    *reinterpret_cast<float4*>(X + b) = make_float4(x[0], x[1], x[2], x[3]);
}

// Scenario group q's current of load e at time t: the breakpoint times are shared, the
// values are each scenario's (held outside the breakpoints, linear in between, as in the
// single-scenario evaluation).
__device__ __forceinline__ void pwl_group(const DevGrid& g, const ScenState& ss, int e, int q, double t,
                                          double (&I)[4]) {
    const long long lo0 = g.pwl_ptr[e], hi0 = g.pwl_ptr[e + 1] - 1;
    const long long npts = g.pwl_ptr[g.n_src];
    const double* T = g.pwl_t;
    long long lo = lo0, hi = hi0;
    int mode = 0;                                  // 0: interpolate, 1: first value, 2: last value
    if (t <= T[lo0]) mode = 1;
    else if (t > T[hi0]) mode = 2;
    else
        while (hi - lo > 1) {
            const long long mid = (lo + hi) >> 1;
            if (t <= T[mid]) hi = mid; else lo = mid;
        }
    const double frac = mode == 0 ? (t - T[lo]) / (T[hi] - T[lo]) : 0.0;
#pragma unroll
    for (int k = 0; k < kGroup; ++k) {
        const int sc = q * kGroup + k;
        if (sc >= ss.n_scen) { I[k] = 0.0; continue; }
        const double* V = ss.pwl_v + (long long)sc * npts;
        I[k] = mode == 1 ? V[lo0] : mode == 2 ? V[hi0] : V[lo] + (V[hi] - V[lo]) * frac;
    }
}

template <bool MIXED>
__global__ void __launch_bounds__(256, 2) scenario_kernel(DevGrid g, ScenState ss, DevCtl ctl, ScenParams sp) {
    using T = typename std::conditional<MIXED, float, double>::type;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const int NG = ss.n_groups;
    const T omega = (T)sp.omega;
    const T* wT = MIXED ? (const T*)g.w32 : (const T*)g.w64;
    const T* iDT = MIXED ? (const T*)g.invD32 : (const T*)g.invD64;
    const T* rT = MIXED ? (const T*)ss.r32 : (const T*)ss.r64;

    int phase = 0;
    auto barrier = [&](bool want, double v) -> BarrierResult {
        const BarrierResult r = grid_barrier(ctl, nblocks, (unsigned)(phase + 1), sp.timeout_ns, false, v,
                                             want ? ctl.red + (phase & 3) : nullptr);
        ++phase;
        if (lead) ctl.red[(phase + 2) & 3] = 0ull;
        return r;
    };
    long long tot_sweeps = 0, tot_outer = 0, steps_done = 0;
    int max_sw = 0, max_out = 0;
    double max_R = 0.0, last_R = 0.0;
    auto publish = [&](long long failed) {
        if (lead) {
            for (int k = 0; k < kStatCount; ++k) ctl.stats[k] = 0.0;
            ctl.stats[kStatSteps] = (double)steps_done;
            ctl.stats[kStatSweeps] = (double)tot_sweeps;
            ctl.stats[kStatMaxSweeps] = (double)max_sw;
            ctl.stats[kStatOuter] = (double)tot_outer;
            ctl.stats[kStatMaxOuter] = (double)max_out;
            ctl.stats[kStatMaxBound] = max_R;
            ctl.stats[kStatFailedStep] = (double)failed;
            ctl.stats[kStatLastR] = last_R;
        }
    };
    // load currents of step S into slot S & 1, per scenario group (as the single-scenario
    // kernel: one thread per source and group for nodes with one load, one per node and
    // group for nodes with several)
    auto eval_sources = [&](long long S) {
        double* dst = ss.inode[S & 1];
        const double tS = (double)S * sp.h;
        for (long long t = gtid; t < (long long)g.n_src * NG; t += nthreads) {
            const int e = (int)(t / NG), q = (int)(t - (long long)e * NG);
            const int a = __ldg(g.src_na + e), b = __ldg(g.src_nb + e);
            if (a < 0 && b < 0) continue;
            double I[4];
            pwl_group(g, ss, e, q, tS, I);
            if (a >= 0) stv(dst, vbase(g, q, a), I);
            if (b >= 0) {
                double m[4] = {-I[0], -I[1], -I[2], -I[3]};
                stv(dst, vbase(g, q, b), m);
            }
        }
        for (long long t = gtid; t < (long long)g.n_multi * NG; t += nthreads) {
            const int k = (int)(t / NG), q = (int)(t - (long long)k * NG);
            const int i = __ldg(g.multi_node + k);
            double sum[4] = {0.0, 0.0, 0.0, 0.0};
            for (int qq = __ldg(g.ld_ptr + i); qq < __ldg(g.ld_ptr + i + 1); ++qq) {
                const int sid = __ldg(g.ld_idx + qq);
                double I[4];
                pwl_group(g, ss, (sid > 0 ? sid : -sid) - 1, q, tS, I);
#pragma unroll
                for (int c = 0; c < 4; ++c) sum[c] += sid > 0 ? I[c] : -I[c];
            }
            stv(dst, vbase(g, q, i), sum);
        }
    };
    unsigned long long* keys = ss.vmin_key;
    for (long long q = gtid; q < (long long)sp.nsteps * ss.n_scen; q += nthreads) keys[q] = ~0ull;
    if (g.n_src > 0) eval_sources(1);
    if (!barrier(false, 0.0).ok) { publish(-1); return; }

    int vL = 0, vP = 1, vF = 2;
    bool have_prev = false;
    const int n_slices = g.n_slices;
    for (int sl = 0; sl < sp.nsteps; ++sl) {
        const long long sabs = sl + 1;
        if (sl > 0 && ss.vmin_key) {
            // the previous step's minima: order keys -> volts
            for (int q = gtid; q < ss.n_scen; q += nthreads) {
                const long long e = (long long)(sl - 1) * ss.n_scen + q;
                reinterpret_cast<double*>(keys)[e] = key_value(keys[e]);
            }
        }
        // ---- right-hand side (Eq. 2), extrapolated warm start, FP64 residual
        double mon = 0.0;
        {
            const double* vl = ss.v[vL];
            const double* vp = ss.v[vP];
            double* vf = ss.v[vF];
            const double* In = ss.inode[sabs & 1];
            T* d0 = (T*)ss.d[0];
            for (long long task = gwarp; task < (long long)n_slices * NG; task += nwarps) {
                const int s = (int)(task / NG), q = (int)(task - (long long)s * NG);
                const SliceDesc sd = global_desc(g, s);
                const int* offs = sd.dpos <= -2 ? g.dia_off + (-2 - sd.dpos) : nullptr;
                const int i0 = s * kSlice + lane * kVec;
                double D[4], iD[4], ch[4], cj[4];
                ldg4(g.D64 + i0, D);
                ldg4(g.invD64 + i0, iD);
                ldg4(g.ch + i0, ch);
                ldg4(g.cinj + i0, cj);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long b0 = vbase(g, q, i0 + j);
                    double a[4], p[4], I[4], x0[4], sig[4] = {0.0, 0.0, 0.0, 0.0};
                    ldv(vl, b0, a);
                    ldv(vp, b0, p);
                    ldv(In, b0, I);
#pragma unroll
                    for (int c = 0; c < 4; ++c) x0[c] = have_prev ? 2.0 * a[c] - p[c] : a[c];
                    for (int k = 0; k < sd.K; ++k) {
                        const long long e = sd.off + (long long)k * kSlice + lane * kVec + j;
                        const double w = __ldg(g.w64 + e);
                        const int col = offs ? i0 + j + offs[k] : __ldg(g.ell_col + e);
                        const long long bc = vbase(g, q, col);
                        double na[4], np_[4];
                        ldv(vl, bc, na);
                        if (have_prev) ldv(vp, bc, np_);
#pragma unroll
                        for (int c = 0; c < 4; ++c) sig[c] = fma(w, have_prev ? 2.0 * na[c] - np_[c] : na[c], sig[c]);
                    }
                    double r[4];
                    T z[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        r[c] = ch[j] * a[c] + cj[j] - I[c] + sig[c] - D[j] * x0[c];
                        mon = nanmax(mon, fabs(r[c]) * iD[j]);
                        z[c] = T(0);
                    }
                    stv(vf, b0, x0);
                    stv(ss.r64, b0, r);
                    if (MIXED) {
                        float r32[4] = {(float)r[0], (float)r[1], (float)r[2], (float)r[3]};
                        stv(ss.r32, b0, r32);
                    }
                    stv(d0, b0, z);
                }
            }
        }
        BarrierResult br = barrier(true, mon);
        if (!br.ok) { publish(-1); return; }
        double R = br.val;
        int sweeps = 0, outer = 0, dsel = 0;
        bool ok = true;
        while (!(R <= sp.target)) {
            if (!(R == R) || isinf(R) || outer >= sp.max_outer || sweeps >= sp.max_sweeps) { ok = false; break; }
            // ---- coloured SOR sweeps on M delta = r (Eq. 16-17), all scenarios at once
            const double inner_tgt = MIXED ? fmax(0.5 * sp.target, sp.inner_reduction * R) : 0.5 * sp.target;
            T* dd = (T*)ss.d[dsel];
            double est_mark = INFINITY;
            int inner = 0;
            bool bad = false;
            while (MIXED && sp.lat_k > 0) {
                // lattice rounds: lat_k exact block sweeps per device barrier, four scenarios per region
                extern __shared__ __align__(16) unsigned char s_dyn[];
                const double m = scen_lattice_round(g, (const float*)ss.d[dsel], (float*)ss.d[dsel ^ 1], ss.r32,
                                                    (float)sp.omega, sp.lat_k, sp.lat_maxnl, NG, s_dyn);
                const BarrierResult be = barrier(true, m);
                if (!be.ok) { publish(-1); return; }
                const double est = be.val;
                dsel ^= 1;
                dd = (T*)ss.d[dsel];
                const int before = inner;
                sweeps += sp.lat_k;
                inner += sp.lat_k;
                if (!(est == est)) { bad = true; break; }
                if (est <= inner_tgt || sweeps >= sp.max_sweeps) break;
                if ((inner >> 4) != (before >> 4)) {
                    if (est > 0.9 * est_mark) break;
                    est_mark = est;
                }
            }
            while (!(MIXED && sp.lat_k > 0)) {
                double est = 0.0;
                for (int c = 0; c < g.ncol; ++c) {
                    const int c0 = __ldg(g.colour_slice + c), c1 = __ldg(g.colour_slice + c + 1);
                    double m = 0.0;
                    for (long long task = gwarp; task < (long long)(c1 - c0) * NG; task += nwarps) {
                        const int s = c0 + (int)(task / NG), q = (int)(task % NG);
                        const SliceDesc sd = global_desc(g, s);
                        const int* offs = sd.dpos <= -2 ? g.dia_off + (-2 - sd.dpos) : nullptr;
                        const int i0 = s * kSlice + lane * kVec;
                        T iD[4];
                        ldg4(iDT + i0, iD);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const long long b0 = vbase(g, q, i0 + j);
                            T dv[4], rv[4], sig[4] = {T(0), T(0), T(0), T(0)};
                            ldv(dd, b0, dv);
                            ldv(rT, b0, rv);
                            for (int k = 0; k < sd.K; ++k) {
                                const long long e = sd.off + (long long)k * kSlice + lane * kVec + j;
                                const T w = __ldg(wT + e);
                                const int col = offs ? i0 + j + offs[k] : __ldg(g.ell_col + e);
                                T dn[4];
                                ldv(dd, vbase(g, q, col), dn);
#pragma unroll
                                for (int cc = 0; cc < 4; ++cc) sig[cc] = fma(w, dn[cc], sig[cc]);
                            }
#pragma unroll
                            for (int cc = 0; cc < 4; ++cc) {
                                const T upd = (rv[cc] + sig[cc]) * iD[j] - dv[cc];
                                dv[cc] = fma(omega, upd, dv[cc]);
                                m = nanmax(m, (double)fabs(upd));
                            }
                            stv(dd, b0, dv);
                        }
                    }
                    const BarrierResult be = barrier(true, m);
                    if (!be.ok) { publish(-1); return; }
                    est = nanmax(est, be.val);
                }
                ++sweeps;
                ++inner;
                if (!(est == est)) { bad = true; break; }
                if (est <= inner_tgt || sweeps >= sp.max_sweeps) break;
                if ((inner & 15) == 0) {           // the inner solve stalls at its precision floor
                    if (est > 0.9 * est_mark) break;
                    est_mark = est;
                }
            }
            if (bad) { ok = false; break; }
            // ---- FP64 defect correction: v += delta, r -= M delta, certified max |r| / D
            double m = 0.0;
            T* dn = (T*)ss.d[dsel ^ 1];
            double* vf = ss.v[vF];
            for (long long task = gwarp; task < (long long)n_slices * NG; task += nwarps) {
                const int s = (int)(task / NG), q = (int)(task - (long long)s * NG);
                const SliceDesc sd = global_desc(g, s);
                const int* offs = sd.dpos <= -2 ? g.dia_off + (-2 - sd.dpos) : nullptr;
                const int i0 = s * kSlice + lane * kVec;
                double D[4], iD[4];
                ldg4(g.D64 + i0, D);
                ldg4(g.invD64 + i0, iD);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long b0 = vbase(g, q, i0 + j);
                    T dv[4];
                    double r[4], vv[4], sig[4] = {0.0, 0.0, 0.0, 0.0};
                    ldv(dd, b0, dv);
                    ldv(ss.r64, b0, r);
                    ldv(vf, b0, vv);
                    for (int k = 0; k < sd.K; ++k) {
                        const long long e = sd.off + (long long)k * kSlice + lane * kVec + j;
                        const double w = __ldg(g.w64 + e);
                        const int col = offs ? i0 + j + offs[k] : __ldg(g.ell_col + e);
                        T dnb[4];
                        ldv(dd, vbase(g, q, col), dnb);
#pragma unroll
                        for (int c = 0; c < 4; ++c) sig[c] = fma(w, (double)dnb[c], sig[c]);
                    }
                    T z[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        r[c] -= D[j] * (double)dv[c] - sig[c];
                        vv[c] += (double)dv[c];
                        m = nanmax(m, fabs(r[c]) * iD[j]);
                        z[c] = T(0);
                    }
                    stv(ss.r64, b0, r);
                    stv(vf, b0, vv);
                    stv(dn, b0, z);
                    if (MIXED) {
                        float r32[4] = {(float)r[0], (float)r[1], (float)r[2], (float)r[3]};
                        stv(ss.r32, b0, r32);
                    }
                }
            }
            br = barrier(true, m);
            if (!br.ok) { publish(-1); return; }
            R = br.val;
            dsel ^= 1;
            ++outer;
        }
        if (!ok) {
            if (lead) {
                cuda::atomic_ref<int, cuda::thread_scope_device> err(*ctl.err);
                int z = 0;
                err.compare_exchange_strong(z, (int)PG_ERR_NOT_CONVERGED);
            }
            publish(sabs);
            return;
        }
        // ---- outputs: every scenario's field, its smallest voltage; the next step's loads
        {
            const double* vnew = ss.v[vF];
            for (long long task = gwarp; task < (long long)n_slices * NG; task += nwarps) {
                const int s = (int)(task / NG), q = (int)(task - (long long)s * NG);
                const int i0 = s * kSlice + lane * kVec;
                unsigned long long kmin[4] = {~0ull, ~0ull, ~0ull, ~0ull};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int o = __ldg(g.orig + i0 + j);
                    if (o < 0) continue;
                    double x[4];
                    ldv(vnew, vbase(g, q, i0 + j), x);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int sc = q * kGroup + c;
                        if (sc >= ss.n_scen) continue;
                        kmin[c] = min(kmin[c], order_key(x[c]));
                        if (sp.v_all) sp.v_all[((long long)sl * ss.n_scen + sc) * g.n_real + o] = x[c];
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    unsigned long long k = kmin[c];
                    for (int o = 16; o; o >>= 1) k = min(k, __shfl_xor_sync(0xffffffffu, k, o));
                    const int sc = q * kGroup + c;
                    if (lane == 0 && sc < ss.n_scen && k != ~0ull) atomicMin(keys + (long long)sl * ss.n_scen + sc, k);
                }
            }
        }
        if (sl + 1 < sp.nsteps && g.n_src > 0) eval_sources(sabs + 1);
        tot_sweeps += sweeps; tot_outer += outer;
        max_sw = max(max_sw, sweeps); max_out = max(max_out, outer);
        max_R = fmax(max_R, R);
        last_R = R;
        ++steps_done;
        vP = vL; vL = vF; vF = 3 - vL - vP;
        have_prev = true;
        if (!barrier(false, 0.0).ok) { publish(-1); return; }
    }
    if (sp.nsteps > 0)
        for (int q = gtid; q < ss.n_scen; q += nthreads) {
            const long long e = (long long)(sp.nsteps - 1) * ss.n_scen + q;
            reinterpret_cast<double*>(keys)[e] = key_value(keys[e]);
        }
    publish(-1);
}

pg_status fail(pg_status s, const std::string& m) {
    set_last_error(m);
    return s;
}

struct Scratch {
    std::vector<void*> p;
    ~Scratch() { for (void* q : p) cudaFree(q); }
    template <typename U>
    U* get(size_t n) {
        void* q = nullptr;
        if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(U)) != cudaSuccess) return nullptr;
        p.push_back(q);
        return static_cast<U*>(q);
    }
};

}  // namespace

}  // namespace pg

using namespace pg;

extern "C" pg_status pg_transient_scenarios(pg_grid* g, double h, int32_t nsteps, int32_t n_scen, const double* i_v,
                                            const pg_scenario_output* out, pg_run_stats* stats) {
    if (!g || nsteps < 1 || n_scen < 1 || !i_v) return fail(PG_ERR_INVALID_ARG, "null grid or values, or no steps");
    if (g->P.n_l > 0) return fail(PG_ERR_UNSUPPORTED, "load scenarios run on RC grids (no inductors)");
    if (g->opt.form != PG_FORM_EXPLICIT) return fail(PG_ERR_UNSUPPORTED, "load scenarios need the explicit form");
    if (g->dg.lwE && !g->mixed)
        return fail(PG_ERR_UNSUPPORTED,
                    "load scenarios in FP64 run on the point inner solve (create the grid with lattice_sweeps = -1)");
    if (g->dg.lwE && g->dg.lat_rows != kLatSide)
        return fail(PG_ERR_UNSUPPORTED, "load scenarios on the lattice inner solve take 34-row regions (tile_rows 0 or 34)");
    const NetCopy& nc = g->nc;
    const size_t npts = nc.i_t.size();
    const bool host = out && out->on_host;
    // the scenarios' PWL values, and the DC point of every scenario: v = Vdd needs one supply
    // level, no branch from a node to ground, and no load current at t = 0
    std::vector<double> hv((size_t)n_scen * npts);
    if (npts) {
        cudaPointerAttributes a{};
        const bool dev = cudaPointerGetAttributes(&a, i_v) == cudaSuccess &&
                         (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
        cudaGetLastError();
        const cudaError_t e = cudaMemcpy(hv.data(), i_v, hv.size() * sizeof(double),
                                         dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost);
        if (e != cudaSuccess) return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    }
    {
        bool one = nc.p > 0;
        for (int k = 1; k < nc.p && one; ++k) one = nc.vdd[k] == nc.vdd[0];
        for (size_t e = 0; e < nc.r_g.size() && one; ++e)
            if ((nc.r_a[e] >= 0) != (nc.r_b[e] >= 0)) one = (nc.r_a[e] >= 0 ? nc.r_b[e] : nc.r_a[e]) != PG_GROUND;
        for (int32_t s = 0; s < n_scen && one; ++s)
            for (size_t e = 0; e + 1 < nc.i_ptr.size() && one; ++e) {
                const int64_t lo = nc.i_ptr[e], hi = nc.i_ptr[e + 1] - 1;
                // the current at t = 0 (held before the first breakpoint)
                double v0 = hv[(size_t)s * npts + lo];
                if (0.0 > nc.i_t[hi]) v0 = hv[(size_t)s * npts + hi];
                else if (0.0 > nc.i_t[lo])
                    for (int64_t k = lo; k < hi; ++k)
                        if (nc.i_t[k] < 0.0 && 0.0 <= nc.i_t[k + 1]) {
                            const double* V = hv.data() + (size_t)s * npts;
                            v0 = V[k] + (V[k + 1] - V[k]) * ((0.0 - nc.i_t[k]) / (nc.i_t[k + 1] - nc.i_t[k]));
                        }
                one = v0 == 0.0;
            }
        for (double x : hv) one = one && std::isfinite(x);
        if (!one)
            return fail(PG_ERR_UNSUPPORTED, "load scenarios start from v = Vdd: one supply level, no resistor to "
                                            "ground and every load current zero at t = 0");
    }
    pg_run_stats st0;
    pg_status s = pg_transient(g, h, 0, nullptr, &st0);      // assemble h (coefficients, omega, bounds)
    if (s) return s;
    const int n_pad = g->P.n_pad;
    const int NG = (n_scen + kGroup - 1) / kGroup;
    const size_t nv = (size_t)NG * n_pad * kGroup;
    Scratch sc;
    ScenState ss{};
    ss.n_groups = NG;
    ss.n_scen = n_scen;
    for (int k = 0; k < 3; ++k) ss.v[k] = sc.get<double>(nv);
    ss.r64 = sc.get<double>(nv);
    ss.r32 = g->mixed ? sc.get<float>(nv) : nullptr;
    const size_t ds = g->mixed ? sizeof(float) : sizeof(double);
    for (int k = 0; k < 2; ++k) ss.d[k] = sc.get<unsigned char>(nv * ds);
    for (int k = 0; k < 2; ++k) ss.inode[k] = sc.get<double>(nv);
    double* pv = sc.get<double>(std::max<size_t>(hv.size(), 1));
    ss.pwl_v = pv;
    ss.vmin_key = sc.get<unsigned long long>((size_t)nsteps * n_scen);
    double* v_all = nullptr;
    const size_t n_all = (size_t)nsteps * n_scen * g->P.n;
    if (out && out->v_all) v_all = host ? sc.get<double>(n_all) : out->v_all;
    if (!ss.v[0] || !ss.v[1] || !ss.v[2] || !ss.r64 || (g->mixed && !ss.r32) || !ss.d[0] || !ss.d[1] ||
        !ss.inode[0] || !ss.inode[1] || !pv || !ss.vmin_key || (out && out->v_all && !v_all))
        return fail(PG_ERR_OOM, "device memory for the scenarios");
    cudaStream_t stream = g->stream;
    auto ck = [&](cudaError_t e) { return e == cudaSuccess ? PG_OK : fail(PG_ERR_CUDA, cudaGetErrorString(e)); };
    // every scenario at v = Vdd (padding at 0), no loads before they are evaluated
    {
        std::vector<double> v0(nv, 0.0);
        for (int q = 0; q < NG; ++q)
            for (int i = 0; i < n_pad; ++i)
                if (g->P.orig[i] >= 0)
                    for (int c = 0; c < kGroup; ++c) v0[((size_t)q * n_pad + i) * kGroup + c] = nc.vdd[0];
        if ((s = ck(cudaMemcpyAsync(ss.v[0], v0.data(), nv * sizeof(double), cudaMemcpyHostToDevice, stream))) ||
            (s = ck(cudaMemcpyAsync(ss.v[1], v0.data(), nv * sizeof(double), cudaMemcpyHostToDevice, stream))) ||
            (s = ck(cudaMemsetAsync(ss.d[0], 0, nv * ds, stream))) ||
            (s = ck(cudaMemsetAsync(ss.d[1], 0, nv * ds, stream))) ||
            (s = ck(cudaMemsetAsync(ss.inode[0], 0, nv * sizeof(double), stream))) ||
            (s = ck(cudaMemsetAsync(ss.inode[1], 0, nv * sizeof(double), stream))) ||
            (hv.size() && (s = ck(cudaMemcpyAsync(pv, hv.data(), hv.size() * sizeof(double), cudaMemcpyHostToDevice,
                                                  stream)))) ||
            (s = ck(cudaStreamSynchronize(stream))))
            return s;
    }
    ScenParams sp{};
    sp.nsteps = nsteps;
    sp.h = h;
    sp.omega = g->omega;
    sp.target = g->target;
    sp.inner_reduction = g->opt.inner_reduction;
    sp.max_sweeps = g->opt.max_sweeps;
    sp.max_outer = 50;
    sp.timeout_ns = (long long)(g->opt.barrier_timeout_s * 1e9);
    sp.v_all = v_all;
    sp.lat_k = g->dg.lwE ? g->lat_k : 0;             // grids built for the lattice inner solve
    sp.lat_maxnl = g->P.lat_maxnl;
    const size_t smem = sp.lat_k > 0 ? scen_region_bytes(sp.lat_maxnl) : 0;
    // launch: at most the co-resident blocks, no more than the work of a colour sweep needs
    const void* fn = g->mixed ? (const void*)scenario_kernel<true> : (const void*)scenario_kernel<false>;
    if (smem > 0 && (s = ck(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))))
        return s;
    int bps = 0;
    if ((s = ck(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, 256, smem)))) return s;
    if (g->opt.blocks_per_sm > 0) bps = std::min(bps, g->opt.blocks_per_sm);
    if (bps < 1) return fail(PG_ERR_CUDA, "scenario kernel does not fit on an SM");
    int smax = 1;
    for (int c = 0; c < g->P.ncol; ++c)
        smax = std::max(smax, (g->P.colour_start[c + 1] - g->P.colour_start[c]) / kSlice);
    const long long warps = (long long)smax * NG;
    long long want = (warps + 7) / 8;
    if (sp.lat_k > 0) want = std::max<long long>(want, (long long)g->dg.lat_tiles * NG);   // one task per block
    const int blocks = (int)std::max<long long>(1, std::min<long long>((long long)g->n_sm * bps, want));
    // the launch's own barrier and reduction words (the grid's, cleared first)
    DevCtl ctl = g->dc;
    if ((s = ck(cudaMemsetAsync(ctl.bar_count, 0, sizeof(unsigned), stream))) ||
        (s = ck(cudaMemsetAsync(ctl.bar_gen, 0, sizeof(unsigned), stream))) ||
        (s = ck(cudaMemsetAsync(ctl.err, 0, sizeof(int32_t), stream))) ||
        (s = ck(cudaMemsetAsync(ctl.red, 0, kRedSlots * sizeof(unsigned long long), stream))))
        return s;
    DevGrid dg = g->dg;
    void* args[] = {(void*)&dg, (void*)&ss, (void*)&ctl, (void*)&sp};
    if ((s = ck(cudaEventRecord(g->ev0, stream))) ||
        (s = ck(cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(256), args, smem, stream))) ||
        (s = ck(cudaEventRecord(g->ev1, stream))))
        return s;
    int32_t err = 0;
    double hst[kStatCount];
    if ((s = ck(cudaMemcpyAsync(&err, ctl.err, sizeof(int32_t), cudaMemcpyDeviceToHost, stream))) ||
        (s = ck(cudaMemcpyAsync(hst, ctl.stats, sizeof(hst), cudaMemcpyDeviceToHost, stream))) ||
        (s = ck(cudaStreamSynchronize(stream))))
        return s;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    const int64_t done = (int64_t)hst[kStatSteps];
    if (out && out->vmin && done > 0) {
        const cudaError_t e = cudaMemcpy(out->vmin, ss.vmin_key, (size_t)done * n_scen * sizeof(double),
                                         host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
        if (e != cudaSuccess) return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    }
    if (out && out->v_all && host && done > 0) {
        const cudaError_t e = cudaMemcpy(out->v_all, v_all, (size_t)done * n_scen * g->P.n * sizeof(double),
                                         cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    }
    fill_run_stats(g, hst, ms, stats, 0.0);     // every scenario starts at the exact DC point
    g->has_state = false;                        // the grid's own transient state is not advanced
    g->inc_ok = false;
    if (err == PG_ERR_TIMEOUT) return fail(PG_ERR_TIMEOUT, "device barrier timed out");
    if (err == PG_ERR_NOT_CONVERGED) return fail(PG_ERR_NOT_CONVERGED, "relaxation did not converge");
    if (err != 0) return fail(PG_ERR_CUDA, "device error");
    return PG_OK;
}
