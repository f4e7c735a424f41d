// Device code: the persistent backward-Euler step driver (Algorithm 1) with
// red-black / multicolour SOR sweeps (Eq. 15-17) over SELL-packed neighbour
// lists, fused residual monitors, FP64 defect correction and the inductor
// current update (Eq. 10).
//
// Work mapping: a warp owns one SELL slice of kSlice = 128 consecutive nodes
// of one colour; lane l handles nodes 4l..4l+3 of the slice, so every
// per-node array and every slot of the weight/column arrays is read with one
// 128-bit (float4 / int4) or two 128-bit (double2) loads per lane, coalesced
// across the warp.  A "diagonal" slice (all columns are the node index plus a
// per-slot constant, which is what a lattice gives in colour-major order)
// carries no column indices at all.
//
// Synchronisation: one cooperative launch; the colour phases are separated
// by a device-wide barrier whose wait is bounded by a globaltimer limit.  On
// timeout the waiting block records PG_ERR_TIMEOUT and every block returns at
// its next barrier, so a failure never leaves the GPU spinning.
#include <cuda/atomic>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "pg_internal.h"

namespace pg {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---- 4-wide loads/stores.  ldg*: read-only for the whole launch (nc path);
//      ld*/st*: state that other blocks write during the launch.
__device__ __forceinline__ void ldg4(const float* p, float (&x)[4]) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void ldg4(const double* p, double (&x)[4]) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}
__device__ __forceinline__ void ldg4(const int32_t* p, int (&x)[4]) {
    int4 v = __ldg(reinterpret_cast<const int4*>(p));
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void ld4(const float* p, float (&x)[4]) {
    float4 v = *reinterpret_cast<const float4*>(p);
    x[0] = v.x; x[1] = v.y; x[2] = v.z; x[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double (&x)[4]) {
    double2 a = reinterpret_cast<const double2*>(p)[0];
    double2 b = reinterpret_cast<const double2*>(p)[1];
    x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float (&x)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void st4(double* p, const double (&x)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(x[0], x[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(x[2], x[3]);
}

// max that lets a NaN win, so a diverged iterate is never mistaken for convergence
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }

// Block-wide max of non-negative values, merged into *slot with one atomic per block.
__device__ __forceinline__ void block_max_into(double v, unsigned long long* slot) {
    __shared__ double sm[32];
    for (int o = 16; o; o >>= 1) v = nanmax(v, __shfl_xor_sync(kFull, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (w == 0) {
        v = (l < (int)(blockDim.x >> 5)) ? sm[l] : 0.0;
        for (int o = 16; o; o >>= 1) v = nanmax(v, __shfl_xor_sync(kFull, v, o));
        if (l == 0 && v != 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(v));
    }
    __syncthreads();
}

// Order-preserving map of a double to an unsigned key (for min reductions).
__device__ __forceinline__ unsigned long long order_key(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Device-wide barrier with a time limit.  .ok is false (for the whole block)
// when this or any other block recorded an error.  .val receives the value of
// `read_slot` (a max-reduction slot filled before the barrier), read once by
// thread 0 after the wait and broadcast, so every block sees the same number.
struct BarrierResult {
    bool ok;
    double val;
};

__device__ __forceinline__ BarrierResult grid_barrier(const DevCtl& c, unsigned nblocks, long long timeout_ns,
                                                      bool skip, const unsigned long long* read_slot) {
    __shared__ int s_ok;
    __shared__ double s_val;
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(*c.bar_gen);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(*c.bar_count);
        cuda::atomic_ref<int, cuda::thread_scope_device> err(*c.err);
        int ok = 1;
        {
            const unsigned g0 = gen.load(cuda::memory_order_relaxed);
            __threadfence();
            // test hook: this block waits without being counted, so the barrier can never open
            const unsigned arrived = skip ? 0u : cnt.fetch_add(1u, cuda::memory_order_acq_rel);
            if (!skip && arrived == nblocks - 1) {
                cnt.store(0u, cuda::memory_order_relaxed);
                gen.fetch_add(1u, cuda::memory_order_release);
            } else {
                const long long t0 = global_ns();
                unsigned ns = 32;
                while (gen.load(cuda::memory_order_acquire) == g0) {
                    if (err.load(cuda::memory_order_relaxed) != 0) { ok = 0; break; }
                    if (global_ns() - t0 > timeout_ns) {
                        int z = 0;
                        err.compare_exchange_strong(z, (int)PG_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(ns);
                    if (ns < 256) ns <<= 1;
                }
            }
            __threadfence();
            if (ok && err.load(cuda::memory_order_acquire) != 0) ok = 0;
        }
        s_ok = ok;
        if (read_slot) {
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(
                *const_cast<unsigned long long*>(read_slot));
            s_val = __longlong_as_double((long long)r.load(cuda::memory_order_acquire));
        }
    }
    __syncthreads();
    return BarrierResult{s_ok != 0, s_val};
}

// Value of current source e at time t (piecewise linear, held outside the breakpoints).
__device__ __forceinline__ double pwl_eval(const DevGrid& g, int e, double t) {
    int64_t lo = g.pwl_ptr[e], hi = g.pwl_ptr[e + 1] - 1;
    const double* T = g.pwl_t;
    const double* V = g.pwl_v;
    if (t <= T[lo]) return V[lo];
    if (t > T[hi]) return V[hi];
    while (hi - lo > 1) {            // keep T[lo] < t <= T[hi]
        int64_t mid = (lo + hi) >> 1;
        if (t <= T[mid]) hi = mid; else lo = mid;
    }
    return V[lo] + (V[hi] - V[lo]) * ((t - T[lo]) / (T[hi] - T[lo]));
}

// Buffer selection by value (no dynamic indexing of kernel-parameter arrays,
// which would force them into local memory).
__device__ __forceinline__ double* vbuf(const DevState& st, int k) {
    return k == 0 ? st.v[0] : (k == 1 ? st.v[1] : st.v[2]);
}
template <typename T>
__device__ __forceinline__ T* dbuf(const DevState& st, int k);
template <>
__device__ __forceinline__ double* dbuf<double>(const DevState& st, int k) { return k ? st.d64[1] : st.d64[0]; }
template <>
__device__ __forceinline__ float* dbuf<float>(const DevState& st, int k) { return k ? st.d32[1] : st.d32[0]; }

__device__ __forceinline__ double term_volt(const DevGrid& g, const double* v, int t) {
    return t >= 0 ? v[t] : (t == PG_GROUND ? 0.0 : g.vdd[-2 - t]);
}

// Columns of the 4 nodes of this lane in slot k of slice s.
__device__ __forceinline__ void slot_cols(const DevGrid& g, bool dia, int dbase, int64_t e, int i0, int k,
                                          int (&c)[4]) {
    if (dia) {
        const int o = __ldg(g.dia_off + dbase + k);
        c[0] = i0 + o; c[1] = i0 + 1 + o; c[2] = i0 + 2 + o; c[3] = i0 + 3 + o;
    } else {
        ldg4(g.ell_col + e, c);
    }
}

// sigma_j = sum_k w[k][j] * x(col[k][j]) for the lane's 4 nodes, accumulated in Acc.
template <typename Acc, typename Wt, typename Load>
__device__ __forceinline__ void sell_row(const DevGrid& g, const Wt* w, int s, int lane, Load xload,
                                         Acc (&sig)[4]) {
    const int64_t base = __ldg(g.slice_off + s) + lane * kVec;
    const int K = __ldg(g.slice_w + s);
    const int d0 = __ldg(g.slice_doff + s);
    const bool dia = __ldg(g.slice_doff + s + 1) > d0;
    const int i0 = s * kSlice + lane * kVec;
    sig[0] = sig[1] = sig[2] = sig[3] = Acc(0);
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
        const int64_t e = base + (int64_t)k * kSlice;
        Wt wv[4];
        ldg4(w + e, wv);
        int c[4];
        slot_cols(g, dia, d0, e, i0, k, c);
#pragma unroll
        for (int j = 0; j < 4; ++j) sig[j] = fma((Acc)wv[j], xload(c[j]), sig[j]);
    }
}

// ---------------------------------------------------------------- phases

// Start of a step: RHS assembly (Eq. 2 / Eq. 10), warm start, FP64 residual.
template <bool MIXED>
__device__ __forceinline__ double phase_rhs(const DevGrid& g, const DevState& st, const RunParams& rp, int s, int lane,
                            int vL, int vP, int vF, bool extrap, double t, int dsel) {
    const int i0 = s * kSlice + lane * kVec;
    const double* vl = vbuf(st, vL);
    const double* vp = vbuf(st, vP);
    double vw[4], b[4], D[4], iD[4];
    ldg4(g.D64 + i0, D);
    ldg4(g.invD64 + i0, iD);
    if (rp.mode == kModeSolve) {
        ldg4(st.rhs + i0, b);
        vw[0] = vw[1] = vw[2] = vw[3] = 0.0;
    } else {
        double a[4], ch[4], cj[4];
        ld4(vl + i0, a);
        ldg4(g.ch + i0, ch);
        ldg4(g.cinj + i0, cj);
        if (extrap) {
            double pp[4];
            ld4(vp + i0, pp);
#pragma unroll
            for (int j = 0; j < 4; ++j) vw[j] = 2.0 * a[j] - pp[j];
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) vw[j] = a[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double bj = ch[j] * a[j] + cj[j];
            const int i = i0 + j;
            for (int q = __ldg(g.ld_ptr + i); q < __ldg(g.ld_ptr + i + 1); ++q) {
                const int sid = __ldg(g.ld_idx + q);
                const double I = pwl_eval(g, (sid > 0 ? sid : -sid) - 1, t);
                bj -= sid > 0 ? I : -I;               // A_i^T I_s(t+h)
            }
            for (int q = __ldg(g.ind_ptr + i); q < __ldg(g.ind_ptr + i + 1); ++q) {
                const int lid = __ldg(g.ind_idx + q);
                const double il = st.il[(lid > 0 ? lid : -lid) - 1];
                bj -= lid > 0 ? il : -il;             // A_l^T i_l(t)
            }
            b[j] = bj;
        }
    }
    double sig[4];
    if (rp.mode == kModeSolve) {
        sig[0] = sig[1] = sig[2] = sig[3] = 0.0;
    } else if (extrap) {
        sell_row<double>(g, g.w64, s, lane, [&](int c) { return 2.0 * vl[c] - vp[c]; }, sig);
    } else {
        sell_row<double>(g, g.w64, s, lane, [&](int c) { return vl[c]; }, sig);
    }
    double r[4], mon = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        r[j] = b[j] + sig[j] - D[j] * vw[j];
        mon = nanmax(mon, fabs(r[j]) * iD[j]);
    }
    st4(vbuf(st, vF) + i0, vw);
    st4(st.r64 + i0, r);
    if (MIXED) {
        float r32[4] = {(float)r[0], (float)r[1], (float)r[2], (float)r[3]};
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        st4(st.r32 + i0, r32);
        st4(dbuf<float>(st, dsel) + i0, z);
    } else {
        double z[4] = {0.0, 0.0, 0.0, 0.0};
        st4(dbuf<double>(st, dsel) + i0, z);
    }
    return mon;
}

// One colour's SOR half-sweep on M delta = r (Eq. 16-17): returns max |unrelaxed update|.
template <typename T>
__device__ __forceinline__ double sweep_slice(const DevGrid& g, const T* w, const T* invD, const T* r, T* d, int s, int lane,
                              T omega) {
    const int i0 = s * kSlice + lane * kVec;
    T dv[4], rv[4], iD[4], sig[4];
    ld4(d + i0, dv);
    ld4(r + i0, rv);
    ldg4(invD + i0, iD);
    sell_row<T>(g, w, s, lane, [&](int c) { return d[c]; }, sig);
    double mon = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T upd = (rv[j] + sig[j]) * iD[j] - dv[j];
        dv[j] = fma(omega, upd, dv[j]);
        mon = nanmax(mon, (double)fabs(upd));
    }
    st4(d + i0, dv);
    return mon;
}

// Outer defect-correction pass: v += delta, r -= M delta (FP64), refresh the FP32 residual.
template <typename T>
__device__ __forceinline__ double outer_slice(const DevGrid& g, const DevState& st, const T* d, T* dnext, float* r32, int s,
                              int lane, double* v) {
    const int i0 = s * kSlice + lane * kVec;
    T dv[4];
    ld4(d + i0, dv);
    double D[4], iD[4], r[4], vv[4], sig[4];
    ldg4(g.D64 + i0, D);
    ldg4(g.invD64 + i0, iD);
    ld4(st.r64 + i0, r);
    ld4(v + i0, vv);
    sell_row<double>(g, g.w64, s, lane, [&](int c) { return (double)d[c]; }, sig);
    double mon = 0.0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double dj = (double)dv[j];
        r[j] = r[j] - (D[j] * dj - sig[j]);
        vv[j] += dj;
        mon = nanmax(mon, fabs(r[j]) * iD[j]);
    }
    st4(st.r64 + i0, r);
    st4(v + i0, vv);
    T z[4] = {T(0), T(0), T(0), T(0)};
    st4(dnext + i0, z);
    if (r32) {
        float f[4] = {(float)r[0], (float)r[1], (float)r[2], (float)r[3]};
        st4(r32 + i0, f);
    }
    return mon;
}

}  // namespace

// ---------------------------------------------------------------- the persistent kernel

template <bool MIXED>
__global__ void __launch_bounds__(256) persistent_kernel(DevGrid g, DevState st, DevCtl ctl, RunParams rp) {
    using T = typename std::conditional<MIXED, float, double>::type;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const T omega = (T)rp.omega;

    // Reduction slots rotate over 4 barrier-delimited phases: phase k merges into
    // slot k%4 and, at its start, clears slot (k+2)%4, whose last readers all
    // passed barrier k-1 (the host clears all four before the launch).
    int phase = 0;
    bool first_bar = true;
    auto barrier = [&](bool want_val) -> BarrierResult {
        const bool skip = first_bar && (rp.debug_flags & PG_DEBUG_SKIP_ARRIVAL) && blockIdx.x == 0;
        first_bar = false;
        const BarrierResult r =
            grid_barrier(ctl, nblocks, rp.timeout_ns, skip, want_val ? ctl.red + (phase & 3) : nullptr);
        ++phase;
        if (lead) ctl.red[(phase + 2) & 3] = 0ull;
        return r;
    };

    // statistics (kept by every thread identically; block 0 thread 0 publishes)
    long long tot_sweeps = 0, tot_outer = 0, steps_done = 0;
    int max_sw = 0, max_out = 0;
    double max_bound_R = 0.0, last_R = 0.0;
    auto publish = [&](long long failed) {
        if (lead) {
            ctl.stats[kStatSteps] = (double)steps_done;
            ctl.stats[kStatSweeps] = (double)tot_sweeps;
            ctl.stats[kStatMaxSweeps] = (double)max_sw;
            ctl.stats[kStatOuter] = (double)tot_outer;
            ctl.stats[kStatMaxOuter] = (double)max_out;
            ctl.stats[kStatMaxBound] = max_bound_R;
            ctl.stats[kStatFailedStep] = (double)failed;
            ctl.stats[kStatLastR] = last_R;
        }
    };
    auto fail = [&](long long step) {
        if (lead) {
            cuda::atomic_ref<int, cuda::thread_scope_device> err(*ctl.err);
            int z = 0;
            err.compare_exchange_strong(z, (int)PG_ERR_NOT_CONVERGED);
        }
        publish(step);
    };
    // per-step min voltage: reduce the per-block partials of step sl
    auto finalize_vmin = [&](int sl) {
        if (blockIdx.x == 0 && threadIdx.x < 32 && rp.vmin) {
            unsigned long long bk = ~0ull;
            int ba = 0x7fffffff;
            const int par = sl & 1;
            for (unsigned b = threadIdx.x; b < nblocks; b += 32) {
                const unsigned long long k = ctl.blk_min[par * nblocks + b];
                const int a = ctl.blk_arg[par * nblocks + b];
                if (k < bk || (k == bk && a < ba)) { bk = k; ba = a; }
            }
            for (int o = 16; o; o >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(kFull, bk, o);
                const int a2 = __shfl_xor_sync(kFull, ba, o);
                if (k2 < bk || (k2 == bk && a2 < ba)) { bk = k2; ba = a2; }
            }
            if (threadIdx.x == 0) {
                rp.vmin[sl] = key_value(bk);
                if (rp.vmin_node) rp.vmin_node[sl] = ba;
            }
        }
    };

    int vL = rp.cur, vP = rp.prev, vF = 3 - rp.cur - rp.prev;
    bool have_prev = rp.have_prev != 0;
    const int nsl = g.n_slices;

    for (int sl = 0; sl < rp.nsteps; ++sl) {
        const long long sabs = rp.step0 + sl + 1;
        const double t = (double)sabs * rp.h;
        const bool extrap = rp.mode == kModeTransient && rp.warm_extrap && have_prev;
        int dsel = 0;
        if (sl > 0) finalize_vmin(sl - 1);

        // ---- phase A: RHS + warm start + residual, all colours
        double mon = 0.0;
        for (int s = gwarp; s < nsl; s += nwarps)
            mon = nanmax(mon, phase_rhs<MIXED>(g, st, rp, s, lane, vL, vP, vF, extrap, t, dsel));
        block_max_into(mon, ctl.red + (phase & 3));
        BarrierResult br = barrier(true);
        if (!br.ok) { publish(-1); return; }
        double R = br.val;

        int sweeps = 0, outer = 0;
        bool ok = true;
        while (!(R <= rp.target)) {
            if (!(R == R) || isinf(R) || outer >= rp.max_outer || sweeps >= rp.max_sweeps) { ok = false; break; }
            // inner relaxation on the correction
            const double inner_tgt = MIXED ? fmax(0.5 * rp.target, rp.inner_reduction * R) : 0.5 * rp.target;
            const T* rr = MIXED ? (const T*)st.r32 : (const T*)st.r64;
            T* dd = dbuf<T>(st, dsel);
            const T* ww = MIXED ? (const T*)g.w32 : (const T*)g.w64;
            const T* iD = MIXED ? (const T*)g.invD32 : (const T*)g.invD64;
            double est_mark = INFINITY;   // monitor value at the last stagnation check
            int inner = 0;
            while (true) {
                double est = 0.0;
                for (int c = 0; c < g.ncol; ++c) {
                    const int s0 = __ldg(g.colour_slice + c), s1 = __ldg(g.colour_slice + c + 1);
                    double m = 0.0;
                    for (int s = s0 + gwarp; s < s1; s += nwarps)
                        m = nanmax(m, sweep_slice<T>(g, ww, iD, rr, dd, s, lane, omega));
                    block_max_into(m, ctl.red + (phase & 3));
                    const BarrierResult be = barrier(true);
                    if (!be.ok) { publish(-1); return; }
                    est = nanmax(est, be.val);
                }
                ++sweeps;
                ++inner;
                if (est <= inner_tgt || !(est == est) || sweeps >= rp.max_sweeps) break;
                // The inner solve stalls at its precision floor (about eps * ||M^-1 D|| of the
                // correction); hand over to the FP64 outer pass when 16 sweeps gain < 10 %.
                if ((inner & 15) == 0) {
                    if (est > 0.9 * est_mark) break;
                    est_mark = est;
                }
            }
            // outer pass
            double m = 0.0;
            T* dn = dbuf<T>(st, dsel ^ 1);
            for (int s = gwarp; s < nsl; s += nwarps)
                m = nanmax(m, outer_slice<T>(g, st, dd, dn, MIXED ? st.r32 : nullptr, s, lane, vbuf(st, vF)));
            block_max_into(m, ctl.red + (phase & 3));
            br = barrier(true);
            if (!br.ok) { publish(-1); return; }
            R = br.val;
            dsel ^= 1;
            ++outer;
        }
        if (!ok) { fail(sabs); return; }

        // ---- post: inductor currents (Eq. 10), outputs
        const double* vnew = vbuf(st, vF);
        if (rp.mode == kModeTransient) {
            for (int e = gtid; e < g.n_l; e += nthreads) {
                const double va = term_volt(g, vnew, __ldg(g.ind_a + e));
                const double vb = term_volt(g, vnew, __ldg(g.ind_b + e));
                const double il = st.il[e] + __ldg(g.ind_hl + e) * (va - vb);
                st.il[e] = il;
                if (rp.il_all) rp.il_all[(long long)sl * g.n_l + e] = il;
            }
        }
        unsigned long long bk = ~0ull;
        int ba = 0x7fffffff;
        for (int i = gtid; i < g.n_pad; i += nthreads) {
            const int o = __ldg(g.orig + i);
            if (o < 0) continue;
            const double x = vnew[i];
            if (rp.v_all) rp.v_all[(long long)sl * g.n_real + o] = x;
            if (rp.solve_out) rp.solve_out[o] = x;
            if (rp.vmin) {
                const unsigned long long k = order_key(x);
                if (k < bk || (k == bk && o < ba)) { bk = k; ba = o; }
            }
        }
        if (rp.probe_v)
            for (int k = gtid; k < rp.n_probes; k += nthreads)
                rp.probe_v[(long long)sl * rp.n_probes + k] = vnew[rp.probes_perm[k]];
        if (rp.vmin) {
            __shared__ unsigned long long s_k[32];
            __shared__ int s_a[32];
            for (int o = 16; o; o >>= 1) {
                const unsigned long long k2 = __shfl_xor_sync(kFull, bk, o);
                const int a2 = __shfl_xor_sync(kFull, ba, o);
                if (k2 < bk || (k2 == bk && a2 < ba)) { bk = k2; ba = a2; }
            }
            const int w = threadIdx.x >> 5;
            if (lane == 0) { s_k[w] = bk; s_a[w] = ba; }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int q = 1; q < (int)(blockDim.x >> 5); ++q)
                    if (s_k[q] < bk || (s_k[q] == bk && s_a[q] < ba)) { bk = s_k[q]; ba = s_a[q]; }
                ctl.blk_min[(sl & 1) * nblocks + blockIdx.x] = bk;
                ctl.blk_arg[(sl & 1) * nblocks + blockIdx.x] = ba;
            }
        }
        tot_sweeps += sweeps; tot_outer += outer;
        max_sw = max(max_sw, sweeps); max_out = max(max_out, outer);
        max_bound_R = fmax(max_bound_R, R);
        last_R = R;
        ++steps_done;
        // rotate: the new state becomes the latest
        vP = vL; vL = vF; vF = 3 - vL - vP;
        have_prev = true;
        if (!barrier(false).ok) { publish(-1); return; }
    }
    if (rp.nsteps > 0) finalize_vmin(rp.nsteps - 1);
    publish(-1);
}

// ---------------------------------------------------------------- power iteration for omega

// y = (x + D^-1 W x) / 2 with x scaled by 1/xmax_prev; accumulates x.(Wx), x.(Dx), max y.
__global__ void __launch_bounds__(256) power_step_kernel(DevGrid g, const double* x, double* y,
                                                        const unsigned long long* xmax_prev, double* acc,
                                                        unsigned long long* ymax) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const double sc = xmax_prev ? 1.0 / __longlong_as_double((long long)*xmax_prev) : 1.0;
    double num = 0.0, den = 0.0, mx = 0.0;
    for (int s = gwarp; s < g.n_slices; s += nwarps) {
        const int i0 = s * kSlice + lane * kVec;
        double xv[4], D[4], iD[4], sig[4], yv[4];
        ld4(x + i0, xv);
        ldg4(g.D64 + i0, D);
        ldg4(g.invD64 + i0, iD);
        sell_row<double>(g, g.w64, s, lane, [&](int c) { return x[c] * sc; }, sig);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const double xs = xv[j] * sc;
            num += xs * sig[j];
            den += D[j] * xs * xs;
            yv[j] = 0.5 * (xs + iD[j] * sig[j]);
            mx = fmax(mx, yv[j]);
        }
        st4(y + i0, yv);
    }
    for (int o = 16; o; o >>= 1) {
        num += __shfl_xor_sync(kFull, num, o);
        den += __shfl_xor_sync(kFull, den, o);
        mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if (lane == 0) {
        atomicAdd(acc + 0, num);
        atomicAdd(acc + 1, den);
        atomicMax(ymax, (unsigned long long)__double_as_longlong(mx));
    }
}

// ---------------------------------------------------------------- state set-up

// dst[i] = src[orig[i]] (caller numbering -> permuted), or `fill` when src is null; padding gets 0.
__global__ void permute_in_kernel(const int32_t* __restrict__ orig, const double* __restrict__ src, double fill,
                                  double* __restrict__ dst, int n_pad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
        const int o = orig[i];
        dst[i] = o < 0 ? 0.0 : (src ? src[o] : fill);
    }
}

// ---------------------------------------------------------------- host-side launch helpers

cudaError_t launch_persistent(bool mixed, const DevGrid& g, const DevState& st, const DevCtl& ctl,
                              const RunParams& rp, int blocks, int threads, cudaStream_t stream) {
    void* args[] = {(void*)&g, (void*)&st, (void*)&ctl, (void*)&rp};
    const void* fn = mixed ? (const void*)persistent_kernel<true> : (const void*)persistent_kernel<false>;
    return cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, 0, stream);
}

cudaError_t persistent_occupancy(bool mixed, int threads, int* blocks_per_sm) {
    const void* fn = mixed ? (const void*)persistent_kernel<true> : (const void*)persistent_kernel<false>;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, 0);
}

cudaError_t launch_power_step(const DevGrid& g, const double* x, double* y, const unsigned long long* xmax_prev,
                              double* acc, unsigned long long* ymax, int blocks, cudaStream_t stream) {
    power_step_kernel<<<blocks, 256, 0, stream>>>(g, x, y, xmax_prev, acc, ymax);
    return cudaGetLastError();
}

cudaError_t launch_permute_in(const int32_t* orig, const double* src, double fill, double* dst, int n_pad,
                              int n_sm, cudaStream_t stream) {
    const int blocks = std::max(1, std::min(4 * n_sm, (n_pad + 255) / 256));
    permute_in_kernel<<<blocks, 256, 0, stream>>>(orig, src, fill, dst, n_pad);
    return cudaGetLastError();
}

}  // namespace pg
