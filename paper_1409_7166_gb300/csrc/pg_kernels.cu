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

#include "pg_device.cuh"

// Minimum resident blocks per SM requested from ptxas for the persistent
// kernel (register budget = 65536 / (256 * PG_MIN_BLOCKS)).
#ifndef PG_MIN_BLOCKS
#define PG_MIN_BLOCKS 2
#endif
// Slots of the SOR sweep issued together (loads in flight per lane).
#ifndef PG_SWEEP_UNROLL
#define PG_SWEEP_UNROLL 4
#endif
constexpr int kSweepUnroll = PG_SWEEP_UNROLL;
constexpr int kIncPeriod = 16;        // full recompute of the step-start residual every 16 steps
constexpr int kIncMaxOuter = 4;       // ... and after any step that needed more outer passes

namespace pg {

namespace {

// ---- slice descriptors
//
// A warp owns a contiguous run of slices of every colour (the same run in
// every pass).  Their descriptors and diagonal column offsets are copied once
// per launch into the warp's part of shared memory, so a sweep reads no
// metadata from global memory: per slice only the weights, the node vectors
// and the neighbour values.
constexpr int kWarpsPerBlock = 8;
constexpr int kCacheSlices = 32;    // descriptors cached per warp
constexpr int kCachePool = 192;     // diagonal offsets cached per warp (32 slices x 6)

struct WarpCache {
    SliceDesc desc[kCacheSlices];
    int pool[kCachePool];
    int base[kMaxColours + 1];   // index of the warp's first slice of colour c in its list
    int lo[kMaxColours];         // first slice of colour c owned by the warp
    int cnt[kMaxColours];        // slices of colour c owned by the warp
};

// Fill the calling warp's cache (once per launch).  Every lane must call it.
__device__ void fill_warp_cache(const DevGrid& g, WarpCache& wc, int gwarp, int nwarps) {
    const int lane = threadIdx.x & 31;
    int j = 0;
    for (int c = 0; c < g.ncol; ++c) {
        const int c0 = __ldg(g.colour_slice + c), c1 = __ldg(g.colour_slice + c + 1);
        const int S = c1 - c0;
        const int R = (S + nwarps - 1) / nwarps;
        const int lo = min(c0 + gwarp * R, c1), hi = min(lo + R, c1);
        if (lane == 0) { wc.base[c] = j; wc.lo[c] = lo; wc.cnt[c] = hi - lo; }
        for (int t = lane; t < hi - lo; t += 32)
            if (j + t < kCacheSlices) wc.desc[j + t] = global_desc(g, lo + t);
        j += hi - lo;
    }
    if (lane == 0) wc.base[g.ncol] = j;
    __syncwarp();
    if (lane == 0) {
        int pos = 0;
        for (int k = 0; k < min(j, kCacheSlices); ++k) {
            SliceDesc& d = wc.desc[k];
            if (d.dpos <= -2) {
                if (pos + d.K <= kCachePool) {
                    const int src = -2 - d.dpos;
                    for (int q = 0; q < d.K; ++q) wc.pool[pos + q] = __ldg(g.dia_off + src + q);
                    d.dpos = pos;
                    pos += d.K;
                }
            }
        }
    }
    __syncwarp();
}

// Descriptor of the t-th slice (slice id s) of colour c in this warp's run.
__device__ __forceinline__ SliceDesc warp_desc(const DevGrid& g, const WarpCache& wc, int c, int t, int s) {
    const int j = wc.base[c] + t;
    return j < kCacheSlices ? wc.desc[j] : global_desc(g, s);
}

// sigma_j = sum_k w[k][j] * x(col[k][j]) for the lane's 4 nodes, accumulated in Acc.
// UNROLL trades registers for loads in flight: the hot FP32 sweep unrolls, the
// once-per-pass FP64 rows do not (they would set the register budget of the whole
// persistent kernel).
template <int UNROLL, typename Acc, typename Wt, typename Load>
__device__ __forceinline__ void sell_row(const DevGrid& g, const WarpCache* wc, const SliceDesc& d, const Wt* w,
                                         int s, int lane, Load xload, Acc (&sig)[4]) {
    const long long base = d.off + lane * kVec;
    const int i0 = s * kSlice + lane * kVec;
    const int* offs = d.dpos >= 0 ? wc->pool + d.dpos : (d.dpos <= -2 ? g.dia_off + (-2 - d.dpos) : nullptr);
    sig[0] = sig[1] = sig[2] = sig[3] = Acc(0);
#pragma unroll UNROLL
    for (int k = 0; k < d.K; ++k) {
        const long long e = base + (long long)k * kSlice;
        Wt wv[4];
        ldg4(w + e, wv);
        int c[4];
        if (offs) {
            const int o = offs[k];
            c[0] = i0 + o; c[1] = i0 + 1 + o; c[2] = i0 + 2 + o; c[3] = i0 + 3 + o;
        } else {
            ldg4(g.ell_col + e, c);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) sig[j] = fma((Acc)wv[j], xload(c[j]), sig[j]);
    }
}

// ---- double-float products for the outer pass (FP32 pairs; GB300's FP64 rate is a
// small fraction of its FP32 rate).  (hi, lo) += (a_hi + a_lo) x for an FP32 x: the
// leading product is split exactly (FMA), the sum kept by TwoSum (Knuth), so the
// result carries about 48 significant bits.
// The error-free steps use the _rn intrinsics, which the compiler never contracts
// into FMAs (a contraction would break the TwoSum identity).
__device__ __forceinline__ void df_acc(float& hi, float& lo, float a_hi, float a_lo, float x) {
    const float p = __fmul_rn(a_hi, x);
    const float e = fmaf(a_hi, x, -p);                 // a_hi x = p + e exactly
    const float t = __fadd_rn(hi, p);
    const float bv = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bv)), __fsub_rn(p, bv));   // hi + p = t + err
    hi = t;
    lo += err + fmaf(a_lo, x, e);
}

// sum_k w_k x_{col_k} of one slice row as a double-float, weights as FP32 pairs; two
// slots' loads in flight at a time (more would spill in the mixed-precision kernel)
template <typename Load>
__device__ __forceinline__ void sell_row_df(const DevGrid& g, const WarpCache* wc, const SliceDesc& d, int s, int lane,
                                            Load xload, float (&hi)[4], float (&lo)[4]) {
    const long long base = d.off + lane * kVec;
    const int i0 = s * kSlice + lane * kVec;
    const int* offs = d.dpos >= 0 ? wc->pool + d.dpos : (d.dpos <= -2 ? g.dia_off + (-2 - d.dpos) : nullptr);
#pragma unroll
    for (int j = 0; j < 4; ++j) hi[j] = lo[j] = 0.f;
#pragma unroll 2
    for (int k = 0; k < d.K; ++k) {
        const long long e = base + (long long)k * kSlice;
        float wh[4], wl[4];
        ldg4(g.w32 + e, wh);
        ldg4(g.w32lo + e, wl);
        int c[4];
        if (offs) {
            const int o = offs[k];
            c[0] = i0 + o; c[1] = i0 + 1 + o; c[2] = i0 + 2 + o; c[3] = i0 + 3 + o;
        } else {
            ldg4(g.ell_col + e, c);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) df_acc(hi[j], lo[j], wh[j], wl[j], xload(c[j]));
    }
}

// ---------------------------------------------------------------- phases

// md = M (x0 - v(s-1)) for a step whose start residual is computed in full: M (v(s-1) -
// v(s-2)) with the extrapolated warm start, 0 without.
__device__ __forceinline__ void md_slice(const DevGrid& g, const WarpCache* wc, const SliceDesc& sd, const DevState& st,
                                         int s, int lane, const double* vl, const double* vp, bool extrap, float th) {
    const int i0 = s * kSlice + lane * kVec;
    double m[4] = {0.0, 0.0, 0.0, 0.0};
    if (extrap) {
        double sig[4], D[4], a[4], p[4];
        sell_row<1, double>(g, wc, sd, g.w64, s, lane, [&](int c) { return vl[c] - vp[c]; }, sig);
        ldg4(g.D64 + i0, D);
        ld4(vl + i0, a);
        ld4(vp + i0, p);
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = D[j] * (a[j] - p[j]) - sig[j];
        if (th != 1.0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) m[j] *= th;       // M (x0 - v(s-1)) = th M (v(s-1) - v(s-2))
        }
    }
    st4(st.md + i0, m);
}

// Warm start v(s-1) + th (v(s-1) - v(s-2)); th = 1 keeps the plain form (same rounding).
__device__ __forceinline__ double warm_value(double a, double p, double th) {
    return th == 1.0 ? 2.0 * a - p : a + th * (a - p);
}

// Start of a step: RHS assembly (Eq. 2 / Eq. 10), warm start, FP64 residual.
template <bool MIXED, bool DAMP>
__device__ __forceinline__ double phase_rhs(const DevGrid& g, const WarpCache* wc, const SliceDesc& sd,
                                            const DevState& st, const RunParams& rp, int s, int lane, int vL, int vP,
                                            int vF, bool extrap, bool three, bool inc, long long sabs, int dsel,
                                            unsigned long long* latR,
                                            LatAccT<typename std::conditional<MIXED, float, double>::type>& lacc,
                                            float th_in) {
    using MonT = typename std::conditional<MIXED, float, double>::type;   // monitored max |r| / D
    const float th = DAMP ? th_in : 1.0f;
    const int i0 = s * kSlice + lane * kVec;
    const double* vl = vbuf(st, vL);
    const double* vp = vbuf(st, vP);
    double vw[4], b[4], D[4];
    MonT iD[4];                                  // 1 / D: FP32 for the mixed kernel's FP32 monitor
    ldg4(g.D64 + i0, D);
    if constexpr (MIXED) ldg4(g.invD32 + i0, iD);
    else ldg4(g.invD64 + i0, iD);

    double base[4] = {0.0, 0.0, 0.0, 0.0};       // the residual is taken of M (x0 - base)
    if (rp.mode == kModeSolve) {
        ldg4(st.rhs + i0, b);
        if (rp.x0) ldg4(rp.x0 + i0, vw);
        else vw[0] = vw[1] = vw[2] = vw[3] = 0.0;
    } else if (three || inc) {
        // Eq. 11 less M v(s-1), an exact rearrangement (the explicit form's incremental step
        // start adds the previous step's final residual to the same increment):
        //   b - M v(s-1) = (C/h)(v(s-1) - v(s-2)) - A_l^T h L^-1 (A_l v(s-1) + A_ls v_d)
        //                  - A_i^T (I_s(t) - I_s(t-h)),
        // and the residual of x0 is that minus M (x0 - v(s-1)).
        double pp[4], ch[4], Ic[4], Ip[4];
        ld4(vl + i0, base);
        ld4(vp + i0, pp);
        ldg4(g.ch + i0, ch);
        ld4(st.inode + (sabs & 1) * (long long)g.n_pad + i0, Ic);          // (A_i^T I_s(t))_i
        ld4(st.inode + ((sabs - 1) & 1) * (long long)g.n_pad + i0, Ip);    // (A_i^T I_s(t - h))_i
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            vw[j] = extrap ? warm_value(base[j], pp[j], th) : base[j];
            double bj = ch[j] * (base[j] - pp[j]) - (Ic[j] - Ip[j]);
            const int i = i0 + j;
            if (g.n_l > 0)
            for (int q = __ldg(g.ind_ptr + i); q < __ldg(g.ind_ptr + i + 1); ++q) {
                const int lid = __ldg(g.ind_idx + q);
                const int e = (lid > 0 ? lid : -lid) - 1;
                const double di = __ldg(g.ind_hl + e) *
                                  (term_volt(g, vl, __ldg(g.ind_a + e)) - term_volt(g, vl, __ldg(g.ind_b + e)));
                bj -= lid > 0 ? di : -di;
            }
            b[j] = bj;
        }
    } else {
        double a[4], ch[4], cj[4], Ic[4];
        ld4(vl + i0, a);
        ldg4(g.ch + i0, ch);
        ldg4(g.cinj + i0, cj);
        ld4(st.inode + (sabs & 1) * (long long)g.n_pad + i0, Ic);          // (A_i^T I_s(t + h))_i
        if (extrap) {
            double pp[4];
            ld4(vp + i0, pp);
#pragma unroll
            for (int j = 0; j < 4; ++j) vw[j] = warm_value(a[j], pp[j], th);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) vw[j] = a[j];
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            double bj = ch[j] * a[j] + cj[j] - Ic[j];
            const int i = i0 + j;
            if (g.n_l > 0)
            for (int q = __ldg(g.ind_ptr + i); q < __ldg(g.ind_ptr + i + 1); ++q) {
                const int lid = __ldg(g.ind_idx + q);
                const double il = st.il[(lid > 0 ? lid : -lid) - 1];
                bj -= lid > 0 ? il : -il;             // A_l^T i_l(t)
            }
            b[j] = bj;
        }
    }
    double sig[4];
    // explicit transient steps keep md = M (x0 - v(s-1)) (the outer passes add M delta)
    const bool track = rp.mode == kModeTransient && !three && st.md != nullptr;
    double mdv[4] = {0.0, 0.0, 0.0, 0.0};
    if (rp.mode == kModeSolve) {
        if (rp.x0) sell_row<1, double>(g, wc, sd, g.w64, s, lane, [&](int c) { return __ldg(rp.x0 + c); }, sig);
        else sig[0] = sig[1] = sig[2] = sig[3] = 0.0;
    } else if (three) {
        if (extrap) sell_row<1, double>(g, wc, sd, g.w64, s, lane, [&](int c) { return vl[c] - vp[c]; }, sig);
        else sig[0] = sig[1] = sig[2] = sig[3] = 0.0;
    } else if (inc) {
        // r = r_final(s-1) + increment - M (x0 - v(s-1)); md carries M (v(s-1) - v(s-2)), and
        // M (x0 - v(s-1)) is th times that
        double rp_[4];
        ld4(st.r64 + i0, rp_);
        if (extrap) {
            ld4(st.md + i0, mdv);
            if (th != 1.0) {
#pragma unroll
                for (int j = 0; j < 4; ++j) mdv[j] *= th;
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] += rp_[j] - mdv[j];
        sig[0] = sig[1] = sig[2] = sig[3] = 0.0;
    } else if (extrap) {
        sell_row<1, double>(g, wc, sd, g.w64, s, lane, [&](int c) { return warm_value(vl[c], vp[c], th); }, sig);
    } else {
        sell_row<1, double>(g, wc, sd, g.w64, s, lane, [&](int c) { return vl[c]; }, sig);
    }
    // a full step's md (M (x0 - v(s-1))) is written by md_slice before phase A; an
    // incremental step stores it here when it differs from the carried value
    if (track && inc && (!extrap || th != 1.0)) st4(st.md + i0, mdv);
    double r[4];
    MonT sc[4], mon = MonT(0);
    float r32[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        r[j] = inc ? b[j] : b[j] + sig[j] - D[j] * (vw[j] - base[j]);
        if constexpr (MIXED) {
            r32[j] = (float)r[j];
            sc[j] = scaled_upper(r32[j], iD[j]);      // an FP32 upper bound of |r| / D
        } else {
            sc[j] = fabs(r[j]) * iD[j];
        }
        mon = nanmax_t<MonT>(mon, sc[j]);
    }
    if (latR) {
        int Lid[4];
        ldg4(g.node_lat + i0, Lid);
        lattice_max(latR, Lid, sc, lacc);
    }
    st4(vbuf(st, vF) + i0, vw);
    st4(st.r64 + i0, r);
    if (MIXED && rp.lat_k > 0 && !g.natural) {
        // the lattice inner solve keeps its FP32 residual and correction in caller order
        float* dz = dbuf<float>(st, dsel);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = __ldg(g.orig + i0 + j);
            if (o >= 0) { st.r32[o] = r32[j]; dz[o] = 0.f; }
        }
    } else if (MIXED) {
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        st4(st.r32 + i0, r32);
        st4(dbuf<float>(st, dsel) + i0, z);
    } else {
        double z[4] = {0.0, 0.0, 0.0, 0.0};
        st4(dbuf<double>(st, dsel) + i0, z);
    }
    return (double)mon;
}

// One colour's SOR half-sweep on M delta = r (Eq. 16-17): returns max |unrelaxed update|.
template <typename T>
__device__ __forceinline__ double sweep_slice(const DevGrid& g, const WarpCache* wc, const SliceDesc& sd, const T* w,
                                              const T* invD, const T* r, T* d, int s, int lane, T omega) {
    const int i0 = s * kSlice + lane * kVec;
    T dv[4], rv[4], iD[4], sig[4];
    ld4(d + i0, dv);
    ld4(r + i0, rv);
    ldg4(invD + i0, iD);
    sell_row<kSweepUnroll, T>(g, wc, sd, w, s, lane, [&](int c) { return d[c]; }, sig);
    T mon = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T upd = (rv[j] + sig[j]) * iD[j] - dv[j];
        dv[j] = fma(omega, upd, dv[j]);
        mon = nanmax_t<T>(mon, fabs(upd));
    }
    st4(d + i0, dv);
    return (double)mon;
}

// One damped-Jacobi sweep over a slice: every node from the previous iterate
// (dold), written to dnew.  Returns max |unrelaxed update|.
template <typename T>
__device__ __forceinline__ double jacobi_slice(const DevGrid& g, const WarpCache* wc, const SliceDesc& sd, const T* w,
                                               const T* invD, const T* r, const T* dold, T* dnew, int s, int lane,
                                               T omega) {
    const int i0 = s * kSlice + lane * kVec;
    T dv[4], rv[4], iD[4], sig[4];
    ld4(dold + i0, dv);
    ld4(r + i0, rv);
    ldg4(invD + i0, iD);
    sell_row<kSweepUnroll, T>(g, wc, sd, w, s, lane, [&](int c) { return dold[c]; }, sig);
    T mon = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T upd = (rv[j] + sig[j]) * iD[j] - dv[j];
        dv[j] = fma(omega, upd, dv[j]);
        mon = nanmax_t<T>(mon, fabs(upd));
    }
    st4(dnew + i0, dv);
    return (double)mon;
}

// ---- TMA-fed sweep (FP32 path)
//
// The streaming operands of a slice (its K weight slots, its own corrections,
// residuals and 1/D: K + 3 contiguous 512-byte runs) are fetched by the
// Tensor Memory Accelerator with cp.async.bulk into a per-warp shared-memory
// stage, completion tracked by an mbarrier (transaction bytes).  Two stages
// per warp: slice t+1 is in flight while slice t is computed, so the warp no
// longer waits on its own streaming loads; only the neighbour gathers remain
// ordinary (L1-cached) loads.  Slices with more than kTmaK slots or explicit
// columns take the direct path.
constexpr int kTmaK = 8;
constexpr int kStageElems = (kTmaK + 3) * kSlice;

__host__ __device__ constexpr int tma_stage_bytes(int elem_size) { return kStageElems * elem_size; }
// per warp: two stages and two mbarriers (padded to keep stages 128-byte aligned)
__host__ __device__ constexpr int tma_warp_bytes(int elem_size) { return 2 * tma_stage_bytes(elem_size) + 128; }


__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// Generic-proxy writes (other blocks' and this warp's stores of the previous
// phases, ordered by the device barrier) become visible to the bulk copies.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Bounded wait on a stage's mbarrier phase; false after the time limit.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, long long timeout_ns) {
    long long t0 = 0;
    for (int it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (it == 256) t0 = global_ns();
        if (it > 256 && global_ns() - t0 > timeout_ns) return false;
    }
}

struct TmaWarp {
    unsigned char* stage[2];
    unsigned long long* bar;   // [2]
    unsigned parity;           // bit b: phase parity to wait for on stage b
};

template <typename T>
__device__ __forceinline__ void tma_issue(const SliceDesc& sd, int s, const T* w, const T* d, const T* r,
                                          const T* invD, T* buf, unsigned long long* bar) {
    const unsigned wb = (unsigned)(sd.K * kSlice * sizeof(T));
    const unsigned vb = (unsigned)(kSlice * sizeof(T));
    mbar_expect_tx(bar, wb + 3 * vb);
    bulk_g2s(buf, w + sd.off, wb, bar);
    bulk_g2s(buf + kTmaK * kSlice, d + (long long)s * kSlice, vb, bar);
    bulk_g2s(buf + (kTmaK + 1) * kSlice, r + (long long)s * kSlice, vb, bar);
    bulk_g2s(buf + (kTmaK + 2) * kSlice, invD + (long long)s * kSlice, vb, bar);
}

// One slice of the SOR half-sweep with its streaming operands already in shared memory.
template <typename T>
__device__ __forceinline__ double sweep_slice_staged(const DevGrid& g, const WarpCache* wc, const SliceDesc& sd,
                                                     const T* buf, T* d, int s, int lane, T omega) {
    const int i0 = s * kSlice + lane * kVec;
    T dv[4], rv[4], iD[4], sig[4];
    ld4(buf + kTmaK * kSlice + lane * kVec, dv);
    ld4(buf + (kTmaK + 1) * kSlice + lane * kVec, rv);
    ld4(buf + (kTmaK + 2) * kSlice + lane * kVec, iD);
    const int* offs = sd.dpos >= 0 ? wc->pool + sd.dpos : g.dia_off + (-2 - sd.dpos);
    sig[0] = sig[1] = sig[2] = sig[3] = T(0);
#pragma unroll kSweepUnroll
    for (int k = 0; k < sd.K; ++k) {
        T wv[4];
        ld4(buf + k * kSlice + lane * kVec, wv);
        const int o = offs[k];
#pragma unroll
        for (int j = 0; j < 4; ++j) sig[j] = fma(wv[j], d[i0 + j + o], sig[j]);
    }
    T mon = T(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const T upd = (rv[j] + sig[j]) * iD[j] - dv[j];
        dv[j] = fma(omega, upd, dv[j]);
        mon = nanmax_t<T>(mon, fabs(upd));
    }
    st4(d + i0, dv);
    return (double)mon;
}

// The warp's run of colour-c slices, double-buffered through the TMA.  Returns
// the max unrelaxed update, or NaN (after recording PG_ERR_TIMEOUT and letting
// its copies land) when a copy does not complete within the time limit.
template <typename T>
__device__ double sweep_colour_tma(const DevGrid& g, const WarpCache* wc, TmaWarp& tw, int c, const T* w,
                                   const T* invD, const T* r, T* d, int lane, T omega, int* err,
                                   long long timeout_ns) {
    const int cnt = wc->cnt[c], lo = wc->lo[c];
    if (cnt == 0) return 0.0;
    auto staged = [&](const SliceDesc& sd) { return sd.dpos != -1 && sd.K <= kTmaK; };
    SliceDesc cur = warp_desc(g, *wc, c, 0, lo);
    bool cur_t = staged(cur);
    if (lane == 0) {
        fence_proxy_async_global();
        if (cur_t) tma_issue<T>(cur, lo, w, d, r, invD, (T*)tw.stage[0], tw.bar + 0);
    }
    double mon = 0.0;
    unsigned pending = cur_t ? 1u : 0u;   // bit b: stage b has a copy in flight
    for (int t = 0; t < cnt; ++t) {
        const int sb = t & 1;
        SliceDesc nxt{};
        bool nxt_t = false;
        if (t + 1 < cnt) {
            nxt = warp_desc(g, *wc, c, t + 1, lo + t + 1);
            nxt_t = staged(nxt);
            if (nxt_t && lane == 0)
                tma_issue<T>(nxt, lo + t + 1, w, d, r, invD, (T*)(sb ? tw.stage[0] : tw.stage[1]), tw.bar + (sb ^ 1));
            if (nxt_t) pending |= 1u << (sb ^ 1);
        }
        if (cur_t) {
            const bool ok = mbar_wait(tw.bar + sb, (tw.parity >> sb) & 1u, timeout_ns);
            if (!ok) {
                if (lane == 0) atomicCAS(err, 0, (int)PG_ERR_TIMEOUT);
                // let every copy still in flight land before the stages are abandoned
                for (int b = 0; b < 2; ++b)
                    if ((pending >> b) & 1u) mbar_wait(tw.bar + b, (tw.parity >> b) & 1u, timeout_ns);
                __syncwarp();
                return __longlong_as_double(0x7ff8000000000000ll);
            }
            tw.parity ^= 1u << sb;
            pending &= ~(1u << sb);
            mon = nanmax(mon, sweep_slice_staged<T>(g, wc, cur, (const T*)(sb ? tw.stage[1] : tw.stage[0]), d, lo + t,
                                                    lane, omega));
        } else {
            mon = nanmax(mon, sweep_slice<T>(g, wc, cur, w, invD, r, d, lo + t, lane, omega));
        }
        __syncwarp();   // stage sb is read by every lane before it is refilled
        cur = nxt;
        cur_t = nxt_t;
    }
    return mon;
}

// ---- TMA-fed step start (incremental explicit step, FP32 inner solve)
//
// Phase A of an incremental step (RC, explicit form, mixed precision, corrections in
// the packing order) streams its operands: no neighbour is read.  The warp walks its
// nodes in chunks of kRhsChunk; the Tensor Memory Accelerator copies the contiguous
// operands of chunk j + 1 (v(s-1), v(s-2), C/h, the load change, the carried residual
// and M (v(s-1) - v(s-2)) in FP64, 1/D in FP32) into one stage of the warp's TMA area
// while chunk j is computed from the other, so the FP64 arithmetic of one chunk
// overlaps the memory traffic of the next.  Each node takes exactly the operations of
// phase_rhs's incremental branch, with the load change Ic - Ip read as formed when the
// load slot was written (the same two operands), so the results are bit-identical.
constexpr int kRhsChunk = 64;
constexpr int kRhsArrays = 6;                                   // FP64 operands per node
constexpr int kRhsStageBytes = kRhsChunk * (8 * kRhsArrays + 4);
static_assert(kRhsStageBytes <= kStageElems * 4, "a step-start chunk fits one TMA stage");

__device__ __forceinline__ double phase_rhs_inc_tma(const DevGrid& g, const WarpCache* wc, TmaWarp& tw,
                                                    const DevState& st, int lane, int vL, int vP, int vF,
                                                    bool extrap, long long sabs, int dsel, float th, int* err,
                                                    long long timeout_ns) {
    const double* vl = vbuf(st, vL);
    const double* vp = vbuf(st, vP);
    double* vf = vbuf(st, vF);
    float* dz = dbuf<float>(st, dsel);
    constexpr unsigned kB8 = kRhsChunk * 8, kB4 = kRhsChunk * 4;
    const unsigned bytes = kB8 * (extrap ? 6u : 5u) + kB4;
    auto issue = [&](long long n0, int sb) {
        unsigned char* buf = sb ? tw.stage[1] : tw.stage[0];   // no dynamic index: tw stays in registers
        unsigned long long* bar = tw.bar + sb;
        mbar_expect_tx(bar, bytes);
        bulk_g2s(buf + 0 * kB8, vl + n0, kB8, bar);
        bulk_g2s(buf + 1 * kB8, vp + n0, kB8, bar);
        bulk_g2s(buf + 2 * kB8, g.ch + n0, kB8, bar);
        bulk_g2s(buf + 3 * kB8, st.dinode + n0, kB8, bar);
        bulk_g2s(buf + 4 * kB8, st.r64 + n0, kB8, bar);
        if (extrap) bulk_g2s(buf + 5 * kB8, st.md + n0, kB8, bar);
        bulk_g2s(buf + 6 * kB8, g.invD32 + n0, kB4, bar);
    };
    float mon = 0.f;
    for (int c = 0; c < g.ncol; ++c) {
        const int cnt = wc->cnt[c];
        if (cnt == 0) continue;
        const long long node0 = (long long)wc->lo[c] * kSlice;
        const int n = cnt * (kSlice / kRhsChunk);
        if (lane == 0) {
            fence_proxy_async_global();
            issue(node0, 0);
        }
        unsigned pending = 1u;
        for (int j = 0; j < n; ++j) {
            const int sb = j & 1;
            if (j + 1 < n) {
                if (lane == 0) issue(node0 + (long long)(j + 1) * kRhsChunk, sb ^ 1);
                pending |= 1u << (sb ^ 1);
            }
            if (!mbar_wait(tw.bar + sb, (tw.parity >> sb) & 1u, timeout_ns)) {
                if (lane == 0) atomicCAS(err, 0, (int)PG_ERR_TIMEOUT);
                for (int b = 0; b < 2; ++b)   // let every copy still in flight land
                    if ((pending >> b) & 1u) mbar_wait(tw.bar + b, (tw.parity >> b) & 1u, timeout_ns);
                __syncwarp();
                return __longlong_as_double(0x7ff8000000000000ll);
            }
            tw.parity ^= 1u << sb;
            pending &= ~(1u << sb);
            const unsigned char* buf = sb ? tw.stage[1] : tw.stage[0];
            const int q = 2 * lane;                               // this lane's two nodes of the chunk
            const long long i = node0 + (long long)j * kRhsChunk + q;
            const double2 a = *reinterpret_cast<const double2*>(buf + 0 * kB8 + q * 8);
            const double2 pp = *reinterpret_cast<const double2*>(buf + 1 * kB8 + q * 8);
            const double2 ch = *reinterpret_cast<const double2*>(buf + 2 * kB8 + q * 8);
            const double2 di = *reinterpret_cast<const double2*>(buf + 3 * kB8 + q * 8);
            const double2 rr = *reinterpret_cast<const double2*>(buf + 4 * kB8 + q * 8);
            double2 md = make_double2(0.0, 0.0);
            if (extrap) md = *reinterpret_cast<const double2*>(buf + 5 * kB8 + q * 8);
            const float2 iD = *reinterpret_cast<const float2*>(buf + 6 * kB8 + q * 4);
            if (extrap && th != 1.0f) {
                md.x *= th;
                md.y *= th;
            }
            // the incremental branch of phase_rhs, node by node
            auto node = [&](double av, double pv, double cv, double div, double rv, double mdv, float iv, double& vw,
                            double& r, float& r32) {
                vw = extrap ? warm_value(av, pv, th) : av;
                double bj = cv * (av - pv) - div;              // div = Ic - Ip, formed when slot S was written
                bj += rv - mdv;
                r = bj;
                r32 = (float)r;
                mon = nanmax_t<float>(mon, scaled_upper(r32, iv));
            };
            double vw0, vw1, r0, r1;
            float r320, r321;
            node(a.x, pp.x, ch.x, di.x, rr.x, md.x, iD.x, vw0, r0, r320);
            node(a.y, pp.y, ch.y, di.y, rr.y, md.y, iD.y, vw1, r1, r321);
            __syncwarp();   // stage sb is read by every lane before it is refilled
            if (!extrap || th != 1.0f) *reinterpret_cast<double2*>(st.md + i) = md;
            *reinterpret_cast<double2*>(vf + i) = make_double2(vw0, vw1);
            *reinterpret_cast<double2*>(st.r64 + i) = make_double2(r0, r1);
            *reinterpret_cast<float2*>(st.r32 + i) = make_float2(r320, r321);
            *reinterpret_cast<float2*>(dz + i) = make_float2(0.f, 0.f);
        }
    }
    return (double)mon;
}

// ---- lattice inner solve (FP32, ghost zones, column blocks)
//
// For a lattice grid (nodes (x, y, l), branches only between lattice
// neighbours) the inner relaxation is block red-black SOR whose blocks are the
// columns (x, y, all l): a column is coloured by the parity of x + y, and its
// update solves the column's tridiagonal block exactly (Thomas factors
// precomputed per h) against the in-plane neighbours of the other colour.
// Gauss-Seidel / SOR over any block partition of an SPD matrix converges for
// 0 < omega < 2 (Theorem 1's argument, with the Ostrowski-Reich theorem for
// blocks), and taking the stiff via couplings into the blocks shrinks the
// spectral radius that the in-plane sweep has to overcome.  With one layer a
// block is a node and this is the point red-black SOR of Eq. 16-17.
//
// The relaxation runs on regions of kLatSide x kLatSide = 34 x 34 columns of all
// layers held in shared memory: a tile of T^2 columns, T = 34 - 2H, plus a ghost
// zone of H = 2k columns, and k exact sweeps (2k half-sweeps) are applied to the
// region: half-sweep j (1-based) updates the columns at distance >= j from the
// region edge, after which every such column holds the exact value (it reads
// only neighbours at distance >= j - 1, updated by every earlier half-sweep), so
// the tile interior (distance >= 2k) equals k global block sweeps.  Tiles read the previous round's corrections
// and write the next buffer: one device barrier per k sweeps, every branch
// weight stored once (E, N, U per node).
//
// The width 34 makes the columns of the first half-sweep (distance >= 1) exactly 32
// wide, 16 column pairs per half-warp row; a region has ROWS = 34 or 66 rows (32 or 64
// of them in the first half-sweep: two or four rows per thread).  A region starts at an
// even column (T and H are even); its rows are staged from the 16-byte boundary at or
// below that column (a lead of 0 or 2 columns), so that on lattices whose width is a
// multiple of 4 every row copies in aligned 16-byte pieces.  Shared-memory rows hold
// kLatW = 36 floats, which keeps the two half-warps (adjacent rows, opposite colours) on
// disjoint banks; each staged array holds lat_astride floats (the grid's largest layer
// count times ROWS rows).
static_assert(kLatSide - 2 == 32, "the first half-sweep covers 32 columns, 16 pairs per half-warp row");

// One tile (region of lattice L): load, 2k half-sweeps, store the interior.
// Returns the max unrelaxed column update of the last sweep over the interior.
// NL (layers) is a template parameter: the column solve unrolls completely.
// V: float (the mixed-precision inner solve on the correction) or double (the FP64 one;
// every staged array in FP64, twice the shared memory).
template <int NL, int ROWS, typename V>
__device__ V lattice_tile(const DevGrid& g, int off, int nx, int ny, int tile, const V* __restrict__ dold,
                          V* __restrict__ dnew, const V* __restrict__ r, V omega, int k, unsigned char* smem) {
    constexpr int kLatPlane = ROWS * kLatW;           // elements per layer of a staged array
    constexpr int J = (ROWS - 2) / 16;                // rows per thread in a half-sweep
    constexpr int kEl = 16 / (int)sizeof(V);          // elements per 16-byte piece
    static_assert(ROWS == 34 || ROWS == 66, "regions of 34 or 66 rows");
    const int H = 2 * k, T = kLatSide - 2 * H, TY = ROWS - 2 * H;
    const int tiles_x = (nx + T - 1) / T;
    const int A = g.lat_astride;                      // elements per array
    V* sd = reinterpret_cast<V*>(smem);
    V* sr = sd + A;
    V* se = sd + 2 * A;
    V* sn = sd + 3 * A;
    V* su = sd + 4 * A;
    V* sm = sd + 5 * A;
    V* sp = sd + 6 * A;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int pair = lane & 15;                        // columns 2 pair, 2 pair + 1 of the slot grid
    const int rsub = lane >> 4;                        // half-warps take adjacent rows (no bank conflicts)
    const long long plane = (long long)nx * ny;
    // region: columns [x0, x0 + 34), rows [y0, y0 + 34); shared column c holds x0 - lead + c
    const int x0 = (tile % tiles_x) * T - H, y0 = (tile / tiles_x) * TY - H;
    const int lead = x0 & (kEl - 1);                   // FP32: 0 or 2 (x0 is even); FP64: 0
    const int xa = x0 - lead;
    auto src_of = [&](int arr) -> const V* {           // by value: no local array
        if constexpr (sizeof(V) == 8)
            return arr == 0 ? dold : arr == 1 ? r : arr == 2 ? g.lwE64 : arr == 3 ? g.lwN64 : arr == 4 ? g.lwU64
                 : arr == 5 ? g.lm64 : g.lip64;
        else
            return arr == 0 ? dold : arr == 1 ? r : arr == 2 ? g.lwE : arr == 3 ? g.lwN : arr == 4 ? g.lwU
                 : arr == 5 ? g.lm : g.lip;
    };
    if ((nx & (kEl - 1)) == 0 && (off & (kEl - 1)) == 0) {
        // rows of 16-byte pieces: a piece (xa + kEl c, ...) is wholly inside the lattice or
        // wholly outside; the (piece, array) pairs are spread over the threads
        constexpr int kChunks = kLatW / kEl;
        constexpr int kPieces = ROWS * kChunks;
        for (int q = threadIdx.x; q < kPieces * kLatArrays; q += blockDim.x) {
            const int arr = q / kPieces, pos = q - arr * kPieces;
            const int ry = pos / kChunks, c4 = kEl * (pos - ry * kChunks);
            const int xx = xa + c4, yy = y0 + ry;
            const bool in = yy >= 0 && yy < ny && xx >= 0 && xx < nx;
            const long long o = in ? off + (long long)yy * nx + xx : 0;
            const V* src = src_of(arr);
            V* dst = sd + arr * A + ry * kLatW + c4;
#pragma unroll
            for (int l = 0; l < NL; ++l)
                cp_async16(dst + l * kLatPlane, src + (in ? o + l * plane : 0), in ? 16u : 0u);
        }
    } else {
        for (int q = threadIdx.x; q < kLatPlane; q += blockDim.x) {
            const int ry = q / kLatW, c = q - ry * kLatW;
            const int xx = xa + c, yy = y0 + ry;
            const bool in = yy >= 0 && yy < ny && xx >= 0 && xx < nx;
            const long long o = in ? off + (long long)yy * nx + xx : 0;
#pragma unroll
            for (int arr = 0; arr < kLatArrays; ++arr)
#pragma unroll
                for (int l = 0; l < NL; ++l)
                    cp_async_elem<V>(sd + arr * A + l * kLatPlane + q, src_of(arr) + (in ? o + l * plane : 0), in);
        }
    }
    cp_async_wait_all();
    __syncthreads();
    V mon = V(0);
    for (int hs = 0; hs < 2 * k; ++hs) {
        const bool last = hs >= 2 * k - 2;
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int ry = 1 + 2 * (warp + 8 * j) + rsub, y = y0 + ry;
            const int cx = 1 + 2 * pair + ((hs + x0 + 1 + y) & 1);   // the column of this colour in the pair
            const int x = x0 + cx;
            const int edge = min(min(cx, ry), min(kLatSide - 1 - cx, ROWS - 1 - ry));
            // half-sweep hs only matters at distance > hs from the region edge: what it
            // would change nearer the edge cannot reach the interior by the last one
            if (edge <= hs || x < 0 || x >= nx || y < 0 || y >= ny) continue;
            const int a0 = ry * kLatW + cx + lead;
            V f[NL], xv[NL];
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const int a = a0 + l * kLatPlane;
                f[l] = sr[a] + se[a] * sd[a + 1] + se[a - 1] * sd[a - 1] + sn[a] * sd[a + kLatW] +
                       sn[a - kLatW] * sd[a - kLatW];
            }
#pragma unroll
            for (int l = 1; l < NL; ++l) f[l] = fma(sm[a0 + l * kLatPlane], f[l - 1], f[l]);
            xv[NL - 1] = f[NL - 1] * sp[a0 + (NL - 1) * kLatPlane];
#pragma unroll
            for (int l = NL - 2; l >= 0; --l)
                xv[l] = fma(su[a0 + l * kLatPlane], xv[l + 1], f[l]) * sp[a0 + l * kLatPlane];
            const bool interior = edge >= H;
#pragma unroll
            for (int l = 0; l < NL; ++l) {
                const int a = a0 + l * kLatPlane;
                const V dv = sd[a];
                const V upd = xv[l] - dv;
                sd[a] = fma(omega, upd, dv);
                if (last && interior) mon = nanmax_t<V>(mon, fabs(upd));
            }
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < T * TY; q += blockDim.x) {
        const int iy = q / T, ix = q - iy * T;
        const int x = x0 + H + ix, y = y0 + H + iy;
        if (x >= nx || y >= ny) continue;
        const long long b = off + (long long)y * nx + x;
        const int a = (H + iy) * kLatW + H + ix + lead;
#pragma unroll
        for (int l = 0; l < NL; ++l) dnew[b + l * plane] = sd[l * kLatPlane + a];
    }
    __syncthreads();   // the next tile overwrites the region
    return mon;
}

// One round over the tiles of every lattice whose residual (latest FP64 pass,
// slots `latR`) is still above the step's target.  The lattices are independent
// sub-circuits (Fig. 1), so a converged one keeps its solution: its correction
// must stay zero in both buffers, which the start buffer is (zeroed by the FP64
// pass) and which the first round of the inner solve (`first`) writes into the
// other one; later rounds skip those tiles entirely.
template <int ROWS, typename V>
__device__ double lattice_round(const DevGrid& g, const V* dold, V* dnew, const V* r, V omega,
                                int k, unsigned char* smem, const unsigned long long* latR, double target,
                                bool first, unsigned* tile_ctr, unsigned round_base) {
    // Tiles are handed out from a launch-wide counter, so a block that finishes early takes
    // the next one: the round ends one tile after the last block starts its final tile,
    // whatever the spread of tile times.  Each block claims its next tile while it works on
    // the current one and stops at its first claim past the round's T tiles, so a round
    // takes exactly T + gridDim.x claims: round n owns the counter values from
    // round_base = n (T + gridDim.x) on, modulo 2^32 like the counter itself (the index
    // claim - round_base is exact while one round takes fewer than 2^32 claims).  Any
    // assignment gives the same result: a tile reads only the previous round's corrections
    // and writes only its own interior.
    __shared__ int s_tile;
    const unsigned T = (unsigned)g.lat_tiles;
    unsigned claim = 0;
    if (threadIdx.x == 0) claim = atomicAdd(tile_ctr, 1u);
    V mon = V(0);
    for (;;) {
        if (threadIdx.x == 0) {
            const unsigned t = claim - round_base;
            s_tile = t < T ? (int)t : -1;
            if (t < T) claim = atomicAdd(tile_ctr, 1u);        // the next one, in flight meanwhile
        }
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t < 0) break;
        int lo = 0, hi = g.n_lats;                      // lattice with lat_tile0[L] <= t < lat_tile0[L+1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(g.lat_tile0 + mid) <= t) lo = mid; else hi = mid;
        }
        const int L = lo;
        const int off = __ldg(g.lat_info + 4 * L), nx = __ldg(g.lat_info + 4 * L + 1),
                  ny = __ldg(g.lat_info + 4 * L + 2), nl = __ldg(g.lat_info + 4 * L + 3);
        const int tile = t - __ldg(g.lat_tile0 + L);
        if (latR && __longlong_as_double((long long)latR[L]) <= target) {
            // converged lattice (uniform across the block: no barrier divergence)
            if (first) {
                const int H = 2 * k, T = kLatSide - 2 * H, TY = ROWS - 2 * H, tiles_x = (nx + T - 1) / T;
                const int tx0 = (tile % tiles_x) * T, ty0 = (tile / tiles_x) * TY;
                const long long plane = (long long)nx * ny;
                for (int q = threadIdx.x; q < T * TY; q += blockDim.x) {
                    const int x = tx0 + q % T, y = ty0 + q / T;
                    if (x >= nx || y >= ny) continue;
                    for (int l = 0; l < nl; ++l) dnew[off + l * plane + (long long)y * nx + x] = V(0);
                }
            }
            continue;
        }
        V m;
        if (nl == 1) m = lattice_tile<1, ROWS, V>(g, off, nx, ny, tile, dold, dnew, r, omega, k, smem);
        else if (nl == 2) m = lattice_tile<2, ROWS, V>(g, off, nx, ny, tile, dold, dnew, r, omega, k, smem);
        else m = lattice_tile<3, ROWS, V>(g, off, nx, ny, tile, dold, dnew, r, omega, k, smem);
        mon = nanmax_t<V>(mon, m);
    }
    return (double)mon;
}

// Outer defect-correction pass: v += delta, r -= M delta (FP64), refresh the FP32 residual.
template <typename T>
__device__ __forceinline__ double outer_slice(const DevGrid& g, const WarpCache* wc, const SliceDesc& sd,
                                              const DevState& st, const T* d, T* dnext, float* r32, int s, int lane,
                                              double* v, bool lat, unsigned long long* latR, LatAccT<T>& lacc,
                                              double* md) {
    // T = float (mixed precision): the monitored max |r| / D is an FP32 upper bound from the
    // FP32 residual copy this pass writes anyway (scaled_upper); T = double: exact FP64
    const int i0 = s * kSlice + lane * kVec;
    T dv[4];
    if (lat) {
        // correction in caller order (lattice inner solve); padding has none
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = __ldg(g.orig + i0 + j);
            dv[j] = o >= 0 ? d[o] : T(0);
        }
    } else {
        ld4(d + i0, dv);
    }
    double r[4], vv[4];
    T iD[4];
    if constexpr (std::is_same<T, float>::value) ldg4(g.invD32 + i0, iD);
    else ldg4(g.invD64 + i0, iD);
    ld4(st.r64 + i0, r);
    ld4(v + i0, vv);
    double Md[4];                                      // (M delta)_i
    if constexpr (std::is_same<T, float>::value) {
        // FP32 correction: M delta as a double-float, minus the neighbour sum, then one
        // FP64 update of r (its error is far below the stopping rule's rounding slack)
        float hi[4], lo[4], dh[4], dl[4];
        if (lat) {
            sell_row_df(g, wc, sd, s, lane, [&](int c) {
                const int o = __ldg(g.orig + c);
                return o >= 0 ? d[o] : 0.f;
            }, hi, lo);
        } else {
            sell_row_df(g, wc, sd, s, lane, [&](int c) { return d[c]; }, hi, lo);
        }
        ldg4(g.D32 + i0, dh);
        ldg4(g.D32lo + i0, dl);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float ph = 0.f, pl = 0.f;
            df_acc(ph, pl, dh[j], dl[j], dv[j]);           // D delta
            // (ph + pl) - (hi + lo): ph - hi = sd + ed exactly (TwoSum), the rest in FP32, so
            // that only two values cross to FP64 (GB300 issues FP64 and conversions slowly)
            const float sd = __fsub_rn(ph, hi[j]);
            const float bd = __fsub_rn(sd, ph);
            const float ed = __fadd_rn(__fsub_rn(ph, __fsub_rn(sd, bd)), __fsub_rn(-hi[j], bd));
            Md[j] = (double)sd + (double)(ed + (pl - lo[j]));
        }
    } else {
        double D[4], sig[4];
        ldg4(g.D64 + i0, D);
        sell_row<1, double>(g, wc, sd, g.w64, s, lane, [&](int c) { return (double)d[c]; }, sig);
#pragma unroll
        for (int j = 0; j < 4; ++j) Md[j] = D[j] * (double)dv[j] - sig[j];
    }
    if (md) {
        double m4[4];
        ld4(md + i0, m4);
#pragma unroll
        for (int j = 0; j < 4; ++j) m4[j] += Md[j];
        st4(md + i0, m4);
    }
    T mon = T(0), sc[4];
    float f[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        r[j] -= Md[j];
        vv[j] += (double)dv[j];
        f[j] = (float)r[j];
        if constexpr (std::is_same<T, float>::value) sc[j] = scaled_upper(f[j], iD[j]);
        else sc[j] = fabs(r[j]) * iD[j];
        mon = nanmax_t<T>(mon, sc[j]);
    }
    if (latR) {
        int Lid[4];
        ldg4(g.node_lat + i0, Lid);
        lattice_max(latR, Lid, sc, lacc);
    }
    st4(st.r64 + i0, r);
    st4(v + i0, vv);
    if (lat) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int o = __ldg(g.orig + i0 + j);
            if (o >= 0) { dnext[o] = T(0); r32[o] = f[j]; }
        }
    } else {
        T z[4] = {T(0), T(0), T(0), T(0)};
        st4(dnext + i0, z);
        if (r32) st4(r32 + i0, f);
    }
    return (double)mon;
}

}  // namespace

// ---------------------------------------------------------------- the persistent kernel

// ROWS: region rows of the lattice inner solve (34, or 66 for tall regions; mixed precision only).
template <bool MIXED, int ROWS>
__global__ void __launch_bounds__(256, PG_MIN_BLOCKS) persistent_kernel(DevGrid g, DevState st, DevCtl ctl, RunParams rp) {
    using T = typename std::conditional<MIXED, float, double>::type;
    const unsigned nblocks = gridDim.x;
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    const int gtid = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    const int nthreads = (int)(gridDim.x * blockDim.x);
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const T omega = (T)rp.omega;
    __shared__ WarpCache s_cache[kWarpsPerBlock];
    WarpCache* wc = &s_cache[threadIdx.x >> 5];
    fill_warp_cache(g, *wc, gwarp, nwarps);
    // TMA stages (mixed precision only; the launch passes the dynamic shared memory)
    extern __shared__ __align__(128) unsigned char s_dyn[];
    TmaWarp tw{};
    if (MIXED) {
        unsigned char* base = s_dyn + (threadIdx.x >> 5) * tma_warp_bytes(sizeof(float));
        tw.stage[0] = base;
        tw.stage[1] = base + tma_stage_bytes(sizeof(float));
        tw.bar = reinterpret_cast<unsigned long long*>(base + 2 * tma_stage_bytes(sizeof(float)));
        tw.parity = 0;
        if (lane == 0 && rp.lat_k == 0) {      // the lattice solve reuses this memory instead
            mbar_init(tw.bar + 0, 1);
            mbar_init(tw.bar + 1, 1);
            fence_proxy_async_smem();
        }
        __syncwarp();
    }

    // Reduction slots rotate over 4 barrier-delimited phases: phase k merges into
    // slot k%4 and, at its start, clears slot (k+2)%4, whose last readers all
    // passed barrier k-1 (the host clears all four before the launch).
    int phase = 0;
    bool first_bar = true;
    auto barrier = [&](bool want_val, double v) -> BarrierResult {
        const bool skip = first_bar && (rp.debug_flags & PG_DEBUG_SKIP_ARRIVAL) && blockIdx.x == 0;
        first_bar = false;
        const BarrierResult r = grid_barrier(ctl, nblocks, (unsigned)(phase + 1), rp.timeout_ns, skip, v,
                                             want_val ? ctl.red + (phase & 3) : nullptr);
        ++phase;
        if (lead) ctl.red[(phase + 2) & 3] = 0ull;
        return r;
    };

    // statistics (kept by every thread identically; block 0 thread 0 publishes)
    long long tot_sweeps = 0, tot_outer = 0, steps_done = 0;
    int max_sw = 0, max_out = 0;
    double max_bound_R = 0.0, last_R = 0.0;
    int last_outer = rp.prev_outer;   // outer passes of the previous step (same in every block)
    // time per phase, read by block 0 right after the barriers that end the phases
    double t_phase[4] = {0.0, 0.0, 0.0, 0.0};
    long long t_mark = lead ? global_ns() : 0ll;
    auto lap = [&](int k) {
        if (lead) {
            const long long t_now = global_ns();
            t_phase[k] += (double)(t_now - t_mark);
            t_mark = t_now;
        }
    };
    auto publish = [&](long long failed) {
        if (lead) {
            ctl.stats[kStatTimeA] = t_phase[0];
            ctl.stats[kStatTimeInner] = t_phase[1];
            ctl.stats[kStatTimeOuter] = t_phase[2];
            ctl.stats[kStatTimePost] = t_phase[3];
            ctl.stats[kStatSteps] = (double)steps_done;
            ctl.stats[kStatSweeps] = (double)tot_sweeps;
            ctl.stats[kStatMaxSweeps] = (double)max_sw;
            ctl.stats[kStatOuter] = (double)tot_outer;
            ctl.stats[kStatMaxOuter] = (double)max_out;
            ctl.stats[kStatMaxBound] = max_bound_R;
            ctl.stats[kStatFailedStep] = (double)failed;
            ctl.stats[kStatLastR] = last_R;
            ctl.stats[kStatLastOuter] = (double)last_outer;
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

    // per-component minima: order keys, all rows set to the largest key before the first
    // barrier; row s receives atomics in step s's post phase and is turned into volts
    // after the barrier that ends step s
    unsigned long long* const comp_key = reinterpret_cast<unsigned long long*>(rp.comp_vmin);
    if (comp_key)
        for (long long q = gtid; q < (long long)rp.nsteps * g.n_comp; q += nthreads) comp_key[q] = ~0ull;
    auto finalize_comp = [&](int sl) {
        if (comp_key)
            for (int q = gtid; q < g.n_comp; q += nthreads) {
                const long long e = (long long)sl * g.n_comp + q;
                rp.comp_vmin[e] = key_value(comp_key[e]);
            }
    };

    const double target = rp.target_scale ? rp.target * __longlong_as_double((long long)*rp.target_scale) : rp.target;
    int vL = rp.cur, vP = rp.prev, vF = 3 - rp.cur - rp.prev;
    bool have_prev = rp.have_prev != 0;
    unsigned lat_rounds = 0;     // lattice rounds run in this launch (the same in every block), modulo 2^32
    // per-lattice residual maxima (lattice inner solve): two buffers, `lat_par` is the one
    // the latest FP64 pass wrote; the host clears both before the launch
    const bool per_lat = rp.lat_k > 0 && ctl.lat_R != nullptr && g.n_lats > 1;   // one lattice: R says it all
    int lat_par = 0;
    auto lat_buf = [&](int b) { return per_lat ? ctl.lat_R + (size_t)b * g.n_lats : nullptr; };
    auto lat_clear = [&](int b) {
        if (per_lat && blockIdx.x == 0)
            for (int q = threadIdx.x; q < g.n_lats; q += blockDim.x) ctl.lat_R[(size_t)b * g.n_lats + q] = 0ull;
    };

    // Load currents of step S into the per-node slot S & 1: (A_i^T I_s(S h))_i, the current
    // drawn from node i by its loads (phase A of step S reads slot S & 1, and slot (S - 1) & 1
    // in the incremental and three-level forms).  A node with one load is written by its
    // source's thread, a node with several by a thread of its own that sums them in CSR order;
    // nodes without loads keep 0.  Each node is always written by the same thread.
    // With the load-aware warm start, word S & 3 of ctl.ld_flags records whether any node's
    // load current changed between (S - 1) h and S h (compared with the other slot, written by
    // the same thread), set at launch for the first two steps as in every post phase, so a run
    // split over launches takes the same decisions.
    const bool damp = rp.mode == kModeTransient && rp.warm_extrap && !rp.three_level &&
                      rp.warm_theta_static < 1.0 && ctl.ld_flags != nullptr;
    auto eval_sources = [&](long long S, bool flag) {
        double* dst = st.inode + (S & 1) * (long long)g.n_pad;
        const double* prev = st.inode + ((S - 1) & 1) * (long long)g.n_pad;
        const double tS = (double)S * rp.h;
        const unsigned long long tk = order_key(tS);
        bool changed = false;
        // kQ sources per thread at once, so their load chains overlap; each starts from the
        // segment of its previous evaluation (time moves forward, so that segment, or the
        // holds before the first and after the last breakpoint, almost always holds t)
        constexpr int kQ = 2;
        for (int e0 = gtid; e0 < g.n_src; e0 += kQ * nthreads) {
            int a[kQ], b[kQ];
            int lo[kQ], hi[kQ], j[kQ];          // breakpoint indices (the host keeps them below 2^31)
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const int e = e0 + q * nthreads;
                const bool ok = e < g.n_src;
                a[q] = ok ? __ldg(g.src_na + e) : -1;
                b[q] = ok ? __ldg(g.src_nb + e) : -1;
                lo[q] = ok ? (int)__ldg(g.pwl_ptr + e) : 0;
                hi[q] = ok ? (int)__ldg(g.pwl_ptr + e + 1) - 1 : 0;
                j[q] = ok ? st.pwl_cur[e] : 0;
            }
            double I[kQ];
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                const int jj = min(max(j[q], lo[q]), hi[q]);
                const int j1 = min(jj + 1, hi[q]);
                const unsigned long long k0 = __ldg(g.pwl_tk + jj), k1 = __ldg(g.pwl_tk + j1);
                const double s0 = __ldg(g.pwl_s + jj), t0 = __ldg(g.pwl_t + jj), v0 = __ldg(g.pwl_v + jj);
                if (jj < hi[q] && k0 < tk && tk <= k1) I[q] = fma(s0, tS - t0, v0);
                else if ((jj == hi[q] && tk > k0) || (jj == lo[q] && tk <= k0)) I[q] = v0;
                else {
                    int64_t jn;
                    I[q] = pwl_eval_search(g, lo[q], hi[q], tS, tk, jn);
                    const int e = e0 + q * nthreads;
                    if (e < g.n_src) st.pwl_cur[e] = (int32_t)jn;
                }
            }
#pragma unroll
            for (int q = 0; q < kQ; ++q) {
                if (a[q] >= 0) {
                    const double p = prev[a[q]];
                    if (flag) changed |= I[q] != p;
                    dst[a[q]] = I[q];
                    st.dinode[a[q]] = I[q] - p;
                }
                if (b[q] >= 0) {
                    const double p = prev[b[q]];
                    if (flag) changed |= -I[q] != p;
                    dst[b[q]] = -I[q];
                    st.dinode[b[q]] = -I[q] - p;
                }
            }
        }
        for (int k = gtid; k < g.n_multi; k += nthreads) {
            const int i = __ldg(g.multi_node + k);
            double sum = 0.0;
            for (int q = __ldg(g.ld_ptr + i); q < __ldg(g.ld_ptr + i + 1); ++q) {
                const int sid = __ldg(g.ld_idx + q);
                const double I = pwl_eval(g, (sid > 0 ? sid : -sid) - 1, tS, tk);
                sum += sid > 0 ? I : -I;
            }
            const double p = prev[i];
            if (flag) changed |= sum != p;
            dst[i] = sum;
            st.dinode[i] = sum - p;
        }
        if (flag && __any_sync(kFull, changed) && lane == 0) atomicOr(ctl.ld_flags + (S & 3), 1u);
    };
    if (rp.mode == kModeTransient && (g.n_src > 0 || damp) && rp.nsteps > 0) {
        const long long S0 = rp.step0;
        if (damp) {                      // with no sources every interval stays static (0)
            if (gtid == 0) {
                ctl.ld_flags[S0 & 3] = 0u;
                ctl.ld_flags[(S0 + 1) & 3] = 0u;
                ctl.ld_flags[(S0 + 2) & 3] = 0u;
            }
            if (g.n_src > 0) eval_sources(S0 - 1, false);
            if (!barrier(false, 0.0).ok) { publish(-1); return; }
            if (g.n_src > 0) {
                eval_sources(S0, true);
                eval_sources(S0 + 1, true);
            }
        } else if (g.n_src > 0) {
            if (rp.three_level || rp.inc_start) eval_sources(S0, false);   // I(t) - I(t - h)
            eval_sources(S0 + 1, false);
        }
        if (!barrier(false, 0.0).ok) { publish(-1); return; }
    }

    for (int sl = 0; sl < rp.nsteps; ++sl) {
        const long long sabs = rp.step0 + sl + 1;
        const bool extrap = rp.mode == kModeTransient && rp.warm_extrap && have_prev;
        // extrapolation weight: damped once no load changed over the last two intervals
        float th = 1.0f;
        if (damp && extrap) {
            const volatile unsigned* f = ctl.ld_flags;
            if (f[sabs & 3] == 0u && f[(sabs - 1) & 3] == 0u) th = (float)rp.warm_theta_static;
        }
        // Eq. 11 needs two levels; a step from a single level is an ordinary backward-Euler step
        const bool three = rp.mode == kModeTransient && rp.three_level && have_prev;
        // explicit form: the step start adds the increment to the previous final residual
        // except every kIncPeriod-th step (by absolute index, so chunked runs repeat a single
        // launch exactly), which recomputes it (bounds the drift of rounding)
        const bool inc = rp.mode == kModeTransient && !rp.three_level && have_prev && st.md != nullptr &&
                         (sl > 0 || rp.inc_start) && (sabs % kIncPeriod) != 0 && last_outer <= kIncMaxOuter;
        int dsel = 0;
        if (sl > 0) { finalize_vmin(sl - 1); finalize_comp(sl - 1); }

        // ---- phase A: RHS + warm start + residual, all colours
        double mon = 0.0;
        if (rp.mode == kModeTransient && !three && !inc && st.md != nullptr) {
            const double* vlp = vbuf(st, vL);
            const double* vpp = vbuf(st, vP);
            for (int c = 0; c < g.ncol; ++c)
                for (int tt = 0; tt < wc->cnt[c]; ++tt) {
                    const int s = wc->lo[c] + tt;
                    md_slice(g, wc, warp_desc(g, *wc, c, tt, s), st, s, lane, vlp, vpp, extrap, th);
                }
        }
        // the incremental explicit RC step streams its operands through the TMA
        const bool staged_rhs = MIXED && inc && !three && rp.mode == kModeTransient && g.n_l == 0 && !per_lat &&
                                !(rp.lat_k > 0 && !g.natural);
        if (staged_rhs) {
            if (rp.lat_k > 0) {
                // the lattice tiles use this shared memory between step starts: fresh barriers
                if (lane == 0) {
                    fence_proxy_async_smem();
                    mbar_init(tw.bar + 0, 1);
                    mbar_init(tw.bar + 1, 1);
                    fence_proxy_async_smem();
                }
                tw.parity = 0;
                __syncwarp();
            }
            mon = phase_rhs_inc_tma(g, wc, tw, st, lane, vL, vP, vF, extrap, sabs, dsel, th, ctl.err, rp.timeout_ns);
            if (rp.lat_k > 0) {
                __syncwarp();
                if (lane == 0) {
                    mbar_inval(tw.bar + 0);
                    mbar_inval(tw.bar + 1);
                }
            }
        } else {
            LatAccT<T> lacc;
            unsigned long long* lb = lat_buf(lat_par ^ 1);
            for (int c = 0; c < g.ncol; ++c)
                for (int tt = 0; tt < wc->cnt[c]; ++tt) {
                    const int s = wc->lo[c] + tt;
                    const SliceDesc d = warp_desc(g, *wc, c, tt, s);
                    if constexpr (MIXED) {   // keeps the undamped mixed path's registers as they were
                        mon = nanmax(mon, th != 1.0f
                                              ? phase_rhs<MIXED, true>(g, wc, d, st, rp, s, lane, vL, vP, vF, extrap,
                                                                       three, inc, sabs, dsel, lb, lacc, th)
                                              : phase_rhs<MIXED, false>(g, wc, d, st, rp, s, lane, vL, vP, vF, extrap,
                                                                        three, inc, sabs, dsel, lb, lacc, 1.0f));
                    } else {
                        mon = nanmax(mon, phase_rhs<MIXED, true>(g, wc, d, st, rp, s, lane, vL, vP, vF, extrap, three,
                                                                 inc, sabs, dsel, lb, lacc, th));
                    }
                }
            if (lb) lat_flush(lb, lacc);
        }
        BarrierResult br = barrier(true, mon);
        if (!br.ok) { publish(-1); return; }
        double R = br.val;
        lat_par ^= 1;
        lap(0);

        int sweeps = 0, outer = 0;
        bool ok = true;
        while (!(R <= target)) {
            if (!(R == R) || isinf(R) || outer >= rp.max_outer || sweeps >= rp.max_sweeps) { ok = false; break; }
            // inner relaxation on the correction
            const double inner_tgt = MIXED ? fmax(0.5 * target, rp.inner_reduction * R) : 0.5 * target;
            const T* rr = MIXED ? (const T*)st.r32 : (const T*)st.r64;
            T* dd = dbuf<T>(st, dsel);
            const T* ww = MIXED ? (const T*)g.w32 : (const T*)g.w64;
            const T* iD = MIXED ? (const T*)g.invD32 : (const T*)g.invD64;
            double est_mark = INFINITY;   // monitor value at the last stagnation check
            bool est_nan = false;         // a non-finite update (diverged, or a failed copy)
            int inner = 0;
            lat_clear(lat_par ^ 1);       // the next FP64 pass writes there; its readers are done
            while (rp.lat_k > 0) {
                // lattice rounds: lat_k exact block sweeps per device barrier (FP32, or FP64 in
                // the FP64 kernel)
                const T* dold = dbuf<T>(st, dsel);
                T* dnew = dbuf<T>(st, dsel ^ 1);
                const double m = lattice_round<ROWS, T>(g, dold, dnew, rr, omega, rp.lat_k, s_dyn,
                                               lat_buf(lat_par), target, inner == 0, ctl.tile_ctr,
                                               lat_rounds * ((unsigned)g.lat_tiles + nblocks));
                ++lat_rounds;
                const BarrierResult be = barrier(true, m);
                if (!be.ok) { publish(-1); return; }
                const double est = be.val;
                dsel ^= 1;
                dd = dbuf<T>(st, dsel);
                const int before = inner;
                sweeps += rp.lat_k;
                inner += rp.lat_k;
                if (!(est == est)) { est_nan = true; break; }
                if (est <= inner_tgt || sweeps >= rp.max_sweeps) break;
                if ((inner >> 4) != (before >> 4)) {
                    if (est > 0.9 * est_mark) break;
                    est_mark = est;
                }
            }
            while (rp.jacobi) {
                // damped Jacobi: all colours from the previous iterate, one barrier per sweep
                const T* dold = dbuf<T>(st, dsel);
                T* dnew = dbuf<T>(st, dsel ^ 1);
                double m = 0.0;
                for (int c = 0; c < g.ncol; ++c)
                    for (int tt = 0; tt < wc->cnt[c]; ++tt) {
                        const int s = wc->lo[c] + tt;
                        m = nanmax(m, jacobi_slice<T>(g, wc, warp_desc(g, *wc, c, tt, s), ww, iD, rr, dold, dnew, s,
                                                      lane, omega));
                    }
                const BarrierResult be = barrier(true, m);
                if (!be.ok) { publish(-1); return; }
                const double est = be.val;
                dsel ^= 1;
                dd = dbuf<T>(st, dsel);
                ++sweeps;
                ++inner;
                if (!(est == est)) { est_nan = true; break; }
                if (est <= inner_tgt || sweeps >= rp.max_sweeps) break;
                if ((inner & 15) == 0) {
                    if (est > 0.9 * est_mark) break;
                    est_mark = est;
                }
            }
            while (!rp.jacobi && !(rp.lat_k > 0)) {
                double est = 0.0;
                for (int c = 0; c < g.ncol; ++c) {
                    double m = 0.0;
                    if (MIXED) {
                        m = sweep_colour_tma<T>(g, wc, tw, c, ww, iD, rr, dd, lane, omega, ctl.err, rp.timeout_ns);
                    } else {
                        for (int tt = 0; tt < wc->cnt[c]; ++tt) {
                            const int s = wc->lo[c] + tt;
                            m = nanmax(m, sweep_slice<T>(g, wc, warp_desc(g, *wc, c, tt, s), ww, iD, rr, dd, s, lane,
                                                         omega));
                        }
                    }
                    const BarrierResult be = barrier(true, m);
                    if (!be.ok) { publish(-1); return; }
                    est = nanmax(est, be.val);
                }
                ++sweeps;
                ++inner;
                if (!(est == est)) { est_nan = true; break; }
                if (est <= inner_tgt || sweeps >= rp.max_sweeps) break;
                // The inner solve stalls at its precision floor (about eps * ||M^-1 D|| of the
                // correction); hand over to the FP64 outer pass when 16 sweeps gain < 10 %.
                if ((inner & 15) == 0) {
                    if (est > 0.9 * est_mark) break;
                    est_mark = est;
                }
            }
            lap(1);
            if (est_nan) { ok = false; break; }
            // outer pass
            double m = 0.0;
            T* dn = dbuf<T>(st, dsel ^ 1);
            {
                LatAccT<T> lacc;
                unsigned long long* lb = lat_buf(lat_par ^ 1);
                for (int c = 0; c < g.ncol; ++c)
                    for (int tt = 0; tt < wc->cnt[c]; ++tt) {
                        const int s = wc->lo[c] + tt;
                        m = nanmax(m, outer_slice<T>(g, wc, warp_desc(g, *wc, c, tt, s), st, dd, dn,
                                                     MIXED ? st.r32 : nullptr, s, lane, vbuf(st, vF),
                                                     MIXED && rp.lat_k > 0 && !g.natural, lb, lacc,
                                                     rp.mode == kModeTransient && !three ? st.md : nullptr));
                    }
                if (lb) lat_flush(lb, lacc);
            }
            br = barrier(true, m);
            if (!br.ok) { publish(-1); return; }
            R = br.val;
            lat_par ^= 1;
            dsel ^= 1;
            ++outer;
            lap(2);
        }
        if (!ok) { fail(sabs); return; }

        // ---- post: inductor currents (Eq. 10), outputs, the next step's load currents
        lat_clear(lat_par ^ 1);           // the next step's phase A writes there
        if (rp.mode == kModeTransient && sl + 1 < rp.nsteps) {
            // the word of step sabs + 2 is next written by the following post phase; nobody
            // reads it before then (step sabs + 1 reads the words of sabs + 1 and sabs)
            if (damp && gtid == 0) ctl.ld_flags[(sabs + 2) & 3] = 0u;
            eval_sources(sabs + 1, damp);
        }
        const double* vnew = vbuf(st, vF);
        if (rp.mode == kModeTransient && !three) {
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
        double objsum = 0.0;
        // four consecutive nodes per thread and iteration (n_pad is a multiple of kSlice):
        // 128-bit loads, a quarter of the dependent iterations
        for (int i4 = 4 * gtid; i4 < g.n_pad; i4 += 4 * nthreads) {
            double x4[4];
            int o4[4];
            ld4(vnew + i4, x4);
            if (g.natural) {               // natural order: node i is caller node i, padding at the end
#pragma unroll
                for (int j = 0; j < 4; ++j) o4[j] = i4 + j < g.n_real ? i4 + j : -1;
            } else {
                ldg4(g.orig + i4, o4);
            }
            if (rp.v_perm_all) st4(rp.v_perm_all + (long long)sl * g.n_pad + i4, x4);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int o = o4[j];
                if (o < 0) continue;
                const double x = x4[j];
                if (rp.obj_partials) {
                    const double sp = softplus_d(rp.obj_vref - x - rp.obj_margin);
                    objsum += sp * sp;
                }
                if (rp.v_all) rp.v_all[(long long)sl * g.n_real + o] = x;
                if (rp.solve_out) rp.solve_out[o] = x;
                if (rp.vmin) {
                    const unsigned long long k = order_key(x);
                    if (k < bk || (k == bk && o < ba)) { bk = k; ba = o; }
                }
            }
        }
        if (rp.probe_v)
            for (int k = gtid; k < rp.n_probes; k += nthreads)
                rp.probe_v[(long long)sl * rp.n_probes + k] = vnew[rp.probes_perm[k]];
        if (comp_key) {
            // warp-aggregated: one atomic when a warp's 32 nodes lie in one component
            unsigned long long* row = comp_key + (long long)sl * g.n_comp;
            for (int base = gwarp * 32; base < g.n_pad; base += nwarps * 32) {
                const int i = base + lane;
                const int c = i < g.n_pad ? __ldg(g.node_comp + i) : -1;
                unsigned long long k = c >= 0 ? order_key(vnew[i]) : ~0ull;
                int chi = c, clo = c >= 0 ? c : 0x7fffffff;
                for (int o = 16; o; o >>= 1) {
                    chi = max(chi, __shfl_xor_sync(kFull, chi, o));
                    clo = min(clo, __shfl_xor_sync(kFull, clo, o));
                }
                if (chi < 0) continue;
                if (clo == chi) {
                    for (int o = 16; o; o >>= 1) k = min(k, __shfl_xor_sync(kFull, k, o));
                    if (lane == 0) atomicMin(row + chi, k);
                } else if (c >= 0) {
                    atomicMin(row + c, k);
                }
            }
        }
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
        if (rp.obj_partials) {
            // fixed-order block sum (deterministic, so finite differences of J are meaningful)
            __shared__ double s_obj[kWarpsPerBlock];
            for (int o = 16; o; o >>= 1) objsum += __shfl_down_sync(kFull, objsum, o);
            if (lane == 0) s_obj[threadIdx.x >> 5] = objsum;
            __syncthreads();
            if (threadIdx.x == 0) {
                double t2 = 0.0;
                for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t2 += s_obj[q];
                rp.obj_partials[(long long)sl * nblocks + blockIdx.x] = t2;
            }
            __syncthreads();
        }
        tot_sweeps += sweeps; tot_outer += outer;
        max_sw = max(max_sw, sweeps); max_out = max(max_out, outer);
        max_bound_R = fmax(max_bound_R, R);
        last_R = R;
        last_outer = outer;
        ++steps_done;
        // rotate: the new state becomes the latest
        vP = vL; vL = vF; vF = 3 - vL - vP;
        have_prev = true;
        if (!barrier(false, 0.0).ok) { publish(-1); return; }
        lap(3);
    }
    if (rp.nsteps > 0) { finalize_vmin(rp.nsteps - 1); finalize_comp(rp.nsteps - 1); }
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
        sell_row<1, double>(g, nullptr, global_desc(g, s), g.w64, s, lane, [&](int c) { return x[c] * sc; }, sig);
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

// Power iteration for the column-block Jacobi operator B^-1 W (lattice form): one
// thread per column (x, y) of any lattice, y = (x + B^-1 W x) / 2 with x scaled by
// 1 / xmax_prev; accumulates x.(W x) and x.(B x), whose ratio is a Rayleigh quotient of
// W v = lambda B v.
template <int NL>
__device__ __forceinline__ void lattice_power_column(const DevGrid& g, int off, int nx, int ny, long long c,
                                                     const double* x, double* y, double sc, double& num,
                                                     double& den, double& mx) {
    const long long plane = (long long)nx * ny;
    const int cx = (int)(c % nx), cy = (int)(c / nx);
    const long long o0 = off + c;
    double xv[NL], wx[NL], f[NL], dl[NL], u[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const long long o = o0 + l * plane;
        xv[l] = x[o] * sc;
        double s = 0.0;
        if (cx + 1 < nx) s += (double)__ldg(g.lwE + o) * x[o + 1] * sc;
        if (cx > 0) s += (double)__ldg(g.lwE + o - 1) * x[o - 1] * sc;
        if (cy + 1 < ny) s += (double)__ldg(g.lwN + o) * x[o + nx] * sc;
        if (cy > 0) s += (double)__ldg(g.lwN + o - nx) * x[o - nx] * sc;
        wx[l] = s;
        u[l] = (double)__ldg(g.lwU + o);
        // block diagonal from the Thomas factors: d_l = d'_l + m_l u_{l-1}
        dl[l] = 1.0 / (double)__ldg(g.lip + o) + (l > 0 ? (double)__ldg(g.lm + o) * u[l - 1] : 0.0);
    }
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        double bx = dl[l] * xv[l];
        if (l > 0) bx -= u[l - 1] * xv[l - 1];
        if (l + 1 < NL) bx -= u[l] * xv[l + 1];
        num += xv[l] * wx[l];
        den += xv[l] * bx;
        f[l] = wx[l];
    }
#pragma unroll
    for (int l = 1; l < NL; ++l) f[l] += (double)__ldg(g.lm + o0 + l * plane) * f[l - 1];
    double z[NL];
    z[NL - 1] = f[NL - 1] * (double)__ldg(g.lip + o0 + (NL - 1) * plane);
#pragma unroll
    for (int l = NL - 2; l >= 0; --l) z[l] = (f[l] + u[l] * z[l + 1]) * (double)__ldg(g.lip + o0 + l * plane);
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        const double yv = 0.5 * (xv[l] + z[l]);
        y[o0 + l * plane] = yv;
        mx = fmax(mx, yv);
    }
}

__global__ void __launch_bounds__(256) lattice_power_kernel(DevGrid g, const double* x, double* y,
                                                           const unsigned long long* xmax_prev, double* acc,
                                                           unsigned long long* ymax) {
    const double sc = xmax_prev ? 1.0 / __longlong_as_double((long long)*xmax_prev) : 1.0;
    double num = 0.0, den = 0.0, mx = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.lat_cols;
         c += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = g.n_lats;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (__ldg(g.lat_col0 + mid) <= c) lo = mid; else hi = mid;
        }
        const int off = __ldg(g.lat_info + 4 * lo), nx = __ldg(g.lat_info + 4 * lo + 1),
                  ny = __ldg(g.lat_info + 4 * lo + 2), nl = __ldg(g.lat_info + 4 * lo + 3);
        const long long cc = c - __ldg(g.lat_col0 + lo);
        if (nl == 1) lattice_power_column<1>(g, off, nx, ny, cc, x, y, sc, num, den, mx);
        else if (nl == 2) lattice_power_column<2>(g, off, nx, ny, cc, x, y, sc, num, den, mx);
        else lattice_power_column<3>(g, off, nx, ny, cc, x, y, sc, num, den, mx);
    }
    for (int o = 16; o; o >>= 1) {
        num += __shfl_xor_sync(kFull, num, o);
        den += __shfl_xor_sync(kFull, den, o);
        mx = fmax(mx, __shfl_xor_sync(kFull, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
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

// ---------------------------------------------------------------- adjoint (not in the paper)

// rhs = dJ/dv_s + (C/h) lambda_{s+1} with dJ/dv = -2 softplus(u) sigmoid(u), u = vref - v - margin;
// also max |rhs| / D into *scale_slot (sets the relative solve target).
// With inductors (explicit form, Eq. 10) the rhs also carries h A_l^T Ldiag^-1 mu_s.
__global__ void __launch_bounds__(256) adjoint_rhs_kernel(DevGrid g, const double* __restrict__ v,
                                                         const double* __restrict__ lam_next,
                                                         const double* __restrict__ mu,
                                                         double* __restrict__ rhs, double vref, double margin,
                                                         unsigned long long* scale_slot) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n_pad; i += gridDim.x * blockDim.x) {
        double r = 0.0;
        if (__ldg(g.orig + i) >= 0) {
            const double u = vref - v[i] - margin;
            r = -2.0 * softplus_d(u) * sigmoid_d(u) + __ldg(g.ch + i) * lam_next[i];
            if (mu)
                for (int q = __ldg(g.ind_ptr + i); q < __ldg(g.ind_ptr + i + 1); ++q) {
                    const int lid = __ldg(g.ind_idx + q);
                    const int e = (lid > 0 ? lid : -lid) - 1;
                    const double t = __ldg(g.ind_hl + e) * mu[e];
                    r += lid > 0 ? t : -t;
                }
            m = fmax(m, fabs(r) * __ldg(g.invD64 + i));
        }
        rhs[i] = r;
    }
    for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(scale_slot, (unsigned long long)__double_as_longlong(m));
}

// Gradient sums of one step (FP64): per neighbour slot with col > node (each edge once)
// acc_slot += (lam_i - lam_j)(v_i - v_j); per node acc_lv += lam v, acc_l += lam,
// acc_dv += lam (v - v_prev).
__global__ void __launch_bounds__(256) adjoint_grad_kernel(DevGrid g, const double* __restrict__ lam,
                                                          const double* __restrict__ v,
                                                          const double* __restrict__ v_prev,
                                                          double* __restrict__ acc_slot, double* __restrict__ acc_lv,
                                                          double* __restrict__ acc_l, double* __restrict__ acc_dv) {
    const int lane = threadIdx.x & 31;
    const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)((gridDim.x * blockDim.x) >> 5);
    for (int s = gwarp; s < g.n_slices; s += nwarps) {
        const SliceDesc d = global_desc(g, s);
        const int i0 = s * kSlice + lane * kVec;
        double li[4], vi[4], vp[4];
        ld4(lam + i0, li);
        ld4(v + i0, vi);
        ld4(v_prev + i0, vp);
        for (int j = 0; j < 4; ++j) {
            acc_lv[i0 + j] += li[j] * vi[j];
            acc_l[i0 + j] += li[j];
            acc_dv[i0 + j] += li[j] * (vi[j] - vp[j]);
        }
        for (int k = 0; k < d.K; ++k) {
            const long long e = d.off + (long long)k * kSlice + lane * kVec;
            int c[4];
            if (d.dpos != -1) {
                const int o = __ldg(g.dia_off + (-2 - d.dpos) + k);
                if (o <= 0) continue;                       // the neighbour with the larger index owns it
                c[0] = i0 + o; c[1] = i0 + 1 + o; c[2] = i0 + 2 + o; c[3] = i0 + 3 + o;
            } else {
                ldg4(g.ell_col + e, c);
            }
            for (int j = 0; j < 4; ++j)
                if (c[j] > i0 + j) acc_slot[e + j] += (li[j] - lam[c[j]]) * (vi[j] - v[c[j]]);
        }
    }
}

// Inductor multipliers of the explicit RLC form: mu_s = mu_(s+1) - A_l lambda_(s+1)
// (a source or ground terminal carries no multiplier).
__global__ void __launch_bounds__(256) adjoint_mu_kernel(DevGrid g, const double* __restrict__ lam_next,
                                                        double* __restrict__ mu) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.n_l; e += gridDim.x * blockDim.x) {
        const int a = __ldg(g.ind_a + e), b = __ldg(g.ind_b + e);
        mu[e] -= (a >= 0 ? lam_next[a] : 0.0) - (b >= 0 ? lam_next[b] : 0.0);
    }
}

// Per inductor: acc_L += u_s (A_l lambda_s - mu_s), u_s = A_l v_s + A_ls v_d (its branch voltage);
// dJ/dL = (h / L^2) acc_L.
__global__ void __launch_bounds__(256) adjoint_lgrad_kernel(DevGrid g, const double* __restrict__ lam,
                                                           const double* __restrict__ v,
                                                           const double* __restrict__ mu,
                                                           double* __restrict__ acc_L) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.n_l; e += gridDim.x * blockDim.x) {
        const int a = __ldg(g.ind_a + e), b = __ldg(g.ind_b + e);
        const double u = term_volt(g, v, a) - term_volt(g, v, b);
        const double dl = (a >= 0 ? lam[a] : 0.0) - (b >= 0 ? lam[b] : 0.0);
        acc_L[e] += u * (dl - mu[e]);
    }
}

// ---------------------------------------------------------------- host-side launch helpers

size_t persistent_smem_bytes(bool mixed, int rows, int nl) {
    const size_t stages = (size_t)kWarpsPerBlock * tma_warp_bytes(sizeof(float));
    if (!mixed) return nl > 0 ? lattice_region_bytes(rows, nl, sizeof(double)) : 0;   // FP64 lattice region
    const size_t region = nl > 0 ? lattice_region_bytes(rows, nl) : 0;
    return std::max(stages, region);
}

static const void* persistent_fn(bool mixed, int rows) {
    return !mixed ? (const void*)persistent_kernel<false, 34>
         : rows == 66 ? (const void*)persistent_kernel<true, 66> : (const void*)persistent_kernel<true, 34>;
}

cudaError_t launch_persistent(bool mixed, const DevGrid& g, const DevState& st, const DevCtl& ctl,
                              const RunParams& rp, int blocks, int threads, size_t smem, cudaStream_t stream) {
    void* args[] = {(void*)&g, (void*)&st, (void*)&ctl, (void*)&rp};
    return cudaLaunchCooperativeKernel(persistent_fn(mixed, g.lat_rows), dim3(blocks), dim3(threads), args, smem,
                                       stream);
}

cudaError_t persistent_occupancy(bool mixed, int rows, int threads, size_t smem, int* blocks_per_sm) {
    const void* fn = persistent_fn(mixed, rows);
    if (smem > 0) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);
}

cudaError_t launch_power_step(const DevGrid& g, const double* x, double* y, const unsigned long long* xmax_prev,
                              double* acc, unsigned long long* ymax, int blocks, cudaStream_t stream) {
    power_step_kernel<<<blocks, 256, 0, stream>>>(g, x, y, xmax_prev, acc, ymax);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_rhs(const DevGrid& g, const double* v, const double* lam_next, const double* mu,
                               double* rhs, double vref, double margin, unsigned long long* scale_slot, int blocks,
                               cudaStream_t stream) {
    adjoint_rhs_kernel<<<blocks, 256, 0, stream>>>(g, v, lam_next, mu, rhs, vref, margin, scale_slot);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_mu(const DevGrid& g, const double* lam_next, double* mu, int blocks, cudaStream_t stream) {
    adjoint_mu_kernel<<<blocks, 256, 0, stream>>>(g, lam_next, mu);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_lgrad(const DevGrid& g, const double* lam, const double* v, const double* mu,
                                 double* acc_L, int blocks, cudaStream_t stream) {
    adjoint_lgrad_kernel<<<blocks, 256, 0, stream>>>(g, lam, v, mu, acc_L);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_grad(const DevGrid& g, const double* lam, const double* v, const double* v_prev,
                                double* acc_slot, double* acc_lv, double* acc_l, double* acc_dv, int blocks,
                                cudaStream_t stream) {
    adjoint_grad_kernel<<<blocks, 256, 0, stream>>>(g, lam, v, v_prev, acc_slot, acc_lv, acc_l, acc_dv);
    return cudaGetLastError();
}

cudaError_t launch_lattice_power(const DevGrid& g, const double* x, double* y, const unsigned long long* xmax_prev,
                                 double* acc, unsigned long long* ymax, int blocks, cudaStream_t stream) {
    lattice_power_kernel<<<blocks, 256, 0, stream>>>(g, x, y, xmax_prev, acc, ymax);
    return cudaGetLastError();
}

cudaError_t launch_permute_in(const int32_t* orig, const double* src, double fill, double* dst, int n_pad,
                              int n_sm, cudaStream_t stream) {
    const int blocks = std::max(1, std::min(4 * n_sm, (n_pad + 255) / 256));
    permute_in_kernel<<<blocks, 256, 0, stream>>>(orig, src, fill, dst, n_pad);
    return cudaGetLastError();
}

}  // namespace pg
