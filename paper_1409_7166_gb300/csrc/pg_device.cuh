// Device helpers shared by the CUDA translation units of the library: vector
// loads and stores, NaN-propagating maxima, order-preserving keys, the bounded
// device-wide barrier, piecewise-linear load evaluation and the SELL slice
// descriptors.  Everything here is inline and local to each translation unit.
#pragma once

#include <cuda/atomic>
#include <cuda_runtime.h>

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

// softplus(u) = log(1 + e^u), evaluated without overflow: max(u, 0) + log1p(e^-|u|)
__device__ __forceinline__ double softplus_d(double u) { return fmax(u, 0.0) + log1p(exp(-fabs(u))); }
__device__ __forceinline__ double sigmoid_d(double u) { return 0.5 * (1.0 + tanh(0.5 * u)); }

// max that lets a NaN win, so a diverged iterate is never mistaken for convergence
__device__ __forceinline__ double nanmax(double a, double b) { return (a > b || a != a) ? a : b; }
// FP32 version for the FP32 sweeps: GB300's FP64 pipe is a small fraction of its FP32
// rate, so even a per-node double compare would cost a large share of a sweep.
__device__ __forceinline__ float nanmaxf(float a, float b) { return (a > b || a != a) ? a : b; }
template <typename T>
__device__ __forceinline__ T nanmax_t(T a, T b) { return (a > b || a != a) ? a : b; }

// Per-lattice maxima of val over the lane's 4 nodes (warp-collective): one atomic
// per warp when the slice lies in one lattice (the common case), else per node.
// Per-lattice maxima of |r|/D (the FP64 passes feed the lattice solve's skip test).
// A warp's slices are contiguous and almost always inside one lattice, so the
// warp keeps a running (lattice, max) pair (warp-uniform) and publishes it with
// one atomic when the lattice changes and at the end of the pass (lat_flush);
// a slice that straddles lattices publishes its values directly.
// V: the type of the maxima (double in the FP64 kernel, float in the mixed one, where
// the monitored values are FP32 upper bounds); published as double bits either way.
template <typename V>
struct LatAccT {
    int L = -1;
    V m = V(0);
};
using LatAcc = LatAccT<double>;
template <typename V>
__device__ __forceinline__ void lat_flush(unsigned long long* latR, LatAccT<V>& acc) {
    if ((threadIdx.x & 31) == 0 && acc.L >= 0 && acc.m != V(0))
        atomicMax(latR + acc.L, (unsigned long long)__double_as_longlong((double)acc.m));
    acc.L = -1;
    acc.m = V(0);
}
// `L` holds node_lat[i0 .. i0 + 3], loaded by the caller with the slice's other operands.
template <typename V>
__device__ __forceinline__ void lattice_max(unsigned long long* latR, const int (&L)[4], const V (&val)[4],
                                            LatAccT<V>& acc) {
    bool same = true;
    const int L0 = __shfl_sync(0xffffffffu, L[0], 0);
    V m = V(0);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        same = same && (L[j] == L0 || L[j] < 0);
        if (L[j] >= 0) m = nanmax_t<V>(m, val[j]);
    }
    if (__all_sync(0xffffffffu, same)) {
        for (int o = 16; o; o >>= 1) m = nanmax_t<V>(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (L0 < 0) return;
        if (L0 != acc.L) lat_flush(latR, acc);
        acc.L = L0;
        acc.m = nanmax_t<V>(acc.m, m);
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (L[j] >= 0 && val[j] != V(0))
                atomicMax(latR + L[j], (unsigned long long)__double_as_longlong((double)val[j]));
    }
}

// Upper bound of |r| / D from the FP32 copies r32 = fl(r) and invD32 = fl(1 / D): each of
// the three roundings (r32, invD32, their product) is within 2^-24 relative, so scaling the
// product by 1 + 2^-21 (itself rounded) can only raise it above the exact value.  The FP32
// monitor costs no FP64 instructions, which GB300 issues at a small fraction of its FP32 rate.
constexpr float kMonUp = 1.0f + 0x1p-21f;
__device__ __forceinline__ float scaled_upper(float r32, float inv_d32) { return fabsf(r32) * inv_d32 * kMonUp; }

// Order-preserving map of a double to an unsigned key (for min reductions).
__device__ __forceinline__ unsigned long long order_key(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double key_value(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

// Device-wide barrier with a time limit, fused with the block's max-reduction.
//
// Every block merges `v` (its threads' partial maxima) into the reduction slot
// `slot` with one atomic, then arrives.  The generation word is cleared by the
// host before each launch, so barrier number k (counted from 0 in every block)
// completes when the generation reaches k + 1: no load is needed before
// arriving.  Arrival is an acq_rel RMW and the wait an acquire load, both at
// device scope, which publishes the block's writes (ordered before the
// arrival by __syncthreads) to every block that passes the barrier.  .ok is
// false for the whole block when an error was recorded (this block's wait
// timed out, or another block's did); .val is the reduced value, read once
// by thread 0 after the wait and broadcast.
struct BarrierResult {
    bool ok;
    double val;
};

__device__ __forceinline__ BarrierResult grid_barrier(const DevCtl& c, unsigned nblocks, unsigned target_gen,
                                                      long long timeout_ns, bool skip, double v,
                                                      unsigned long long* slot) {
    __shared__ double s_part[32];
    __shared__ int s_ok;
    __shared__ double s_val;
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (slot) {
        for (int o = 16; o; o >>= 1) v = nanmax(v, __shfl_xor_sync(kFull, v, o));
        if (l == 0) s_part[w] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(*c.bar_gen);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(*c.bar_count);
        cuda::atomic_ref<int, cuda::thread_scope_device> err(*c.err);
        if (slot) {
            double m = s_part[0];
            for (int q = 1; q < (int)(blockDim.x >> 5); ++q) m = nanmax(m, s_part[q]);
            if (m != 0.0) atomicMax(slot, (unsigned long long)__double_as_longlong(m));
        }
        int ok = 1;
        // test hook: a skipping block waits without being counted, so the barrier never opens
        const unsigned arrived = skip ? 0u : cnt.fetch_add(1u, cuda::memory_order_acq_rel);
        if (!skip && arrived == nblocks - 1) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.store(target_gen, cuda::memory_order_release);
        } else {
            long long t0 = 0;
            unsigned ns = 0;
            for (int it = 0; gen.load(cuda::memory_order_acquire) < target_gen; ++it) {
                if (err.load(cuda::memory_order_relaxed) != 0) { ok = 0; break; }
                if (it == 64) t0 = global_ns();
                if (it > 64) {
                    if (global_ns() - t0 > timeout_ns) {
                        int z = 0;
                        err.compare_exchange_strong(z, (int)PG_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                    __nanosleep(ns);
                    ns = ns < 128 ? ns + 16 : 128;
                }
            }
        }
        s_ok = ok;
        if (slot) {
            cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> r(*slot);
            s_val = __longlong_as_double((long long)r.load(cuda::memory_order_relaxed));
        }
    }
    __syncthreads();
    return BarrierResult{s_ok != 0, slot ? s_val : 0.0};
}

// Value of current source e at time t (piecewise linear, held outside the breakpoints).
// Value of PWL source e at time t (tk = order_key(t)): held before the first and after
// the last breakpoint, linear in between.  The segment is found by integer compares of
// order keys and interpolated with its precomputed slope (no FP64 compare or divide: both
// issue slowly on GB300's FP64 pipe).
__device__ __forceinline__ double pwl_eval(const DevGrid& g, int e, double t, unsigned long long tk) {
    int64_t lo = g.pwl_ptr[e], hi = g.pwl_ptr[e + 1] - 1;
    const unsigned long long* K = g.pwl_tk;
    if (tk <= K[lo]) return g.pwl_v[lo];
    if (tk > K[hi]) return g.pwl_v[hi];
    while (hi - lo > 1) {            // keep t[lo] < t <= t[hi]
        const int64_t mid = (lo + hi) >> 1;
        if (tk <= K[mid]) hi = mid; else lo = mid;
    }
    return fma(g.pwl_s[lo], t - g.pwl_t[lo], g.pwl_v[lo]);
}

// Value of PWL source e (breakpoints lo..hi) at t when the cursor segment j does not hold
// it: the search of pwl_eval, also returning the segment (hi past the last breakpoint).
__device__ __forceinline__ double pwl_eval_search(const DevGrid& g, int64_t lo, int64_t hi, double t,
                                                  unsigned long long tk, int64_t& j) {
    const unsigned long long* K = g.pwl_tk;
    if (tk <= K[lo]) { j = lo; return g.pwl_v[lo]; }
    if (tk > K[hi]) { j = hi; return g.pwl_v[hi]; }
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (tk <= K[mid]) hi = mid; else lo = mid;
    }
    j = lo;
    return fma(g.pwl_s[lo], t - g.pwl_t[lo], g.pwl_v[lo]);
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

// ---- shared-memory staging
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Asynchronous global -> shared copies (no registers held while in flight);
// src_bytes = 0 fills the destination with zeros.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, unsigned src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// One element (4 or 8 bytes) or a 16-byte piece.
template <typename V>
__device__ __forceinline__ void cp_async_elem(V* dst, const V* src, bool in) {
    if constexpr (sizeof(V) == 8) cp_async8(dst, src, in ? 8u : 0u);
    else cp_async4(dst, src, in ? 4u : 0u);
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// ---- SELL slice descriptors

struct SliceDesc {
    long long off;   // element offset of the slice's slot 0
    int K;           // slots per node
    int dpos;        // >= 0: offsets at pool[dpos]; -1: explicit columns; <= -2: offsets at dia_off[-2 - dpos]
};

__device__ __forceinline__ SliceDesc global_desc(const DevGrid& g, int s) {
    SliceDesc d;
    d.off = __ldg(g.slice_off + s);
    d.K = __ldg(g.slice_w + s);
    const int d0 = __ldg(g.slice_doff + s);
    d.dpos = __ldg(g.slice_doff + s + 1) > d0 ? -2 - d0 : -1;
    return d;
}

}  // namespace

}  // namespace pg
