// pg_solve_noalloc: a solve entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the point where they need a solve:
// processes whose device memory is reserved up front by another allocator or
// capped by a budget (so a fresh cudaMalloc fails or fragments it), and
// steady-state loops that must not allocate at all.  For them this entry point
// runs the same persistent relaxation kernel as pg_solve, but takes every
// scratch buffer the solve needs (the permuted right-hand side, the iterate,
// the residuals, the corrections, the barrier and reduction words and the
// statistics) from one file-scope device array of fixed size, instead of from
// allocations.  The grid itself (its read-only coefficients) is still created
// with pg_create_grid beforehand.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "pg_grid.h"

namespace {

// Maximum scratch shared by all calls: 32 MiB.  CUDA loads this file's module,
// and with it reserves the array on a device, at the first lookup of its address
// on that device, which pg_create_grid makes; from then on the device holds it
// until the process exits.
constexpr size_t kScratchBytes = size_t(32) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {nullptr};
bool g_tried[kMaxDevices] = {false};
std::string g_bind_error[kMaxDevices];

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Byte layout of the scratch for a grid with n_pad permuted nodes and `blocks` CTAs.
struct Layout {
    size_t ctl, red, tile, stats, blk_min, blk_arg, rhs, v, r64, r32, d0, d1, total;
};

Layout layout(int n_pad, int blocks, bool mixed) {
    Layout L{};
    size_t o = 0;
    L.ctl = o;      o = align256(o + 3 * sizeof(uint32_t));              // barrier count, generation, error
    L.red = o;      o = align256(o + pg::kRedSlots * sizeof(unsigned long long));
    L.tile = o;     o = align256(o + sizeof(unsigned));                      // lattice tile counter
    L.stats = o;    o = align256(o + pg::kStatCount * sizeof(double));
    L.blk_min = o;  o = align256(o + 2 * size_t(blocks) * sizeof(unsigned long long));
    L.blk_arg = o;  o = align256(o + 2 * size_t(blocks) * sizeof(int32_t));
    L.rhs = o;      o = align256(o + size_t(n_pad) * sizeof(double));
    L.v = o;        o = align256(o + size_t(n_pad) * sizeof(double));
    L.r64 = o;      o = align256(o + size_t(n_pad) * sizeof(double));
    const size_t ds = mixed ? sizeof(float) : sizeof(double);
    L.r32 = o;      o = align256(o + (mixed ? size_t(n_pad) * sizeof(float) : 0));
    L.d0 = o;       o = align256(o + size_t(n_pad) * ds);
    L.d1 = o;       o = align256(o + size_t(n_pad) * ds);
    L.total = o;
    return L;
}

pg_status fail(pg_status s, const std::string& m) {
    pg::set_last_error(m);
    return s;
}

}  // namespace

void pg::noalloc_bind_device(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lk(g_addr_mu);
    if (g_tried[dev]) return;
    g_tried[dev] = true;
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();            // the grid does not depend on this array
        g_bind_error[dev] = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return;
    }
    g_addr[dev] = p;
}

extern "C" pg_status pg_solve_noalloc(pg_grid* g, double h, const double* b, double* x, double tol,
                                      pg_run_stats* stats) {
    if (!g || !b || !x || !(tol > 0.0)) return fail(PG_ERR_INVALID_ARG, "null argument or tol <= 0");
    if (g->h != h)
        return fail(PG_ERR_INVALID_ARG,
                    "pg_solve_noalloc needs the coefficients of this h assembled first "
                    "(call pg_solve or pg_transient with the same h once)");
    const Layout L = layout(g->P.n_pad, g->blocks, g->mixed);
    if (L.total > kScratchBytes)
        return fail(PG_ERR_INVALID_ARG,
                    "grid too large for the fixed scratch of pg_solve_noalloc: needs " + std::to_string(L.total) +
                        " bytes, the maximum is " + std::to_string(kScratchBytes) +
                        " (about 830k padded nodes in FP64, 930k in mixed precision)");
    const double target = tol / g->kappa - 1e-13;
    if (!(target > 0.0)) return fail(PG_ERR_INVALID_ARG, "tol below the rounding floor");

    // The array's device address was looked up when the grid was created (with the grid's
    // device current); this call only reads it, so it never loads a module or reserves memory.
    const int dev = g->device;
    if (dev < 0 || dev >= kMaxDevices) return fail(PG_ERR_CUDA, "device ordinal out of range");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_addr_mu);
        if (!g_addr[dev])
            return fail(PG_ERR_CUDA, "the fixed scratch array could not be set up when the grid was created" +
                                         (g_bind_error[dev].empty() ? std::string() : ": " + g_bind_error[dev]));
        base = static_cast<unsigned char*>(g_addr[dev]);
    }

    pg::DevCtl c{};
    c.bar_count = reinterpret_cast<unsigned*>(base + L.ctl);
    c.bar_gen = c.bar_count + 1;
    c.err = reinterpret_cast<int32_t*>(c.bar_count + 2);
    c.red = reinterpret_cast<unsigned long long*>(base + L.red);
    c.tile_ctr = reinterpret_cast<unsigned*>(base + L.tile);
    c.stats = reinterpret_cast<double*>(base + L.stats);
    c.blk_min = reinterpret_cast<unsigned long long*>(base + L.blk_min);
    c.blk_arg = reinterpret_cast<int32_t*>(base + L.blk_arg);
    pg::DevState st{};
    double* rhs = reinterpret_cast<double*>(base + L.rhs);
    double* v = reinterpret_cast<double*>(base + L.v);
    st.v[0] = st.v[1] = st.v[2] = v;           // a solve touches only the buffer it writes
    st.il = nullptr;
    st.r64 = reinterpret_cast<double*>(base + L.r64);
    if (g->mixed) {
        st.r32 = reinterpret_cast<float*>(base + L.r32);
        st.d32[0] = reinterpret_cast<float*>(base + L.d0);
        st.d32[1] = reinterpret_cast<float*>(base + L.d1);
    } else {
        st.d64[0] = reinterpret_cast<double*>(base + L.d0);
        st.d64[1] = reinterpret_cast<double*>(base + L.d1);
    }
    st.rhs = rhs;

    // The array keeps the previous call's contents: clear what must start at zero.
    cudaStream_t s = g->stream;
    cudaError_t e = cudaSuccess;
    if ((e = cudaMemsetAsync(base + L.ctl, 0, 3 * sizeof(uint32_t), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + L.red, 0, pg::kRedSlots * sizeof(unsigned long long), s)) != cudaSuccess ||
        (e = cudaMemsetAsync(base + L.tile, 0, sizeof(unsigned), s)) != cudaSuccess)
        return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    if ((e = pg::launch_permute_in(g->dg.orig, b, 0.0, rhs, g->P.n_pad, g->n_sm, s)) != cudaSuccess)
        return fail(PG_ERR_CUDA, cudaGetErrorString(e));

    pg::RunParams rp = pg::base_params(g);
    rp.mode = pg::kModeSolve;
    rp.nsteps = 1;
    rp.step0 = 0;
    rp.cur = 0; rp.prev = 1;
    rp.have_prev = 0;
    rp.warm_extrap = 0;
    rp.target = target;
    rp.solve_out = x;
    rp.debug_flags = 0;
    if ((e = cudaEventRecord(g->ev0, s)) != cudaSuccess ||
        (e = pg::launch_persistent(g->mixed, g->dg, st, c, rp, g->blocks, g->threads, g->smem, s)) != cudaSuccess ||
        (e = cudaEventRecord(g->ev1, s)) != cudaSuccess)
        return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    int32_t err = 0;
    double hs[pg::kStatCount];
    if ((e = cudaMemcpyAsync(&err, c.err, sizeof(int32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(hs, c.stats, sizeof(hs), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, g->ev0, g->ev1);
    pg::fill_run_stats(g, hs, ms, stats, 0.0);     // the same report as pg_solve
    if (err == PG_ERR_TIMEOUT) return fail(PG_ERR_TIMEOUT, "device barrier timed out");
    if (err == PG_ERR_NOT_CONVERGED) return fail(PG_ERR_NOT_CONVERGED, "relaxation did not converge");
    if (err != 0) return fail(PG_ERR_CUDA, "device error");
    return PG_OK;
}
