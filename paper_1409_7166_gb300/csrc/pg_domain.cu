// Device half of the row-block domain decomposition of one lattice grid.
//
// The node update of Eq. 16-17 reads only the node's own value and those of
// its neighbours, so one red-black half-sweep over a block of lattice rows
// needs, from the other colour, only the row just below and the row just above
// the block.  A block holds its rows of every layer (the vias stay inside it)
// plus one halo row on each side, which the caller refreshes from the
// neighbouring blocks between half-sweeps (device copies within one process,
// or point-to-point messages between GPUs).  The red-black order puts the two
// colours in separate half-sweeps, so the decomposed iteration makes exactly
// the updates of the undecomposed one: every node's update reads the same
// neighbour values and adds its terms in the same fixed order.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "pg_grid.h"

namespace {

// One thread per node of the colour: row k (1..rows) of layer l holds the nodes x with
// x + y + l of the given parity, y = y0 + k - 1 the global row.
__global__ void __launch_bounds__(256) block_half_sweep_kernel(pg_row_block b, int colour, double omega,
                                                               unsigned long long* max_update) {
    const int nx = b.nx, rows = b.rows, nl = b.nl;
    const int half = (nx + 1) / 2;                   // nodes of one parity per row, at most
    const long long total = (long long)nl * rows * half;
    const long long plane = (long long)rows * nx;    // one layer of w_e, w_u, inv_d, rhs
    const long long xplane = (long long)(rows + 2) * nx;   // one layer of x (with halos)
    const long long nplane = (long long)(rows + 1) * nx;   // one layer of w_n
    double m = 0.0;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(t / ((long long)rows * half));
        const int rem = (int)(t - (long long)l * rows * half);
        const int k = 1 + rem / half;                  // local row of x (0 and rows + 1 are halos)
        const int q = rem - (k - 1) * half;
        const int y = b.y0 + k - 1;
        const int x = 2 * q + ((colour - y - l) & 1);  // the q-th node of this colour in the row
        if (x >= nx) continue;
        const long long o = l * plane + (long long)(k - 1) * nx + x;      // w_e, w_u, inv_d, rhs
        const long long ox = l * xplane + (long long)k * nx + x;          // x
        const long long on = l * nplane + (long long)k * nx + x;          // w_n couples rows k, k + 1
        const double* X = b.x;
        // Eq. 16: the neighbour sum, in a fixed order (E, W, N, S, up, down)
        double s = 0.0;
        if (x + 1 < nx) s = fma(b.w_e[o], X[ox + 1], s);
        if (x > 0) s = fma(b.w_e[o - 1], X[ox - 1], s);
        s = fma(b.w_n[on], X[ox + nx], s);              // the halo above for k = rows
        s = fma(b.w_n[on - nx], X[ox - nx], s);         // the halo below for k = 1
        if (l + 1 < nl) s = fma(b.w_u[o], X[ox + xplane], s);
        if (l > 0) s = fma(b.w_u[o - plane], X[ox - xplane], s);
        // Eq. 17: over-relaxed update
        const double xo = X[ox];
        const double upd = (b.rhs[o] + s) * b.inv_d[o] - xo;
        b.x[ox] = fma(omega, upd, xo);
        m = fmax(m, fabs(upd));
    }
    for (int off = 16; off; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(max_update, (unsigned long long)__double_as_longlong(m));
}

pg_status fail(pg_status s, const std::string& m) {
    pg::set_last_error(m);
    return s;
}

}  // namespace

extern "C" pg_status pg_block_half_sweep(const pg_row_block* blk, int32_t colour, double omega, double* max_update,
                                         void* stream) {
    if (!blk || !blk->x || !blk->w_e || !blk->w_n || !blk->w_u || !blk->inv_d || !blk->rhs || !max_update)
        return fail(PG_ERR_INVALID_ARG, "pg_block_half_sweep: null block array");
    if (blk->nx < 1 || blk->rows < 1 || blk->nl < 1 || blk->y0 < 0)
        return fail(PG_ERR_INVALID_ARG, "pg_block_half_sweep: empty block or negative first row");
    if (colour != 0 && colour != 1) return fail(PG_ERR_INVALID_ARG, "pg_block_half_sweep: colour must be 0 or 1");
    if (!(omega > 0.0 && omega < 2.0)) return fail(PG_ERR_INVALID_ARG, "pg_block_half_sweep: omega must be in (0, 2)");
    const long long total = (long long)blk->nl * blk->rows * ((blk->nx + 1) / 2);
    if (total > (long long)1 << 40) return fail(PG_ERR_INVALID_ARG, "pg_block_half_sweep: block too large");
    int dev = 0, n_sm = 1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    const long long want = (total + 255) / 256;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(want, 8LL * n_sm));
    block_half_sweep_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(
        *blk, colour, omega, reinterpret_cast<unsigned long long*>(max_update));
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(PG_ERR_CUDA, cudaGetErrorString(e));
    return PG_OK;
}
