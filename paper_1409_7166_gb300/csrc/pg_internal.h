// Internal structures shared by the host builder, the C ABI and the kernels.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/pg.h"

namespace pg {

constexpr int kVec = 4;                 // nodes per thread (128-bit vector loads)
constexpr int kSlice = 32 * kVec;       // nodes per SELL slice (one warp)
constexpr int kMaxColours = 16;
constexpr int kRedSlots = 4;            // rotating reduction slots

// ---------------------------------------------------------------- host side

// Result of validation, colouring and packing (independent of h).
struct Packed {
    int32_t n = 0;          // caller's nodes
    int32_t n_pad = 0;      // permuted nodes incl. padding (multiple of kSlice)
    int32_t p = 0;          // source nodes
    int32_t ncol = 0;
    int32_t colour_start[kMaxColours + 1] = {0};  // node index, multiple of kSlice
    std::vector<int32_t> perm;        // caller id -> permuted index
    std::vector<int32_t> orig;        // permuted index -> caller id (-1 = padding)
    std::vector<double> vdd;

    // merged neighbour lists in caller numbering (CSR): conductance part and 1/L part
    std::vector<int64_t> adj_ptr;
    std::vector<int32_t> adj_nbr;
    std::vector<double> adj_g, adj_il;
    // per caller node: grounded parts
    std::vector<double> g_gnd, il_gnd, cap, inj_g, inj_il;

    // SELL slices over the permuted index space
    int32_t n_slices = 0;
    std::vector<int64_t> slice_off;   // [n_slices+1] element offset of the slice's slots
    std::vector<int32_t> slice_w;     // slots per node in the slice
    std::vector<int32_t> slice_doff;  // [n_slices+1] offset into dia_off (== itself if explicit)
    std::vector<int32_t> dia_off;     // per diagonal slice: slice_w column offsets
    std::vector<int32_t> ell_col;     // explicit columns (only explicit slices fill them)
    std::vector<int64_t> ell_adj;     // slot -> adjacency entry (-1 = empty slot)
    int64_t n_ell = 0;
    int32_t n_dia_slices = 0;

    // loads: per permuted node CSR of signed source ids (+(e+1) leaves the node, -(e+1) enters)
    std::vector<int32_t> ld_ptr, ld_idx;
    std::vector<int64_t> pwl_ptr;
    std::vector<double> pwl_t, pwl_v;
    std::vector<double> pwl_s;              // per-breakpoint segment slopes (pwl_aux)
    std::vector<unsigned long long> pwl_tk; // order keys of pwl_t (pwl_aux)

    // inductors
    int32_t n_l = 0;
    std::vector<int32_t> ind_a, ind_b;        // permuted node, or terminal code (< 0)
    std::vector<double> ind_invL;
    std::vector<int32_t> ind_ptr, ind_idx;    // per permuted node CSR of signed inductor ids

    // lattice form (optional): nodes (x, y, l) with id (l*ny + y)*nx + x and every
    // branch between lattice neighbours; adj_dir marks the +x / +y / +l entries
    bool lattice = false;
    std::vector<int32_t> lats;     // 4 per lattice: first node id, nx, ny, nl
    int32_t lat_maxnl = 0;
    std::vector<int8_t> adj_dir;   // 0: +x, 1: +y, 2: +l, -1: the reverse entries
    std::vector<int32_t> node_lat; // permuted node -> lattice (-1 for padding)

    // components (connected sub-circuits, Fig. 1)
    int32_t n_comp = 0;
    std::vector<uint8_t> comp_has_r_anchor;
    std::vector<int32_t> comp_of;             // caller id -> component
};

// lattice_policy: the lattice_sweeps option when the grid runs in mixed precision (the
// lattice inner solve will be used when the netlist is a lattice), INT32_MIN otherwise.
// Grids that take the lattice inner solve are packed in natural (caller) order with one
// colour: no point sweep runs on them, and the FP64 passes then read the lattice-ordered
// corrections contiguously.
// colouring: PG_COLOUR_* (the order of the neighbour-list sweeps).
// Slopes and time keys of the PWL sources: slope[k] = (v[k+1] - v[k]) / (t[k+1] - t[k]) for a
// segment of positive width inside one source, else 0; key[k] orders like t[k] (ordering as
// unsigned integers: sign-magnitude flipped), so the device searches with integer compares.
void pwl_aux(const std::vector<int64_t>& ptr, const std::vector<double>& t, const std::vector<double>& v,
             std::vector<double>* slope, std::vector<unsigned long long>* key);
pg_status build_packed(const pg_netlist* nl, Packed* out, std::string* why, int32_t lattice_policy,
                       int32_t colouring = PG_COLOUR_AUTO);

// Lattice inner solve chosen automatically (lattice_sweeps = 0): k = 3 block sweeps per
// barrier for lattices of 2-3 layers, and for single-layer lattices small enough that a
// round is about one tile pass (up to kSmallLattice nodes), where several sweeps per
// barrier pay; larger single-layer grids run the point SOR faster.
constexpr int32_t kSmallLattice = 200000;
inline int32_t auto_lattice_k(int32_t lat_maxnl, int32_t n_nodes) {
    return lat_maxnl >= 2 || (lat_maxnl == 1 && n_nodes <= kSmallLattice) ? 3 : 0;
}
// Tile geometry of the lattice inner solve: a region of kLatSide columns by `rows` rows
// (34 or 66) whose tile owns (kLatSide - 4k) x (rows - 4k) interior columns for k exact
// sweeps per round (a ghost zone of 2k columns on every side), so that the columns its
// first half-sweep updates are exactly 32 x (rows - 2), 16 pairs of them per half-warp row.
constexpr int kLatSide = 34;
constexpr int kLatW = 36;                          // shared-memory row stride (floats)
constexpr int kLatArrays = 7;                      // delta, r, wE, wN, wU, Thomas m, 1/pivot
inline int lattice_tile_side(int k) { return kLatSide - 4 * k; }
inline int lattice_tile_rows(int k, int rows) { return rows - 4 * k; }
// Dynamic shared memory of one lattice region: kLatArrays arrays of nl layers of rows x kLatW
// elements of elem bytes (4 in mixed precision, 8 for the FP64 lattice solve).
inline size_t lattice_region_bytes(int rows, int nl, size_t elem = sizeof(float)) {
    return (size_t)kLatArrays * nl * rows * kLatW * elem;
}
// Refill the value-dependent parts of a packed grid (merged weights, grounded
// parts, capacitances, 1/L) from a netlist with the same topology.
pg_status refill_values(const pg_netlist* nl, Packed* P, std::string* why);

// ---------------------------------------------------------------- device side

// Everything one launch of the persistent kernel reads or writes.
struct DevGrid {
    int32_t n_pad, ncol, n_slices, n_real;
    const int32_t* colour_slice;   // [ncol + 1] first slice of each colour (device copy)
    const int64_t* slice_off;
    const int32_t* slice_w;
    const int32_t* slice_doff;
    const int32_t* dia_off;
    const int32_t* ell_col;
    const double* w64;
    const float* w32;
    const float* w32lo;      // w64 - w32 (FP32): w32 + w32lo carries w64 to about 2^-48
    const float* D32;        // D as an FP32 pair (D32 + D32lo), for the outer pass
    const float* D32lo;
    const double* D64;
    const double* invD64;
    const float* invD32;
    const double* ch;        // C_i / h
    const double* cinj;      // constant source injection: sum g Vk + h sum Vk / L
    const int32_t* orig;
    const int32_t* ld_ptr;
    const int32_t* ld_idx;
    int32_t n_src;           // PWL load sources
    // per source and terminal: the permuted node whose only load this source is (its total
    // load current is the source's, written directly), kLoadMulti for a node with several
    // loads (summed per node over ld_ptr / ld_idx), kLoadNone for a terminal that is not a node
    const int32_t* src_na;   // terminal the current leaves (its node's injection is -I)
    const int32_t* src_nb;   // terminal the current enters (+I)
    int32_t n_multi;         // permuted nodes with several loads
    const int32_t* multi_node;
    const int64_t* pwl_ptr;
    const double* pwl_t;
    const double* pwl_v;
    const double* pwl_s;                 // slope of the segment that starts at each breakpoint (0 if none)
    const unsigned long long* pwl_tk;    // order keys of the breakpoint times (integer search)
    int32_t n_l;
    const int32_t* ind_a;
    const int32_t* ind_b;
    const double* ind_hl;    // h / L
    const int32_t* ind_ptr;
    const int32_t* ind_idx;
    const double* vdd;
    // lattice form of the FP32 inner solve (caller order), or null
    int32_t n_lats;          // independent lattices, 4 ints each in lat_info: first id, nx, ny, nl
    const int32_t* lat_info;
    const int32_t* lat_tile0;   // [n_lats + 1] first tile of each lattice (for the round's tile size)
    int32_t lat_tiles;
    const int64_t* lat_col0;    // [n_lats + 1] first column (x, y) of each lattice
    int64_t lat_cols;
    const int32_t* node_lat;    // [n_pad] lattice of each permuted node, -1 for padding
    const float* lwE;        // weight to (x+1, y, l); 0 on the last column
    const float* lwN;        // weight to (x, y+1, l)
    const float* lwU;        // weight to (x, y, l+1)
    const float* lm;         // column block (via couplings): Thomas multiplier u_{l-1} / d'_{l-1} (0 for l = 0)
    const float* lip;        // column block: inverse Thomas pivot 1 / d'_l
    // the same five arrays in FP64, for the FP64 lattice inner solve (null in mixed precision)
    const double* lwE64;
    const double* lwN64;
    const double* lwU64;
    const double* lm64;
    const double* lip64;
    int32_t lat_rows;        // region rows of the lattice solve (34 or 66)
    int32_t lat_astride;     // floats per staged array in shared memory: max layers x rows x kLatW
    int32_t natural;         // 1: the permutation is the identity on the real nodes (padding after them)
    // connected components (independent sub-circuits, Fig. 1)
    int32_t n_comp;
    const int32_t* node_comp;   // [n_pad] component of each permuted node, -1 for padding
};

enum Mode : int32_t { kModeTransient = 0, kModeSolve = 1 };
constexpr int32_t kLoadNone = -1;      // src_na / src_nb: the terminal is ground or a source node
constexpr int32_t kLoadMulti = -2;     // src_na / src_nb: the node has several loads

struct DevState {
    double* v[3];            // rotating node-voltage buffers (permuted)
    double* il;              // inductor currents
    double* r64;             // FP64 residual b - M v
    float* r32;              // FP32 copy of the residual (mixed precision)
    double* d64[2];          // correction buffers (FP64 sweeps)
    float* d32[2];           // correction buffers (FP32 sweeps)
    const double* rhs;       // kModeSolve: right-hand side (permuted)
    double* inode;           // [2 x n_pad] total load current drawn from each node, (A_i^T I_s(S h))_i,
                             // slot S & 1 (transient mode); nodes without loads stay 0
    double* md;              // [n_pad] M (v(s) - v(s-1)) by the end of step s (incremental step start)
    double* dinode;          // [n_pad] slot S minus slot S - 1 of inode, written with slot S (the load
                             // change the incremental step start adds); nodes without loads stay 0
    int32_t* pwl_cur;        // [n_src] breakpoint segment of each source's latest evaluation (a hint:
                             // checked before use, any value is safe)
};

struct DevCtl {
    unsigned int* bar_count;
    unsigned int* bar_gen;
    int32_t* err;
    unsigned long long* red;        // [kRedSlots] max reductions (double bits)
    unsigned long long* blk_min;    // [2 * nblocks] per-block min keys (double bits, ordered)
    int32_t* blk_arg;               // [2 * nblocks]
    double* stats;                  // device statistics, see kStat*
    unsigned long long* lat_R;      // [2 * n_lats] per-lattice max |r| / D of the latest FP64 pass
    unsigned int* tile_ctr;         // lattice tiles handed out so far in the launch, modulo 2^32 (cleared before it)
    unsigned int* ld_flags;         // [4] ring: word S & 3 is nonzero if a load current changed
                                    // between (S-1) h and S h; null disables the damped warm start
};

enum Stat : int {
    kStatSteps = 0, kStatSweeps, kStatMaxSweeps, kStatOuter, kStatMaxOuter,
    kStatMaxBound, kStatFailedStep, kStatLastR,
    kStatTimeA, kStatTimeInner, kStatTimeOuter, kStatTimePost,   // ns on block 0's clock
    kStatLastOuter,                                              // outer passes of the last step
    kStatCount
};

struct RunParams {
    int32_t mode;
    int32_t mixed;            // 1: FP32 sweeps
    int32_t nsteps;
    int64_t step0;            // absolute index of the state at launch (time = step * h)
    double h;
    int32_t cur, prev, prev2; // buffer indices of v at launch: current (= step0), previous
    int32_t have_prev;        // previous step exists (for extrapolation)
    int32_t warm_extrap;
    double warm_theta_static; // extrapolation weight on steps whose last two load intervals are
                              // static (1: plain linear extrapolation on every step)
    double omega;
    double kappa;             // bound constant ||M^-1 D||_inf
    double target;            // per-step target on max |r_i| / D_i  (= step_tol / kappa)
    double inner_reduction;
    int32_t max_sweeps;
    int32_t max_outer;
    double slack;             // rounding allowance added to the certified bound
    long long timeout_ns;
    int32_t debug_flags;
    // outputs (device pointers, may be null)
    double* v_all;
    double* il_all;
    double* vmin;
    int32_t* vmin_node;
    int32_t n_probes;
    const int32_t* probes_perm;
    double* probe_v;
    double* solve_out;        // kModeSolve: x in caller numbering
    double* comp_vmin;        // [nsteps x n_comp] smallest voltage per component (keys until converted)
    // kModeSolve extras
    const double* x0;                              // initial guess (permuted) or null (x = 0)
    const unsigned long long* target_scale;        // if set, target *= this double (device)
    // transient extras
    double* v_perm_all;       // [nsteps x n_pad] voltages in permuted order (adjoint recompute)
    double* obj_partials;     // [nsteps x nblocks] per-block sums of softplus(vref - v - margin)^2
    double obj_vref, obj_margin;
    int32_t lat_k;            // > 0: lattice inner solve, lat_k exact red-black sweeps per round
    int32_t three_level;      // 1: right-hand side of Eq. 11 (state v(s-1), v(s-2); no i_l)
    int32_t jacobi;           // 1: damped-Jacobi inner sweeps instead of coloured SOR
    int32_t inc_start;        // 1: the residual and M d of the previous launch's last step are current
    int32_t prev_outer;       // outer passes of the step before the launch's first one (inc_start)
};

}  // namespace pg

// ---------------------------------------------------------------- launch helpers (pg_kernels.cu)
#include <cuda_runtime.h>

namespace pg {
// smem: dynamic shared memory of the launch (persistent_smem_bytes for the grid)
cudaError_t launch_persistent(bool mixed, const DevGrid& g, const DevState& st, const DevCtl& ctl,
                              const RunParams& rp, int blocks, int threads, size_t smem, cudaStream_t stream);
cudaError_t persistent_occupancy(bool mixed, int rows, int threads, size_t smem, int* blocks_per_sm);
// Dynamic shared memory the persistent kernel needs: the TMA stages of the FP32 point sweep,
// or (the same memory) the lattice region of `rows` rows and `nl` layers.
size_t persistent_smem_bytes(bool mixed, int rows, int nl);
cudaError_t launch_power_step(const DevGrid& g, const double* x, double* y, const unsigned long long* xmax_prev,
                              double* acc, unsigned long long* ymax, int blocks, cudaStream_t stream);
cudaError_t launch_lattice_power(const DevGrid& g, const double* x, double* y, const unsigned long long* xmax_prev,
                                 double* acc, unsigned long long* ymax, int blocks, cudaStream_t stream);
cudaError_t launch_permute_in(const int32_t* orig, const double* src, double fill, double* dst, int n_pad,
                              int n_sm, cudaStream_t stream);
cudaError_t launch_adjoint_rhs(const DevGrid& g, const double* v, const double* lam_next, const double* mu,
                               double* rhs, double vref, double margin, unsigned long long* scale_slot, int blocks,
                               cudaStream_t stream);
cudaError_t launch_adjoint_mu(const DevGrid& g, const double* lam_next, double* mu, int blocks, cudaStream_t stream);
cudaError_t launch_adjoint_lgrad(const DevGrid& g, const double* lam, const double* v, const double* mu,
                                 double* acc_L, int blocks, cudaStream_t stream);
cudaError_t launch_adjoint_grad(const DevGrid& g, const double* lam, const double* v, const double* v_prev,
                                double* acc_slot, double* acc_lv, double* acc_l, double* acc_dv, int blocks,
                                cudaStream_t stream);
}  // namespace pg
