/*
 * pg.h -- C ABI of the GB300 power-grid transient library (libpg).
 *
 * What it computes (Yang, Wang, Azevedo, Wang, "An Efficient Topology-Based
 * Algorithm for Transient Analysis of Power Grid"):
 *
 *   For an RC or RLC power grid with trivial nodes v, ideal supply nodes v_d,
 *   grounded capacitors C, conductance matrix G (pads included), inductor
 *   matrix L = A_l^T Ldiag^-1 A_l and piecewise-linear load currents I_s,
 *   each backward-Euler step of length h solves the SPD system
 *
 *       M v(t+h) = (C/h) v(t) - A_l^T i_l(t) - A_i^T I_s(t+h) - G_s v_d - h L_s v_d,
 *       M = C/h + G + h L                                   (Eq. 2, Eq. 10-11)
 *
 *   then advances the inductor currents
 *
 *       i_l(t+h) = i_l(t) + h Ldiag^-1 (A_l v(t+h) + A_ls v_d)     (Eq. 10).
 *
 *   The system is solved without assembling M, by the node-local update of
 *   Eq. 15-17 (Gauss-Seidel / SOR, Theorem 1) in red-black or multicolour
 *   order on the GPU.  The signs of the source terms follow KVL (Eq. 7).
 *
 * Conventions shared by every call:
 *   - Units are SI: S, F, H, s, A, V.
 *   - A branch terminal is an int32: t >= 0 is trivial node t, PG_GROUND (-1)
 *     is ground, PG_SOURCE(k) = -2-k is source node k (the split of the
 *     incidence matrix into A and A_s, Eq. 4-5).
 *   - "device" pointers are CUDA device (or managed) memory on the grid's
 *     device; "host" pointers are ordinary or pinned host memory.  The library
 *     never frees memory it did not allocate.
 *   - Calls are ordered on the grid's stream (pg_set_stream); calls that
 *     return statistics synchronise that stream before returning.
 *   - Errors are returned as pg_status; pg_status_str names them.  A failed
 *     call leaves the grid usable unless it returned PG_ERR_CUDA.
 */
#ifndef PG_H
#define PG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PG_GROUND (-1)
#define PG_SOURCE(k) (-2 - (k))

typedef enum pg_status {
    PG_OK = 0,
    PG_ERR_INVALID_ARG = 1,    /* bad index, non-positive element value, bad option */
    PG_ERR_FLOATING_NODE = 2,  /* topological assumption 2 or 3 violated (Section III-B) */
    PG_ERR_OOM = 3,            /* device or host allocation failed */
    PG_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    PG_ERR_NOT_CONVERGED = 5,  /* relaxation hit its sweep cap or produced a non-finite value */
    PG_ERR_TIMEOUT = 6,        /* the device-wide barrier exceeded its time limit */
    PG_ERR_UNSUPPORTED = 7     /* input outside the per-node form, e.g. node-to-node capacitor */
} pg_status;

/*
 * Netlist (Section III-A, Eq. 4-8).  Structure of arrays; every branch is
 * oriented a -> b.  Capacitors must have exactly one trivial terminal (the
 * grounded C_i of Eq. 12).  A current source drives its PWL current from a
 * to b through the source, so a load drawing I(t) from node k is a = k,
 * b = PG_GROUND.  Source e owns PWL breakpoints i_t/i_v[i_ptr[e] .. i_ptr[e+1]);
 * times must be non-decreasing; the value is held constant before the first
 * and after the last breakpoint and is linear in between.
 * lat_nx/lat_ny/lat_nl: optional lattice shape (node (x,y,l) = (l*ny+y)*nx+x)
 * or 0.  n_lat / lat_desc: optional list of n_lat lattices (independent grids
 * side by side), lat_desc[4k .. 4k+3] = (first node id, nx, ny, nl), node
 * (x, y, l) of lattice k having id first + (l*ny + y)*nx + x.  When the lattices
 * cover every node and every branch joins lattice neighbours, the mixed-precision
 * inner solve can use the lattice form (see pg_options.lattice_sweeps); results
 * do not depend on it.
 * pg_create_grid copies everything; the caller may free the arrays after it
 * returns.  All pointers are host pointers.
 */
typedef struct pg_netlist {
    int32_t n_nodes;
    int32_t n_sources;
    const double* vdd;                 /* [n_sources] source-node voltages */
    int64_t n_r; const int32_t* r_a; const int32_t* r_b; const double* r_g;
    int64_t n_c; const int32_t* c_a; const int32_t* c_b; const double* c_val;
    int64_t n_l; const int32_t* l_a; const int32_t* l_b; const double* l_val;
    int64_t n_i; const int32_t* i_a; const int32_t* i_b;
    const int64_t* i_ptr;              /* [n_i + 1]; i_ptr[n_i] (all breakpoints) <= 2^31 - 2 */
    const double* i_t; const double* i_v;
    int32_t lat_nx, lat_ny, lat_nl;
    int32_t n_lat;
    const int32_t* lat_desc;           /* [4 * n_lat] or NULL */
} pg_netlist;

typedef enum pg_precision {
    PG_PREC_FP64 = 0,   /* FP64 sweeps */
    PG_PREC_MIXED = 1   /* FP32 sweeps on the correction, FP64 residual and defect correction */
} pg_precision;

#define PG_DEBUG_SKIP_ARRIVAL 1  /* test hook: block 0 never arrives at the first device barrier */

typedef struct pg_options {
    int32_t precision;        /* pg_precision */
    double omega;             /* SOR factor (Eq. 17) in (0, 2); 0 = Young's formula from an estimated
                                 Jacobi spectral radius, with omega - 1 taken 1 % high */
    double tol;               /* target max-abs voltage error of every step against the exact
                                 backward-Euler trajectory, V (0 -> 1e-6) */
    double step_tol;          /* per-step solve target, V; 0 -> derived from tol: RC grids use
                                 0.9 tol / kacc (see pg_run_stats), grids with inductors 1e-4 tol */
    int32_t max_sweeps;       /* cap on relaxation sweeps per step (0 -> 20000) */
    int32_t warm_start;       /* 0: V(s-1) as in Algorithm 1; 1: linear extrapolation;
                                 2: linear extrapolation while the load currents change, damped to
                                 V(s-1) + (V(s-1) - V(s-2)) / 2 once they have been constant for
                                 two steps (explicit form; the three-level form extrapolates fully);
                                 -1 (default): 2 for grids without inductors, 1 with inductors
                                 (an RC grid relaxes monotonically once its loads are quiet; an
                                 RLC grid keeps ringing, and full extrapolation follows it) */
    double inner_reduction;   /* PG_PREC_MIXED: residual reduction asked of one FP32 inner solve;
                                 0 (default) -> 1e-1 for netlists of more than 8 lattices (a batch:
                                 more frequent FP64 passes let converged grids drop out sooner), else
                                 1e-3; an inner solve also ends when it stalls */
    int32_t threads_per_block;/* 0 -> 256 */
    int32_t blocks_per_sm;    /* 0 -> as many as fit */
    double barrier_timeout_s; /* device barrier time limit (0 -> 2 s) */
    int32_t debug_flags;      /* PG_DEBUG_* test hooks; 0 in production */
    int32_t lattice_sweeps;   /* On a lattice netlist (lat_nx/ny/nl given, <= 3 layers, branches only
                                 between lattice neighbours) the inner solve (FP32 in PG_PREC_MIXED, FP64
                                 otherwise) becomes column-block red-black SOR (each (x, y) column's
                                 layers solved exactly) on shared-memory tiles with ghost zones, k exact
                                 block sweeps per device barrier.  k > 0 (<= 7): that k; 0 (default):
                                 k = 3 for 2-3 layers and for single-layer lattices of at most 200k
                                 nodes, in FP64 only for netlists of at most 8 lattices, else off;
                                 < 0: off (neighbour-list point SOR) */
    int32_t jacobi;           /* 0 (default): coloured Gauss-Seidel / SOR inner sweeps (Eq. 16-17);
                                 1: damped Jacobi, every node updated from the previous iterate with
                                 omega <= 1 (default 1), one device barrier per sweep; no lattice solve */
    int32_t form;             /* PG_FORM_EXPLICIT (default): inductor currents kept as state (Eq. 10);
                                 PG_FORM_THREE_LEVEL: the three-level recurrence of Eq. 11 / Eq. 14,
                                 whose state is v(s-1), v(s-2) alone.  A step from a single level (the
                                 DC point, pg_set_state) is an ordinary backward-Euler step with the
                                 state's inductor currents; pg_initial_conditions gives the paper's two
                                 levels instead.  No il_all output; step errors add up over the steps
                                 instead of decaying, so err_bound is NaN */
    int32_t colouring;        /* update order of the neighbour-list (point) sweeps, which Section IV-A
                                 leaves open (any order converges, Theorem 1):
                                 PG_COLOUR_AUTO (0, default): red-black where the netlist is
                                 bipartite, else greedy multicolour; PG_COLOUR_RED_BLACK: the same,
                                 named; PG_COLOUR_FOUR: on lattice netlists four colours
                                 ((x + l) mod 2) + 2 (y mod 2), swept in that order (omega as for
                                 red-black), elsewhere greedy multicolour.  The lattice inner solve
                                 keeps its column red-black order whatever this says */
    int32_t tile_rows;        /* rows of the lattice inner solve's shared-memory region: 0 (default)
                                 or 34 (34 x 34 columns), or 66 (34 columns x 66 rows, one block per
                                 SM: twice the interior per region load) */
} pg_options;

#define PG_COLOUR_AUTO 0
#define PG_COLOUR_RED_BLACK 1
#define PG_COLOUR_FOUR 2

#define PG_FORM_EXPLICIT 0
#define PG_FORM_THREE_LEVEL 1

/* Fill *opt with the defaults listed above. */
void pg_default_options(pg_options* opt);

typedef struct pg_grid pg_grid;

/*
 * Validate a netlist against the paper's topological assumptions
 * (Section III-B: every trivial node has a non-current-source branch; each
 * connected sub-circuit, Fig. 1, reaches a source or ground through a
 * resistor or inductor), colour it, pack it for the device, and allocate the
 * grid's device memory on the current CUDA device.  *out receives the handle
 * (NULL on error).  opt may be NULL for defaults.
 * Errors: PG_ERR_INVALID_ARG, PG_ERR_FLOATING_NODE, PG_ERR_UNSUPPORTED,
 * PG_ERR_OOM, PG_ERR_CUDA.
 */
pg_status pg_create_grid(const pg_netlist* nl, const pg_options* opt, pg_grid** out);

/* Free every resource of the grid (synchronises its stream).  NULL is a no-op. */
void pg_destroy(pg_grid* g);

/* Static string naming a status code. */
const char* pg_status_str(pg_status s);

/* Detail message of the last failing call on the calling thread (valid until
 * that thread's next failing call). */
const char* pg_last_error(void);

/* Order subsequent work on this cudaStream_t (NULL = legacy default stream). */
pg_status pg_set_stream(pg_grid* g, void* stream);

/*
 * Connected components: sub-circuits that share no element (Section III-B,
 * Fig. 1), numbered in the order of their smallest node id.  *n_comp receives
 * the count; comp_of (host, [n_nodes], may be NULL) each node's component.
 */
pg_status pg_grid_components(const pg_grid* g, int32_t* n_comp, int32_t* comp_of);

/* Node count, inductor count, colour count and permuted (padded) node count. */
pg_status pg_grid_info(const pg_grid* g, int32_t* n_nodes, int32_t* n_inductors,
                       int32_t* n_colours, int32_t* n_padded);

/*
 * Set the transient state: node voltages v[n_nodes] and inductor currents
 * il[n_l] (either may be NULL: NULL v keeps the DC operating point rule, NULL il
 * means zero currents), at step index `step` (time = step * h).  Pointers are
 * host memory when on_host != 0, else device memory.
 */
pg_status pg_set_state(pg_grid* g, const double* v, const double* il, int64_t step, int32_t on_host);

/* Copy the current state out (same conventions); *step receives the step index. */
pg_status pg_get_state(pg_grid* g, double* v, double* il, int64_t* step, int32_t on_host);

/* Forget the state: the next pg_transient starts from the DC operating point at t = 0. */
pg_status pg_reset(pg_grid* g);

/*
 * Replace the PWL breakpoint values of the current sources (same i_ptr layout
 * as the netlist).  i_t and/or i_v may be NULL to keep them.  Host or device
 * memory per on_host.  Used to run many current scenarios on one grid.
 */
pg_status pg_update_sources(pg_grid* g, const double* i_t, const double* i_v, int32_t on_host);

/* Per-step outputs of pg_transient.  Any pointer may be NULL.  Rows are in
 * step order, columns in the caller's node numbering. */
typedef struct pg_output {
    int32_t on_host;      /* 0: the pointers below are device memory; 1: host memory */
    double* v_all;        /* [nsteps x n_nodes] node voltages after each step */
    double* il_all;       /* [nsteps x n_l] inductor currents after each step */
    double* vmin;         /* [nsteps] smallest node voltage (worst IR drop) */
    int32_t* vmin_node;   /* [nsteps] node attaining it (smallest id on ties) */
    int32_t n_probes;
    const int32_t* probes;/* [n_probes] node ids (same memory kind as the outputs) */
    double* probe_v;      /* [nsteps x n_probes] */
    double* comp_vmin;    /* [nsteps x n_components] smallest voltage of each connected component
                             (independent sub-circuit, Fig. 1; numbering of pg_grid_components) */
} pg_output;

typedef struct pg_run_stats {
    int64_t steps_done;
    int64_t total_sweeps;       /* relaxation sweeps summed over the steps */
    int32_t max_sweeps_step;    /* most sweeps any single step needed */
    int32_t max_outer_step;     /* most defect-correction passes any step needed */
    int64_t total_outer;
    double max_step_bound;      /* largest certified per-step error bound, V */
    double err_bound;           /* bound on the accumulated error, V (RC): kacc times the largest
                                   per-step bound since the state was set, the DC solve included */
    int64_t failed_step;        /* step index of a failure, -1 if none */
    double omega;               /* SOR factor used */
    double rho_jacobi;          /* estimated Jacobi spectral radius (lower bound) */
    double kappa;               /* upper bound of ||M^-1 D||_inf used by the stopping rule */
    double q;                   /* upper bound of ||M^-1 C/h||_inf (RC error gain per step) */
    double step_tol;            /* per-step target actually used, V */
    double device_ms;           /* device time of the persistent launch(es), ms */
    double kacc;                /* RC: upper bound of ||1 + (G + G0)^-1 (C/h) 1||_inf, the factor
                                   turning per-step errors into the accumulated error; inf for RLC */
    int32_t lattice_sweeps;     /* inner solve: 0 = neighbour-list point SOR, k > 0 = lattice
                                   column-block SOR with k sweeps per device barrier */
    double phase_ms[4];         /* device time of the launch by phase, ms: step start (RHS, warm start,
                                   FP64 residual), inner solves, FP64 outer passes, step end (inductor
                                   update, outputs); each ends at a device barrier */
} pg_run_stats;

/*
 * Run nsteps backward-Euler steps of length h (Algorithm 1) from the current
 * state; if no state is set, first compute the DC operating point at t = 0
 * (capacitors open, inductors carrying i_l(0) = 0; Section IV-B) and take it
 * as step 0.  Changing h re-assembles the per-h coefficients (D, weights,
 * C/h, h/L) and the stopping-rule constants.  Each step is solved until its
 * certified error bound is below the per-step target.  out and stats may be
 * NULL.  Errors: PG_ERR_INVALID_ARG, PG_ERR_NOT_CONVERGED (stats->failed_step
 * set; the state is left at the last good step), PG_ERR_TIMEOUT, PG_ERR_CUDA.
 */
pg_status pg_transient(pg_grid* g, double h, int32_t nsteps, const pg_output* out,
                       pg_run_stats* stats);

/*
 * Option search by timed trials (the paper leaves omega and the sweep schedule
 * open, Section IV).  Builds the netlist once per structural candidate (lattice
 * block sweeps per barrier k in {off, 1, 2, 3} when the netlist describes
 * lattices and the precision is mixed; with k > 0 region rows in {34, 66}, with
 * the point sweeps colouring in {automatic, four colours} on lattice netlists;
 * blocks per SM in {as many as fit, 1})
 * and, on each, times trial_steps transient steps from the DC point (best of
 * two runs, CUDA events) for every runtime candidate (inner reduction in {1e-3,
 * 1e-2, 1e-1} when mixed; omega - 1 of the automatic value scaled by {1, 1.01,
 * 0.98} when omega is not fixed), then damped Jacobi (jacobi = 1, omega 1) with
 * at most 4x the winner's sweeps per step.  Every trial runs under the certified
 * stopping rule of `base` (tol), so only time is compared.  `base` (NULL ->
 * defaults) supplies every other field.  On success *best is `base` with
 * lattice_sweeps, tile_rows, colouring, blocks_per_sm, inner_reduction, jacobi and omega (0 = the automatic value;
 * a scaled value is tied to this h) set to the fastest candidate and *best_ms
 * (may be NULL) to its trial time.  stream: cudaStream_t for the trials or
 * NULL.  Errors: PG_ERR_INVALID_ARG, or the last failure when no candidate ran.
 */
pg_status pg_autotune(const pg_netlist* nl, const pg_options* base, double h, int32_t trial_steps, void* stream,
                      pg_options* best, double* best_ms);

/* Size in bytes of the device record pg_transient_async writes (dstats). */
#define PG_ASYNC_STATS_BYTES 128

/*
 * pg_transient as pure stream-ordered work, for replay under a CUDA graph (the
 * paper's Algorithm 1 loop as one persistent launch; the graph packaging has no
 * counterpart in the paper).  Runs nsteps backward-Euler steps (Eq. 2 / Eq. 10)
 * starting at step 0 from v0 (device, [n_nodes], caller numbering) with zero
 * inductor currents; v0 = NULL puts every node at the supply voltage, which is
 * the DC point when all loads are zero at t = 0 (needs a single supply level).
 * Only memsets, kernel launches and device-to-device copies are issued on the
 * grid's stream and nothing waits on the host, so the call can be captured
 * (cudaStreamBeginCapture, torch.cuda.graph) and the graph replayed: each replay
 * reads the source waveforms and element values current at replay time
 * (pg_update_sources between replays), but the grid must be assembled for h
 * beforehand (pg_transient(g, h, 0, NULL, NULL)) and must not be used by another
 * call while a replay runs.  out: device pointers only (on_host = 0, no probes).
 * dstats (device, PG_ASYNC_STATS_BYTES, may be NULL) receives the launch's
 * statistics and error word; decode it with pg_async_stats.  The grid's host
 * transient state is left undefined: the next pg_transient starts from the DC
 * point.  Errors at the call: PG_ERR_INVALID_ARG, PG_ERR_CUDA.
 */
pg_status pg_transient_async(pg_grid* g, double h, int32_t nsteps, const double* v0, const pg_output* out,
                             void* dstats);

/*
 * Decode a record written by pg_transient_async once the work that wrote it has
 * finished (synchronise the stream the graph was replayed on first).  Returns
 * the launch's status (PG_OK, PG_ERR_NOT_CONVERGED, PG_ERR_TIMEOUT); stats may be
 * NULL (device_ms is 0: not timed).
 */
pg_status pg_async_stats(pg_grid* g, const void* dstats, pg_run_stats* stats);

/*
 * The initial-condition procedure of Section IV-B: (1) DC at t = 0 with every
 * capacitor a voltage source v_c(0) and every inductor a current source i_l(0);
 * (2) v_c(h) = v_c(0) + h i_c(0) / C, i_l(h) = i_l(0) + h v_l(0) / L;
 * (3) DC at t = h with the capacitors at v_c(h) and the inductors carrying
 * i_l(h).  Both DC analyses are relaxation solves of derived grids (the
 * capacitor nodes fixed) to the grid's per-step target.  The grid's state
 * becomes v(h) at step 1 with v(0) as the previous level and i_l(h) as the
 * inductor currents, which is what both forms continue from.  vc0 ([n_c], one
 * voltage per capacitor element; parallel capacitors on one node must agree) or
 * NULL for the DC operating point with the capacitors open; il0 ([n_l]) or NULL
 * for zero; host or device per on_host.  Errors: PG_ERR_INVALID_ARG,
 * PG_ERR_FLOATING_NODE (a node with no conductive path to a source, a capacitor
 * node or ground once the inductors are current sources), PG_ERR_CUDA.
 */
pg_status pg_initial_conditions(pg_grid* g, double h, const double* vc0, const double* il0, int32_t on_host);

/*
 * One backward-Euler step: the body of Algorithm 1's time loop once (the RHS of
 * Eq. 2 / Eq. 10 at t = (s + 1) h, the warm start from v(s), relaxation by
 * Eq. 16-17 to the certified per-step target, the inductor update of Eq. 10).
 * Same as pg_transient with nsteps = 1; v_out (device, [n_nodes]) may be NULL.
 * Errors as pg_transient.
 */
pg_status pg_step(pg_grid* g, double h, double* v_out, pg_run_stats* stats);

/*
 * Solve M x = b once for the assembled h (b, x: device, [n_nodes], caller
 * numbering) to the absolute error target `tol` (V-like units of x), starting
 * from x = 0: the relaxation of Section IV (Eq. 14-17, with the coefficients of
 * Eq. 14 for this h) on its own, outside the time loop, under the same
 * certified stopping rule as a step.  b is read on the
 * grid's stream; the first call allocates one [n_nodes]-sized device buffer that
 * the grid keeps.  tol must exceed kappa * 1e-13 (the rounding allowance of the
 * stopping rule), else PG_ERR_INVALID_ARG.
 */
pg_status pg_solve(pg_grid* g, double h, const double* b, double* x, double tol,
                   pg_run_stats* stats);

/*
 * Replace element values on the same topology (netlist order; any pointer may
 * be NULL to keep those values).  The next call re-assembles the per-h
 * coefficients.  Host or device memory per on_host.  Errors:
 * PG_ERR_INVALID_ARG for a non-positive or non-finite value.
 */
pg_status pg_update_values(pg_grid* g, const double* r_g, const double* c_val, const double* l_val,
                           int32_t on_host);

/* Objective of pg_adjoint. */
#define PG_OBJ_SOFTPLUS_DROP 0   /* J = sum_{s=1..nsteps} sum_i softplus(vref - v_{s,i} - margin)^2 */

typedef struct pg_objective {
    int32_t kind;     /* PG_OBJ_SOFTPLUS_DROP */
    double vref;      /* reference voltage, V (the supply) */
    double margin;    /* tolerated drop before the penalty grows, V */
} pg_objective;

/*
 * Gradient of a worst-IR-drop objective over an RC or RLC transient (no
 * counterpart in the paper; it differentiates the backward-Euler recurrence the
 * paper solves, Eq. 2 / Eq. 10 with explicit inductor currents).  Runs nsteps
 * steps from the DC operating point with a checkpoint (v_s, v_{s-1}, i_l) every
 * ckpt_every steps (0 -> 50), then the discrete adjoint backwards:
 *     mu_s = mu_{s+1} - A_l lambda_{s+1}                      (inductors; mu_nsteps = 0)
 *     M lambda_s = dJ/dv_s + (C/h) lambda_{s+1} + h A_l^T Ldiag^-1 mu_s,  lambda_{nsteps+1} = 0,
 * each solve by the same relaxation kernel (relative residual 1e-9), recomputing
 * each segment's states from its checkpoint.  Outputs (netlist order, each may be
 * NULL): dJ_dG[n_r] = -sum_s (lambda_a - lambda_b)(v_a - v_b) per resistor, plus
 * the DC point's own adjoint term when the DC point depends on the resistors;
 * dJ_dC[n_c] = -sum_s lambda_k (v_{s,k} - v_{s-1,k}) / h per capacitor;
 * dJ_dL[n_l] = (h / L^2) sum_s u_s (lambda_a - lambda_b - mu_s) per inductor,
 * u_s its branch voltage.  *J (host) receives the objective.  Host or device
 * outputs per on_host.  The grid's transient state is reset afterwards.  Errors:
 * PG_ERR_UNSUPPORTED for the three-level form; otherwise as pg_transient.
 */
pg_status pg_adjoint(pg_grid* g, double h, int32_t nsteps, const pg_objective* obj, int32_t ckpt_every,
                     double* J, double* dJ_dG, double* dJ_dC, double* dJ_dL, int32_t on_host, pg_run_stats* stats);

/*
 * pg_solve without device allocations.  The paper has no counterpart: this
 * serves callers that cannot call cudaMalloc when they solve, e.g. processes
 * whose device memory is reserved up front by another allocator or capped,
 * or steady-state loops that must not allocate.  Same arguments, result and
 * errors as pg_solve, with these differences:
 *   - All scratch (permuted right-hand side, iterate, residuals, corrections,
 *     barrier and reduction words, statistics) lives in one file-scope device
 *     array of 32 MiB inside the library.  CUDA loads the array's module, and
 *     reserves its memory on a device, when its address is first looked up on
 *     that device (cudaGetSymbolAddress, with the device current).  The first
 *     pg_create_grid on each device makes that lookup, so the reservation
 *     belongs to grid creation; the device then holds the array until the
 *     process exits.  If the lookup failed there, this call returns
 *     PG_ERR_CUDA naming the cause, and never retries it.  Grids whose scratch
 *     would not fit (about 830k padded nodes in FP64, 930k in mixed precision)
 *     are rejected with PG_ERR_INVALID_ARG and a message naming the limit.
 *   - The coefficients for h must already be assembled (one earlier pg_solve
 *     or pg_transient with the same h); otherwise PG_ERR_INVALID_ARG.  The
 *     call itself allocates no device memory, loads no module and calls no
 *     allocating routine.  Its statistics are filled exactly as pg_solve's.
 *   - Every call shares the one array and it keeps the last call's contents;
 *     the call clears what must start at zero.  Calls that overlap on the GPU
 *     (other streams, other threads, other grids) race on it: serialise them.
 * b and x are device pointers in the caller's node numbering.
 */
pg_status pg_solve_noalloc(pg_grid* g, double h, const double* b, double* x, double tol,
                           pg_run_stats* stats);

/* Outputs of pg_transient_scenarios (each may be NULL). */
typedef struct pg_scenario_output {
    int32_t on_host;          /* 1: the pointers below are host memory, 0: device memory */
    double* v_all;            /* [nsteps][n_scen][n_nodes] every scenario's node voltages */
    double* vmin;             /* [nsteps][n_scen] every scenario's smallest node voltage */
} pg_scenario_output;

/*
 * Many load scenarios of one RC grid in one persistent launch: n_scen right-hand
 * sides of the same backward-Euler system (Eq. 2, M = C/h + G + G0), relaxed
 * together (Eq. 16-17) so that every coefficient is read once for all of them.
 * Scenario k's load currents are the grid's PWL sources with the breakpoint times
 * of the netlist and the breakpoint values i_v[k * n_points .. (k + 1) * n_points)
 * (n_points = the netlist's i_ptr[n_i]; host or device memory, found by address).
 * Every scenario starts at v = Vdd, the DC point of a grid with one supply level, no
 * resistor to ground and no load current at t = 0, and runs nsteps steps of length h
 * with the grid's precision, tolerance and stopping rule; a step ends when the
 * certified bound of its worst scenario meets the step target, so stats (the work
 * of all scenarios together; err_bound covers every scenario) reads as for
 * pg_transient.  The grid's own transient state is reset.  The paper solves one
 * right-hand side per step; sharing the matrix across load patterns has no
 * counterpart there.  Errors: PG_ERR_INVALID_ARG; PG_ERR_UNSUPPORTED for grids with
 * inductors, the three-level form, grids built for the lattice inner solve (create
 * them with lattice_sweeps = -1), or a start other than v = Vdd; PG_ERR_OOM;
 * PG_ERR_NOT_CONVERGED; PG_ERR_TIMEOUT; PG_ERR_CUDA.
 */
pg_status pg_transient_scenarios(pg_grid* g, double h, int32_t nsteps, int32_t n_scen, const double* i_v,
                                 const pg_scenario_output* out, pg_run_stats* stats);

/*
 * Row-block domain decomposition of one lattice grid (the device half).  The node
 * update of Eq. 16-17 reads only the node and its neighbours, so a grid cut along y
 * into blocks of rows (all layers of each column kept together) can be relaxed
 * block by block: each block holds its rows plus one halo row on each side, and
 * the halos are refreshed from the neighbouring blocks between half-sweeps.  The
 * red-black order puts the colours in separate half-sweeps, so the decomposed
 * iteration makes exactly the updates of the undecomposed one (a single block
 * holding every row).  Layout: node (x, local row k, layer l) at (l*R + k)*nx + x,
 * with R the row count of the array.  All pointers are device memory owned by the
 * caller, FP64.
 */
typedef struct pg_row_block {
    int32_t nx, rows, nl;     /* the block: rows [y0, y0 + rows) of an nx-wide lattice, nl layers */
    int32_t y0;               /* its first global row: colours are the parity of x + y + l */
    const double* w_e;        /* [nl][rows][nx] conductance to (x + 1, y, l); 0 on the last column */
    const double* w_n;        /* [nl][rows + 1][nx] row k couples local rows k and k + 1 (row 0: the
                                 halo below and the first row; row rows: the last row and the halo
                                 above); 0 across the grid's outer edges */
    const double* w_u;        /* [nl][rows][nx] conductance to layer l + 1; 0 on the top layer */
    const double* inv_d;      /* [nl][rows][nx] 1 / D of Eq. 14 */
    const double* rhs;        /* [nl][rows][nx] right-hand side */
    double* x;                /* [nl][rows + 2][nx] iterate; local rows 0 and rows + 1 are the halos
                                 (zero at the grid's outer edges) */
} pg_row_block;

/*
 * One colour half-sweep (Eq. 16-17) over a block: every node of the colour (x + y + l
 * of that parity) in rows 1..rows is over-relaxed with factor omega in (0, 2); the
 * neighbour sum is formed in a fixed order.  *max_update (device, a non-negative
 * double the caller zeroes) receives the largest unrelaxed update |(rhs + sum)/D - x|
 * merged by max.  Stream-ordered on `stream` (a cudaStream_t, or NULL).  The paper
 * has no multi-GPU schedule: this is the device step of the decomposition that
 * Eq. 16-17's locality allows.  Errors: PG_ERR_INVALID_ARG (null array, empty
 * block, colour not 0 or 1, omega outside (0, 2)), PG_ERR_CUDA (launch).
 */
pg_status pg_block_half_sweep(const pg_row_block* blk, int32_t colour, double omega, double* max_update,
                              void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PG_H */
