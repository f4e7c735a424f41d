/* Red-black SOR for one backward-Euler step of a power grid, on all host cores.
 *
 * TEST AND BENCHMARK INFRASTRUCTURE ONLY.  This is the multicore CPU baseline of
 * the paper's method: the node update of Eq. 16 with the SOR blend of Eq. 17,
 * in a red-black node order.  It is timed beside the GPU path and shares no code
 * with the CUDA library.
 *
 * The step's nodal system M x = b is given by its diagonal D and its
 * off-diagonal couplings in CSR form (M = C/h + G + h L, an M-matrix by
 * Lemma 1).  The couplings are w_ij = -M_ij > 0.  Nodes are listed colour by
 * colour, and no two nodes of one colour are coupled, so the nodes of a colour
 * update independently: one OpenMP loop per colour.  The result is therefore
 * the same for any thread count.
 *
 * Every `check_every` sweeps the scaled residual
 *     R = max_i |b_i + sum_j w_ij x_j - D_i x_i| / D_i
 * is formed.  The solve stops once R <= target.  The caller derives `target`
 * from the certified rule: kappa R bounds the step's voltage error, with
 * kappa = ||M^-1 D||_inf.
 *
 * Returns the sweeps used, -1 if max_sweeps ran out, or -2 on a non-finite
 * residual.  *R_out receives the last residual formed.
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double scaled_residual(int n, const int* rowptr, const int* col, const double* w, const double* D,
                              const double* b, const double* x, int* nonfinite) {
    double R = 0.0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(max : R) reduction(| : bad)
    for (int i = 0; i < n; ++i) {
        double s = b[i] - D[i] * x[i];
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s += w[e] * x[col[e]];
        const double a = fabs(s) / D[i];
        if (isfinite(a)) {
            if (a > R) R = a;
        } else {
            bad = 1;
        }
    }
    *nonfinite = bad;
    return R;
}

int rbsor_step(int n, const int* rowptr, const int* col, const double* w, const double* D, const int* order,
               int n_first, const double* b, double* x, double omega, double target, int max_sweeps,
               int check_every, double* R_out) {
    if (check_every < 1) check_every = 1;
    {
        int bad = 0;
        const double R = scaled_residual(n, rowptr, col, w, D, b, x, &bad);   /* the warm start may do */
        *R_out = bad ? NAN : R;
        if (bad) return -2;
        if (R <= target) return 0;
    }
    for (int k = 1; k <= max_sweeps; ++k) {
        for (int c = 0; c < 2; ++c) {
            const int lo = c ? n_first : 0, hi = c ? n : n_first;
#pragma omp parallel for schedule(static)
            for (int q = lo; q < hi; ++q) {
                const int i = order[q];
                double s = b[i];
                for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s += w[e] * x[col[e]];
                x[i] += omega * (s / D[i] - x[i]);
            }
        }
        if (k % check_every == 0 || k == max_sweeps) {
            int bad = 0;
            const double R = scaled_residual(n, rowptr, col, w, D, b, x, &bad);
            *R_out = bad ? NAN : R;
            if (bad) return -2;
            if (R <= target) return k;
        }
    }
    return -1;
}

/* Threads an OpenMP parallel region gets (for the report). */
int rbsor_threads(void) {
    int t = 1;
#ifdef _OPENMP
#pragma omp parallel
    {
#pragma omp single
        t = omp_get_num_threads();
    }
#endif
    return t;
}

/* Thread count of the following parallel regions (0 or less: leave as is). */
void rbsor_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ---- column-block form on a lattice ------------------------------------------------
 *
 * Nodes (x, y, l) with id (l ny + y) nx + x, couplings only between lattice
 * neighbours: wE[i] to (x + 1, y, l), wN[i] to (x, y + 1, l), wU[i] to
 * (x, y, l + 1).  The block of column (x, y) is its nl layers coupled by the
 * vias.  The block update solves that tridiagonal block exactly, against the
 * in-plane neighbours of the other colour (columns are coloured by the parity
 * of x + y).  This is block Gauss-Seidel / SOR over a partition of the SPD
 * system, which converges for 0 < omega < 2.  Tm and Tip are the block's
 * elimination factors (multiplier and reciprocal pivot per layer).
 */
#define RBSOR_MAX_LAYERS 8

static double lattice_residual(int nx, int ny, int nl, const double* wE, const double* wN, const double* wU,
                               const double* D, const double* b, const double* x, int* nonfinite) {
    const long plane = (long)nx * ny, n = plane * nl;
    double R = 0.0;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(max : R) reduction(| : bad)
    for (long i = 0; i < n; ++i) {
        const int xx = (int)(i % nx), yy = (int)((i / nx) % ny), ll = (int)(i / plane);
        double s = b[i] - D[i] * x[i];
        if (xx + 1 < nx) s += wE[i] * x[i + 1];
        if (xx > 0) s += wE[i - 1] * x[i - 1];
        if (yy + 1 < ny) s += wN[i] * x[i + nx];
        if (yy > 0) s += wN[i - nx] * x[i - nx];
        if (ll + 1 < nl) s += wU[i] * x[i + plane];
        if (ll > 0) s += wU[i - plane] * x[i - plane];
        const double a = fabs(s) / D[i];
        if (isfinite(a)) {
            if (a > R) R = a;
        } else {
            bad = 1;
        }
    }
    *nonfinite = bad;
    return R;
}

int rbsor_block_step(int nx, int ny, int nl, const double* wE, const double* wN, const double* wU,
                     const double* D, const double* Tm, const double* Tip, const double* b, double* x,
                     double omega, double target, int max_sweeps, int check_every, double* R_out) {
    if (nl < 1 || nl > RBSOR_MAX_LAYERS) return -3;
    if (check_every < 1) check_every = 1;
    const long plane = (long)nx * ny;
    int bad = 0;
    double R = lattice_residual(nx, ny, nl, wE, wN, wU, D, b, x, &bad);
    *R_out = bad ? NAN : R;
    if (bad) return -2;
    if (R <= target) return 0;
    for (int k = 1; k <= max_sweeps; ++k) {
        for (int c = 0; c < 2; ++c) {
#pragma omp parallel for schedule(static)
            for (int yy = 0; yy < ny; ++yy) {
                for (int xx = (c + yy) & 1; xx < nx; xx += 2) {
                    double f[RBSOR_MAX_LAYERS], z[RBSOR_MAX_LAYERS];
                    const long i0 = (long)yy * nx + xx;
                    for (int l = 0; l < nl; ++l) {
                        const long i = i0 + l * plane;
                        double s = b[i];
                        if (xx + 1 < nx) s += wE[i] * x[i + 1];
                        if (xx > 0) s += wE[i - 1] * x[i - 1];
                        if (yy + 1 < ny) s += wN[i] * x[i + nx];
                        if (yy > 0) s += wN[i - nx] * x[i - nx];
                        f[l] = s;
                    }
                    for (int l = 1; l < nl; ++l) f[l] += Tm[i0 + l * plane] * f[l - 1];
                    z[nl - 1] = f[nl - 1] * Tip[i0 + (nl - 1) * plane];
                    for (int l = nl - 2; l >= 0; --l)
                        z[l] = (wU[i0 + l * plane] * z[l + 1] + f[l]) * Tip[i0 + l * plane];
                    for (int l = 0; l < nl; ++l) {
                        const long i = i0 + l * plane;
                        x[i] += omega * (z[l] - x[i]);
                    }
                }
            }
        }
        if (k % check_every == 0 || k == max_sweeps) {
            R = lattice_residual(nx, ny, nl, wE, wN, wU, D, b, x, &bad);
            *R_out = bad ? NAN : R;
            if (bad) return -2;
            if (R <= target) return k;
        }
    }
    return -1;
}
