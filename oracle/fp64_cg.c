/* Plain FP64 matrix-free kernel MVM and preconditioned CG on the host cores.
 *
 * TEST INFRASTRUCTURE ONLY: part of the oracle package.  Only the tests, the
 * smoke() self-check and the benchmark's CPU-baseline leg may load it.  It
 * shares no code, header or constant with the CUDA path; it is the same
 * arithmetic as oracle/gp_oracle.py (kmvm, precond_apply, cg_standard),
 * written in C with OpenMP so that full-size problems (N = 65,536 and more)
 * finish in seconds per MVM instead of hours.
 *
 * Definitions (Sec. 2.2 and Eq. mvm of the paper):
 *   r^2_ij = sum_k ((x_ik - x_jk) / l_k)^2
 *   (Ktilde v)_i = a^2 sum_j k(r^2_ij) v_j + sigma^2 v_i
 *   k: 0 RBF exp(-r^2/2), 1 Matern-3/2 (1 + sqrt3 r) exp(-sqrt3 r),
 *      2 Matern-1/2 exp(-r), 3 Matern-5/2 (1 + sqrt5 r + 5 r^2/3) exp(-sqrt5 r)
 *   P^{-1} w = w / sigma^2 - L C^{-1} L^T w / sigma^4,  C = I + L^T L / sigma^2
 *   (Eq. woodbury; Cc is the lower Cholesky factor of C).
 * The CG is Alg. 1 (App. A) run per column with per-column scalars, with the
 * preconditioned direction update d = -z + beta d.
 *
 * Layouts: every matrix is row-major FP64.  X: N x d.  V, out, B, U: N x R
 * (the R values of one row are contiguous).  L: N x k.  Cc: k x k.
 * Return value 0 on success, -1 on invalid arguments, -2 on allocation failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

static double unit_kernel(double r2, int kernel) {
    if (r2 < 0.0) r2 = 0.0;
    if (kernel == 0) return exp(-0.5 * r2);
    const double r = sqrt(r2);
    if (kernel == 1) {
        const double s = sqrt(3.0) * r;
        return (1.0 + s) * exp(-s);
    }
    if (kernel == 2) return exp(-r);
    const double s = sqrt(5.0) * r;
    return (1.0 + s + s * s / 3.0) * exp(-s);
}

/* dk/d(r^2): the derivative every hyperparameter gradient uses.
 * RBF -k/2; Matern-3/2 -(3/2) exp(-sqrt3 r); Matern-1/2 -exp(-r)/(2r), taken as
 * 0 at r = 0 where the (x_i - x_j) factors it multiplies vanish; Matern-5/2
 * -(5/6)(1 + sqrt5 r) exp(-sqrt5 r). */
static double unit_kernel_dr2(double r2, int kernel) {
    if (r2 < 0.0) r2 = 0.0;
    if (kernel == 0) return -0.5 * exp(-0.5 * r2);
    const double r = sqrt(r2);
    if (kernel == 1) return -1.5 * exp(-sqrt(3.0) * r);
    if (kernel == 2) return r > 0.0 ? -exp(-r) / (2.0 * r) : 0.0;
    const double s = sqrt(5.0) * r;
    return -(5.0 / 6.0) * (1.0 + s) * exp(-s);
}

int orc_threads(void) { return omp_get_max_threads(); }

/* out[t] = (Ktilde V)[rows[t]] for t < nrows (rows == NULL: every row, nrows = N).
 * The noise term sigma^2 v_i is added when add_noise != 0. */
int orc_kmvm(const double* X, int64_t N, int d, const double* ls, int kernel, double a2, double s2,
             const double* V, int R, const int64_t* rows, int64_t nrows, int add_noise, double* out) {
    if (!X || !ls || !V || !out || N <= 0 || d <= 0 || R <= 0 || kernel < 0 || kernel > 3) return -1;
    if (!rows) nrows = N;
    double* inv_l = (double*)malloc(sizeof(double) * (size_t)d);
    if (!inv_l) return -2;
    for (int k = 0; k < d; ++k) inv_l[k] = 1.0 / ls[k];
    int bad = 0;
#pragma omp parallel
    {
        double* acc = (double*)malloc(sizeof(double) * (size_t)R);
        if (!acc) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t t = 0; t < nrows; ++t) {
            if (!acc) continue;
            const int64_t i = rows ? rows[t] : t;
            const double* xi = X + i * d;
            for (int c = 0; c < R; ++c) acc[c] = 0.0;
            for (int64_t j = 0; j < N; ++j) {
                const double* xj = X + j * d;
                double r2 = 0.0;
                for (int k = 0; k < d; ++k) {
                    const double diff = (xi[k] - xj[k]) * inv_l[k];
                    r2 += diff * diff;
                }
                const double kv = a2 * unit_kernel(r2, kernel);
                const double* vj = V + j * R;
                for (int c = 0; c < R; ++c) acc[c] += kv * vj[c];
            }
            for (int c = 0; c < R; ++c) out[t * R + c] = acc[c] + (add_noise ? s2 * V[i * R + c] : 0.0);
        }
        free(acc);
    }
    free(inv_l);
    return bad ? -2 : 0;
}

/* Z = P^{-1} W (Eq. woodbury) for W, Z: N x R.  k = 0: Z = W / sigma^2. */
static int precond_apply(const double* L, const double* Cc, int64_t N, int k, double s2, const double* W, int R,
                         double* Z) {
    if (k == 0) {
        for (int64_t e = 0; e < N * R; ++e) Z[e] = W[e] / s2;
        return 0;
    }
    double* LtW = (double*)calloc((size_t)k * R, sizeof(double));
    if (!LtW) return -2;
    /* L^T W, reduced over rows in per-thread copies */
#pragma omp parallel
    {
        double* part = (double*)calloc((size_t)k * R, sizeof(double));
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i) {
            if (!part) continue;
            for (int m = 0; m < k; ++m) {
                const double l = L[i * k + m];
                for (int c = 0; c < R; ++c) part[m * R + c] += l * W[i * R + c];
            }
        }
        if (part) {
#pragma omp critical
            for (int e = 0; e < k * R; ++e) LtW[e] += part[e];
            free(part);
        }
    }
    /* c = C^{-1} L^T W via Cc (forward) and Cc^T (back) substitution, per column */
    for (int c = 0; c < R; ++c) {
        for (int m = 0; m < k; ++m) {
            double s = LtW[m * R + c];
            for (int q = 0; q < m; ++q) s -= Cc[m * k + q] * LtW[q * R + c];
            LtW[m * R + c] = s / Cc[m * k + m];
        }
        for (int m = k - 1; m >= 0; --m) {
            double s = LtW[m * R + c];
            for (int q = m + 1; q < k; ++q) s -= Cc[q * k + m] * LtW[q * R + c];
            LtW[m * R + c] = s / Cc[m * k + m];
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int c = 0; c < R; ++c) {
            double lc = 0.0;
            for (int m = 0; m < k; ++m) lc += L[i * k + m] * LtW[m * R + c];
            Z[i * R + c] = W[i * R + c] / s2 - lc / (s2 * s2);
        }
    }
    free(LtW);
    return 0;
}

/* per-column dot products out[c] = sum_i A[i][c] B[i][c] */
static void col_dots(const double* A, const double* B, int64_t N, int R, double* out) {
    for (int c = 0; c < R; ++c) out[c] = 0.0;
#pragma omp parallel
    {
        double part[256];
        for (int c = 0; c < R; ++c) part[c] = 0.0;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < N; ++i)
            for (int c = 0; c < R; ++c) part[c] += A[i * R + c] * B[i * R + c];
#pragma omp critical
        for (int c = 0; c < R; ++c) out[c] += part[c];
    }
}

/* Preconditioned CG (Alg. 1) from x_0 = 0 on every column of B, at most
 * max_iter iterations; a column stops once ||r|| / ||b|| <= tol.  Stops early
 * (after the iteration in progress) when time_limit_s > 0 is exceeded.
 * U: solution.  iters_out: iterations run.  relres: per-column ||r|| / ||b||
 * of the recursive residual.  sec_per_iter: mean wall time of an iteration. */
int orc_pcg(const double* X, int64_t N, int d, const double* ls, int kernel, double a2, double s2,
            const double* B, int R, const double* L, int k, const double* Cc, double tol, int max_iter,
            double time_limit_s, double* U, int* iters_out, double* relres, double* sec_per_iter) {
    if (!X || !B || !U || R <= 0 || R > 256 || k < 0 || (k > 0 && (!L || !Cc))) return -1;
    const size_t nv = (size_t)N * (size_t)R;
    double* r = (double*)malloc(nv * sizeof(double));
    double* z = (double*)malloc(nv * sizeof(double));
    double* dd = (double*)malloc(nv * sizeof(double));
    double* Kd = (double*)malloc(nv * sizeof(double));
    if (!r || !z || !dd || !Kd) {
        free(r); free(z); free(dd); free(Kd);
        return -2;
    }
    double gamma[256], bnorm[256], dKd[256], tmp[256];
    int active[256];
    int rc = 0;
    /* x_0 = 0: r_0 = K x_0 - b = -b */
    for (size_t e = 0; e < nv; ++e) { U[e] = 0.0; r[e] = -B[e]; }
    col_dots(B, B, N, R, bnorm);
    for (int c = 0; c < R; ++c) { bnorm[c] = sqrt(bnorm[c]); relres[c] = 1.0; active[c] = bnorm[c] > 0.0; }
    rc = precond_apply(L, Cc, N, k, s2, r, R, z);
    for (size_t e = 0; e < nv; ++e) dd[e] = -z[e];
    col_dots(r, z, N, R, gamma);
    const double t0 = omp_get_wtime();
    int it = 0;
    while (rc == 0 && it < max_iter) {
        int any = 0;
        for (int c = 0; c < R; ++c) any |= active[c];
        if (!any) break;
        if (time_limit_s > 0.0 && it > 0 && omp_get_wtime() - t0 > time_limit_s) break;
        rc = orc_kmvm(X, N, d, ls, kernel, a2, s2, dd, R, NULL, N, 1, Kd);
        if (rc) break;
        col_dots(dd, Kd, N, R, dKd);
        double alpha[256];
        for (int c = 0; c < R; ++c) alpha[c] = active[c] ? gamma[c] / dKd[c] : 0.0;
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i)
            for (int c = 0; c < R; ++c) {
                U[i * R + c] += alpha[c] * dd[i * R + c];
                r[i * R + c] += alpha[c] * Kd[i * R + c];
            }
        rc = precond_apply(L, Cc, N, k, s2, r, R, z);
        if (rc) break;
        col_dots(r, z, N, R, tmp);
        double beta[256];
        for (int c = 0; c < R; ++c) {
            beta[c] = active[c] ? tmp[c] / gamma[c] : 0.0;
            if (active[c]) gamma[c] = tmp[c];
        }
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < N; ++i)
            for (int c = 0; c < R; ++c)
                if (active[c]) dd[i * R + c] = -z[i * R + c] + beta[c] * dd[i * R + c];
        col_dots(r, r, N, R, tmp);
        for (int c = 0; c < R; ++c) {
            if (!active[c]) continue;
            relres[c] = sqrt(tmp[c]) / bnorm[c];
            if (relres[c] <= tol) active[c] = 0;
        }
        ++it;
    }
    const double t1 = omp_get_wtime();
    *iters_out = it;
    *sec_per_iter = it > 0 ? (t1 - t0) / it : 0.0;
    free(r); free(z); free(dd); free(Kd);
    return rc;
}

/* Gradient of q = sum_c u_c^T Ktilde w_c with u, w held fixed (the quantity a
 * backward pass through Eq. mvm returns), G_ij = sum_c u_ic w_jc:
 *   g[m]   = dq/dl_m  = sum_ij G_ij a^2 k'(r^2_ij) (-2 (x_im - x_jm)^2 / l_m^3)
 *   g[d]   = dq/da^2  = sum_ij G_ij k(r^2_ij)
 *   g[d+1] = dq/dsigma^2 = sum_c u_c^T w_c
 *   gX[i][m] (optional) = sum_j (G_ij + G_ji) a^2 k'(r^2_ij) 2 (x_im - x_jm) / l_m^2.
 * U, W: N x R row-major; g: d + 2 doubles; gX: N x d row-major or NULL. */
int orc_quad_form_grad(const double* X, int64_t N, int d, const double* ls, int kernel, double a2,
                       const double* U, const double* W, int R, double* g, double* gX) {
    if (!X || !ls || !U || !W || !g || N <= 0 || d <= 0 || d > 128 || R <= 0 || kernel < 0 || kernel > 3) return -1;
    for (int m = 0; m < d + 2; ++m) g[m] = 0.0;
    int bad = 0;
#pragma omp parallel
    {
        double* acc = (double*)calloc((size_t)d + 2, sizeof(double));
        double diff[128], gxi[128];
        if (!acc) {
#pragma omp atomic write
            bad = 1;
        }
#pragma omp for schedule(dynamic, 16)
        for (int64_t i = 0; i < N; ++i) {
            if (!acc) continue;
            const double* xi = X + i * d;
            for (int m = 0; m < d; ++m) gxi[m] = 0.0;
            double uw = 0.0;
            for (int c = 0; c < R; ++c) uw += U[i * R + c] * W[i * R + c];
            acc[d + 1] += uw;
            for (int64_t j = 0; j < N; ++j) {
                const double* xj = X + j * d;
                double r2 = 0.0;
                for (int m = 0; m < d; ++m) {
                    diff[m] = xi[m] - xj[m];
                    const double t = diff[m] / ls[m];
                    r2 += t * t;
                }
                double gij = 0.0, gji = 0.0;
                for (int c = 0; c < R; ++c) {
                    gij += U[i * R + c] * W[j * R + c];
                    gji += U[j * R + c] * W[i * R + c];
                }
                const double k = unit_kernel(r2, kernel);
                const double wk = a2 * unit_kernel_dr2(r2, kernel);
                acc[d] += gij * k;
                for (int m = 0; m < d; ++m) {
                    acc[m] += gij * wk * (-2.0 * diff[m] * diff[m] / (ls[m] * ls[m] * ls[m]));
                    gxi[m] += (gij + gji) * wk * 2.0 * diff[m] / (ls[m] * ls[m]);
                }
            }
            if (gX)
                for (int m = 0; m < d; ++m) gX[i * d + m] = gxi[m];
        }
        if (acc) {
#pragma omp critical
            for (int m = 0; m < d + 2; ++m) g[m] += acc[m];
            free(acc);
        }
    }
    return bad ? -2 : 0;
}
