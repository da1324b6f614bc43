// Negative log marginal likelihood and its gradient (Sec. 4.3).
//
// The solves K [u_0, u_1 .. u_M] = [y, z_1 .. z_M] of Eq. cg run through the
// stable CG (Alg. 2).  With the solutions detached, the gradient of the
// pseudo-loss (Eq. approx_loss, Eq. approx)
//     1/(2M) sum_j u_j^T (dKtilde w_j) - 1/2 u_0^T (dKtilde u_0)
// is one bilinear-form backward sum_c u'_c^T dKtilde w'_c with
// u' = [u_1 .. u_M, u_0] and w' = [w_1/(2M) .. w_M/(2M), -u_0/2]; w_j = z_j
// for probes with E[z z^T] = I, and w_j = P^{-1} z_j for probes drawn as
// z = L e1 + sigma e2 (E[z z^T] = P), which keeps the trace estimate
// unbiased under preconditioning.
//
// The loss value  1/2 log|Ktilde| + 1/2 y^T u_0 + N/2 log(2 pi)  (Eq. loss)
// needs the log-determinant, which the paper avoids; it is estimated by
// stochastic Lanczos quadrature from the CG step sizes of the probe columns
// (the Lanczos tridiagonal that CG builds implicitly), plus log|P| for
// P-distributed probes:
//     log|Ktilde| ~ log|P| + 1/M sum_j gamma0_j e1^T log(T_j) e1,
//     T_kk = 1/alpha_k + beta_k/alpha_{k-1},  T_{k,k+1} = sqrt(beta_{k+1})/alpha_k.
// e1^T log(T) e1 comes from the eigen-decomposition of T (implicit-shift QL,
// FP64, on the host: T is at most max_iter x max_iter).
#include "gpk_internal.cuh"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <vector>

namespace gpk {

// Eigenvalues of the symmetric tridiagonal matrix (diag d[0..n), off-diagonal
// e[0..n-1)) and the first components of its normalised eigenvectors, by the
// implicit QL method with Wilkinson shifts (Bowdler, Martin, Reinsch and
// Wilkinson, 1968), tracking only the first row of the accumulated rotations.
// On return d holds the eigenvalues and z the first components.  Returns 0,
// or -1 if an eigenvalue fails to converge in 60 sweeps.
static int tridiag_eig_first_row(int n, double* d, double* e, double* z) {
    for (int i = 0; i < n; ++i) z[i] = (i == 0) ? 1.0 : 0.0;
    if (n == 0) return 0;
    e[n - 1] = 0.0;
    for (int l = 0; l < n; ++l) {
        int sweeps = 0;
        while (true) {
            // find the first negligible off-diagonal at or after l
            int m = l;
            for (; m < n - 1; ++m) {
                const double scale = fabs(d[m]) + fabs(d[m + 1]);
                if (fabs(e[m]) <= 1e-16 * scale) break;
            }
            if (m == l) break;
            if (++sweeps > 60) return -1;
            // Wilkinson shift from the leading 2 x 2 block
            double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
            double r = hypot(g, 1.0);
            g = d[m] - d[l] + e[l] / (g + (g >= 0.0 ? r : -r));
            double s = 1.0, c = 1.0, p = 0.0;
            int i = m - 1;
            bool deflated = false;
            for (; i >= l; --i) {
                const double f = s * e[i];
                const double b = c * e[i];
                r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) {   // the rotation underflowed: split the matrix here
                    d[i + 1] -= p;
                    e[m] = 0.0;
                    deflated = true;
                    break;
                }
                s = f / r;
                c = g / r;
                g = d[i + 1] - p;
                r = (d[i] - g) * s + 2.0 * c * b;
                p = s * r;
                d[i + 1] = g + p;
                g = c * r - b;
                // apply the same plane rotation to the first row of the eigenvectors
                const double zf = z[i + 1];
                z[i + 1] = s * z[i] + c * zf;
                z[i] = c * z[i] - s * zf;
            }
            if (deflated) continue;
            d[l] -= p;
            e[l] = g;
            e[m] = 0.0;
        }
    }
    return 0;
}

// gamma0 * e1^T log(T) e1 for the Lanczos tridiagonal of CG step sizes
// alpha[0..J), beta[0..J-1) (beta[k] = beta_{k+1}).
int slq_quadrature_host(const double* alpha, const double* beta, int J, double gamma0, double* out) {
    if (J < 1) return GP_ERR_INVALID;
    std::vector<double> d(J), e(J), z(J);
    for (int k = 0; k < J; ++k) {
        if (!(alpha[k] > 0.0)) return GP_ERR_BREAKDOWN;
        d[k] = 1.0 / alpha[k] + (k > 0 ? beta[k - 1] / alpha[k - 1] : 0.0);
        e[k] = (k + 1 < J) ? sqrt(beta[k]) / alpha[k] : 0.0;
    }
    if (tridiag_eig_first_row(J, d.data(), e.data(), z.data()) != 0) return GP_ERR_NOT_CONVERGED;
    double q = 0.0;
    for (int k = 0; k < J; ++k) {
        if (!(d[k] > 0.0)) return GP_ERR_BREAKDOWN;
        q += z[k] * z[k] * log(d[k]);
    }
    *out = gamma0 * q;
    return GP_OK;
}

namespace {

// B[:,0] = y; B[:,j] = sigma Z_j + L E_j (precond probes) or Z_j (j = 1..M)
__global__ void build_rhs_kernel(const float* __restrict__ y, const float* __restrict__ Z, const float* __restrict__ E,
                                 const float* __restrict__ L, int rank, float sigma, int64_t N, int M,
                                 float* __restrict__ B) {
    const int c = blockIdx.y;   // 0..M
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float v;
        if (c == 0) {
            v = y[i];
        } else if (E) {
            v = sigma * Z[(int64_t)(c - 1) * N + i];
            for (int a = 0; a < rank; ++a) v = fmaf(L[(int64_t)a * N + i], E[(int64_t)(c - 1) * rank + a], v);
        } else {
            v = Z[(int64_t)(c - 1) * N + i];
        }
        B[(int64_t)c * N + i] = v;
    }
}

// U' = [u_1 .. u_M, u_0];  W' = [w_1 s .. w_M s, -u_0 / 2],  s = 1 / (2M)
__global__ void pseudo_loss_operands_kernel(const float* __restrict__ U, const float* __restrict__ Wp, int64_t N,
                                            int M, float* __restrict__ Uo, float* __restrict__ Wo) {
    const int c = blockIdx.y;   // 0..M
    const float s = 0.5f / (float)M;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        if (c < M) {
            Uo[(int64_t)c * N + i] = U[(int64_t)(c + 1) * N + i];
            Wo[(int64_t)c * N + i] = s * Wp[(int64_t)(c + 1) * N + i];
        } else {
            const float u0 = U[i];
            Uo[(int64_t)c * N + i] = u0;
            Wo[(int64_t)c * N + i] = -0.5f * u0;
        }
    }
}

__global__ void dot_kernel(const float* __restrict__ a, const float* __restrict__ b, int64_t N, double* out) {
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) acc = fma((double)a[i], (double)b[i], acc);
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        *out = t;
    }
}

}  // namespace

size_t mll_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t N, int M, int rank, const gp_cg_opts_t* o) {
    WsCounter c;
    const size_t NR = (size_t)N * (M + 1);
    c.take<float>(NR);   // B
    c.take<float>(NR);   // U (when not supplied)
    c.take<float>(NR);   // P^{-1} Z
    c.take<float>(NR);   // U'
    c.take<float>(NR);   // W'
    c.take<double>(4);
    size_t s = c.off;
    const size_t cgw = cg_workspace(ctx, hyp, N, M + 1, rank, o);
    const bool tc = (o->precision & 0xff) != GP_PREC_FP32 && vjp_tc_supported(hyp, M + 1);
    const size_t vw = tc ? vjp_tc_workspace(ctx, hyp, N, M + 1) : vjp_workspace(N, hyp->d, M + 1);
    const size_t ww = rank > 0 ? woodbury_workspace(ctx, N, rank, M + 1) : 0;
    size_t m = cgw > vw ? cgw : vw;
    m = m > ww ? m : ww;
    return s + m;
}

int mll_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, const float* y, int64_t N, const float* Z,
            int M, const float* E, const gp_precond_t* pc, const gp_cg_opts_t* o, int flags, double* mll,
            double* grad, float* gradX, float* U_user, gp_cg_stats_t* stats, cudaStream_t s) {
    const int R = M + 1;
    const size_t NR = (size_t)N * R;
    const int rank = (pc && pc->rank > 0) ? pc->rank : 0;
    const bool pprobe = (flags & GP_MLL_PRECOND_PROBES) != 0;
    if (pprobe && (rank == 0 || !E)) return GP_ERR_INVALID;
    float* B = wc.take<float>(NR);
    float* U = U_user ? U_user : wc.take<float>(NR);
    float* W = pprobe ? wc.take<float>(NR) : nullptr;
    float* Uo = wc.take<float>(NR);
    float* Wo = wc.take<float>(NR);
    double* dsc = wc.take<double>(4);
    if (!wc.ok) return GP_ERR_WORKSPACE;
    const int vg = (int)((N + 255) / 256 < 1024 ? (N + 255) / 256 : 1024);
    build_rhs_kernel<<<dim3(vg, R), 256, 0, s>>>(y, Z, pprobe ? E : nullptr, rank ? pc->L : nullptr, rank,
                                                 (float)sqrt(hyp->noise), N, M, B);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;

    // ---- solves (Eq. cg) ----
    std::vector<double> alpha((size_t)o->max_iter * R), beta((size_t)o->max_iter * R), g0(R), rel(R);
    std::vector<int> it(R), lz(R);
    gp_cg_stats_t st;
    memset(&st, 0, sizeof(st));
    st.col_iters = it.data();
    st.rel_resid = rel.data();
    st.alpha = alpha.data();
    st.beta = beta.data();
    st.gamma0 = g0.data();
    st.lanczos_len = lz.data();
    gp_cg_opts_t oo = *o;
    const int depth = (flags >> 8) & 0xff;   // GP_MLL_SLQ_MIN_ITER
    if ((flags & GP_MLL_WANT_LOGDET) && depth > oo.min_iter) oo.min_iter = depth < oo.max_iter ? depth : oo.max_iter;
    {
        WsCarver w2 = wc;
        const int cs = cg_run(ctx, w2, hyp, X, N, B, R, U, pc, &oo, &st, s);
        if (cs != GP_OK && cs != GP_ERR_NOT_CONVERGED) return cs;
    }
    if (stats) {
        stats->iters = st.iters;
        stats->converged = st.converged;
        stats->breakdowns = st.breakdowns;
        stats->restarts = st.restarts;
        for (int c = 0; c < R; ++c) {
            if (stats->col_iters) stats->col_iters[c] = it[c];
            if (stats->rel_resid) stats->rel_resid[c] = rel[c];
            if (stats->gamma0) stats->gamma0[c] = g0[c];
            if (stats->lanczos_len) stats->lanczos_len[c] = lz[c];
        }
    }

    // ---- gradient of the pseudo-loss (Eq. approx) ----
    if (pprobe) {
        WsCarver w2 = wc;
        GPK_TRY(woodbury_apply(ctx, w2, pc->L, pc->core, nullptr, rank, hyp->noise, N, B, R, nullptr, W, s));
    }
    pseudo_loss_operands_kernel<<<dim3(vg, R), 256, 0, s>>>(U, pprobe ? W : B, N, M, Uo, Wo);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    {
        // the backward runs on the tensor cores in FP16 when the solve's MVM does
        WsCarver w2 = wc;
        if ((o->precision & 0xff) != GP_PREC_FP32 && vjp_tc_supported(hyp, R))
            GPK_TRY(vjp_tc_run(ctx, w2, hyp, X, N, Uo, Wo, R, grad, gradX, s));
        else
            GPK_TRY(vjp_run(ctx, w2, hyp, X, N, Uo, Wo, R, grad, gradX, s));
    }

    // ---- loss value (Eq. loss) with the SLQ log-determinant ----
    dot_kernel<<<1, 1024, 0, s>>>(y, U, N, dsc);
    ctx->launches++;
    double yu = 0.0;
    if (cudaMemcpyAsync(&yu, dsc, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GP_ERR_CUDA;
    double logdet = NAN;
    if ((flags & GP_MLL_WANT_LOGDET) && (pprobe || rank == 0)) {
        double acc = 0.0;
        int used = 0;
        for (int c = 1; c < R; ++c) {
            const int J = lz[c];
            if (J < 1) continue;
            std::vector<double> a(J), b(J > 1 ? J - 1 : 1);
            for (int k = 0; k < J; ++k) a[k] = alpha[(size_t)k * R + c];
            for (int k = 0; k + 1 < J; ++k) b[k] = beta[(size_t)k * R + c];
            double q = 0.0;
            if (slq_quadrature_host(a.data(), b.data(), J, g0[c], &q) == GP_OK) {
                acc += q;
                ++used;
            }
        }
        if (used > 0) {
            logdet = acc / used;
            if (pprobe) {
                std::vector<double> core((size_t)rank * rank);
                if (cudaMemcpy(core.data(), pc->core, sizeof(double) * rank * rank, cudaMemcpyDeviceToHost) !=
                    cudaSuccess)
                    return GP_ERR_CUDA;
                double ldc = 0.0;
                for (int a = 0; a < rank; ++a) ldc += log(core[(size_t)a * rank + a]);
                logdet += (double)N * log(hyp->noise) + 2.0 * ldc;
            }
        }
    }
    if (mll) *mll = 0.5 * logdet + 0.5 * yu + 0.5 * (double)N * log(2.0 * M_PI);
    return GP_OK;
}

}  // namespace gpk

extern "C" {

int gp_slq_quadrature(const double* alpha, const double* beta, int J, double gamma0, double* out) {
    if (!alpha || !out || (J > 1 && !beta)) return GP_ERR_INVALID;
    return gpk::slq_quadrature_host(alpha, beta, J, gamma0, out);
}

size_t gp_mll_workspace_size(const gp_hyp_t* hyp, int64_t N, int M, int rank, const gp_cg_opts_t* opts) {
    if (gpk::check_hyp(hyp) != GP_OK || !opts || N < 1 || M < 1 || M > 31 || hyp->d > 32) return 0;
    gpk::Ctx probe;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) probe.num_sms = 148;
    return gpk::mll_workspace(&probe, hyp, N, M, rank, opts);
}

int gp_mll_and_grad(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, const float* y, int64_t N, const float* Z,
                    int M, const float* E, const gp_precond_t* precond, const gp_cg_opts_t* opts, int flags,
                    double* mll, double* grad, float* grad_X, float* U, gp_cg_stats_t* stats, void* stream) {
    if (!ctx || !X || !y || !Z || !grad || !opts) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_hyp(hyp));
    if (N < 1 || M < 1 || M > 31 || hyp->d > 32 || !(hyp->noise > 0.0)) return GP_ERR_INVALID;
    if (flags & ~(GP_MLL_PRECOND_PROBES | GP_MLL_WANT_LOGDET | GP_MLL_SLQ_MIN_ITER(255))) return GP_ERR_INVALID;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return GP_ERR_CUDA;
    gpk::WsCarver wc(ctx->ws, ctx->ws_bytes);
    int st = gpk::mll_run(ctx, wc, hyp, X, y, N, Z, M, E, precond, opts, flags, mll, grad, grad_X, U, stats,
                          (cudaStream_t)stream);
    if (prev != ctx->device) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
