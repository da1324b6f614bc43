// Backward of the kernel MVM -- the gradient of
//     q(theta, X) = sum_c u_c^T Ktilde(theta, X) w_c
// with respect to theta = (l_1..l_d, a^2, sigma^2) and, optionally, X
// (what Eq. approx needs: the pseudo-loss is such a bilinear form with the
// solves detached).  With r^2 = sum_m (x_im - x_jm)^2 / l_m^2,
// K_ij = a^2 k(r^2), G_ij = sum_c u_ic w_jc and k' = dk/d(r^2):
//     dq/da^2    = sum_ij G_ij k(r_ij^2)
//     dq/dl_m    = -(2 / l_m) sum_ij G_ij a^2 k'(r_ij^2) (x_im - x_jm)^2 / l_m^2
//     dq/dsigma^2 = sum_c u_c^T w_c
//     dq/dx_im   = (2 / l_m) sum_j (G_ij + G_ji) a^2 k'(r_ij^2) (x_im - x_jm) / l_m
// Every pair is evaluated on the fly in FP32 on the CUDA cores (one row per
// thread, column tiles of the scaled inputs and of W / U in shared memory);
// per-row sums are reduced per block and the block partials are summed in
// FP64 in a fixed order, so the result is deterministic.
#include "gpk_internal.cuh"

#include <math.h>

namespace gpk {

namespace {

constexpr int kVjpThreads = 128;
constexpr int kVjpTile = 32;

template <int KIND>
__device__ __forceinline__ void kernel_and_deriv(float r2, float& k, float& kp) {
    // unit-outputscale k(r^2) and dk/d(r^2) from the FP32 squared distance
    if constexpr (KIND == GP_KERNEL_RBF) {
        k = __expf(-0.5f * r2);
        kp = -0.5f * k;
    } else {
        const float r = sqrtf(fmaxf(r2, 0.0f));
        if constexpr (KIND == GP_KERNEL_MATERN32) {
            const float e = __expf(-1.7320508075688772f * r);
            k = (1.0f + 1.7320508075688772f * r) * e;
            kp = -1.5f * e;
        } else if constexpr (KIND == GP_KERNEL_MATERN12) {
            const float e = __expf(-r);
            k = e;
            kp = r > 0.0f ? -e / (2.0f * r) : 0.0f;   // the (x_i - x_j) factors vanish with r
        } else {
            const float s = 2.23606797749979f * r;
            const float e = __expf(-s);
            k = (1.0f + s + s * s / 3.0f) * e;
            kp = -(5.0f / 6.0f) * (1.0f + s) * e;
        }
    }
}

// part[blk][0..d) : sum over the block's rows of sum_j a^2 k' G_ij dx_m^2   (dx = x^_i - x^_j)
// part[blk][d]    : sum over the block's rows of sum_j k G_ij
// gX (optional)   : per row i and dim m, sum_j (G_ij + G_ji) a^2 k' dx_m
template <int KIND, int DPM, int RPM, int WITH_X>
__global__ void __launch_bounds__(kVjpThreads)
vjp_kernel(const float* __restrict__ Xs, int64_t N, int dp, const float* __restrict__ U,
           const float* __restrict__ W, int R, float a2, double* __restrict__ part, float* __restrict__ gX) {
    __shared__ float sx[kVjpTile][DPM];
    __shared__ float sw[kVjpTile][RPM];
    __shared__ float su[WITH_X ? kVjpTile : 1][WITH_X ? RPM : 1];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kVjpThreads + tid;
    const bool valid = i < N;
    float xi[DPM], ui[RPM], wi[WITH_X ? RPM : 1], accl[DPM], accx[WITH_X ? DPM : 1];
    float acca = 0.0f;
#pragma unroll
    for (int m = 0; m < DPM; ++m) {
        xi[m] = (valid && m < dp) ? Xs[i * dp + m] : 0.0f;
        accl[m] = 0.0f;
        if constexpr (WITH_X) accx[m] = 0.0f;
    }
#pragma unroll
    for (int c = 0; c < RPM; ++c) {
        ui[c] = (valid && c < R) ? U[(int64_t)c * N + i] : 0.0f;
        if constexpr (WITH_X) wi[c] = (valid && c < R) ? W[(int64_t)c * N + i] : 0.0f;
    }
    for (int64_t jb = 0; jb < N; jb += kVjpTile) {
        __syncthreads();
        for (int e = tid; e < kVjpTile * DPM; e += kVjpThreads) {
            const int jj = e / DPM, m = e % DPM;
            const int64_t j = jb + jj;
            sx[jj][m] = (j < N && m < dp) ? Xs[j * dp + m] : 0.0f;
        }
        for (int e = tid; e < kVjpTile * RPM; e += kVjpThreads) {
            const int c = e / kVjpTile, jj = e % kVjpTile;
            const int64_t j = jb + jj;
            sw[jj][c] = (j < N && c < R) ? W[(int64_t)c * N + j] : 0.0f;
            if constexpr (WITH_X) su[jj][c] = (j < N && c < R) ? U[(int64_t)c * N + j] : 0.0f;
        }
        __syncthreads();
        const int jn = (int)((N - jb) < kVjpTile ? (N - jb) : kVjpTile);
        for (int jj = 0; jj < jn; ++jj) {
            float dx[DPM];
            float r2 = 0.0f;
#pragma unroll
            for (int m = 0; m < DPM; ++m) {
                dx[m] = xi[m] - sx[jj][m];
                r2 = fmaf(dx[m], dx[m], r2);
            }
            float k, kp;
            kernel_and_deriv<KIND>(r2, k, kp);
            float g = 0.0f;
#pragma unroll
            for (int c = 0; c < RPM; ++c) g = fmaf(ui[c], sw[jj][c], g);
            acca = fmaf(k, g, acca);
            const float wgt = a2 * kp * g;
#pragma unroll
            for (int m = 0; m < DPM; ++m) accl[m] = fmaf(wgt, dx[m] * dx[m], accl[m]);
            if constexpr (WITH_X) {
                float gt = 0.0f;
#pragma unroll
                for (int c = 0; c < RPM; ++c) gt = fmaf(wi[c], su[jj][c], gt);
                const float wx = a2 * kp * (g + gt);
#pragma unroll
                for (int m = 0; m < DPM; ++m) accx[m] = fmaf(wx, dx[m], accx[m]);
            }
        }
    }
    if constexpr (WITH_X) {
        if (valid)
            for (int m = 0; m < dp; ++m) gX[i * dp + m] = accx[m];
    }
    // block reduction of the d + 1 sums, FP64
    __shared__ double red[kVjpThreads / 32][DPM + 1];
    const int w = tid >> 5, l = tid & 31;
    for (int m = 0; m <= DPM; ++m) {
        double v = (m < DPM) ? (double)accl[m] : (double)acca;
        if (!valid) v = 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) red[w][m] = v;
    }
    __syncthreads();
    if (tid <= DPM) {
        double t = 0.0;
        for (int q = 0; q < kVjpThreads / 32; ++q) t += red[q][tid];
        const int slot = tid < DPM ? tid : dp;   // a^2 term goes to slot dp
        if (tid < dp || tid == DPM) part[(int64_t)blockIdx.x * (dp + 1) + slot] = t;
    }
}

// out[s] = sum_b part[b][s] in block order (FP64); one thread per slot.
__global__ void sum_parts_kernel(const double* __restrict__ part, int nblk, int nslot, double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nslot) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += part[(int64_t)b * nslot + s];
    out[s] = t;
}

// out[c] = u_c^T w_c in FP64 (one block per column, fixed-order tree)
__global__ void coldot_kernel(const float* __restrict__ U, const float* __restrict__ W, int64_t N,
                              double* __restrict__ out) {
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) acc = fma((double)U[(int64_t)c * N + i], (double)W[(int64_t)c * N + i], acc);
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
        out[c] = t;
    }
}

template <int KIND, int DPM, int RPM>
cudaError_t vjp_launch3(bool with_x, unsigned grid, const float* Xs, int64_t N, int dp, const float* U,
                        const float* W, int R, float a2, double* part, float* gX, cudaStream_t s) {
    if (with_x)
        vjp_kernel<KIND, DPM, RPM, 1><<<grid, kVjpThreads, 0, s>>>(Xs, N, dp, U, W, R, a2, part, gX);
    else
        vjp_kernel<KIND, DPM, RPM, 0><<<grid, kVjpThreads, 0, s>>>(Xs, N, dp, U, W, R, a2, part, gX);
    return cudaGetLastError();
}

template <int KIND, int DPM>
cudaError_t vjp_launch2(int RPM, bool with_x, unsigned grid, const float* Xs, int64_t N, int dp, const float* U,
                        const float* W, int R, float a2, double* part, float* gX, cudaStream_t s) {
    switch (RPM) {
        case 4: return vjp_launch3<KIND, DPM, 4>(with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        case 8: return vjp_launch3<KIND, DPM, 8>(with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        case 16: return vjp_launch3<KIND, DPM, 16>(with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        default: return vjp_launch3<KIND, DPM, 32>(with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
    }
}

template <int KIND>
cudaError_t vjp_launch1(int DPM, int RPM, bool with_x, unsigned grid, const float* Xs, int64_t N, int dp,
                        const float* U, const float* W, int R, float a2, double* part, float* gX, cudaStream_t s) {
    switch (DPM) {
        case 4: return vjp_launch2<KIND, 4>(RPM, with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        case 8: return vjp_launch2<KIND, 8>(RPM, with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        case 12: return vjp_launch2<KIND, 12>(RPM, with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        case 16: return vjp_launch2<KIND, 16>(RPM, with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        case 20: return vjp_launch2<KIND, 20>(RPM, with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
        default: return vjp_launch2<KIND, 32>(RPM, with_x, grid, Xs, N, dp, U, W, R, a2, part, gX, s);
    }
}

}  // namespace

size_t vjp_workspace(int64_t N, int d, int R) {
    WsCounter c;
    const int dp = ((d + 3) / 4) * 4;
    const int64_t nblk = (N + kVjpThreads - 1) / kVjpThreads;
    c.take<float>((size_t)N * dp);
    c.take<double>((size_t)nblk * (dp + 1));
    c.take<double>((size_t)(dp + 1));
    c.take<double>((size_t)R);
    c.take<float>((size_t)N * dp);
    (void)R;
    return c.off;
}

// grad_theta (host, d + 2 doubles) = d/dtheta sum_c u_c^T Ktilde w_c; gX (device, N x d, optional)
int vjp_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U, const float* W,
            int R, double* grad_theta_host, float* gX_dev, cudaStream_t s) {
    const int d = hyp->d;
    const int dp = ((d + 3) / 4) * 4;
    if (dp > 32 || R > 32) return GP_ERR_UNSUPPORTED;
    const int64_t nblk = (N + kVjpThreads - 1) / kVjpThreads;
    float* Xs = wc.take<float>((size_t)N * dp);
    double* part = wc.take<double>((size_t)nblk * (dp + 1));
    double* sums = wc.take<double>((size_t)(dp + 1));
    double* dots = wc.take<double>((size_t)R);
    float* gXs = gX_dev ? wc.take<float>((size_t)N * dp) : nullptr;
    if (!wc.ok) return GP_ERR_WORKSPACE;
    ScaleVec inv;
    for (int k = 0; k < 64; ++k) inv.v[k] = k < d ? (float)(1.0 / hyp->lengthscale[k]) : 0.0f;
    GPK_TRY(launch_prep_x_f32(ctx, X, N, N, d, dp, inv, Xs, s));
    const int DPM = dp <= 4 ? 4 : dp <= 8 ? 8 : dp <= 12 ? 12 : dp <= 16 ? 16 : dp <= 20 ? 20 : 32;
    const int RPM = R <= 4 ? 4 : R <= 8 ? 8 : R <= 16 ? 16 : 32;
    const float a2 = (float)hyp->outputscale;
    cudaError_t e;
    switch (hyp->kernel) {
        case GP_KERNEL_RBF:
            e = vjp_launch1<GP_KERNEL_RBF>(DPM, RPM, gX_dev != nullptr, (unsigned)nblk, Xs, N, dp, U, W, R, a2, part, gXs, s);
            break;
        case GP_KERNEL_MATERN32:
            e = vjp_launch1<GP_KERNEL_MATERN32>(DPM, RPM, gX_dev != nullptr, (unsigned)nblk, Xs, N, dp, U, W, R, a2, part, gXs, s);
            break;
        case GP_KERNEL_MATERN12:
            e = vjp_launch1<GP_KERNEL_MATERN12>(DPM, RPM, gX_dev != nullptr, (unsigned)nblk, Xs, N, dp, U, W, R, a2, part, gXs, s);
            break;
        default:
            e = vjp_launch1<GP_KERNEL_MATERN52>(DPM, RPM, gX_dev != nullptr, (unsigned)nblk, Xs, N, dp, U, W, R, a2, part, gXs, s);
            break;
    }
    ctx->launches++;
    if (e != cudaSuccess) return GP_ERR_CUDA;
    sum_parts_kernel<<<1, 64, 0, s>>>(part, (int)nblk, dp + 1, sums);
    coldot_kernel<<<R, 256, 0, s>>>(U, W, N, dots);
    ctx->launches += 2;
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    double hs[64 + 1];
    double hd[32];
    if (cudaMemcpyAsync(hs, sums, sizeof(double) * (dp + 1), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hd, dots, sizeof(double) * R, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GP_ERR_CUDA;
    // sums[m] = sum_ij a^2 k' G (x^_im - x^_jm)^2 with x^ = x / l, so dq/dl_m = -(2 / l_m) sums[m]
    for (int m = 0; m < d; ++m) grad_theta_host[m] = -2.0 / (double)hyp->lengthscale[m] * hs[m];
    grad_theta_host[d] = hs[dp];
    double sg = 0.0;
    for (int c = 0; c < R; ++c) sg += hd[c];
    grad_theta_host[d + 1] = sg;
    if (gX_dev) {
        // dq/dx_im = (2 / l_m) sum_j (G_ij + G_ji) a^2 k' (x^_im - x^_jm): scale and compact to N x d
        const float* src = gXs;
        GPK_TRY(launch_scale_cols(ctx, src, N, dp, d, hyp->lengthscale, gX_dev, s));
    }
    return GP_OK;
}

namespace {
__global__ void scale_cols_kernel(const float* __restrict__ src, int64_t N, int dp, int d, ScaleVec sc,
                                  float* __restrict__ dst) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * d; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d;
        const int m = (int)(e % d);
        dst[e] = src[i * dp + m] * sc.v[m];
    }
}
}  // namespace

int launch_scale_cols(Ctx* ctx, const float* src, int64_t N, int dp, int d, const float* ls_host, float* dst,
                      cudaStream_t s) {
    ScaleVec sc;
    for (int k = 0; k < 64; ++k) sc.v[k] = k < d ? (float)(2.0 / ls_host[k]) : 0.0f;
    int64_t g = (N * d + 255) / 256;
    if (g > 4096) g = 4096;
    scale_cols_kernel<<<(unsigned)g, 256, 0, s>>>(src, N, dp, d, sc, dst);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

}  // namespace gpk

extern "C" {

size_t gp_kmvm_vjp_workspace_size(const gp_hyp_t* hyp, int64_t N, int R) {
    if (gpk::check_hyp(hyp) != GP_OK || N < 1 || R < 1 || R > 32 || hyp->d > 32) return 0;
    return gpk::vjp_workspace(N, hyp->d, R);
}

int gp_kmvm_vjp(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U, const float* W, int R,
                double* grad_theta, float* grad_X, void* stream) {
    if (!ctx || !X || !U || !W || !grad_theta) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_hyp(hyp));
    if (N < 1 || R < 1 || R > 32 || hyp->d > 32) return GP_ERR_INVALID;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return GP_ERR_CUDA;
    gpk::WsCarver wc(ctx->ws, ctx->ws_bytes);
    int st = gpk::vjp_run(ctx, wc, hyp, X, N, U, W, R, grad_theta, grad_X, (cudaStream_t)stream);
    if (prev != ctx->device) cudaSetDevice(prev);
    return st;
}

size_t gp_kmvm_vjp_prec_workspace_size(const gp_hyp_t* hyp, int64_t N, int R, int precision) {
    if (gpk::check_hyp(hyp) != GP_OK || N < 1 || R < 1 || R > 32 || hyp->d > 32) return 0;
    if (precision == GP_PREC_FP32) return gpk::vjp_workspace(N, hyp->d, R);
    if (precision != GP_PREC_FP16 || !gpk::vjp_tc_supported(hyp, R)) return 0;
    gpk::Ctx probe;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) probe.num_sms = 148;
    return gpk::vjp_tc_workspace(&probe, hyp, N, R);
}

int gp_kmvm_vjp_prec(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U, const float* W,
                     int R, int precision, double* grad_theta, float* grad_X, void* stream) {
    if (precision == GP_PREC_FP32) return gp_kmvm_vjp(ctx, hyp, X, N, U, W, R, grad_theta, grad_X, stream);
    if (!ctx || !X || !U || !W || !grad_theta) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_hyp(hyp));
    if (N < 1 || R < 1 || R > 32 || hyp->d > 32) return GP_ERR_INVALID;
    if (precision != GP_PREC_FP16) return GP_ERR_INVALID;
    if (!gpk::vjp_tc_supported(hyp, R)) return GP_ERR_UNSUPPORTED;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return GP_ERR_CUDA;
    gpk::WsCarver wc(ctx->ws, ctx->ws_bytes);
    int st = gpk::vjp_tc_run(ctx, wc, hyp, X, N, U, W, R, grad_theta, grad_X, (cudaStream_t)stream);
    if (prev != ctx->device) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
