// The summation-variant study of the half-precision MVM (Sec. 4.1,
// Fig. 4b; App. B, Fig. A.1a).  The paper's FP16 MVM runs on CUDA cores and
// compares how the row sums sum_j k_ij v_j are accumulated.  This engine does
// the same on this GPU: per pair the kernel value is rounded to FP16 and
// multiplied by the FP16 (column-scaled) v_j in FP16, and the products are
// accumulated by one of four schemes (GP_MVM_SUM(x) of include/gpk.h):
//   1  FP32 accumulation of the FP16 products   (the tensor-core engines' order)
//   2  FP16 accumulation, one running sum        (naive half precision)
//   3  FP16 block sums: an FP16 sum per 128-column tile, added in FP32
//   4  Kahan compensated summation in FP16       (sum and correction in half)
// One thread per output row, the column tiles of the scaled inputs (FP32) and
// of V (FP16) staged in shared memory; up to 8 right-hand sides.  It is a study
// engine: the hot path's MVM is the tensor-core one.
#include "gpk_internal.cuh"
#include "kfun.cuh"

namespace gpk {

namespace {

constexpr int kSumThreads = 128;
constexpr int kSumTile = 128;
constexpr int kSumMaxR = 8;
constexpr int kSumMaxDp = 32;

template <int KIND, int SCHEME>
__global__ void __launch_bounds__(kSumThreads)
kmvm_sum_kernel(const float* __restrict__ Xr, const float* __restrict__ Xc, int64_t Nr, int64_t Nc, int dp,
                const float* __restrict__ V, int R, const unsigned* __restrict__ cmax_bits, float a2, float noise,
                int diag, float* __restrict__ out, int64_t ld_out) {
    __shared__ float sx[kSumTile][kSumMaxDp + 1];
    __shared__ __half sv[kSumTile][kSumMaxR];
    __shared__ float vs[kSumMaxR];
    const int tid = threadIdx.x;
    const int64_t i = (int64_t)blockIdx.x * kSumThreads + tid;
    if (tid < kSumMaxR) {
        float sc = 1.0f;
        if (tid < R) {
            const float cm = __uint_as_float(cmax_bits[tid]);
            if (cm > 0.0f && cm <= 3.0e38f) {
                int e;
                frexpf(cm, &e);
                sc = ldexpf(1.0f, -e);   // max |v| s_c in [1/2, 1)
            }
        }
        vs[tid] = sc;
    }
    float xi[kSumMaxDp];
#pragma unroll
    for (int m = 0; m < kSumMaxDp; ++m) xi[m] = (i < Nr && m < dp) ? Xr[i * dp + m] : 0.0f;
    float acc32[kSumMaxR];
    __half acc16[kSumMaxR], comp[kSumMaxR];
#pragma unroll
    for (int c = 0; c < kSumMaxR; ++c) {
        acc32[c] = 0.0f;
        acc16[c] = __float2half(0.0f);
        comp[c] = __float2half(0.0f);
    }
    for (int64_t jb = 0; jb < Nc; jb += kSumTile) {
        __syncthreads();
        for (int e = tid; e < kSumTile * dp; e += kSumThreads) {
            const int jj = e / dp, m = e % dp;
            sx[jj][m] = (jb + jj < Nc) ? Xc[(jb + jj) * dp + m] : 0.0f;
        }
        for (int e = tid; e < kSumTile * kSumMaxR; e += kSumThreads) {
            const int jj = e % kSumTile, c = e / kSumTile;
            const float v = (c < R && jb + jj < Nc) ? V[(int64_t)c * Nc + jb + jj] * vs[c] : 0.0f;
            sv[jj][c] = __float2half_rn(v);
        }
        __syncthreads();
        const int jn = (int)((Nc - jb) < kSumTile ? (Nc - jb) : kSumTile);
        for (int jj = 0; jj < jn; ++jj) {
            float q = 0.0f;
#pragma unroll
            for (int m = 0; m < kSumMaxDp; ++m) {
                if (m < dp) {
                    const float t = xi[m] - sx[jj][m];
                    q = fmaf(t, t, q);
                }
            }
            float k = kernel_from_s<KIND>(-q);
            if (diag && jb + jj == i) k = 0.0f;   // square Matern-1/2: exact diagonal added with the noise term
            const __half kh = __float2half_rn(k);
#pragma unroll
            for (int c = 0; c < kSumMaxR; ++c) {
                if (c < R) {
                    const __half p = __hmul(kh, sv[jj][c]);
                    if constexpr (SCHEME == 1) {
                        acc32[c] += __half2float(p);
                    } else if constexpr (SCHEME == 2 || SCHEME == 3) {
                        acc16[c] = __hadd(acc16[c], p);
                    } else {
                        const __half y = __hsub(p, comp[c]);
                        const __half t = __hadd(acc16[c], y);
                        comp[c] = __hsub(__hsub(t, acc16[c]), y);
                        acc16[c] = t;
                    }
                }
            }
        }
        if constexpr (SCHEME == 3) {
#pragma unroll
            for (int c = 0; c < kSumMaxR; ++c) {
                acc32[c] += __half2float(acc16[c]);
                acc16[c] = __float2half(0.0f);
            }
        }
    }
    if (i >= Nr) return;
#pragma unroll
    for (int c = 0; c < kSumMaxR; ++c) {
        if (c < R) {
            const float sum = (SCHEME == 2 || SCHEME == 4) ? __half2float(acc16[c]) : acc32[c];
            float o = a2 * sum / vs[c];
            if (noise != 0.0f) o += noise * V[(int64_t)c * Nc + i];
            out[(int64_t)c * ld_out + i] = o;
        }
    }
}

template <int KIND>
cudaError_t launch_sum_kind(int scheme, unsigned grid, cudaStream_t s, const float* Xr, const float* Xc, int64_t Nr,
                            int64_t Nc, int dp, const float* V, int R, const unsigned* cm, float a2, float noise,
                            int diag, float* out, int64_t ld_out) {
    switch (scheme) {
        case 1: kmvm_sum_kernel<KIND, 1><<<grid, kSumThreads, 0, s>>>(Xr, Xc, Nr, Nc, dp, V, R, cm, a2, noise, diag, out, ld_out); break;
        case 2: kmvm_sum_kernel<KIND, 2><<<grid, kSumThreads, 0, s>>>(Xr, Xc, Nr, Nc, dp, V, R, cm, a2, noise, diag, out, ld_out); break;
        case 3: kmvm_sum_kernel<KIND, 3><<<grid, kSumThreads, 0, s>>>(Xr, Xc, Nr, Nc, dp, V, R, cm, a2, noise, diag, out, ld_out); break;
        default: kmvm_sum_kernel<KIND, 4><<<grid, kSumThreads, 0, s>>>(Xr, Xc, Nr, Nc, dp, V, R, cm, a2, noise, diag, out, ld_out); break;
    }
    return cudaGetLastError();
}

}  // namespace

int launch_kmvm_sum(Ctx* ctx, int scheme, const MvmArgs& a, float outputscale, const float* Xrs, const float* Xcs,
                    int dp, const float* V, const unsigned* cmax_bits, cudaStream_t s) {
    if (a.R > kSumMaxR || dp > kSumMaxDp || scheme < 1 || scheme > 4) return GP_ERR_UNSUPPORTED;
    const unsigned grid = (unsigned)((a.Nr + kSumThreads - 1) / kSumThreads);
    const int diag = a.diag_coef != 0.0f ? 1 : 0;
    const float noise = a.noise + a.diag_coef;
    cudaError_t e;
    prof_begin(ctx, s);
    switch (a.kernel) {
        case GP_KERNEL_RBF:
            e = launch_sum_kind<GP_KERNEL_RBF>(scheme, grid, s, Xrs, Xcs, a.Nr, a.Nc, dp, V, a.R, cmax_bits,
                                               outputscale, noise, diag, a.out, a.ld_out);
            break;
        case GP_KERNEL_MATERN32:
            e = launch_sum_kind<GP_KERNEL_MATERN32>(scheme, grid, s, Xrs, Xcs, a.Nr, a.Nc, dp, V, a.R, cmax_bits,
                                                    outputscale, noise, diag, a.out, a.ld_out);
            break;
        case GP_KERNEL_MATERN12:
            e = launch_sum_kind<GP_KERNEL_MATERN12>(scheme, grid, s, Xrs, Xcs, a.Nr, a.Nc, dp, V, a.R, cmax_bits,
                                                    outputscale, noise, diag, a.out, a.ld_out);
            break;
        default:
            e = launch_sum_kind<GP_KERNEL_MATERN52>(scheme, grid, s, Xrs, Xcs, a.Nr, a.Nc, dp, V, a.R, cmax_bits,
                                                    outputscale, noise, diag, a.out, a.ld_out);
            break;
    }
    prof_end(ctx, s);
    ctx->launches++;
    return e == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

}  // namespace gpk
