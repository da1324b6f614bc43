// The comparator arm: the same matrix-free MVM (Eq. mvm) in plain FP32 on the
// CUDA cores -- the "single precision" side of the paper's half-vs-single
// comparison (Sec. 4.1, Fig. 4a).  Squared distances are formed from
// differences of the scaled inputs (no expanded-norm cancellation), the kernel
// function uses the same special-function-unit forms as the tensor-core
// engine, and the contraction with V is an FP32 FMA chain per output.
//
// Each thread owns two output rows; a 128-thread block covers 256 rows and
// walks a range of columns in 64-column tiles staged in shared memory (all
// threads read the same column: broadcast, no bank conflicts).  Column ranges
// are split across blockIdx.y so the grid fills the 152 SMs many times over;
// split partials are summed by launch_split_reduce in a fixed order.
//
// The arithmetic runs on packed FP32 pairs (__fadd2_rn / __ffma2_rn, two
// IEEE round-to-nearest operations per instruction): a row's squared distance
// as two interleaved partial sums over even and odd dimensions, and its
// accumulators as pairs of adjacent output columns.  Shared memory holds the
// negated column inputs so the difference is one packed add.
#include "gpk_internal.cuh"
#include "kfun.cuh"

namespace gpk {

namespace {

constexpr int kSimtThreads = 128;
constexpr int kSimtRows = 2 * kSimtThreads;
constexpr int kSimtTile = 64;

template <int KIND, int DPM, int RPM>
__global__ void __launch_bounds__(kSimtThreads)
kmvm_simt_kernel(const float* __restrict__ Xr, const float* __restrict__ Xc, const float* __restrict__ V,
                 int64_t Nr, int64_t Nc, int dp, int R, int n_split, float a2, float noise,
                 const float* __restrict__ Vnoise, float* __restrict__ out, int64_t ld_out,
                 float* __restrict__ partial, int64_t ld_part) {
    // staged column tile; rows padded by 4 floats (16-byte aligned float4 reads,
    // fewer bank conflicts on the transposing stores of V).  sx holds -x_j.
    __shared__ __align__(16) float sx[kSimtTile][DPM + 4];
    __shared__ __align__(16) float sv[kSimtTile][RPM + 4];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * kSimtRows + tid;
    const int64_t i1 = i0 + kSimtThreads;
    float2 x0[DPM / 2], x1[DPM / 2], acc0[RPM / 2], acc1[RPM / 2];
#pragma unroll
    for (int h = 0; h < DPM / 2; ++h) {
        const int k = 2 * h;   // dp is a multiple of 4, so k < dp covers k + 1 too
        x0[h] = (i0 < Nr && k < dp) ? make_float2(Xr[i0 * dp + k], Xr[i0 * dp + k + 1]) : make_float2(0.0f, 0.0f);
        x1[h] = (i1 < Nr && k < dp) ? make_float2(Xr[i1 * dp + k], Xr[i1 * dp + k + 1]) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int h = 0; h < RPM / 2; ++h) { acc0[h] = make_float2(0.0f, 0.0f); acc1[h] = make_float2(0.0f, 0.0f); }

    const int64_t ntiles = (Nc + kSimtTile - 1) / kSimtTile;
    const int64_t t0 = (ntiles * blockIdx.y) / n_split, t1 = (ntiles * (blockIdx.y + 1)) / n_split;
    for (int64_t t = t0; t < t1; ++t) {
        const int64_t jb = t * kSimtTile;
        for (int e = tid; e < kSimtTile * DPM; e += kSimtThreads) {
            const int jj = e / DPM, k = e % DPM;
            const int64_t j = jb + jj;
            sx[jj][k] = (j < Nc && k < dp) ? -Xc[j * dp + k] : 0.0f;
        }
        for (int e = tid; e < kSimtTile * RPM; e += kSimtThreads) {
            const int c = e / kSimtTile, jj = e % kSimtTile;
            const int64_t j = jb + jj;
            sv[jj][c] = (j < Nc && c < R) ? V[(int64_t)c * Nc + j] : 0.0f;
        }
        __syncthreads();
        const int jn = (int)((Nc - jb) < kSimtTile ? (Nc - jb) : kSimtTile);
        for (int jj = 0; jj < jn; ++jj) {
            float2 q0 = make_float2(0.0f, 0.0f), q1 = make_float2(0.0f, 0.0f);
#pragma unroll
            for (int k = 0; k < DPM; k += 4) {
                if (k < dp) {
                    const float4 x4 = *reinterpret_cast<const float4*>(&sx[jj][k]);   // broadcast
                    const float2 xa = make_float2(x4.x, x4.y), xb = make_float2(x4.z, x4.w);
                    const float2 d0a = __fadd2_rn(x0[k / 2], xa), d0b = __fadd2_rn(x0[k / 2 + 1], xb);
                    const float2 d1a = __fadd2_rn(x1[k / 2], xa), d1b = __fadd2_rn(x1[k / 2 + 1], xb);
                    q0 = __ffma2_rn(d0a, d0a, q0);
                    q1 = __ffma2_rn(d1a, d1a, q1);
                    q0 = __ffma2_rn(d0b, d0b, q0);
                    q1 = __ffma2_rn(d1b, d1b, q1);
                }
            }
            const float k0 = kernel_from_s<KIND>(-(q0.x + q0.y));
            const float k1 = kernel_from_s<KIND>(-(q1.x + q1.y));
            const float2 kk0 = make_float2(k0, k0), kk1 = make_float2(k1, k1);
#pragma unroll
            for (int c = 0; c < RPM; c += 4) {
                if (c < R) {
                    const float4 v4 = *reinterpret_cast<const float4*>(&sv[jj][c]);   // broadcast
                    const float2 va = make_float2(v4.x, v4.y), vb = make_float2(v4.z, v4.w);
                    acc0[c / 2] = __ffma2_rn(kk0, va, acc0[c / 2]);
                    acc1[c / 2] = __ffma2_rn(kk1, va, acc1[c / 2]);
                    acc0[c / 2 + 1] = __ffma2_rn(kk0, vb, acc0[c / 2 + 1]);
                    acc1[c / 2 + 1] = __ffma2_rn(kk1, vb, acc1[c / 2 + 1]);
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < RPM; ++c) {
        if (c < R) {
            const float s0 = (c & 1) ? acc0[c / 2].y : acc0[c / 2].x;
            const float s1 = (c & 1) ? acc1[c / 2].y : acc1[c / 2].x;
            if (n_split == 1) {
                if (i0 < Nr) {
                    float v = a2 * s0;
                    if (noise != 0.0f) v = fmaf(noise, Vnoise[(int64_t)c * Nc + i0], v);
                    out[(int64_t)c * ld_out + i0] = v;
                }
                if (i1 < Nr) {
                    float v = a2 * s1;
                    if (noise != 0.0f) v = fmaf(noise, Vnoise[(int64_t)c * Nc + i1], v);
                    out[(int64_t)c * ld_out + i1] = v;
                }
            } else {
                float* pp = partial + ((int64_t)blockIdx.y * RPM + c) * ld_part;
                if (i0 < Nr) pp[i0] = s0;
                if (i1 < Nr) pp[i1] = s1;
            }
        }
    }
}

// out[c][i] = scale_c * sum_s partial[s][c][i] + noise * Vnoise[c][i];
// scale_c = outscale[c] if outscale != null, else scale_const.
__global__ void split_reduce_kernel(const float* __restrict__ partial, int n_split, int64_t ld_part, int RP,
                                    int64_t Nr, int R, const float* __restrict__ outscale, float scale_const,
                                    float noise, const float* __restrict__ Vnoise, int64_t ld_v,
                                    float* __restrict__ out, int64_t ld_out) {
    const int c = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Nr || c >= R) return;
    float s = 0.0f;
    for (int sp = 0; sp < n_split; ++sp) s += partial[((int64_t)sp * RP + c) * ld_part + i];
    float v = s * (outscale ? outscale[c] : scale_const);
    if (noise != 0.0f) v = fmaf(noise, Vnoise[(int64_t)c * ld_v + i], v);
    out[(int64_t)c * ld_out + i] = v;
}

template <int KIND, int DPM>
cudaError_t simt_dispatch_r(const SimtPlan& pl, int RPM, dim3 grid, const float* Xr, const float* Xc,
                            const float* V, int64_t Nr, int64_t Nc, int R, float a2, float noise,
                            const float* Vn, float* out, int64_t ld_out, float* part, int64_t ld_part,
                            cudaStream_t s) {
    switch (RPM) {
#define GPK_SIMT_CASE(RP)                                                                                        \
        case RP:                                                                                                 \
            kmvm_simt_kernel<KIND, DPM, RP><<<grid, kSimtThreads, 0, s>>>(Xr, Xc, V, Nr, Nc, pl.dp, R, pl.n_split, \
                                                                          a2, noise, Vn, out, ld_out, part,     \
                                                                          ld_part);                              \
            break;
        GPK_SIMT_CASE(4) GPK_SIMT_CASE(8) GPK_SIMT_CASE(12) GPK_SIMT_CASE(16)
        GPK_SIMT_CASE(20) GPK_SIMT_CASE(24) GPK_SIMT_CASE(28) GPK_SIMT_CASE(32)
#undef GPK_SIMT_CASE
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int KIND>
cudaError_t simt_dispatch(const SimtPlan& pl, dim3 grid, const float* Xr, const float* Xc, const float* V,
                          int64_t Nr, int64_t Nc, int R, float a2, float noise, const float* Vn, float* out,
                          int64_t ld_out, float* part, int64_t ld_part, cudaStream_t s) {
    const int DPMr = pl.dp <= 8 ? 8 : (pl.dp <= 16 ? 16 : (pl.dp <= 32 ? 32 : 64));
    switch (DPMr) {
        case 8: return simt_dispatch_r<KIND, 8>(pl, pl.R_pad, grid, Xr, Xc, V, Nr, Nc, R, a2, noise, Vn, out, ld_out, part, ld_part, s);
        case 16: return simt_dispatch_r<KIND, 16>(pl, pl.R_pad, grid, Xr, Xc, V, Nr, Nc, R, a2, noise, Vn, out, ld_out, part, ld_part, s);
        case 32: return simt_dispatch_r<KIND, 32>(pl, pl.R_pad, grid, Xr, Xc, V, Nr, Nc, R, a2, noise, Vn, out, ld_out, part, ld_part, s);
        default: return simt_dispatch_r<KIND, 64>(pl, pl.R_pad, grid, Xr, Xc, V, Nr, Nc, R, a2, noise, Vn, out, ld_out, part, ld_part, s);
    }
}

}  // namespace

SimtPlan simt_plan(const Ctx* ctx, int64_t Nr, int64_t Nc, int d, int R) {
    SimtPlan p;
    p.dp = ((d + 3) / 4) * 4;
    p.R_pad = ((R + 3) / 4) * 4;   // accumulators for the columns in use only (R <= 32)
    p.n_rowblk = (int)((Nr + kSimtRows - 1) / kSimtRows);
    const int64_t ntiles = (Nc + kSimtTile - 1) / kSimtTile;
    const int64_t target = (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148) * 16;
    int64_t sp = (target + p.n_rowblk - 1) / p.n_rowblk;
    const int64_t max_sp = ntiles / 4 > 0 ? ntiles / 4 : 1;
    if (sp > max_sp) sp = max_sp;
    if (sp > 64) sp = 64;
    if (sp < 1) sp = 1;
    p.n_split = (int)sp;
    return p;
}

size_t simt_partial_floats(const SimtPlan& p, int64_t Nr) {
    return p.n_split > 1 ? (size_t)p.n_split * p.R_pad * (size_t)Nr : 0;
}

int launch_kmvm_simt(Ctx* ctx, const SimtPlan& pl, const MvmArgs& a, float outputscale, const float* Xrs,
                     const float* Xcs, const float* V, float* partial, cudaStream_t s) {
    if (a.R > 32) return GP_ERR_UNSUPPORTED;
    dim3 grid((unsigned)pl.n_rowblk, (unsigned)pl.n_split);
    cudaError_t e;
    switch (a.kernel) {
        case GP_KERNEL_RBF:
            e = simt_dispatch<GP_KERNEL_RBF>(pl, grid, Xrs, Xcs, V, a.Nr, a.Nc, a.R, outputscale, a.noise, a.Vnoise,
                                             a.out, a.ld_out, partial, a.Nr, s);
            break;
        case GP_KERNEL_MATERN32:
            e = simt_dispatch<GP_KERNEL_MATERN32>(pl, grid, Xrs, Xcs, V, a.Nr, a.Nc, a.R, outputscale, a.noise,
                                                  a.Vnoise, a.out, a.ld_out, partial, a.Nr, s);
            break;
        case GP_KERNEL_MATERN12:
            e = simt_dispatch<GP_KERNEL_MATERN12>(pl, grid, Xrs, Xcs, V, a.Nr, a.Nc, a.R, outputscale, a.noise,
                                                  a.Vnoise, a.out, a.ld_out, partial, a.Nr, s);
            break;
        case GP_KERNEL_MATERN52:
            e = simt_dispatch<GP_KERNEL_MATERN52>(pl, grid, Xrs, Xcs, V, a.Nr, a.Nc, a.R, outputscale, a.noise,
                                                  a.Vnoise, a.out, a.ld_out, partial, a.Nr, s);
            break;
        default: return GP_ERR_INVALID;
    }
    ctx->launches++;
    if (e != cudaSuccess) return GP_ERR_CUDA;
    if (pl.n_split > 1) {
        dim3 g2((unsigned)((a.Nr + 255) / 256), (unsigned)a.R);
        split_reduce_kernel<<<g2, 256, 0, s>>>(partial, pl.n_split, a.Nr, pl.R_pad, a.Nr, a.R, nullptr, outputscale,
                                               a.noise, a.Vnoise, a.Nc, a.out, a.ld_out);
        ctx->launches++;
        if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    }
    return GP_OK;
}

int launch_split_reduce(Ctx* ctx, const float* partial, int n_split, int64_t ld_part, int64_t Nr, int R,
                        int RP, const float* outscale, float outscale_const, float noise, const float* Vnoise,
                        int64_t ld_v, float* out, int64_t ld_out, cudaStream_t s) {
    dim3 g((unsigned)((Nr + 255) / 256), (unsigned)R);
    split_reduce_kernel<<<g, 256, 0, s>>>(partial, n_split, ld_part, RP, Nr, R, outscale, outscale_const, noise,
                                          Vnoise, ld_v, out, ld_out);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

}  // namespace gpk
