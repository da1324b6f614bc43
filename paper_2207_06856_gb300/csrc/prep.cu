// Operand preparation for the kernel MVM (Sec. 4.1 "Half Precision
// Matrix Vector Multiplies" and the downscaling paragraph that follows it).
//
// Tensor-core operands.  For point i with scaled inputs x^_i = c x_i / l (c
// from kernel_from_s) and t_i = -|x^_i|^2 / 2, two K-major rows are written:
//     XA[i] = [ x^_i , 1 .. 1 (nt) , t_i^(0) .. t_i^(nt-1) , 0 .. ]   (row side)
//     XB[i] = [ x^_i , t_i^(0) .. t_i^(nt-1) , 1 .. 1 (nt) , 0 .. ]   (column side)
// so one tensor-core contraction XA[i] . XB[j] yields
//     s_ij = x^_i . x^_j + t_i + t_j = -c^2 r_ij^2 / 2
// directly (the row norms ride along in the contraction dimension).  t is
// carried as nt terms of the operand type (t = sum of terms to ~2^-22
// relative for FP16, ~2^-24 for BF16), and |x^|^2 is taken, in FP64, from the
// rounded operands the tensor core sees, so a point paired with itself gives
// s = 0 up to FP32 accumulation rounding.  With the hi+lo split the scaled
// input is x^ = hi + lo and the contraction carries hi.hi + hi.lo + lo.hi.
//
// Right-hand sides.  The paper downscales every MVM input by N^{-1/2} to keep
// half-precision values in range.  With FP32 accumulation the output cannot
// overflow, so only the operand range matters; by default each column c is
// scaled by the power of two s_c that brings max|v_c| into [1/2, 1) (exact,
// no rounding), and the result is multiplied back by a^2 / s_c in FP32.  The
// paper-literal N^{-1/2} scaling is available as an option.
#include "gpk_internal.cuh"

namespace gpk {

template <typename T> __device__ __forceinline__ T to_op(float x);
template <> __device__ __forceinline__ __half to_op<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 to_op<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <typename T> __device__ __forceinline__ float from_op(T x);
template <> __device__ __forceinline__ float from_op<__half>(__half x) { return __half2float(x); }
template <> __device__ __forceinline__ float from_op<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

OperandLayout make_layout(int d, int prec, int xsplit, int vsplit, int psplit) {
    OperandLayout L;
    L.prec = prec;
    L.xsplit = xsplit;
    L.vsplit = vsplit;
    L.psplit = psplit;
    L.nt = (prec == GP_PREC_BF16) ? 3 : 2;
    L.kdim = (xsplit ? 3 * d : d) + 2 * L.nt;
    L.k_pad = L.kdim <= 16 ? 16 : (L.kdim <= 32 ? 32 : (L.kdim <= 64 ? 64 : (L.kdim <= 128 ? 128 : 0)));
    return L;
}

float kernel_input_scale(int kernel) {
    switch (kernel) {
        case GP_KERNEL_RBF: return 1.2011224087864498f;       // sqrt(log2 e)
        case GP_KERNEL_MATERN32: return 2.449489742783178f;   // sqrt(6)
        case GP_KERNEL_MATERN12: return 1.4142135623730951f;  // sqrt(2)
        case GP_KERNEL_MATERN52: return 3.1622776601683795f;  // sqrt(10)
    }
    return 0.0f;
}

// One thread per (padded) point.  XA or XB may be null.
__device__ __forceinline__ unsigned float_order(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float order_float(unsigned s) {
    return __uint_as_float((s & 0x80000000u) ? (s & 0x7FFFFFFFu) : ~s);
}

__global__ void bbox_kernel(const float* __restrict__ X, int64_t total, int d, unsigned* __restrict__ bb) {
    __shared__ unsigned smin[64], smax[64];
    for (int k = threadIdx.x; k < d; k += blockDim.x) { smin[k] = 0xFFFFFFFFu; smax[k] = 0u; }
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned o = float_order(X[e]);
        const int k = (int)(e % d);
        atomicMin(&smin[k], o);
        atomicMax(&smax[k], o);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        atomicMin(&bb[k], smin[k]);
        atomicMax(&bb[d + k], smax[k]);
    }
}

int launch_bbox(Ctx* ctx, const float* X, int64_t N, int d, unsigned* bb, cudaStream_t s) {
    if (cudaMemsetAsync(bb, 0xFF, sizeof(unsigned) * d, s) != cudaSuccess) return GP_ERR_CUDA;
    if (cudaMemsetAsync(bb + d, 0x00, sizeof(unsigned) * d, s) != cudaSuccess) return GP_ERR_CUDA;
    const int64_t total = N * d;
    int64_t blocks = (total + 256 * 16 - 1) / (256 * 16);
    if (blocks > 512) blocks = 512;
    bbox_kernel<<<(unsigned)blocks, 256, 0, s>>>(X, total, d, bb);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

template <typename T>
__global__ void prep_x_kernel(const float* __restrict__ X, int64_t N, int64_t N_pad, int d, ScaleVec inv,
                              const unsigned* __restrict__ bb, int xsplit, int nt, int k_pad, T* __restrict__ XA,
                              T* __restrict__ XB, int* err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    T* a = XA ? XA + i * k_pad : nullptr;
    T* b = XB ? XB + i * k_pad : nullptr;
    const T zero = to_op<T>(0.0f);
    if (i >= N) {
        for (int k = 0; k < k_pad; ++k) {
            if (a) a[k] = zero;
            if (b) b[k] = zero;
        }
        return;
    }
    const float* x = X + i * d;
    double nrm = 0.0;
    for (int k = 0; k < d; ++k) {
        const float ctr = bb ? 0.5f * (order_float(bb[k]) + order_float(bb[d + k])) : 0.0f;
        const float xh = (x[k] - ctr) * inv.v[k];
        const T hi = to_op<T>(xh);
        const float fhi = from_op<T>(hi);
        if (xsplit) {
            const T lo = to_op<T>(xh - fhi);
            const float flo = from_op<T>(lo);
            if (a) { a[k] = hi; a[d + k] = hi; a[2 * d + k] = lo; }
            if (b) { b[k] = hi; b[d + k] = lo; b[2 * d + k] = hi; }
            nrm += (double)fhi * fhi + 2.0 * (double)fhi * flo;
        } else {
            if (a) a[k] = hi;
            if (b) b[k] = hi;
            nrm += (double)fhi * fhi;
        }
    }
    const int col = xsplit ? 3 * d : d;
    double t = -0.5 * nrm;
    if (sizeof(T) == 2 && nt == 2 && !(t > -60000.0)) {
        // FP16 cannot carry this norm (inputs hundreds of lengthscales out):
        // record a range error instead of returning a meaningless result.
        atomicCAS(err, 0, (int)DEV_NONFINITE);
    }
    const T one = to_op<T>(1.0f);
    for (int m = 0; m < nt; ++m) {
        const T q = to_op<T>((float)t);
        t -= (double)from_op<T>(q);
        if (a) { a[col + m] = one; a[col + nt + m] = q; }
        if (b) { b[col + m] = q; b[col + nt + m] = one; }
    }
    for (int k = col + 2 * nt; k < k_pad; ++k) {
        if (a) a[k] = zero;
        if (b) b[k] = zero;
    }
}

int launch_prep_x(Ctx* ctx, const OperandLayout& L, const float* X, int64_t N, int64_t N_pad, int d,
                  const ScaleVec& inv, const unsigned* bb, void* XA, void* XB, cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = (N_pad + threads - 1) / threads;
    if (L.prec == GP_PREC_BF16) {
        prep_x_kernel<__nv_bfloat16><<<(unsigned)blocks, threads, 0, s>>>(
            X, N, N_pad, d, inv, bb, L.xsplit, L.nt, L.k_pad, (__nv_bfloat16*)XA, (__nv_bfloat16*)XB, ctx->dev_err);
    } else {
        prep_x_kernel<__half><<<(unsigned)blocks, threads, 0, s>>>(X, N, N_pad, d, inv, bb, L.xsplit, L.nt, L.k_pad,
                                                                   (__half*)XA, (__half*)XB, ctx->dev_err);
    }
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

// FP32 SIMT operand: Xs[i*dp + k] = x_ik * inv_ls[k] for k < d, 0 up to dp.
__global__ void prep_x_f32_kernel(const float* __restrict__ X, int64_t N, int64_t N_pad, int d, int dp,
                                  ScaleVec inv, float* __restrict__ Xs) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N_pad) return;
    float* o = Xs + i * dp;
    for (int k = 0; k < dp; ++k) o[k] = (i < N && k < d) ? X[i * d + k] * inv.v[k] : 0.0f;
}

int launch_prep_x_f32(Ctx* ctx, const float* X, int64_t N, int64_t N_pad, int d, int dp, const ScaleVec& inv,
                      float* Xs, cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = (N_pad + threads - 1) / threads;
    prep_x_f32_kernel<<<(unsigned)blocks, threads, 0, s>>>(X, N, N_pad, d, dp, inv, Xs);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

// Per-column max |v| as float bits (non-negative floats order like unsigned ints).
// grid = (chunks, R); cmax_bits must be zeroed before the launch.
__global__ void v_colmax_kernel(const float* __restrict__ V, int64_t N, unsigned* __restrict__ cmax_bits) {
    const int c = blockIdx.y;
    const float* v = V + (int64_t)c * N;
    float m = 0.0f;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
        const float a = fabsf(v[j]);
        m = (a > m || a != a) ? a : m;   // NaN propagates
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float q = __shfl_xor_sync(0xffffffffu, m, o);
        m = (q > m || q != q) ? q : m;
    }
    __shared__ float wm[32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) wm[w] = m;
    __syncthreads();
    if (w == 0) {
        m = (l < (int)(blockDim.x >> 5)) ? wm[l] : 0.0f;
        for (int o = 16; o > 0; o >>= 1) {
            const float q = __shfl_xor_sync(0xffffffffu, m, o);
            m = (q > m || q != q) ? q : m;
        }
        if (l == 0) atomicMax(cmax_bits + c, __float_as_uint(m));
    }
}

int launch_v_colmax(Ctx* ctx, const float* V, int64_t N, int R, unsigned* cmax_bits, cudaStream_t s) {
    if (cudaMemsetAsync(cmax_bits, 0, sizeof(unsigned) * R, s) != cudaSuccess) return GP_ERR_CUDA;
    const int threads = 256;
    int64_t chunks = (N + threads * 8 - 1) / (threads * 8);
    if (chunks > 1024) chunks = 1024;
    v_colmax_kernel<<<dim3((unsigned)chunks, (unsigned)R), threads, 0, s>>>(V, N, cmax_bits);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

// Cast V (N x R col-major FP32) to Vt (R_pad x N_pad, operand type), each
// column scaled by s_c; outscale[c] = a^2 / s_c.  Two elements per thread.
template <typename T>
__global__ void v_cast_kernel(const float* __restrict__ V, int64_t N, int64_t N_pad, int R, int R_pad,
                              const unsigned* __restrict__ cmax_bits, int scale_mode, int vsplit, float a2,
                              T* __restrict__ Vt, float* __restrict__ outscale, int* err) {
    const int c = blockIdx.y;
    float sc = 1.0f, os = a2;
    if (c < R) {
        if (scale_mode == 1) {
            sc = rsqrtf((float)N);
            os = a2 * sqrtf((float)N);
        } else {
            const float cm = __uint_as_float(cmax_bits[c]);
            if (!(cm <= 3.0e38f)) {
                if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(err, 0, (int)DEV_NONFINITE);
                sc = 0.0f;
                os = 0.0f;
            } else if (cm > 0.0f) {
                int e;
                frexpf(cm, &e);          // cm = m 2^e, m in [1/2, 1)
                sc = ldexpf(1.0f, -e);
                os = ldexpf(a2, e);
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) outscale[c] = (c < R) ? os : 0.0f;
    const int64_t j = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (j >= N_pad) return;
    const float* v = V + (int64_t)c * N;
    const float v0 = (c < R && j < N) ? v[j] * sc : 0.0f;
    const float v1 = (c < R && j + 1 < N) ? v[j + 1] * sc : 0.0f;
    T* o = Vt + (int64_t)c * N_pad + j;
    const T h0 = to_op<T>(v0), h1 = to_op<T>(v1);
    o[0] = h0;
    o[1] = h1;
    if (vsplit) {
        T* q = Vt + (int64_t)(R_pad + c) * N_pad + j;
        q[0] = to_op<T>(v0 - from_op<T>(h0));
        q[1] = to_op<T>(v1 - from_op<T>(h1));
    }
}

// FP32 right-hand sides for the FP32 value product of the pair engine:
// V32 (4 rows x N_pad, row stride N_pad) = V (R x N) zero-padded in rows and
// columns; outscale = a^2 (the epilogue's sums are of unscaled v), or 0 with
// DEV_NONFINITE recorded for a column holding a non-finite value.
__global__ void v_pack32_kernel(const float* __restrict__ V, int64_t N, int64_t N_pad, int R,
                                const unsigned* __restrict__ cmax_bits, float a2, float* __restrict__ V32,
                                float* __restrict__ outscale, int* err) {
    const int c = blockIdx.y;
    bool ok = true;
    if (c < R) ok = __uint_as_float(cmax_bits[c]) <= 3.0e38f;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        outscale[c] = (c < R && ok) ? a2 : 0.0f;
        if (!ok) atomicCAS(err, 0, (int)DEV_NONFINITE);
    }
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < N_pad; j += (int64_t)gridDim.x * blockDim.x)
        V32[(int64_t)c * N_pad + j] = (c < R && ok && j < N) ? V[(int64_t)c * N + j] : 0.0f;
}

int launch_v_pack32(Ctx* ctx, const float* V, int64_t N, int64_t N_pad, int R, const unsigned* cmax_bits,
                    double outputscale, float* V32, float* outscale, cudaStream_t s) {
    if (R > 4) return GP_ERR_UNSUPPORTED;
    const int64_t want = (N_pad + 255) / 256;
    const unsigned blocks = (unsigned)(want < 1024 ? want : 1024);
    v_pack32_kernel<<<dim3(blocks, 4), 256, 0, s>>>(V, N, N_pad, R, cmax_bits, (float)outputscale, V32, outscale,
                                                     ctx->dev_err);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

int launch_v_cast(Ctx* ctx, int prec, int scale_mode, int vsplit, const float* V, int64_t N, int64_t N_pad, int R,
                  int R_pad, const unsigned* cmax_bits, double outputscale, void* Vt, float* outscale,
                  cudaStream_t s) {
    const int threads = 256;
    const int64_t blocks = (N_pad / 2 + threads - 1) / threads;
    dim3 grid((unsigned)blocks, (unsigned)R_pad);
    if (prec == GP_PREC_BF16) {
        v_cast_kernel<__nv_bfloat16><<<grid, threads, 0, s>>>(V, N, N_pad, R, R_pad, cmax_bits, scale_mode, vsplit,
                                                              (float)outputscale, (__nv_bfloat16*)Vt,
                                                              outscale, ctx->dev_err);
    } else {
        v_cast_kernel<__half><<<grid, threads, 0, s>>>(V, N, N_pad, R, R_pad, cmax_bits, scale_mode, vsplit,
                                                       (float)outputscale, (__half*)Vt, outscale,
                                                       ctx->dev_err);
    }
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

}  // namespace gpk
