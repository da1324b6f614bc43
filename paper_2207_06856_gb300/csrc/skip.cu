// Compact-support tile skipping for the tensor-core MVM (Sec. 3.1, "finite
// precision kernels have finite support", Fig. 2c; App. C.1).
//
// In a finite format a stationary kernel is exactly zero beyond the distance at
// which its value drops below half the smallest subnormal: the kernel tile P of
// the tensor-core MVM stores FP16 (or BF16) values rounded to nearest, so every
// pair with k(r) < tau (tau = 2^-25 for FP16, 2^-134 for BF16) contributes an
// exact 0.  For each 128-row tile the bounding box of its scaled operands
// x^ = c (x - centre) / l (as the MMA sees them: the FP16 value, plus the lo
// term when the inputs are split) bounds every pair distance from below:
//     |x^_i - x^_j|^2 >= sum_k gap_k^2,  gap_k = max(0, lo_J,k - hi_I,k, lo_I,k - hi_J,k),
// and the exp2 argument s = -|x^_i - x^_j|^2 / 2 from above.  A (row-tile pair,
// column tile) whose bound lies below s*, the argument beyond which the kernel
// value underflows (with a margin of 0.5 for the approximate SFU functions and
// the MMA's accumulation), is skipped: its P would be all zeros, so the result
// is bit-identical to the full MVM.
#include "gpk_internal.cuh"

#include <math.h>

namespace gpk {

namespace {

// The float value of operand element k of a row (hi, plus lo when split): A
// rows hold [hi | hi | lo], B rows [hi | lo | hi] (prep_x_kernel).
template <typename T>
__device__ __forceinline__ float op_value(const T* row, int k, int d, int xsplit, int is_b) {
    float v = (float)row[k];
    if (xsplit) v += (float)row[(is_b ? d : 2 * d) + k];
    return v;
}

// box[t][0..d) = per-dimension minimum, box[t][d..2d) = maximum over the real
// rows of 128-row tile t (an empty tile gets +inf / -inf).
template <typename T>
__global__ void tile_box_kernel(const T* __restrict__ Xop, int64_t N, int k_pad, int d, int xsplit, int is_b,
                                float* __restrict__ box) {
    const int t = blockIdx.x;
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        float lo = INFINITY, hi = -INFINITY;
        for (int r = 0; r < 128; ++r) {
            const int64_t i = (int64_t)t * 128 + r;
            if (i >= N) break;
            const float v = op_value(Xop + i * k_pad, k, d, xsplit, is_b);
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
        box[(int64_t)t * 2 * d + k] = lo;
        box[(int64_t)t * 2 * d + d + k] = hi;
    }
}

__device__ __forceinline__ double gap2(const float* a, const float* b, int d) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        const double g = fmax(0.0, fmax((double)b[k] - (double)a[d + k], (double)a[k] - (double)b[d + k]));
        s += g * g;
    }
    return s;
}

// mask[ip][w] bit l: column tile 32 w + l of row-tile pair ip is evaluated.
// count: number of evaluated (pair, tile) entries.
__global__ void skip_mask_kernel(const float* __restrict__ rbox, int n_rtiles, const float* __restrict__ cbox,
                                 int n_jt, int n_ip, int words, int d, double two_thr, uint32_t* __restrict__ mask,
                                 unsigned long long* __restrict__ count) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int64_t wid = gid >> 5;   // (ip, w)
    const bool in = wid < (int64_t)n_ip * words;
    bool on = false;
    if (in) {
        const int ip = (int)(wid / words), w = (int)(wid % words);
        const int jt = w * 32 + lane;
        if (jt < n_jt) {
            const float* cb = cbox + (int64_t)jt * 2 * d;
            for (int a = 0; a < 2; ++a) {
                const int rt = 2 * ip + a;
                if (rt < n_rtiles && gap2(rbox + (int64_t)rt * 2 * d, cb, d) < two_thr) on = true;
            }
        }
    }
    const unsigned bits = __ballot_sync(0xffffffffu, on);
    if (in && lane == 0) {
        mask[wid] = bits;
        atomicAdd(count, (unsigned long long)__popc(bits));
    }
}

}  // namespace

// -s* for the kernel and the P tile's format: every s <= s* gives a kernel
// value that rounds to zero.  RBF: k = 2^s.  Matern: k = poly(u) e^-u with
// u = sqrt(-s) (the forms of kernel_from_s); u* from bisection on the monotone
// tail, then a margin of 0.5 in u.
double skip_threshold(int kernel, int prec) {
    const double log2_tau = prec == GP_PREC_BF16 ? -134.0 : -25.0;
    if (kernel == GP_KERNEL_RBF) return -log2_tau + 0.5;
    auto logk = [kernel](double u) {
        double poly = 1.0;
        if (kernel == GP_KERNEL_MATERN32) poly = 1.0 + u;
        else if (kernel == GP_KERNEL_MATERN52) poly = 1.0 + u + u * u / 3.0;
        return (log(poly) - u) / log(2.0);
    };
    double lo = 0.0, hi = 1.0;
    while (logk(hi) >= log2_tau) hi *= 2.0;
    for (int i = 0; i < 200; ++i) {
        const double mid = 0.5 * (lo + hi);
        if (logk(mid) >= log2_tau) lo = mid; else hi = mid;
    }
    const double u = hi + 0.5;
    return u * u;
}

size_t skip_words(const TcPlan& p) { return (size_t)p.n_it * (size_t)((p.n_jt + 31) / 32); }

int prepare_skip(Ctx* ctx, KOp& op, cudaStream_t s) {
    const TcPlan& p = op.tp;
    const int d = op.d;
    const int n_rtiles = (int)((op.Nr + 127) / 128);
    const int words = (p.n_jt + 31) / 32;
    if (cudaMemsetAsync(op.skip_count, 0, sizeof(unsigned long long), s) != cudaSuccess) return GP_ERR_CUDA;
    if (op.prec == GP_PREC_BF16) {
        tile_box_kernel<__nv_bfloat16><<<n_rtiles, 32, 0, s>>>((const __nv_bfloat16*)op.XA, op.Nr, op.lay.k_pad, d,
                                                               op.lay.xsplit, 0, op.rbox);
        tile_box_kernel<__nv_bfloat16><<<p.n_jt, 32, 0, s>>>((const __nv_bfloat16*)op.XB, op.Nc, op.lay.k_pad, d,
                                                             op.lay.xsplit, 1, op.cbox);
    } else {
        tile_box_kernel<__half><<<n_rtiles, 32, 0, s>>>((const __half*)op.XA, op.Nr, op.lay.k_pad, d, op.lay.xsplit, 0,
                                                        op.rbox);
        tile_box_kernel<__half><<<p.n_jt, 32, 0, s>>>((const __half*)op.XB, op.Nc, op.lay.k_pad, d, op.lay.xsplit, 1,
                                                      op.cbox);
    }
    const double two_thr = 2.0 * skip_threshold(op.kernel, op.prec);
    const int64_t threads = (int64_t)p.n_it * words * 32;
    skip_mask_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(op.rbox, n_rtiles, op.cbox, p.n_jt, p.n_it,
                                                                      words, d, two_thr, op.mask, op.skip_count);
    ctx->launches += 3;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

}  // namespace gpk
