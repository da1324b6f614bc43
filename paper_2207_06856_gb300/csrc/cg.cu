// Enhanced-stability preconditioned CG (Alg. 2) and textbook
// preconditioned CG (Alg. 1), for R right-hand sides at once with per-column
// scalars (mBCG, App. A).
//
// Alg. 2 as run here (r = K x - b sign convention of the paper):
//   r_0 = K(x_0) - b,  z_0 = P^{-1} r_0,  d_0 = -z_0,  log gamma_0 = LSE(r_0^T z_0)
//   repeat:  log alpha = log gamma - LSE(d^T K d);  x += alpha d;  r += alpha K d
//            r <- r - sum_j (zeta_j^T r) rho_j        (re-orthogonalisation)
//            z = P^{-1} r;  log gamma' = LSE(r^T z);  beta = exp(log gamma' - log gamma)
//            d = -z + beta d
// The loop condition is read as "relative residual above tol" (the printed
// condition is inverted), d is formed from z (the printed -r is the P = I
// case), and P(.) applies P^{-1} (Eq. woodbury).
//
// LSE.  The paper's transformation log w^T z = y_max + log sum s_i
// exp(y_i - y_max), y_i = log|w_i| + log|z_i|, holds for any shift.  The GPU
// takes the shift as a power of two: each thread sums its FP32 x FP32
// products exactly as float-float pairs, converts the pair to (e, s) with
// |s| < 1 and partial sum = s 2^e in FP64, partial pairs are merged in a
// fixed order, and LSE = log(s) + e log 2.  No per-element transcendental is
// needed and nothing can overflow or underflow.  A non-positive s is a
// breakdown of that column.
//
// Re-orthogonalisation.  In PCG the residuals are mutually orthogonal in the
// P^{-1} inner product, so the default stores rho_j = r_j / sqrt(gamma_j),
// zeta_j = z_j / sqrt(gamma_j) and projects r <- r - sum_j (zeta_j^T r) rho_j
// (classical Gram-Schmidt, optionally twice; coefficients accumulated in
// FP64).  GP_REORTH_EUCLID stores u_j = r_j / ||r_j|| (the literal form).
//
// The only host/device round trip per iteration is a 4-byte copy of the
// number of still-active columns.
#include "gpk_internal.cuh"

#include <math.h>
#include <string.h>
#include <vector>

namespace gpk {

namespace {

constexpr int kDotThreads = 256;
constexpr int kDotPerThread = 8;
constexpr int kDotChunk = kDotThreads * kDotPerThread;
constexpr int kEmptyExp = -100000;


struct Lse {
    double s;
    int e;
};

__device__ __forceinline__ void lse_add(Lse& a, double p) {
    if (p == 0.0) return;
    int ep;
    frexp(p, &ep);   // |p| < 2^ep
    if (ep > a.e) {
        a.s = (a.e == kEmptyExp) ? 0.0 : ldexp(a.s, a.e - ep);
        a.e = ep;
    }
    a.s += ldexp(p, -a.e);
}

__device__ __forceinline__ void lse_merge(Lse& a, const Lse& b) {
    if (b.e == kEmptyExp) return;
    if (a.e == kEmptyExp) { a = b; return; }
    if (b.e > a.e) {
        a.s = ldexp(a.s, a.e - b.e) + b.s;
        a.e = b.e;
    } else {
        a.s += ldexp(b.s, b.e - a.e);
    }
}

__device__ __forceinline__ Lse lse_shfl(const Lse& a, int o) {
    Lse b;
    b.s = __shfl_xor_sync(0xffffffffu, a.s, o);
    b.e = __shfl_xor_sync(0xffffffffu, a.e, o);
    return b;
}

// (hi, lo) += a * b exactly up to float-float rounding: TwoProd via FMA, then
// Knuth's TwoSum of hi with the product's high part and a plain add of the
// low parts.  Explicit round-to-nearest operations keep the compiler from
// contracting or reassociating the error terms.
__device__ __forceinline__ void ff_add_prod(float& hi, float& lo, float a, float b) {
    const float p = __fmul_rn(a, b);
    const float pe = __fmaf_rn(a, b, -p);          // a * b = p + pe exactly
    const float s = __fadd_rn(hi, p);
    const float bb = __fsub_rn(s, hi);
    const float se = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));   // hi + p = s + se
    hi = s;
    lo = __fadd_rn(lo, __fadd_rn(se, pe));
}

// Float-float addition (a_hi, a_lo) += (b_hi, b_lo): TwoSum of the high parts,
// low parts and the rounding error added (the pair is not renormalised).
__device__ __forceinline__ void ff_add(float& hi, float& lo, float bh, float bl) {
    const float s = __fadd_rn(hi, bh);
    const float bb = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, bl), e);
}

// part[(c * nblk + blk) * 3 + {0,1,2}] = (s, e, sum a^2) of column c over this chunk.
__global__ void __launch_bounds__(kDotThreads)
dots_kernel(const float* __restrict__ A, const float* __restrict__ B, int64_t N, int nblk,
            const int* __restrict__ active, double* __restrict__ part) {
    const int c = blockIdx.y;
    if (active && !active[c]) return;
    const float* a = A + (int64_t)c * N;
    const float* b = B + (int64_t)c * N;
    // The chunk's products are formed exactly as float-float pairs (TwoProd
    // with an FMA) and reduced with TwoSum on the FP32 pipe, through the warp
    // and the block in a fixed order (FP64 arithmetic is scarce on this GPU);
    // only the block's pair enters the FP64 (s, e) form.  The pair carries a
    // 48-bit significand; FP32 range bounds the chunk sums (|sum| < 2^127).
    float sh = 0.0f, sl = 0.0f, nh = 0.0f, nl = 0.0f;
    const int64_t base = (int64_t)blockIdx.x * kDotChunk;
#pragma unroll
    for (int q = 0; q < kDotPerThread; ++q) {
        const int64_t i = base + q * kDotThreads + threadIdx.x;
        if (i < N) {
            const float av = a[i], bv = b[i];
            ff_add_prod(sh, sl, av, bv);
            ff_add_prod(nh, nl, av, av);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const float h1 = __shfl_xor_sync(0xffffffffu, sh, o), l1 = __shfl_xor_sync(0xffffffffu, sl, o);
        const float h2 = __shfl_xor_sync(0xffffffffu, nh, o), l2 = __shfl_xor_sync(0xffffffffu, nl, o);
        ff_add(sh, sl, h1, l1);
        ff_add(nh, nl, h2, l2);
    }
    __shared__ float4 sw[kDotThreads / 32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sw[w] = make_float4(sh, sl, nh, nl);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 t = sw[0];
        for (int q = 1; q < kDotThreads / 32; ++q) {
            ff_add(t.x, t.y, sw[q].x, sw[q].y);
            ff_add(t.z, t.w, sw[q].z, sw[q].w);
        }
        Lse acc{0.0, kEmptyExp};
        lse_add(acc, (double)t.x + (double)t.y);
        double* o = part + ((int64_t)c * nblk + blockIdx.x) * 3;
        o[0] = acc.s;
        o[1] = (double)acc.e;
        o[2] = (double)t.z + (double)t.w;
    }
}

enum ScalarMode { SC_INIT = 0, SC_ALPHA = 1, SC_BETA = 2, SC_BNORM = 3 };

// One block of one warp per column, so the FP64 merges and recurrences of the
// columns run on different SMs (FP64 throughput is per SM and low on this
// GPU): merge the partials of column c in a fixed order, then run the scalar
// step of Alg. 1 / Alg. 2.  The last block to finish counts the active
// columns (n_active[2] is its ticket, returned to 0 by that block).
__global__ void __launch_bounds__(32)
scalar_kernel(int mode, int stable, const double* __restrict__ part, int nblk, int R, ColState* __restrict__ st,
              int k, double tol, int min_iter, double* __restrict__ ahist, double* __restrict__ bhist,
              double* __restrict__ rhist, int* __restrict__ n_active, int* __restrict__ aflags) {
    const int l = threadIdx.x;
    {
        const int c = blockIdx.x;
        ColState& S = st[c];
        const bool act = (mode == SC_INIT || mode == SC_BNORM) ? true : (S.active != 0);
        if (act) {
            Lse acc{0.0, kEmptyExp};
            double n2 = 0.0;
            for (int b = l; b < nblk; b += 32) {
                const double* o = part + ((int64_t)c * nblk + b) * 3;
                lse_merge(acc, Lse{o[0], (int)o[1]});
                n2 += o[2];
            }
            // fixed-order tree merge across lanes
            for (int off = 16; off > 0; off >>= 1) {
                lse_merge(acc, lse_shfl(acc, off));
                n2 += __shfl_xor_sync(0xffffffffu, n2, off);
            }
            if (l == 0) {
                // acc = (s, e) with LSE = log s + e log 2; Alg. 2's
                // exp(LSE_1 - LSE_2) is formed as ldexp(s_1 / s_2, e_1 - e_2):
                // the same quotient, no transcendental, no overflow.
                const bool pos = acc.e != kEmptyExp && acc.s > 0.0;
                const double val = pos ? ldexp(acc.s, acc.e) : 0.0;
                if (mode == SC_BNORM) {
                    S.bnorm = sqrt(n2);
                } else if (mode == SC_INIT) {
                    S.rnorm = sqrt(n2);
                    S.relres = S.bnorm > 0.0 ? S.rnorm / S.bnorm : 0.0;
                    S.gamma_s = pos ? acc.s : 0.0;
                    S.gamma_e = pos ? acc.e : 0;
                    S.gamma = val;
                    // r_0^T z_0 of the first run only: it weights the SLQ quadrature
                    // of the Lanczos process that run's step sizes describe, and a
                    // true-residual restart (k > 0) must not overwrite it
                    if (k == 0) S.gamma0 = val;
                    S.alpha = 0.0;
                    S.beta = 0.0;
                    S.iters = k;
                    S.breakdown = 0;
                    const bool work = S.bnorm > 0.0 && S.rnorm > 0.0 && (S.relres > tol || min_iter > k);
                    if (work && !pos) S.breakdown = 1;
                    S.active = (work && pos) ? 1 : 0;
                    if (rhist) rhist[(int64_t)k * R + c] = S.relres;
                } else if (mode == SC_ALPHA) {
                    // alpha_k = gamma_k / d^T K d  (Alg. 2: from the LSE forms)
                    if (!pos) {
                        S.breakdown = 1;
                        S.active = 0;
                        S.alpha = 0.0;
                    } else {
                        S.alpha = stable ? ldexp(S.gamma_s / acc.s, S.gamma_e - acc.e) : S.gamma / val;
                    }
                    if (ahist) ahist[(int64_t)k * R + c] = S.alpha;
                } else {   // SC_BETA
                    S.rnorm = sqrt(n2);
                    S.relres = S.bnorm > 0.0 ? S.rnorm / S.bnorm : 0.0;
                    S.iters = k + 1;
                    if (rhist) rhist[(int64_t)(k + 1) * R + c] = S.relres;
                    if (S.rnorm == 0.0) {
                        S.active = 0;           // exact solution reached
                        S.beta = 0.0;
                    } else if (!pos) {
                        S.breakdown = 1;
                        S.active = 0;
                        S.beta = 0.0;
                    } else {
                        S.beta = stable ? ldexp(acc.s / S.gamma_s, acc.e - S.gamma_e) : val / S.gamma;
                        S.gamma_s = acc.s;
                        S.gamma_e = acc.e;
                        S.gamma = val;
                        if (bhist) bhist[(int64_t)k * R + c] = S.beta;
                        if (S.relres <= tol && k + 1 >= min_iter) S.active = 0;
                    }
                }
                if (S.breakdown && n_active) atomicAdd(&n_active[1], 1);   // breakdowns of this run
            }
        }
        if (l == 0 && aflags) aflags[c] = S.active;   // the masks of the masked kernels
    }
    if (n_active) {
        int last = 0;
        if (l == 0) {
            __threadfence();
            last = atomicAdd(&n_active[2], 1) == (int)gridDim.x - 1;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
            __threadfence();
            int cnt = 0;
            float rmax = 0.0f;   // largest recursive relative residual of the active columns
            for (int q = l; q < R; q += 32) {
                if (*(volatile const int*)&st[q].active != 0) {
                    ++cnt;
                    rmax = fmaxf(rmax, (float)*(volatile const double*)&st[q].relres);
                }
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            const unsigned rbits = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));   // non-negative floats
            if (l == 0) {
                n_active[0] = cnt;
                n_active[2] = 0;
                n_active[3] = (int)rbits;
            }
        }
    }
}

// x += alpha d; r += alpha Kd   (active columns)
__global__ void update_xr_kernel(float* __restrict__ x, float* __restrict__ r, const float* __restrict__ d,
                                 const float* __restrict__ Kd, int64_t N, const ColState* __restrict__ st) {
    const int c = blockIdx.y;
    if (!st[c].active) return;
    const float a = (float)st[c].alpha;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)c * N + i;
        x[o] = fmaf(a, d[o], x[o]);
        r[o] = fmaf(a, Kd[o], r[o]);
    }
}

// r = s * src - b ; x = 0 (x0 not given) or r = Kx0 - b
__global__ void init_r_kernel(float* __restrict__ r, const float* __restrict__ Kx, const float* __restrict__ b,
                              float* __restrict__ x, int64_t total, int zero_x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        r[i] = (Kx ? Kx[i] : 0.0f) - b[i];
        if (zero_x) x[i] = 0.0f;
    }
}

__global__ void copy_active_kernel(float* __restrict__ dst, const float* __restrict__ src, int64_t N,
                                   const ColState* __restrict__ st) {
    const int c = blockIdx.y;
    if (st && !st[c].active) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        dst[(int64_t)c * N + i] = src[(int64_t)c * N + i];
}

// d = -z + beta d (beta = 0 at the start), then store the basis vectors of
// this iterate: pinv: rho = r / sqrt(gamma), zeta = z / sqrt(gamma); euclid:
// u = r / ||r||.
__global__ void update_d_kernel(float* __restrict__ d, const float* __restrict__ z, const float* __restrict__ r,
                                int64_t N, const ColState* __restrict__ st, int first, int reorth,
                                float* __restrict__ rho, float* __restrict__ zeta) {
    const int c = blockIdx.y;
    const ColState& S = st[c];
    if (!S.active) return;
    // the column's scalars once per block: FP64 is slow on this GPU
    __shared__ float s_beta, s_sg;
    if (threadIdx.x == 0) {
        s_beta = first ? 0.0f : (float)S.beta;
        s_sg = (reorth == GP_REORTH_PINV) ? (float)(1.0 / sqrt(S.gamma))
                                          : (float)(S.rnorm > 0.0 ? 1.0 / S.rnorm : 0.0);
    }
    __syncthreads();
    const float beta = s_beta, sg = s_sg;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = (int64_t)c * N + i;
        const float zi = z[o];
        d[o] = first ? -zi : fmaf(beta, d[o], -zi);
        if (reorth != GP_REORTH_NONE) {
            rho[o] = r[o] * sg;
            if (reorth == GP_REORTH_PINV) zeta[o] = zi * sg;
        }
    }
}

// gpart[(c * nblk + blk) * nb + j] = sum over the chunk of ZB_j[c][i] r[c][i]
// (FP32 products summed over a warp's 256 elements, FP64 across warps and,
// in gram_finalize_kernel, across blocks).  Dynamic shared memory: 8 x nb floats.
__global__ void __launch_bounds__(kDotThreads)
gram_kernel(const float* __restrict__ ZB, int nb, int R, const float* __restrict__ r, int64_t N, int nblk,
            const ColState* __restrict__ st, double* __restrict__ gpart) {
    const int c = blockIdx.y;
    if (!st[c].active) return;
    extern __shared__ float sred[];   // [warp][j]
    const int64_t base = (int64_t)blockIdx.x * kDotChunk;
    float rv[kDotPerThread];
#pragma unroll
    for (int q = 0; q < kDotPerThread; ++q) {
        const int64_t i = base + q * kDotThreads + threadIdx.x;
        rv[q] = i < N ? r[(int64_t)c * N + i] : 0.0f;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    // four basis vectors per step: their 32 loads per thread in flight together
    // (the sums of each vector in the same order as one at a time)
    int j = 0;
    for (; j + 4 <= nb; j += 4) {
        const float* z0 = ZB + ((int64_t)j * R + c) * N;
        const int64_t stride = (int64_t)R * N;
        float a[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int q = 0; q < kDotPerThread; ++q) {
            const int64_t i = base + q * kDotThreads + threadIdx.x;
            if (i < N) {
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = fmaf(z0[u * stride + i], rv[q], a[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            for (int o = 16; o > 0; o >>= 1) a[u] += __shfl_xor_sync(0xffffffffu, a[u], o);
            if (l == 0) sred[w * nb + j + u] = a[u];
        }
    }
    for (; j < nb; ++j) {
        const float* zb = ZB + ((int64_t)j * R + c) * N;
        float a = 0.0f;
#pragma unroll
        for (int q = 0; q < kDotPerThread; ++q) {
            const int64_t i = base + q * kDotThreads + threadIdx.x;
            if (i < N) a = fmaf(zb[i], rv[q], a);
        }
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (l == 0) sred[w * nb + j] = a;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < kDotThreads / 32; ++q) t += (double)sred[q * nb + j];
        gpart[((int64_t)c * nblk + blockIdx.x) * nb + j] = t;
    }
}

// coef[j * R + c] = sum_blk gpart  (fixed order)
__global__ void gram_finalize_kernel(const double* __restrict__ gpart, int nblk, int nb, int R,
                                     const ColState* __restrict__ st, double* __restrict__ coef) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nb * R) return;
    const int j = e / R, c = e % R;
    if (!st[c].active) return;
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += gpart[((int64_t)c * nblk + b) * nb + j];
    coef[e] = t;
}

// r -= sum_j coef[j][c] RB_j[c]
__global__ void reorth_update_kernel(const float* __restrict__ RB, int nb, int R, const double* __restrict__ coef,
                                     float* __restrict__ r, int64_t N, const ColState* __restrict__ st) {
    const int c = blockIdx.y;
    if (!st[c].active) return;
    __shared__ float sc[1024];
    for (int j = threadIdx.x; j < nb; j += blockDim.x) sc[j] = (float)coef[j * R + c];
    __syncthreads();
    const int64_t stride = (int64_t)R * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float v = r[(int64_t)c * N + i];
        const float* rb = RB + (int64_t)c * N + i;
        int j = 0;
        for (; j + 4 <= nb; j += 4) {   // four loads in flight; the same order of updates
            const float b0 = rb[(int64_t)j * stride], b1 = rb[(int64_t)(j + 1) * stride];
            const float b2 = rb[(int64_t)(j + 2) * stride], b3 = rb[(int64_t)(j + 3) * stride];
            v = fmaf(-sc[j], b0, v);
            v = fmaf(-sc[j + 1], b1, v);
            v = fmaf(-sc[j + 2], b2, v);
            v = fmaf(-sc[j + 3], b3, v);
        }
        for (; j < nb; ++j) v = fmaf(-sc[j], rb[(int64_t)j * stride], v);
        r[(int64_t)c * N + i] = v;
    }
}



int vec_grid(const Ctx* ctx, int64_t N) {
    int64_t g = (N + 255) / 256;
    const int64_t cap = 2 * (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148);
    return (int)(g < cap ? g : cap);
}

template <class A>
void cg_layout(A& a, const Ctx* ctx, int64_t N, int R, int rank, const gp_cg_opts_t* o) {
    const size_t NR = (size_t)N * R;
    a.template take<float>(NR);   // r
    a.template take<float>(NR);   // z
    a.template take<float>(NR);   // d
    a.template take<float>(NR);   // Kd
    const bool re = o->algorithm == GP_CG_STABLE && o->reorth != GP_REORTH_NONE;
    const int nb_max = o->max_iter + 1;   // a restart starts a fresh basis, so this bounds every run
    if (re) a.template take<float>((size_t)nb_max * NR);
    if (re && o->reorth == GP_REORTH_PINV) a.template take<float>((size_t)nb_max * NR);
    const int nblk = (int)((N + kDotChunk - 1) / kDotChunk);
    a.template take<double>((size_t)nblk * R * 3);
    if (re) {
        a.template take<double>((size_t)nblk * R * nb_max);
        a.template take<double>((size_t)nb_max * R);
    }
    a.template take<double>((size_t)o->max_iter * R);
    a.template take<double>((size_t)o->max_iter * R);
    a.template take<double>((size_t)(o->max_iter + 1) * R);
    a.template take<ColState>((size_t)R);
    a.template take<int>(4);
    a.template take<int>((size_t)R);
    a.template take<int>((size_t)R);
    if (rank > 0) a.template take<double>((size_t)rank * rank);   // C^{-1}
    (void)ctx;
}

int check_cg_args(const gp_hyp_t* hyp, int64_t N, int R, const gp_cg_opts_t* o) {
    GPK_TRY(check_hyp(hyp));
    if (!o || N < 1 || R < 1 || R > 64 || !(hyp->noise > 0.0)) return GP_ERR_INVALID;
    if (o->max_iter < 1 || o->max_iter > 1000 || o->min_iter < 0 || !(o->tol >= 0.0)) return GP_ERR_INVALID;
    if (o->algorithm != GP_CG_STABLE && o->algorithm != GP_CG_STANDARD) return GP_ERR_INVALID;
    if (o->restarts < 0 || o->restarts > 16) return GP_ERR_INVALID;
    // the solve's and the check's MVM: a precision and optionally operand flags
    GPK_TRY(check_mvm_flags(o->check_precision, false));
    if (o->reorth < GP_REORTH_NONE || o->reorth > GP_REORTH_EUCLID) return GP_ERR_INVALID;
    GPK_TRY(check_mvm_flags(o->precision, false));
    if (o->refine_precision != 0) {
        GPK_TRY(check_mvm_flags(o->refine_precision, false));
        if (!(o->refine_resid >= 0.0) || (o->refine_resid == 0.0 && o->restarts < 1)) return GP_ERR_INVALID;
    }
    return GP_OK;
}

// The refine MVM needs its own operator unless it is the solve's or the check's.
bool refine_own(const gp_cg_opts_t* o) {
    return o->refine_precision != 0 && o->refine_precision != o->precision &&
           !(o->restarts > 0 && o->refine_precision == o->check_precision);
}

}  // namespace

size_t cg_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t N, int R, int rank, const gp_cg_opts_t* o) {
    WsCounter c;
    cg_layout(c, ctx, N, R, rank, o);
    size_t s = c.off + kop_workspace(ctx, hyp, N, N, R, o->precision, true);
    if (o->restarts > 0 && o->check_precision != o->precision)
        s += kop_workspace(ctx, hyp, N, N, R, o->check_precision, true);
    if (refine_own(o)) s += kop_workspace(ctx, hyp, N, N, R, o->refine_precision, true);
    if (rank > 0) s += woodbury_workspace(ctx, N, rank, R);
    return s;
}

// ---- step-able solver ---------------------------------------------------------------
// The solve is a sequence of enqueued phases (set-up, one iteration, a
// true-residual check), each ending with an asynchronous copy of the number of
// still-active columns into pinned host memory.  step() decides the next phase
// from that number once the previous phase has completed, so a caller may
// block on it (gp_cg_solve) or poll an event and interleave many solves.

int CgSolver::launched(int n) {
    ctx->launches += n;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

int CgSolver::flag_copy() {
    // [0] active columns, [1] breakdown count of the current run, [2] 0 (the
    // scalar step's ticket), [3] largest relative residual of the active columns
    // (float bits)
    if (cudaMemcpyAsync(flag_host, b.nact, 4 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GP_ERR_CUDA;
    if (ev && cudaEventRecord(ev, s) != cudaSuccess) return GP_ERR_CUDA;
    return GP_OK;
}

int CgSolver::wait() {
    const cudaError_t e = ev ? cudaEventSynchronize(ev) : cudaStreamSynchronize(s);
    return e == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

int CgSolver::precond(const float* W, float* Z, bool masked) {
    const dim3 gcol((unsigned)vg, (unsigned)R);
    if (rank == 0) {
        copy_active_kernel<<<gcol, 256, 0, s>>>(Z, W, N, masked ? b.st : nullptr);
        return launched(1);
    }
    WsCarver wtmp = wc_rest;   // Woodbury scratch; the active flags come from the last scalar step
    return woodbury_apply(ctx, wtmp, pc.L, pc.core, b.cinv, rank, hyp.noise, N, W, R, masked ? b.aflags : nullptr,
                          Z, s);
}

int CgSolver::dots(const float* A, const float* Bv, bool masked) {
    dots_kernel<<<dim3((unsigned)b.nblk_dot, (unsigned)R), kDotThreads, 0, s>>>(A, Bv, N, b.nblk_dot,
                                                                                 masked ? b.aflags : nullptr, b.dpart);
    return launched(1);
}

int CgSolver::scalar(int mode, int kk) {
    scalar_kernel<<<(unsigned)R, 32, 0, s>>>(mode, stable, b.dpart, b.nblk_dot, R, b.st, kk, o.tol, o.min_iter, b.ahist,
                                     b.bhist, b.rhist, b.nact, b.aflags);
    return launched(1);
}

int CgSolver::start(bool from_x, int k0) {
    const dim3 gcol((unsigned)vg, (unsigned)R);
    const size_t NR = (size_t)N * R;
    GPK_CUDA_TRY(cudaMemsetAsync(b.nact, 0, 2 * sizeof(int), s));
    if (from_x) {
        // the first start uses the solve's MVM; a restart the check MVM
        GPK_TRY(kop_apply(ctx, k0 > 0 ? *op_chk : op, U, R, b.Kd, N, true, s));
        init_r_kernel<<<vg, 256, 0, s>>>(b.r, b.Kd, B, U, (int64_t)NR, 0);
    } else {
        init_r_kernel<<<vg, 256, 0, s>>>(b.r, nullptr, B, U, (int64_t)NR, 1);
    }
    GPK_TRY(launched(1));
    GPK_TRY(precond(b.r, b.z, false));
    GPK_TRY(dots(b.r, b.z, false));
    GPK_TRY(scalar(SC_INIT, k0));
    update_d_kernel<<<gcol, 256, 0, s>>>(b.d, b.z, b.r, N, b.st, 1, reorth, b.rho, b.zeta);
    GPK_TRY(launched(1));
    return flag_copy();
}

int CgSolver::iterate() {
    const dim3 gcol((unsigned)vg, (unsigned)R);
    const dim3 gdot((unsigned)b.nblk_dot, (unsigned)R);
    const size_t NR = (size_t)N * R;
    // Kd = Ktilde d
    GPK_TRY(kop_apply(ctx, escalated ? *op_chk : refined ? *op_ref : op, b.d, R, b.Kd, N, true, s));
    GPK_TRY(dots(b.d, b.Kd, true));   // masked by the flags of the last scalar step
    GPK_TRY(scalar(SC_ALPHA, k));
    update_xr_kernel<<<gcol, 256, 0, s>>>(U, b.r, b.d, b.Kd, N, b.st);
    GPK_TRY(launched(1));
    if (reorth != GP_REORTH_NONE) {
        const int nb = k - nb0 + 1;   // basis vectors r_0 .. r_k of this run
        const float* ZB = reorth == GP_REORTH_PINV ? b.zeta : b.rho;
        for (int p = 0; p < passes; ++p) {
            gram_kernel<<<gdot, kDotThreads, (size_t)(kDotThreads / 32) * nb * sizeof(float), s>>>(
                ZB, nb, R, b.r, N, b.nblk_dot, b.st, b.gpart);
            // 32-thread blocks: the FP64 sums spread over many SMs
            gram_finalize_kernel<<<(nb * R + 31) / 32, 32, 0, s>>>(b.gpart, b.nblk_dot, nb, R, b.st, b.coef);
            reorth_update_kernel<<<gcol, 256, 0, s>>>(b.rho, nb, R, b.coef, b.r, N, b.st);
            GPK_TRY(launched(3));
        }
    }
    GPK_TRY(precond(b.r, b.z, true));
    GPK_TRY(dots(b.r, b.z, true));
    GPK_TRY(scalar(SC_BETA, k));
    const size_t slot = (size_t)(k - nb0 + 1);
    float* rho_k = b.rho ? b.rho + slot * NR : nullptr;
    float* zeta_k = b.zeta ? b.zeta + slot * NR : nullptr;
    update_d_kernel<<<gcol, 256, 0, s>>>(b.d, b.z, b.r, N, b.st, 0, reorth, rho_k, zeta_k);
    GPK_TRY(launched(1));
    ++k;
    iters = k;
    return flag_copy();
}

int CgSolver::setup(Ctx* c, WsCarver& wc, const gp_hyp_t* h, const float* X_, int64_t N_, const float* B_, int R_,
                    float* U_, const gp_precond_t* pc_, const gp_cg_opts_t* o_, cudaStream_t s_, int* flag_host_,
                    cudaEvent_t ev_) {
    ctx = c;
    s = s_;
    flag_host = flag_host_;
    ev = ev_;
    hyp = *h;
    X = X_;
    N = N_;
    B = B_;
    R = R_;
    U = U_;
    o = *o_;
    pc = pc_ ? *pc_ : gp_precond_t{nullptr, nullptr, 0};
    rank = pc.rank > 0 ? pc.rank : 0;
    stable = o.algorithm == GP_CG_STABLE;
    reorth = stable ? o.reorth : GP_REORTH_NONE;
    passes = o.reorth_passes >= 2 ? 2 : 1;
    const size_t NR = (size_t)N * R;
    b.r = wc.take<float>(NR);
    b.z = wc.take<float>(NR);
    b.d = wc.take<float>(NR);
    b.Kd = wc.take<float>(NR);
    b.nb_max = o.max_iter + 1;
    b.rho = reorth != GP_REORTH_NONE ? wc.take<float>((size_t)b.nb_max * NR) : nullptr;
    b.zeta = reorth == GP_REORTH_PINV ? wc.take<float>((size_t)b.nb_max * NR) : nullptr;
    b.nblk_dot = (int)((N + kDotChunk - 1) / kDotChunk);
    b.dpart = wc.take<double>((size_t)b.nblk_dot * R * 3);
    b.gpart = reorth != GP_REORTH_NONE ? wc.take<double>((size_t)b.nblk_dot * R * b.nb_max) : nullptr;
    b.coef = reorth != GP_REORTH_NONE ? wc.take<double>((size_t)b.nb_max * R) : nullptr;
    b.ahist = wc.take<double>((size_t)o.max_iter * R);
    b.bhist = wc.take<double>((size_t)o.max_iter * R);
    b.rhist = wc.take<double>((size_t)(o.max_iter + 1) * R);
    b.st = wc.take<ColState>((size_t)R);
    b.nact = wc.take<int>(4);
    b.aflags = wc.take<int>((size_t)R);
    b.len0 = wc.take<int>((size_t)R);
    b.cinv = rank > 0 ? wc.take<double>((size_t)rank * rank) : nullptr;
    if (!wc.ok) return GP_ERR_WORKSPACE;
    GPK_CUDA_TRY(cudaMemsetAsync(b.nact, 0, 4 * sizeof(int), s));   // counts and the scalar step's ticket
    if (rank > 0) GPK_TRY(woodbury_prepare(ctx, pc.core, rank, b.cinv, s));
    GPK_TRY(kop_prepare(ctx, wc, op, &hyp, X, N, X, N, R, o.precision, s));
    op_chk = &op;
    if (o.restarts > 0 && o.check_precision != o.precision) {
        GPK_TRY(kop_prepare(ctx, wc, op_chk_own, &hyp, X, N, X, N, R, o.check_precision, s));
        op_chk = &op_chk_own;
    }
    op_ref = &op;
    if (o.refine_precision != 0) {
        if (refine_own(&o)) {
            GPK_TRY(kop_prepare(ctx, wc, op_ref_own, &hyp, X, N, X, N, R, o.refine_precision, s));
            op_ref = &op_ref_own;
        } else if (o.refine_precision != o.precision) {
            op_ref = op_chk;
        }
    }
    wc_rest = wc;
    vg = vec_grid(ctx, N);
    k = nb0 = restarts = iters = 0;
    last_check = false;
    len_recorded = false;
    escalated = false;
    refined = false;
    relax_off = false;
    k_sw = 0;
    r_sw = 0.0f;
    GPK_TRY(dots(B, B, false));
    GPK_TRY(scalar(SC_BNORM, 0));
    return start(o.x0_given != 0, 0);
}

// Decide and enqueue the next phase; the previous phase must have completed.
int CgSolver::step(bool* done) {
    const int n = *flag_host;
    *done = false;
    if (o.refine_precision != 0 && o.refine_resid > 0.0 && n > 0 && !relax_off) {
        uint32_t bits;
        memcpy(&bits, &flag_host[3], sizeof(bits));
        float rmax;
        memcpy(&rmax, &bits, sizeof(rmax));
        if (!refined) {
            // relaxation: the refine MVM once every active column's recursive
            // residual is at most refine_resid
            if ((double)rmax <= o.refine_resid) {
                refined = true;
                k_sw = k;
                r_sw = rmax;
            }
        } else {
            // stagnation guard, for a switch made after the residual fell below its start
            // (early CG residuals rise well above it): on the cheaper operator the largest
            // residual must halve within max(20, k_sw / 4) iterations and never double;
            // otherwise (its rounding is too large for this system) the rest of the solve
            // returns to the solve's MVM
            const int W = k_sw / 4 > 20 ? k_sw / 4 : 20;
            if (r_sw < 1.0f && (rmax > 2.0f * r_sw || (k - k_sw >= W && rmax > 0.5f * r_sw))) {
                refined = false;
                relax_off = true;
            }
        }
    }
    if (n > 0 && k < o.max_iter) {
        last_check = false;
        return iterate();
    }
    if (last_check) {   // a true-residual check left nothing to do
        *done = true;
        return GP_OK;
    }
    if (!len_recorded) {
        // lengths of the first (unrestarted) run: the Lanczos process its step sizes describe
        if (cudaMemcpy2DAsync(b.len0, sizeof(int), &b.st[0].iters, sizeof(ColState), sizeof(int), (size_t)R,
                              cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return GP_ERR_CUDA;
        len_recorded = true;
    }
    if (restarts < o.restarts && k < o.max_iter) {
        // A breakdown means the MVM's operator is not positive definite to the
        // accuracy reached: with escalation the rest of the solve uses the
        // check MVM (the restart below already does).
        if (o.escalate && flag_host[1] > 0 && op_chk != &op) escalated = true;
        // mixed-precision refinement: the restarts run on the refine MVM
        if (o.refine_precision != 0 && o.refine_resid == 0.0) refined = true;
        // True-residual check: recompute r = K x - b; columns above tol restart.
        ++restarts;
        nb0 = k;
        last_check = true;
        return start(true, k);
    }
    *done = true;
    return GP_OK;
}

int CgSolver::enqueue_state(ColState* host_st) {
    return cudaMemcpyAsync(host_st, b.st, sizeof(ColState) * R, cudaMemcpyDeviceToHost, s) == cudaSuccess
               ? GP_OK : GP_ERR_CUDA;
}

int CgSolver::summarize(const ColState* hs, gp_cg_stats_t* stats) const {
    int conv = 0, brk = 0;
    for (int c = 0; c < R; ++c) {
        if (hs[c].breakdown) ++brk;
        else if (hs[c].relres <= o.tol) ++conv;
    }
    if (stats) {
        stats->iters = iters;
        stats->converged = conv;
        stats->breakdowns = brk;
        stats->restarts = restarts;
        stats->escalated = escalated ? 1 : 0;
        for (int c = 0; c < R; ++c) {
            if (stats->col_iters) stats->col_iters[c] = hs[c].iters;
            if (stats->rel_resid) stats->rel_resid[c] = hs[c].relres;
            if (stats->gamma0) stats->gamma0[c] = hs[c].gamma0;
        }
    }
    if (brk > 0) return GP_ERR_BREAKDOWN;
    return conv == R ? GP_OK : GP_ERR_NOT_CONVERGED;
}

int CgSolver::finish(gp_cg_stats_t* stats) {
    std::vector<ColState> hs(R);
    GPK_TRY(enqueue_state(hs.data()));
    cudaError_t ce = cudaSuccess;
    if (stats) {
        if (stats->alpha) ce = cudaMemcpyAsync(stats->alpha, b.ahist, sizeof(double) * o.max_iter * R, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess && stats->beta)
            ce = cudaMemcpyAsync(stats->beta, b.bhist, sizeof(double) * o.max_iter * R, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess && stats->resid_hist)
            ce = cudaMemcpyAsync(stats->resid_hist, b.rhist, sizeof(double) * (o.max_iter + 1) * R,
                                 cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess && stats->lanczos_len && len_recorded)
            ce = cudaMemcpyAsync(stats->lanczos_len, b.len0, sizeof(int) * R, cudaMemcpyDeviceToHost, s);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return GP_ERR_CUDA;
    if (stats && stats->lanczos_len && !len_recorded)
        for (int c = 0; c < R; ++c) stats->lanczos_len[c] = hs[c].iters;
    return summarize(hs.data(), stats);
}

int cg_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, const float* B, int R,
           float* U, const gp_precond_t* pc, const gp_cg_opts_t* o, gp_cg_stats_t* stats, cudaStream_t s) {
    CgSolver S;
    GPK_TRY(S.setup(ctx, wc, hyp, X, N, B, R, U, pc, o, s, ctx->host_pinned, nullptr));
    bool done = false;
    while (!done) {
        GPK_TRY(S.wait());
        GPK_TRY(S.step(&done));
    }
    return S.finish(stats);
}

}  // namespace gpk

extern "C" {

size_t gp_cg_workspace_size(const gp_hyp_t* hyp, int64_t N, int R, int rank, const gp_cg_opts_t* opts) {
    if (gpk::check_cg_args(hyp, N, R, opts) != GP_OK) return 0;
    gpk::Ctx probe;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) probe.num_sms = 148;
    return gpk::cg_workspace(&probe, hyp, N, R, rank, opts);
}

int gp_cg_solve(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* B, int R, float* U,
                const gp_precond_t* precond, const gp_cg_opts_t* opts, gp_cg_stats_t* stats, void* stream) {
    if (!ctx || !X || !B || !U) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_cg_args(hyp, N, R, opts));
    if (precond && precond->rank > 0 && (!precond->L || !precond->core || precond->rank > 512)) return GP_ERR_INVALID;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return GP_ERR_CUDA;
    gpk::WsCarver wc(ctx->ws, ctx->ws_bytes);
    int st = gpk::cg_run(ctx, wc, hyp, X, N, B, R, U, precond, opts, stats, (cudaStream_t)stream);
    if (prev != ctx->device) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
