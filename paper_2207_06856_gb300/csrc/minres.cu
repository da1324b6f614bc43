// Low-precision preconditioned MINRES (the Conclusion names MINRES as a
// further iterative method for the paper's low- and mixed-precision approach).
//
// MINRES for Ktilde U = B, Ktilde = K + sigma^2 I, preconditioned by the SPD
// pivoted-Cholesky/Woodbury operator P (Eq. woodbury), all R columns at once:
// each column runs the Lanczos process of P^-1 Ktilde in the P inner product
// in the form of Paige and Saunders' MINRES (r1, r2: the last two unnormalised
// Lanczos vectors, y = P^-1 r2, v = y / beta with beta = sqrt(r2^T y), the
// next vector from Ktilde v - (alpha / beta) r2 - (beta / beta_old) r1),
// and updates the QR factorisation of its tridiagonal matrix with one Givens
// rotation per step; the search direction w and the iterate x follow from
// the rotation, and phibar is the residual's P^-1 norm (the quantity MINRES
// minimises over the Krylov space of P^-1 Ktilde).
//
// Per iteration: v = y / beta; Ktilde v (one MVM for all columns, the low
// precision engine of the solve); y = Ktilde v - (beta / beta_old) r1 with
// the partial dot v^T y fused in; alpha; y -= (alpha / beta) r2; rotate the
// three Lanczos buffers; y = P^-1 r2 (Woodbury); r2^T y; the FP64 scalar step
// (beta, the rotation, phi, phibar); w and x.  The dot products are reduced in
// FP64 in a fixed order (deterministic), the scalar recurrences run in FP64
// one warp per column, and the host reads the number of still-active columns
// after every iteration.  True-residual checks recompute r = B - Ktilde x with
// the check MVM and restart the columns still above the tolerance.
#include "gpk_internal.cuh"

#include <math.h>
#include <string.h>

#include <vector>

namespace gpk {

namespace {

constexpr int kMrThreads = 256;
constexpr int kMrPerThread = 8;
constexpr int kMrChunk = kMrThreads * kMrPerThread;

struct MrState {
    double bnorm_p;   // ||b||_{P^-1}: beta_1 of the first run
    double bnorm2;    // ||b||_2
    double beta, oldb, alfa;
    double dbar, epsln, oldeps, delta;
    double cs, sn, phi, phibar, denom;
    double relres;    // P^-1-norm relative residual: the recurrence's, or the recomputed one after a start
    double rel2;      // 2-norm relative residual of the last recomputed residual
    double tolc;      // the recurrence's stopping level for this column (P^-1 norm)
    int active;       // column still iterating
    int iters;
    int breakdown;
    int upd;          // the w / x update of the current iteration applies
};

enum MrMode { MR_BNORM = 0, MR_START = 1, MR_ALPHA = 2, MR_BETA = 3, MR_FINAL = 4 };

int mr_grid(const Ctx* ctx, int64_t N) {
    const int64_t want = (N + 255) / 256;
    const int64_t cap = (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148) * 8;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

// Block-level FP64 reduction of two sums in a fixed order (threads, then warps).
__device__ __forceinline__ void block_sum2(double& a, double& b, double* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sh[2 * w] = a;
        sh[2 * w + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0.0, sb = 0.0;
        for (int q = 0; q < kMrThreads / 32; ++q) {
            sa += sh[2 * q];
            sb += sh[2 * q + 1];
        }
        a = sa;
        b = sb;
    }
}

// part[(c * nblk + blk) * 2 + {0, 1}] = (sum a_i b_i, sum a_i^2) over this block's chunk.
__global__ void __launch_bounds__(kMrThreads)
mr_dots_kernel(const float* __restrict__ A, const float* __restrict__ B, int64_t N, int nblk,
               const MrState* __restrict__ st, int all, double* __restrict__ part) {
    __shared__ double sh[2 * kMrThreads / 32];
    const int c = blockIdx.y;
    if (!all && !st[c].active) return;
    const float* a = A + (int64_t)c * N;
    const float* b = B + (int64_t)c * N;
    double sab = 0.0, saa = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kMrChunk;
#pragma unroll
    for (int q = 0; q < kMrPerThread; ++q) {
        const int64_t i = base + q * kMrThreads + threadIdx.x;
        if (i < N) {
            const double av = a[i], bv = b[i];
            sab = fma(av, bv, sab);
            saa = fma(av, av, saa);
        }
    }
    block_sum2(sab, saa, sh);
    if (threadIdx.x == 0) {
        double* o = part + ((int64_t)c * nblk + blockIdx.x) * 2;
        o[0] = sab;
        o[1] = saa;
    }
}

// y = Av - (beta / beta_old) r1 (no r1 term in a run's first step), with the
// partial sums of v^T y (and y^T y) for alpha.
__global__ void __launch_bounds__(kMrThreads)
mr_lanczos1_kernel(float* __restrict__ Y, const float* __restrict__ AV, const float* __restrict__ R1,
                   const float* __restrict__ V, int64_t N, int nblk, const MrState* __restrict__ st,
                   double* __restrict__ part) {
    __shared__ double sh[2 * kMrThreads / 32];
    const int c = blockIdx.y;
    const MrState& S = st[c];
    if (!S.active) return;
    const float coef = S.oldb > 0.0 ? (float)(S.beta / S.oldb) : 0.0f;
    const int64_t off = (int64_t)c * N;
    double svy = 0.0, syy = 0.0;
    const int64_t base = (int64_t)blockIdx.x * kMrChunk;
#pragma unroll
    for (int q = 0; q < kMrPerThread; ++q) {
        const int64_t i = base + q * kMrThreads + threadIdx.x;
        if (i < N) {
            const float y = fmaf(-coef, R1[off + i], AV[off + i]);
            Y[off + i] = y;
            const double yd = y;
            svy = fma((double)V[off + i], yd, svy);
            syy = fma(yd, yd, syy);
        }
    }
    block_sum2(svy, syy, sh);
    if (threadIdx.x == 0) {
        double* o = part + ((int64_t)c * nblk + blockIdx.x) * 2;
        o[0] = svy;
        o[1] = syy;
    }
}

// v = y / beta (active columns; 0 elsewhere, so the shared MVM sees finite input)
__global__ void mr_scale_kernel(float* __restrict__ V, const float* __restrict__ Y, int64_t N,
                                const MrState* __restrict__ st) {
    const int c = blockIdx.y;
    const MrState& S = st[c];
    const float s = (S.active && S.beta > 0.0) ? (float)(1.0 / S.beta) : 0.0f;
    const int64_t off = (int64_t)c * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        V[off + i] = s * Y[off + i];
}

// y -= (alpha / beta) r2
__global__ void mr_lanczos2_kernel(float* __restrict__ Y, const float* __restrict__ R2, int64_t N,
                                   const MrState* __restrict__ st) {
    const int c = blockIdx.y;
    const MrState& S = st[c];
    if (!S.active) return;
    const float coef = (float)(S.alfa / S.beta);
    const int64_t off = (int64_t)c * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        Y[off + i] = fmaf(-coef, R2[off + i], Y[off + i]);
}

// w_new = (v - oldeps w1 - delta w2) / gamma with w1 = the direction before last
// (buffer W2) and w2 = the last one (buffer W); w_new overwrites W2; x += phi w_new.
__global__ void mr_update_kernel(float* __restrict__ X, float* __restrict__ W2, const float* __restrict__ W,
                                 const float* __restrict__ V, int64_t N, const MrState* __restrict__ st) {
    const int c = blockIdx.y;
    const MrState& S = st[c];
    if (!S.upd) return;
    const float oe = (float)S.oldeps, de = (float)S.delta, dn = (float)S.denom, ph = (float)S.phi;
    const int64_t off = (int64_t)c * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const float wn = dn * fmaf(-de, W[off + i], fmaf(-oe, W2[off + i], V[off + i]));
        W2[off + i] = wn;
        X[off + i] = fmaf(ph, wn, X[off + i]);
    }
}

// r = b - Av (from_x) or r = b
__global__ void mr_init_r_kernel(float* __restrict__ R, const float* __restrict__ AV, const float* __restrict__ B,
                                 int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        R[i] = AV ? B[i] - AV[i] : B[i];
}

__global__ void mr_copy_active_kernel(float* __restrict__ dst, const float* __restrict__ src, int64_t N,
                                      const MrState* __restrict__ st, int all) {
    const int c = blockIdx.y;
    if (!all && !st[c].active) return;
    const int64_t off = (int64_t)c * N;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        dst[off + i] = src[off + i];
}

// The active flags as ints for the Woodbury apply's column mask.
__global__ void mr_flags_kernel(const MrState* __restrict__ st, int R, int* __restrict__ act) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c < R) act[c] = st[c].active;
}

// FP64 scalar step, one warp per column: merge the partial sums of column c in
// a fixed order, then
//   MR_BNORM  ||b||_2;
//   MR_START  a run's start from r (r = b, or b - Ktilde x at a true-residual
//             check): beta_1 = sqrt(r^T P^-1 r), the rotation reset, the
//             relative residuals; the column is active while above tol;
//   MR_ALPHA  alpha_k = v_k^T (Ktilde v_k - ...);
//   MR_BETA   beta_{k+1}, then the Givens rotation that annihilates beta_{k+1}
//             in the tridiagonal's QR factorisation: (cs, sn), gamma, the
//             coefficients of the direction update (oldeps, delta, 1 / gamma),
//             the step phi along it and the new residual norm phibar;
//   MR_FINAL  the relative residuals of a recomputed r, nothing else.
// The last block to finish counts the active columns and the breakdowns.
__global__ void __launch_bounds__(32)
mr_scalar_kernel(int mode, const double* __restrict__ part, int nblk, int R, MrState* __restrict__ st, int k,
                 int first, double tol, int norm2, double* __restrict__ rhist, int* __restrict__ nact) {
    const int c = blockIdx.x, l = threadIdx.x;
    MrState& S = st[c];
    const bool use = (mode == MR_ALPHA || mode == MR_BETA) ? (S.active != 0) : true;
    double s0 = 0.0, s1 = 0.0;
    if (use) {
        for (int b = l; b < nblk; b += 32) {
            s0 += part[((int64_t)c * nblk + b) * 2];
            s1 += part[((int64_t)c * nblk + b) * 2 + 1];
        }
        for (int o = 16; o > 0; o >>= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
    }
    if (l == 0) {
        if (mode == MR_BETA && !use) S.upd = 0;
        if (use) {
            if (mode == MR_BNORM) {
                S.bnorm2 = sqrt(s1);
            } else if (mode == MR_START) {
                const bool ok = s0 >= 0.0 && isfinite(s0);
                if (first) {
                    S.bnorm_p = ok ? sqrt(s0) : 0.0;
                    S.iters = 0;
                }
                S.beta = ok ? sqrt(s0) : 0.0;
                S.oldb = 0.0;
                S.alfa = 0.0;
                S.dbar = 0.0;
                S.epsln = 0.0;
                S.oldeps = 0.0;
                S.delta = 0.0;
                S.cs = -1.0;
                S.sn = 0.0;
                S.phi = 0.0;
                S.phibar = S.beta;
                S.denom = 0.0;
                S.upd = 0;
                S.breakdown = ok ? 0 : 1;
                S.relres = S.bnorm_p > 0.0 ? S.beta / S.bnorm_p : 0.0;
                S.rel2 = S.bnorm2 > 0.0 ? sqrt(s1) / S.bnorm2 : 0.0;
                if (norm2 && !first) {
                    // a true-residual check in the 2-norm: the recurrence's P^-1-norm target
                    // follows the ratio of the two norms seen on this residual
                    S.tolc = S.rel2 > 0.0 ? 0.95 * tol * S.relres / S.rel2 : tol;
                    S.active = (ok && S.beta > 0.0 && S.rel2 > tol) ? 1 : 0;
                } else {
                    S.tolc = tol;
                    S.active = (ok && S.beta > 0.0 && S.relres > tol) ? 1 : 0;
                }
                if (rhist) rhist[(int64_t)k * R + c] = S.relres;
            } else if (mode == MR_ALPHA) {
                S.alfa = s0;
            } else if (mode == MR_BETA) {
                if (!(s0 >= 0.0) || !isfinite(s0) || !isfinite(S.alfa)) {
                    S.breakdown = 1;
                    S.active = 0;
                    S.upd = 0;
                } else {
                    S.oldb = S.beta;
                    S.beta = sqrt(s0);
                    S.oldeps = S.epsln;
                    S.delta = S.cs * S.dbar + S.sn * S.alfa;
                    const double gbar = S.sn * S.dbar - S.cs * S.alfa;
                    S.epsln = S.sn * S.beta;
                    S.dbar = -S.cs * S.beta;
                    double gamma = hypot(gbar, S.beta);
                    if (gamma < 1e-300) gamma = 1e-300;
                    S.cs = gbar / gamma;
                    S.sn = S.beta / gamma;
                    S.phi = S.cs * S.phibar;
                    S.phibar = S.sn * S.phibar;
                    S.denom = 1.0 / gamma;
                    S.iters += 1;
                    S.upd = 1;
                    S.relres = S.bnorm_p > 0.0 ? fabs(S.phibar) / S.bnorm_p : 0.0;
                    if (rhist) rhist[(int64_t)(k + 1) * R + c] = S.relres;
                    // beta = 0: the Krylov space is invariant and this step is exact
                    if (S.relres <= S.tolc || S.beta == 0.0) S.active = 0;
                }
            } else {   // MR_FINAL
                S.relres = S.bnorm_p > 0.0 ? sqrt(fmax(s0, 0.0)) / S.bnorm_p : 0.0;
                S.rel2 = S.bnorm2 > 0.0 ? sqrt(s1) / S.bnorm2 : 0.0;
            }
        }
    }
    if (nact) {
        int last = 0;
        if (l == 0) {
            __threadfence();
            last = atomicAdd(&nact[2], 1) == (int)gridDim.x - 1;
        }
        if (__shfl_sync(0xffffffffu, last, 0)) {
            __threadfence();
            int cnt = 0, brk = 0;
            float rmax = 0.0f;   // largest relative residual of the active columns
            for (int q = l; q < R; q += 32) {
                const bool a = *(volatile const int*)&st[q].active != 0;
                cnt += a;
                brk += *(volatile const int*)&st[q].breakdown != 0;
                if (a) rmax = fmaxf(rmax, (float)*(volatile const double*)&st[q].relres);
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            brk = __reduce_add_sync(0xffffffffu, brk);
            const unsigned rbits = __reduce_max_sync(0xffffffffu, __float_as_uint(rmax));
            if (l == 0) {
                nact[0] = cnt;
                nact[1] = brk;
                nact[2] = 0;
                nact[3] = (int)rbits;
            }
        }
    }
}

template <class A>
void mr_layout(A& a, int64_t N, int R, int rank, const gp_minres_opts_t* o) {
    const size_t NR = (size_t)N * R;
    for (int q = 0; q < 7; ++q) a.template take<float>(NR);   // r1, r2, y, v, Av, w, w2
    const int nblk = (int)((N + kMrChunk - 1) / kMrChunk);
    a.template take<double>((size_t)nblk * R * 2);
    a.template take<MrState>((size_t)R);
    a.template take<int>((size_t)R);
    a.template take<int>(4);
    a.template take<double>((size_t)(o->max_iter + 1) * R);
    if (rank > 0) a.template take<double>((size_t)rank * rank);   // C^{-1}
}

int check_minres_args(const gp_hyp_t* hyp, int64_t N, int R, const gp_minres_opts_t* o) {
    GPK_TRY(check_hyp(hyp));
    if (!o || N < 1 || R < 1 || R > 64 || !(hyp->noise > 0.0)) return GP_ERR_INVALID;
    if (o->max_iter < 1 || o->max_iter > 1000 || !(o->tol >= 0.0)) return GP_ERR_INVALID;
    if (o->restarts < 0 || o->restarts > 16) return GP_ERR_INVALID;
    if (o->norm != GP_MINRES_NORM_P && o->norm != GP_MINRES_NORM_2) return GP_ERR_INVALID;
    if (o->norm == GP_MINRES_NORM_2 && o->restarts < 1) return GP_ERR_INVALID;
    if (o->refine_precision != 0) {
        GPK_TRY(check_mvm_flags(o->refine_precision, false));
        if (!(o->refine_resid > 0.0)) return GP_ERR_INVALID;
    }
    GPK_TRY(check_mvm_flags(o->precision, false));
    GPK_TRY(check_mvm_flags(o->check_precision, false));
    return GP_OK;
}

size_t minres_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t N, int R, int rank, const gp_minres_opts_t* o) {
    WsCounter c;
    mr_layout(c, N, R, rank, o);
    size_t s = c.off + kop_workspace(ctx, hyp, N, N, R, o->precision, true);
    if (o->check_precision != o->precision) s += kop_workspace(ctx, hyp, N, N, R, o->check_precision, true);
    if (o->refine_precision != 0 && o->refine_precision != o->precision && o->refine_precision != o->check_precision)
        s += kop_workspace(ctx, hyp, N, N, R, o->refine_precision, true);
    if (rank > 0) s += woodbury_workspace(ctx, N, rank, R);
    return s;
}

struct MrSolve {
    Ctx* ctx;
    cudaStream_t s;
    gp_hyp_t hyp;
    const float* X;
    const float* B;
    float* U;
    int64_t N;
    int R;
    gp_minres_opts_t o;
    gp_precond_t pc{};
    int rank = 0, vg = 1, nblk = 1;
    float *r1, *r2, *y, *v, *av, *w, *w2;
    double* part;
    MrState* st;
    int* act;
    int* nact;
    double* rhist;
    double* cinv = nullptr;
    KOp op, op_chk_own, op_ref_own;
    KOp* op_chk = nullptr;
    KOp* op_ref = nullptr;     // the relaxed schedule's MVM
    bool refined = false, relax_off = false;
    int k_sw = 0;
    float r_sw = 0.0f;
    WsCarver wc_rest{nullptr, 0};

    int launched(int n) {
        ctx->launches += n;
        return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
    }
    int dots(const float* A, const float* Bv, bool all) {
        mr_dots_kernel<<<dim3((unsigned)nblk, (unsigned)R), kMrThreads, 0, s>>>(A, Bv, N, nblk, st, all ? 1 : 0, part);
        return launched(1);
    }
    int scalar(int mode, int k, int first) {
        mr_scalar_kernel<<<(unsigned)R, 32, 0, s>>>(mode, part, nblk, R, st, k, first, o.tol,
                                                    o.norm == GP_MINRES_NORM_2 ? 1 : 0, rhist, nact);
        return launched(1);
    }
    // Z = P^-1 W on the active columns (all columns when `all`)
    int precond(const float* W, float* Z, bool all) {
        const dim3 gcol((unsigned)vg, (unsigned)R);
        if (rank == 0) {
            mr_copy_active_kernel<<<gcol, 256, 0, s>>>(Z, W, N, st, all ? 1 : 0);
            return launched(1);
        }
        const int* mask = nullptr;
        if (!all) {
            mr_flags_kernel<<<(unsigned)((R + 63) / 64), 64, 0, s>>>(st, R, act);
            GPK_TRY(launched(1));
            mask = act;
        }
        WsCarver wtmp = wc_rest;
        return woodbury_apply(ctx, wtmp, pc.L, pc.core, cinv, rank, hyp.noise, N, W, R, mask, Z, s);
    }
    int flag_copy_wait() {
        GPK_CUDA_TRY(cudaMemcpyAsync(ctx->host_pinned, nact, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        GPK_CUDA_TRY(cudaStreamSynchronize(s));
        return GP_OK;
    }
    // A run's start: r1 = b (x = 0) or b - Ktilde x with the check MVM; y = P^-1 r1.
    int start(bool from_x, int k, int first) {
        const size_t NR = (size_t)N * R;
        if (from_x) {
            GPK_TRY(kop_apply(ctx, *op_chk, U, R, av, N, true, s));
            mr_init_r_kernel<<<vg, 256, 0, s>>>(r1, av, B, (int64_t)NR);
        } else {
            mr_init_r_kernel<<<vg, 256, 0, s>>>(r1, nullptr, B, (int64_t)NR);
        }
        GPK_TRY(launched(1));
        GPK_TRY(precond(r1, y, true));
        GPK_TRY(dots(r1, y, true));
        GPK_TRY(scalar(MR_START, k, first));
        GPK_CUDA_TRY(cudaMemcpyAsync(r2, r1, sizeof(float) * NR, cudaMemcpyDeviceToDevice, s));
        GPK_CUDA_TRY(cudaMemsetAsync(w, 0, sizeof(float) * NR, s));
        GPK_CUDA_TRY(cudaMemsetAsync(w2, 0, sizeof(float) * NR, s));
        return flag_copy_wait();
    }
    // the relaxed schedule of gp_cg_opts_t: switch once every active residual is at
    // most refine_resid; after a switch below the start, return to the solve's MVM
    // if the largest residual has not halved within max(20, k_sw / 4) iterations or
    // has doubled
    void relax_step(int k) {
        if (o.refine_precision == 0 || !(o.refine_resid > 0.0) || relax_off || ctx->host_pinned[0] == 0) return;
        float rmax;
        memcpy(&rmax, &ctx->host_pinned[3], sizeof(rmax));
        if (!refined) {
            if ((double)rmax <= o.refine_resid) {
                refined = true;
                k_sw = k;
                r_sw = rmax;
            }
        } else {
            const int W = k_sw / 4 > 20 ? k_sw / 4 : 20;
            if (r_sw < 1.0f && (rmax > 2.0f * r_sw || (k - k_sw >= W && rmax > 0.5f * r_sw))) {
                refined = false;
                relax_off = true;
            }
        }
    }
    int iterate(int k) {
        const dim3 gcol((unsigned)vg, (unsigned)R);
        const dim3 gdot((unsigned)nblk, (unsigned)R);
        mr_scale_kernel<<<gcol, 256, 0, s>>>(v, y, N, st);
        GPK_TRY(launched(1));
        GPK_TRY(kop_apply(ctx, refined ? *op_ref : op, v, R, av, N, true, s));
        mr_lanczos1_kernel<<<gdot, kMrThreads, 0, s>>>(y, av, r1, v, N, nblk, st, part);
        GPK_TRY(launched(1));
        GPK_TRY(scalar(MR_ALPHA, k, 0));
        mr_lanczos2_kernel<<<gcol, 256, 0, s>>>(y, r2, N, st);
        GPK_TRY(launched(1));
        float* t = r1;   // (r1, r2, y) <- (r2, y, r1): y is the new Lanczos vector
        r1 = r2;
        r2 = y;
        y = t;
        GPK_TRY(precond(r2, y, false));
        GPK_TRY(dots(r2, y, false));
        GPK_TRY(scalar(MR_BETA, k, 0));
        mr_update_kernel<<<gcol, 256, 0, s>>>(U, w2, w, v, N, st);
        GPK_TRY(launched(1));
        t = w;           // the new direction (in w2's buffer) becomes w
        w = w2;
        w2 = t;
        return flag_copy_wait();
    }
};

int minres_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, const float* B, int R,
               float* U, const gp_precond_t* pc, const gp_minres_opts_t* o, gp_minres_stats_t* stats,
               cudaStream_t s) {
    GPK_TRY(check_minres_args(hyp, N, R, o));
    MrSolve S;
    S.ctx = ctx;
    S.s = s;
    S.hyp = *hyp;
    S.X = X;
    S.B = B;
    S.U = U;
    S.N = N;
    S.R = R;
    S.o = *o;
    if (pc && pc->rank > 0) {
        S.pc = *pc;
        S.rank = pc->rank;
    }
    const size_t NR = (size_t)N * R;
    float** vecs[7] = {&S.r1, &S.r2, &S.y, &S.v, &S.av, &S.w, &S.w2};
    for (float** p : vecs) *p = wc.take<float>(NR);
    S.nblk = (int)((N + kMrChunk - 1) / kMrChunk);
    S.part = wc.take<double>((size_t)S.nblk * R * 2);
    S.st = wc.take<MrState>((size_t)R);
    S.act = wc.take<int>((size_t)R);
    S.nact = wc.take<int>(4);
    S.rhist = wc.take<double>((size_t)(o->max_iter + 1) * R);
    S.cinv = S.rank > 0 ? wc.take<double>((size_t)S.rank * S.rank) : nullptr;
    if (!wc.ok) return GP_ERR_WORKSPACE;
    GPK_CUDA_TRY(cudaMemsetAsync(S.nact, 0, 4 * sizeof(int), s));
    GPK_CUDA_TRY(cudaMemsetAsync(S.st, 0, sizeof(MrState) * R, s));
    GPK_CUDA_TRY(cudaMemsetAsync(S.rhist, 0, sizeof(double) * (o->max_iter + 1) * R, s));
    GPK_CUDA_TRY(cudaMemsetAsync(U, 0, sizeof(float) * NR, s));
    if (S.rank > 0) GPK_TRY(woodbury_prepare(ctx, S.pc.core, S.rank, S.cinv, s));
    GPK_TRY(kop_prepare(ctx, wc, S.op, hyp, X, N, X, N, R, o->precision, s));
    S.op_chk = &S.op;
    if (o->check_precision != o->precision) {
        GPK_TRY(kop_prepare(ctx, wc, S.op_chk_own, hyp, X, N, X, N, R, o->check_precision, s));
        S.op_chk = &S.op_chk_own;
    }
    S.op_ref = &S.op;
    if (o->refine_precision != 0 && o->refine_precision != o->precision) {
        if (o->refine_precision == o->check_precision) {
            S.op_ref = S.op_chk;
        } else {
            GPK_TRY(kop_prepare(ctx, wc, S.op_ref_own, hyp, X, N, X, N, R, o->refine_precision, s));
            S.op_ref = &S.op_ref_own;
        }
    }
    S.wc_rest = wc;
    S.vg = mr_grid(ctx, N);
    GPK_TRY(S.dots(B, B, true));
    GPK_TRY(S.scalar(MR_BNORM, 0, 0));
    GPK_TRY(S.start(false, 0, 1));
    int k = 0, restarts = 0;
    bool checked = false;   // the state holds recomputed residuals of the final iterate
    for (;;) {
        if (ctx->host_pinned[0] > 0 && k < o->max_iter) {
            S.relax_step(k);
            GPK_TRY(S.iterate(k));
            ++k;
            checked = false;
            continue;
        }
        if (restarts < o->restarts && k < o->max_iter && !checked) {
            ++restarts;
            GPK_TRY(S.start(true, k, 0));   // true-residual check; columns above tol restart
            checked = true;
            continue;
        }
        break;
    }
    if (!checked) {
        // residuals of the final iterate, recomputed with the check MVM
        GPK_TRY(kop_apply(ctx, *S.op_chk, U, R, S.av, N, true, s));
        mr_init_r_kernel<<<S.vg, 256, 0, s>>>(S.r1, S.av, B, (int64_t)NR);
        GPK_TRY(S.launched(1));
        GPK_TRY(S.precond(S.r1, S.y, true));
        GPK_TRY(S.dots(S.r1, S.y, true));
        GPK_TRY(S.scalar(MR_FINAL, k, 0));
    }
    std::vector<MrState> hs(R);
    GPK_CUDA_TRY(cudaMemcpyAsync(hs.data(), S.st, sizeof(MrState) * R, cudaMemcpyDeviceToHost, s));
    if (stats && stats->resid_hist)
        GPK_CUDA_TRY(cudaMemcpyAsync(stats->resid_hist, S.rhist, sizeof(double) * (o->max_iter + 1) * R,
                                     cudaMemcpyDeviceToHost, s));
    GPK_CUDA_TRY(cudaStreamSynchronize(s));
    int conv = 0, brk = 0;
    for (int c = 0; c < R; ++c) {
        if (hs[c].breakdown) ++brk;
        else if ((o->norm == GP_MINRES_NORM_2 ? hs[c].rel2 : hs[c].relres) <= o->tol) ++conv;
    }
    if (stats) {
        stats->iters = k;
        stats->converged = conv;
        stats->breakdowns = brk;
        stats->restarts = restarts;
        for (int c = 0; c < R; ++c) {
            if (stats->col_iters) stats->col_iters[c] = hs[c].iters;
            if (stats->rel_resid) stats->rel_resid[c] = hs[c].rel2;
            if (stats->rel_resid_p) stats->rel_resid_p[c] = hs[c].relres;
        }
    }
    if (brk > 0) return GP_ERR_BREAKDOWN;
    return conv == R ? GP_OK : GP_ERR_NOT_CONVERGED;
}

}  // namespace

}  // namespace gpk

extern "C" {

size_t gp_minres_workspace_size(const gp_hyp_t* hyp, int64_t N, int R, int rank, const gp_minres_opts_t* opts) {
    if (gpk::check_minres_args(hyp, N, R, opts) != GP_OK || rank < 0 || rank > 512) return 0;
    gpk::Ctx probe;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) probe.num_sms = 148;
    return gpk::minres_workspace(&probe, hyp, N, R, rank, opts);
}

int gp_minres_solve(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, const float* B, int R, float* U,
                    const gp_precond_t* precond, const gp_minres_opts_t* opts, gp_minres_stats_t* stats,
                    void* stream) {
    if (!ctx || !X || !B || !U) return GP_ERR_INVALID;
    if (precond && precond->rank > 0 && (!precond->L || !precond->core || precond->rank > 512)) return GP_ERR_INVALID;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != ctx->device && cudaSetDevice(ctx->device) != cudaSuccess) return GP_ERR_CUDA;
    gpk::WsCarver wc(ctx->ws, ctx->ws_bytes);
    const int st = gpk::minres_run(ctx, wc, hyp, X, N, B, R, U, precond, opts, stats, (cudaStream_t)stream);
    if (prev != ctx->device) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
