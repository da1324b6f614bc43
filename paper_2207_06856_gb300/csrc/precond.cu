// S3 + S4: pivoted-Cholesky preconditioner and its Woodbury application
// (Sec. 4.2 "Preconditioning", Eq. woodbury).
//
// Factor.  k steps of partial pivoted Cholesky of K (no noise), using only
// kernel rows K e_p and the diagonal, which is the constant a^2 for a
// stationary kernel.  Step m picks p = argmax of the remaining diagonal
// (lowest index on ties), forms
//     l_m = (K e_p - L_{:,<m} L_{p,<m}^T) / sqrt(diag_p),   diag -= l_m^2,
// in FP32.  One launch per step: every block first reduces the previous
// step's per-block argmax candidates (a few hundred pairs), so no separate
// global argmax pass is needed; the kernel row is evaluated on the fly from
// the scaled inputs (SIMT FP32, same kernel forms as the MVM).
//
// Core.  C = I + sigma^-2 L^T L is accumulated in FP64 from exact FP64
// products and factored C = Lc Lc^T in FP64 by one CTA.
//
// Apply.  P^{-1} w = sigma^-2 w - sigma^-4 L C^{-1} L^T w: t = L^T w (FP32
// within 256-row blocks, FP64 across blocks, fixed order), u = C^{-1} t by
// FP64 triangular solves (one warp per right-hand side), then the N x k
// product with u fused with the scaling.
#include "gpk_internal.cuh"
#include "kfun.cuh"

#include <math.h>

namespace gpk {

namespace {

struct Cand {
    float val;
    int idx;
};

__device__ __forceinline__ bool cand_better(float v, int i, float bv, int bi) {
    return v > bv || (v == bv && (unsigned)i < (unsigned)bi);
}

__device__ void block_argmax(float& v, int& i) {
    __shared__ float sv[32];
    __shared__ int si[32];
    for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (cand_better(ov, oi, v, i)) { v = ov; i = oi; }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) { sv[w] = v; si[w] = i; }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        v = l < nw ? sv[l] : -INFINITY;
        i = l < nw ? si[l] : 0x7fffffff;
        for (int o = 16; o > 0; o >>= 1) {
            const float ov = __shfl_xor_sync(0xffffffffu, v, o);
            const int oi = __shfl_xor_sync(0xffffffffu, i, o);
            if (cand_better(ov, oi, v, i)) { v = ov; i = oi; }
        }
        if (l == 0) { sv[0] = v; si[0] = i; }
    }
    __syncthreads();
    v = sv[0];
    i = si[0];
    __syncthreads();
}

constexpr int kPcThreads = 256;

template <int KIND>
__global__ void __launch_bounds__(kPcThreads)
pivchol_step_kernel(const float* __restrict__ Xs, int64_t N, int dp, int m, float a2, float tol_abs,
                    float* __restrict__ L, float* __restrict__ diag, const Cand* __restrict__ cin, int g_in,
                    Cand* __restrict__ cout, int* __restrict__ piv, int* __restrict__ rank_out) {
    __shared__ float sxp[64];
    __shared__ float slp[512];
    if (*rank_out >= 0) return;   // an earlier step stopped the factorisation
    float dmax;
    int p;
    if (m == 0) {
        dmax = a2;
        p = 0;
    } else {
        dmax = -INFINITY;
        p = 0x7fffffff;
        for (int g = threadIdx.x; g < g_in; g += blockDim.x) {
            const Cand c = cin[g];
            if (cand_better(c.val, c.idx, dmax, p)) { dmax = c.val; p = c.idx; }
        }
        block_argmax(dmax, p);
    }
    if (!(dmax > tol_abs)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *rank_out = m;
        return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) piv[m] = p;
    for (int k = threadIdx.x; k < dp; k += blockDim.x) sxp[k] = Xs[(int64_t)p * dp + k];
    for (int q = threadIdx.x; q < m; q += blockDim.x) slp[q] = L[(int64_t)q * N + p];
    __syncthreads();
    const float inv = 1.0f / sqrtf(dmax);
    float bv = -INFINITY;
    int bi = 0x7fffffff;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float q2 = 0.0f;
        for (int k = 0; k < dp; ++k) {
            const float df = Xs[i * dp + k] - sxp[k];
            q2 = fmaf(df, df, q2);
        }
        const float kv = a2 * kernel_from_s<KIND>(-q2);
        float dot = 0.0f;
        for (int q = 0; q < m; ++q) dot = fmaf(L[(int64_t)q * N + i], slp[q], dot);
        const float lv = (kv - dot) * inv;
        L[(int64_t)m * N + i] = lv;
        const float dn = (i == p) ? 0.0f : diag[i] - lv * lv;
        diag[i] = dn;
        if (cand_better(dn, (int)i, bv, bi)) { bv = dn; bi = (int)i; }
    }
    block_argmax(bv, bi);
    if (threadIdx.x == 0) cout[blockIdx.x] = Cand{bv, bi};
}

__global__ void fill_kernel(float* p, int64_t n, float v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// partial[s][a][b] = sum over rows of split s of L[a][i] L[b][i], FP64.
// grid = (tiles of 16 x 16 over k x k, splits); L column-major (ld N).
__global__ void gram_ll_kernel(const float* __restrict__ L, int64_t N, int k, int nsplit,
                               double* __restrict__ partial) {
    __shared__ float sa[64][17];
    __shared__ float sb[64][17];
    const int tiles = (k + 15) / 16;
    const int ta = blockIdx.x / tiles, tb = blockIdx.x % tiles;
    const int s = blockIdx.y;
    const int la = threadIdx.x >> 4, lb = threadIdx.x & 15;   // 256 threads: 16 x 16
    const int a = ta * 16 + la, b = tb * 16 + lb;
    const int64_t r0 = (N * s) / nsplit, r1 = (N * (s + 1)) / nsplit;
    double acc = 0.0;
    for (int64_t i0 = r0; i0 < r1; i0 += 64) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            const int ii = e % 64, cc = e / 64;
            const int64_t i = i0 + ii;
            const int ca = ta * 16 + cc, cb = tb * 16 + cc;
            sa[ii][cc] = (i < r1 && ca < k) ? L[(int64_t)ca * N + i] : 0.0f;
            sb[ii][cc] = (i < r1 && cb < k) ? L[(int64_t)cb * N + i] : 0.0f;
        }
        __syncthreads();
        for (int ii = 0; ii < 64; ++ii) acc = fma((double)sa[ii][la], (double)sb[ii][lb], acc);
        __syncthreads();
    }
    if (a < k && b < k) partial[((int64_t)s * k + a) * k + b] = acc;
}

// One CTA: C = I + sigma^-2 sum_s partial[s], then in-place FP64 Cholesky.
// core (k x k, column-major) receives the lower factor (upper part zeroed).
__global__ void core_chol_kernel(const double* __restrict__ partial, int nsplit, int k, double inv_noise,
                                 double* __restrict__ core, int* err) {
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int a = e % k, b = e / k;   // row a, column b
        double g = 0.0;
        for (int s = 0; s < nsplit; ++s) g += partial[((int64_t)s * k + a) * k + b];
        core[(int64_t)b * k + a] = (a == b ? 1.0 : 0.0) + inv_noise * g;
    }
    __syncthreads();
    __shared__ double piv;
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            const double djj = core[(int64_t)j * k + j];
            if (!(djj > 0.0)) atomicCAS(err, 0, (int)DEV_BREAKDOWN);
            piv = sqrt(djj > 0.0 ? djj : 1.0);
            core[(int64_t)j * k + j] = piv;
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) core[(int64_t)j * k + i] /= piv;
        __syncthreads();
        const int rem = k - j - 1;
        for (int e = threadIdx.x; e < rem * rem; e += blockDim.x) {
            const int i = j + 1 + e % rem, l = j + 1 + e / rem;
            if (l <= i) core[(int64_t)l * k + i] -= core[(int64_t)j * k + i] * core[(int64_t)j * k + l];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
        const int a = e % k, b = e / k;
        if (a < b) core[(int64_t)b * k + a] = 0.0;
    }
}

// ---- Woodbury apply ---------------------------------------------------------------------
constexpr int kWbRows = 256;

// tpart[blk][a][c] = sum_{i in blk rows} L[a][i] W[c][i]   (FP32 in-block, stored FP64)
__global__ void __launch_bounds__(256)
wb_ltw_kernel(const float* __restrict__ L, int64_t N, int k, const float* __restrict__ W, int R,
              const int* __restrict__ active, int64_t rows_per_blk, double* __restrict__ tpart) {
    extern __shared__ float sh[];
    constexpr int ST = kWbRows + 1;    // padded row stride: conflict-free column reads
    float* sw = sh;                    // [R][ST]
    float* sl = sh + R * ST;           // [16][ST]
    const int64_t r0 = rows_per_blk * blockIdx.x;
    const int64_t r1 = (r0 + rows_per_blk < N) ? r0 + rows_per_blk : N;
    const int npair = 16 * R;
    for (int a0 = 0; a0 < k; a0 += 16) {
        // each thread owns up to 2 (a, c) pairs of this 16-column slab
        float acc0 = 0.0f, acc1 = 0.0f;
        for (int64_t i0 = r0; i0 < r1; i0 += kWbRows) {
            __syncthreads();
            for (int e = threadIdx.x; e < R * kWbRows; e += blockDim.x) {
                const int c = e / kWbRows, ii = e % kWbRows;
                const int64_t i = i0 + ii;
                sw[c * ST + ii] = (i < r1) ? W[(int64_t)c * N + i] : 0.0f;
            }
            for (int e = threadIdx.x; e < 16 * kWbRows; e += blockDim.x) {
                const int aa = e / kWbRows, ii = e % kWbRows;
                const int64_t i = i0 + ii;
                sl[aa * ST + ii] = (i < r1 && a0 + aa < k) ? L[(int64_t)(a0 + aa) * N + i] : 0.0f;
            }
            __syncthreads();
            for (int q = 0; q < 2; ++q) {
                const int pr = threadIdx.x + q * blockDim.x;
                if (pr < npair) {
                    const int aa = pr % 16, c = pr / 16;
                    const float* wl = sw + c * ST;
                    const float* ll = sl + aa * ST;
                    float acc = 0.0f;
                    for (int ii = 0; ii < kWbRows; ++ii) acc = fmaf(ll[ii], wl[ii], acc);
                    if (q == 0) acc0 += acc; else acc1 += acc;
                }
            }
        }
        for (int q = 0; q < 2; ++q) {
            const int pr = threadIdx.x + q * blockDim.x;
            if (pr < npair) {
                const int aa = pr % 16, c = pr / 16;
                if (a0 + aa < k)
                    tpart[((int64_t)blockIdx.x * k + a0 + aa) * R + c] = (double)(q == 0 ? acc0 : acc1);
            }
        }
    }
}

// One warp per right-hand side: t = sum of partials (fixed order),
// u = C^{-1} t with C = Lc Lc^T (forward then backward substitution, FP64).
// grid = ceil(R / 8) CTAs of 8 warps; CTA b solves columns 8b .. 8b+7.
constexpr int kWbSolveWarps = 8;
__global__ void __launch_bounds__(kWbSolveWarps * 32)
wb_solve_kernel(const double* __restrict__ tpart, int nblk, int k, int R, const double* __restrict__ core,
                float* __restrict__ u_out, double* __restrict__ ybuf) {
    const int c0 = blockIdx.x * kWbSolveWarps;
    const int nc = (R - c0) < kWbSolveWarps ? (R - c0) : kWbSolveWarps;
    // t = sum over row blocks (fixed order) for this CTA's columns, layout [a][c]
    for (int e = threadIdx.x; e < k * nc; e += blockDim.x) {
        const int a = e / nc, c = c0 + e % nc;
        double t = 0.0;
        for (int b = 0; b < nblk; ++b) t += tpart[((int64_t)b * k + a) * R + c];
        ybuf[a * R + c] = t;
    }
    __syncthreads();
    // One warp per right-hand side; lane l keeps rows a = l + 32 m in registers
    // (k <= 512).  core holds Lc column-major: Lc(a, b) = core[b * k + a].
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kMaxPer = 16;
    if (w < nc) {
        const int c = c0 + w;
        double y[kMaxPer];
#pragma unroll
        for (int m = 0; m < kMaxPer; ++m) {
            const int a = lane + 32 * m;
            y[m] = a < k ? ybuf[a * R + c] : 0.0;
        }
        // forward, column-oriented: y_a /= Lc(a,a); y_i -= Lc(i,a) y_a for i > a
        for (int a = 0; a < k; ++a) {
            const double* col = core + (int64_t)a * k;
            double ya = 0.0;
#pragma unroll
            for (int m = 0; m < kMaxPer; ++m)
                if (lane + 32 * m == a) ya = y[m] / col[a];
            ya = __shfl_sync(0xffffffffu, ya, a & 31);
#pragma unroll
            for (int m = 0; m < kMaxPer; ++m) {
                const int i = lane + 32 * m;
                if (i == a) y[m] = ya;
                else if (i > a && i < k) y[m] = fma(-col[i], ya, y[m]);
            }
        }
        // backward, row-oriented: u_a = (y_a - sum_{j > a} Lc(j,a) u_j) / Lc(a,a)
        for (int a = k - 1; a >= 0; --a) {
            const double* col = core + (int64_t)a * k;
            double sacc = 0.0;
#pragma unroll
            for (int m = 0; m < kMaxPer; ++m) {
                const int j = lane + 32 * m;
                if (j > a && j < k) sacc = fma(col[j], y[m], sacc);
            }
            for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
#pragma unroll
            for (int m = 0; m < kMaxPer; ++m)
                if (lane + 32 * m == a) y[m] = (y[m] - sacc) / col[a];
        }
#pragma unroll
        for (int m = 0; m < kMaxPer; ++m) {
            const int a = lane + 32 * m;
            if (a < k) u_out[a * R + c] = (float)y[m];
        }
    }
}

// z[c][i] = inv_s2 w[c][i] - inv_s4 sum_a L[a][i] u[a][c]   (active columns only)
template <int RB>
__global__ void __launch_bounds__(256)
wb_out_kernel(const float* __restrict__ L, int64_t N, int k, const float* __restrict__ W, int R, int c0,
              const float* __restrict__ u, float inv_s2, float inv_s4, const int* __restrict__ active,
              float* __restrict__ Z) {
    extern __shared__ float su[];   // [k][RB]
    const int rc = (R - c0) < RB ? (R - c0) : RB;
    for (int e = threadIdx.x; e < k * RB; e += blockDim.x) {
        const int a = e / RB, cc = e % RB;
        su[e] = cc < rc ? u[a * R + c0 + cc] : 0.0f;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float acc[RB];
#pragma unroll
        for (int cc = 0; cc < RB; ++cc) acc[cc] = 0.0f;
        for (int a = 0; a < k; ++a) {
            const float la = L[(int64_t)a * N + i];
#pragma unroll
            for (int cc = 0; cc < RB; ++cc) acc[cc] = fmaf(la, su[a * RB + cc], acc[cc]);
        }
#pragma unroll
        for (int cc = 0; cc < RB; ++cc) {
            const int c = c0 + cc;
            if (cc < rc && (!active || active[c])) {
                const int64_t o = (int64_t)c * N + i;
                Z[o] = inv_s2 * W[o] - inv_s4 * acc[cc];
            }
        }
    }
}

}  // namespace

// ---- host side -----------------------------------------------------------------------------
int pivchol_grid(const Ctx* ctx, int64_t N) {
    int64_t g = (N + kPcThreads - 1) / kPcThreads;
    const int64_t cap = 2 * (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148);
    return (int)(g < cap ? g : cap);
}

size_t pivchol_workspace(const Ctx* ctx, int64_t N, int d, int rank) {
    WsCounter c;
    const int dp = ((d + 3) / 4) * 4;
    const int G = pivchol_grid(ctx, N);
    c.take<float>((size_t)N * dp);
    c.take<float>((size_t)N);
    c.take<Cand>((size_t)G);
    c.take<Cand>((size_t)G);
    c.take<int>(4);
    const int nsplit = 64;
    c.take<double>((size_t)nsplit * rank * rank);
    return c.off;
}

int pivchol_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, int rank, float* L,
                int32_t* piv, double* core, int* rank_out_host, cudaStream_t s) {
    const int dp = ((hyp->d + 3) / 4) * 4;
    const int G = pivchol_grid(ctx, N);
    float* Xs = wc.take<float>((size_t)N * dp);
    float* diag = wc.take<float>((size_t)N);
    Cand* ca = wc.take<Cand>((size_t)G);
    Cand* cb = wc.take<Cand>((size_t)G);
    int* rk = wc.take<int>(4);
    const int nsplit = 64;
    double* part = wc.take<double>((size_t)nsplit * rank * rank);
    if (!wc.ok) return GP_ERR_WORKSPACE;
    ScaleVec inv;
    const float c = kernel_input_scale(hyp->kernel);
    for (int k = 0; k < 64; ++k) inv.v[k] = k < hyp->d ? (float)((double)c / sqrt(2.0) / hyp->lengthscale[k]) : 0.0f;
    GPK_TRY(launch_prep_x_f32(ctx, X, N, N, hyp->d, dp, inv, Xs, s));
    const float a2 = (float)hyp->outputscale;
    fill_kernel<<<G, 256, 0, s>>>(diag, N, a2);
    ctx->launches++;
    if (cudaMemsetAsync(rk, 0xFF, sizeof(int), s) != cudaSuccess) return GP_ERR_CUDA;   // -1 = running
    // Without a host readback of the reached rank the factor is used at its
    // full width: columns an early stop leaves unwritten must be zero (they add
    // nothing to L L^T and an identity block to the core).
    if (!rank_out_host && cudaMemsetAsync(L, 0, sizeof(float) * (size_t)N * rank, s) != cudaSuccess)
        return GP_ERR_CUDA;
    const float tol_abs = 1e-6f * a2;
    for (int m = 0; m < rank; ++m) {
        const Cand* cin = (m & 1) ? ca : cb;
        Cand* cout = (m & 1) ? cb : ca;
        switch (hyp->kernel) {
            case GP_KERNEL_RBF:
                pivchol_step_kernel<GP_KERNEL_RBF><<<G, kPcThreads, 0, s>>>(Xs, N, dp, m, a2, tol_abs, L, diag, cin, G,
                                                                            cout, piv, rk);
                break;
            case GP_KERNEL_MATERN32:
                pivchol_step_kernel<GP_KERNEL_MATERN32><<<G, kPcThreads, 0, s>>>(Xs, N, dp, m, a2, tol_abs, L, diag,
                                                                                 cin, G, cout, piv, rk);
                break;
            case GP_KERNEL_MATERN12:
                pivchol_step_kernel<GP_KERNEL_MATERN12><<<G, kPcThreads, 0, s>>>(Xs, N, dp, m, a2, tol_abs, L, diag,
                                                                                 cin, G, cout, piv, rk);
                break;
            default:
                pivchol_step_kernel<GP_KERNEL_MATERN52><<<G, kPcThreads, 0, s>>>(Xs, N, dp, m, a2, tol_abs, L, diag,
                                                                                 cin, G, cout, piv, rk);
                break;
        }
        ctx->launches++;
    }
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    int kr = rank;
    if (rank_out_host) {
        if (cudaMemcpyAsync(ctx->host_pinned, rk, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return GP_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return GP_ERR_CUDA;
        const int rk_host = ctx->host_pinned[0];
        kr = rk_host < 0 ? rank : rk_host;
        *rank_out_host = kr;
    }
    if (kr == 0) return GP_OK;
    const int tiles = (kr + 15) / 16;
    gram_ll_kernel<<<dim3(tiles * tiles, nsplit), 256, 0, s>>>(L, N, kr, nsplit, part);
    ctx->launches++;
    core_chol_kernel<<<1, 1024, 0, s>>>(part, nsplit, kr, 1.0 / hyp->noise, core, ctx->dev_err);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

// ---- Woodbury apply ----
size_t woodbury_workspace(const Ctx* ctx, int64_t N, int k, int R) {
    (void)ctx;
    WsCounter c;
    const int64_t rows_per = N < 65536 ? kWbRows : ((N / 256 + kWbRows - 1) / kWbRows) * kWbRows;
    const int64_t nblk = (N + rows_per - 1) / rows_per;
    c.take<double>((size_t)nblk * k * R);
    c.take<double>((size_t)k * R);
    c.take<float>((size_t)k * R);
    return c.off;
}

int woodbury_apply(Ctx* ctx, WsCarver& wc, const float* L, const double* core, int k, double noise, int64_t N,
                   const float* W, int R, const int* active, float* Z, cudaStream_t s) {
    const int64_t rows_per = N < 65536 ? kWbRows : ((N / 256 + kWbRows - 1) / kWbRows) * kWbRows;
    const int64_t nblk = (N + rows_per - 1) / rows_per;
    double* tpart = wc.take<double>((size_t)nblk * k * R);
    double* ybuf = wc.take<double>((size_t)k * R);
    float* u = wc.take<float>((size_t)k * R);
    if (!wc.ok) return GP_ERR_WORKSPACE;
    const size_t sh1 = (size_t)(R + 16) * (kWbRows + 1) * sizeof(float);
    if (sh1 > 48 * 1024) {
        if (cudaFuncSetAttribute(wb_ltw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh1) != cudaSuccess)
            return GP_ERR_CUDA;
    }
    if (16 * R > 512) return GP_ERR_UNSUPPORTED;
    wb_ltw_kernel<<<(unsigned)nblk, 256, sh1, s>>>(L, N, k, W, R, active, rows_per, tpart);
    ctx->launches++;
    wb_solve_kernel<<<(unsigned)((R + kWbSolveWarps - 1) / kWbSolveWarps), kWbSolveWarps * 32, 0, s>>>(
        tpart, (int)nblk, k, R, core, u, ybuf);
    ctx->launches++;
    const float inv_s2 = (float)(1.0 / noise), inv_s4 = (float)(1.0 / (noise * noise));
    int64_t g = (N + 255) / 256;
    const int64_t cap = 4 * (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148);
    if (g > cap) g = cap;
    const int RB = R <= 8 ? 8 : (R <= 16 ? 16 : 32);
    for (int c0 = 0; c0 < R; c0 += RB) {
        const size_t sh = (size_t)k * RB * sizeof(float);
        if (RB == 8)
            wb_out_kernel<8><<<(unsigned)g, 256, sh, s>>>(L, N, k, W, R, c0, u, inv_s2, inv_s4, active, Z);
        else if (RB == 16)
            wb_out_kernel<16><<<(unsigned)g, 256, sh, s>>>(L, N, k, W, R, c0, u, inv_s2, inv_s4, active, Z);
        else
            wb_out_kernel<32><<<(unsigned)g, 256, sh, s>>>(L, N, k, W, R, c0, u, inv_s2, inv_s4, active, Z);
        ctx->launches++;
    }
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

}  // namespace gpk

extern "C" {

size_t gp_pivchol_workspace_size(const gp_hyp_t* hyp, int64_t N, int rank) {
    if (gpk::check_hyp(hyp) != GP_OK || N < 1 || rank < 1 || rank > 512) return 0;
    gpk::Ctx probe;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) probe.num_sms = 148;
    return gpk::pivchol_workspace(&probe, N, hyp->d, rank);
}

int gp_pivchol_precond(gp_ctx* ctx, const gp_hyp_t* hyp, const float* X, int64_t N, int rank, float* L,
                       int32_t* piv, double* core, int* rank_out, void* stream) {
    if (!ctx || !X || !L || !piv || !core || !rank_out) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_hyp(hyp));
    if (N < 1 || rank < 1 || rank > 512 || rank > N || !(hyp->noise > 0.0)) return GP_ERR_INVALID;
    gpk::Ctx* c = ctx;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != c->device && cudaSetDevice(c->device) != cudaSuccess) return GP_ERR_CUDA;
    gpk::WsCarver wc(c->ws, c->ws_bytes);
    int st = gpk::pivchol_run(c, wc, hyp, X, N, rank, L, piv, core, rank_out, (cudaStream_t)stream);
    if (prev != c->device) cudaSetDevice(prev);
    return st;
}

}  // extern "C"
