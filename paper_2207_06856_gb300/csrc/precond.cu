// Pivoted-Cholesky preconditioner and its Woodbury application
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
// Core.  C = I + sigma^-2 L^T L is accumulated in FP64 from FP32 sums of
// 64-row chunks and factored C = Lc Lc^T in FP64 by one CTA.
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
        // 64 products in FP32, the chunk sums in FP64 (FP64 is scarce on this GPU)
        float cs = 0.0f;
#pragma unroll 16
        for (int ii = 0; ii < 64; ++ii) cs = fmaf(sa[ii][la], sb[ii][lb], cs);
        acc += (double)cs;
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
// FP64 instructions are scarce on this GPU (a warp-wide FP64 FMA occupies its
// pipe for tens of cycles), so the FP64 parts of the apply are spread over
// many warps and never sit on a sequential path: C^{-1} is formed once per
// solve, and every apply is  t = L^T w (FP32 within row blocks, FP64 across
// them), u = C^{-1} t (one warp per output), z = (w - L u / sigma^2) / sigma^2.

// Column j of C^{-1} = Lc^{-T} Lc^{-1} e_j: forward and backward substitution,
// one warp per column, lane l holding rows l + 32 m (k <= 32 PER).
// Lc is column-major: Lc(a, b) = core[b * k + a].
template <int PER>
__global__ void __launch_bounds__(256)
core_inverse_kernel(const double* __restrict__ core, int k, double* __restrict__ cinv) {
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (j >= k) return;
    double y[PER];
#pragma unroll
    for (int m = 0; m < PER; ++m) y[m] = (lane + 32 * m == j) ? 1.0 : 0.0;
    // forward, column-oriented (entries above j stay zero)
    for (int a = j; a < k; ++a) {
        const double* col = core + (int64_t)a * k;
        double ya = 0.0;
#pragma unroll
        for (int m = 0; m < PER; ++m)
            if (lane + 32 * m == a) ya = y[m] / col[a];
        ya = __shfl_sync(0xffffffffu, ya, a & 31);
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int i = lane + 32 * m;
            if (i == a) y[m] = ya;
            else if (i > a && i < k) y[m] = fma(-col[i], ya, y[m]);
        }
    }
    // backward, row-oriented: x_a = (y_a - sum_{i > a} Lc(i, a) x_i) / Lc(a, a)
    for (int a = k - 1; a >= 0; --a) {
        const double* col = core + (int64_t)a * k;
        double sacc = 0.0;
#pragma unroll
        for (int m = 0; m < PER; ++m) {
            const int i = lane + 32 * m;
            if (i > a && i < k) sacc = fma(col[i], y[m], sacc);
        }
        for (int o = 16; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
#pragma unroll
        for (int m = 0; m < PER; ++m)
            if (lane + 32 * m == a) y[m] = (y[m] - sacc) / col[a];
    }
#pragma unroll
    for (int m = 0; m < PER; ++m) {
        const int a = lane + 32 * m;
        if (a < k) cinv[(int64_t)j * k + a] = y[m];
    }
}

// tpart[blk][a][c] = sum over this CTA's rows of L[a][i] W[c][i]: FP32
// register blocks of 4 a x 4 c per thread over 32-row tiles staged in shared
// memory (row-major, a or c fastest, float4 reads), stored as FP64.  The next
// tile's global loads are issued into registers before the current tile is
// multiplied, so the memory latency overlaps the arithmetic.
constexpr int kLtwTile = 32;
constexpr int kLtwMaxL = 16;   // prefetched L elements per thread: nab_pass <= 32
constexpr int kLtwMaxW = 8;    // prefetched W elements per thread: R <= 64
__global__ void __launch_bounds__(256, 3)
wb_ltw_kernel(const float* __restrict__ L, int64_t N, int k, const float* __restrict__ W, int R,
              int64_t rows_per_blk, int nab_pass, double* __restrict__ tpart) {
    extern __shared__ float4 sh4[];
    const int ncb = (R + 3) / 4;
    const int lstride = nab_pass + 1;   // float4 units per staged row (one pad)
    const int wstride = ncb + 1;
    float4* sL = sh4;                              // [kLtwTile][lstride]
    float4* sW = sh4 + kLtwTile * lstride;         // [kLtwTile][wstride]
    float* sLf = reinterpret_cast<float*>(sL);
    float* sWf = reinterpret_cast<float*>(sW);
    const int64_t r0 = rows_per_blk * blockIdx.x;
    const int64_t r1 = (r0 + rows_per_blk < N) ? r0 + rows_per_blk : N;
    const int ab = threadIdx.x % nab_pass, cb = threadIdx.x / nab_pass;
    const bool worker = cb < ncb;
    const int nLe = 4 * nab_pass * kLtwTile, nWe = 4 * ncb * kLtwTile;
    float pl[kLtwMaxL], pw[kLtwMaxW];
    for (int a0 = 0; a0 < k; a0 += 4 * nab_pass) {
        float acc[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] = 0.0f;
        auto fetch = [&](int64_t i0) {
#pragma unroll
            for (int q = 0; q < kLtwMaxL; ++q) {
                const int e = threadIdx.x + q * 256;
                const int aa = e / kLtwTile, ii = e % kLtwTile;
                const int64_t i = i0 + ii;
                pl[q] = (e < nLe && i < r1 && a0 + aa < k) ? L[(int64_t)(a0 + aa) * N + i] : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < kLtwMaxW; ++q) {
                const int e = threadIdx.x + q * 256;
                const int cc = e / kLtwTile, ii = e % kLtwTile;
                const int64_t i = i0 + ii;
                pw[q] = (e < nWe && i < r1 && cc < R) ? W[(int64_t)cc * N + i] : 0.0f;
            }
        };
        if (r0 < r1) fetch(r0);
        for (int64_t i0 = r0; i0 < r1; i0 += kLtwTile) {
            __syncthreads();
            // stage the prefetched tile as [row][a] and [row][c]
#pragma unroll
            for (int q = 0; q < kLtwMaxL; ++q) {
                const int e = threadIdx.x + q * 256;
                if (e < nLe) sLf[(e % kLtwTile) * 4 * lstride + e / kLtwTile] = pl[q];
            }
#pragma unroll
            for (int q = 0; q < kLtwMaxW; ++q) {
                const int e = threadIdx.x + q * 256;
                if (e < nWe) sWf[(e % kLtwTile) * 4 * wstride + e / kLtwTile] = pw[q];
            }
            __syncthreads();
            if (i0 + kLtwTile < r1) fetch(i0 + kLtwTile);   // next tile in flight during the products
            if (worker) {
#pragma unroll 8
                for (int ii = 0; ii < kLtwTile; ++ii) {
                    const float4 l4 = sL[ii * lstride + ab];
                    const float4 w4 = sW[ii * wstride + cb];
                    const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
                    const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(lv[x], wv[y], acc[x][y]);
                }
            }
        }
        if (worker) {
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const int a = a0 + 4 * ab + x;
#pragma unroll
                for (int y = 0; y < 4; ++y) {
                    const int c = 4 * cb + y;
                    if (a < k && c < R) tpart[((int64_t)blockIdx.x * k + a) * R + c] = (double)acc[x][y];
                }
            }
        }
    }
}

// t[a][c] = sum over blocks of tpart (fixed order within each lane, fixed
// shuffle tree across lanes); one warp per (a, c).
__global__ void __launch_bounds__(256)
wb_reduce_kernel(const double* __restrict__ tpart, int nblk, int k, int R, double* __restrict__ t) {
    const int e = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= k * R) return;
    double v = 0.0;
    for (int b = lane; b < nblk; b += 32) v += tpart[(int64_t)b * k * R + e];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) t[e] = v;
}

// u[a][c] = sum_b C^{-1}[a][b] t[b][c] (FP64), stored FP32; one warp per (a, c).
__global__ void __launch_bounds__(256)
wb_gemv_kernel(const double* __restrict__ cinv, const double* __restrict__ t, int k, int R, float* __restrict__ u) {
    const int e = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (e >= k * R) return;
    const int a = e / R, c = e % R;
    double v = 0.0;
    for (int b = lane; b < k; b += 32) v = fma(cinv[(int64_t)a * k + b], t[b * R + c], v);   // C^{-1} symmetric
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) u[e] = (float)v;
}

// z[c][i] = inv_s2 w[c][i] - inv_s4 sum_a L[a][i] u[a][c]   (active columns only)
// u staged in shared memory as [a][RB] (RB a multiple of 4: float4 reads,
// the same address across the warp).
// grid.y: column groups of RB (c0 = RB * blockIdx.y): more threads in flight
// than one per row.
template <int RB>
__global__ void __launch_bounds__(256)
wb_out_kernel(const float* __restrict__ L, int64_t N, int k, const float* __restrict__ W, int R,
              const float* __restrict__ u, float inv_s2, float inv_s4, const int* __restrict__ active,
              float* __restrict__ Z) {
    const int c0 = RB * (int)blockIdx.y;
    extern __shared__ float4 su4[];   // [k][RB / 4]
    float* su = reinterpret_cast<float*>(su4);
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
#pragma unroll 4
        for (int a = 0; a < k; ++a) {
            const float la = L[(int64_t)a * N + i];
#pragma unroll
            for (int q = 0; q < RB / 4; ++q) {
                const float4 u4 = su4[a * (RB / 4) + q];
                acc[4 * q] = fmaf(la, u4.x, acc[4 * q]);
                acc[4 * q + 1] = fmaf(la, u4.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(la, u4.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(la, u4.w, acc[4 * q + 3]);
            }
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
namespace {
int ltw_grid(const Ctx* ctx, int64_t N, int64_t* rows_per) {
    // two CTAs per SM, each walking its rows in dependent 32-row tiles: more
    // CTAs hide more latency but each adds k x R FP64 partials to reduce
    // (measured on the precision workload: 2 per SM beat 3, 4 and 6)
    const int64_t G = 2 * (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148);
    int64_t rp = (N + G - 1) / G;
    rp = ((rp + kLtwTile - 1) / kLtwTile) * kLtwTile;
    if (rp < kLtwTile) rp = kLtwTile;
    *rows_per = rp;
    return (int)((N + rp - 1) / rp);
}
}  // namespace

size_t woodbury_workspace(const Ctx* ctx, int64_t N, int k, int R) {
    WsCounter c;
    int64_t rp = 0;
    const int nblk = ltw_grid(ctx, N, &rp);
    c.take<double>((size_t)nblk * k * R);   // partials
    c.take<double>((size_t)k * R);          // t
    c.take<float>((size_t)k * R);           // u
    c.take<double>((size_t)k * k);          // C^{-1} when the caller has none
    return c.off;
}

int woodbury_prepare(Ctx* ctx, const double* core, int k, double* cinv, cudaStream_t s) {
    const unsigned g = (unsigned)((k + 7) / 8);
    if (k <= 128) core_inverse_kernel<4><<<g, 256, 0, s>>>(core, k, cinv);
    else if (k <= 256) core_inverse_kernel<8><<<g, 256, 0, s>>>(core, k, cinv);
    else core_inverse_kernel<16><<<g, 256, 0, s>>>(core, k, cinv);
    ctx->launches++;
    return cudaGetLastError() == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

int woodbury_apply(Ctx* ctx, WsCarver& wc, const float* L, const double* core, const double* cinv, int k,
                   double noise, int64_t N, const float* W, int R, const int* active, float* Z, cudaStream_t s) {
    int64_t rows_per = 0;
    const int nblk = ltw_grid(ctx, N, &rows_per);
    double* tpart = wc.take<double>((size_t)nblk * k * R);
    double* t = wc.take<double>((size_t)k * R);
    float* u = wc.take<float>((size_t)k * R);
    double* cinv_own = wc.take<double>((size_t)k * k);
    if (!wc.ok) return GP_ERR_WORKSPACE;
    if (R > 64 || k > 512) return GP_ERR_UNSUPPORTED;
    if (!cinv) {
        GPK_TRY(woodbury_prepare(ctx, core, k, cinv_own, s));
        cinv = cinv_own;
    }
    const int ncb = (R + 3) / 4;
    const int nab_all = (k + 3) / 4;
    int nab_pass = 256 / ncb;
    if (nab_pass > 32) nab_pass = 32;   // the prefetch registers of wb_ltw_kernel
    if (nab_pass > nab_all) nab_pass = nab_all;
    const size_t sh1 = (size_t)kLtwTile * ((nab_pass + 1) + (ncb + 1)) * sizeof(float4);
    if (sh1 > 48 * 1024 &&
        cudaFuncSetAttribute(wb_ltw_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh1) != cudaSuccess)
        return GP_ERR_CUDA;
    wb_ltw_kernel<<<(unsigned)nblk, 256, sh1, s>>>(L, N, k, W, R, rows_per, nab_pass, tpart);
    ctx->launches++;
    const unsigned gw = (unsigned)((k * R + 7) / 8);
    wb_reduce_kernel<<<gw, 256, 0, s>>>(tpart, nblk, k, R, t);
    wb_gemv_kernel<<<gw, 256, 0, s>>>(cinv, t, k, R, u);
    ctx->launches += 2;
    const float inv_s2 = (float)(1.0 / noise), inv_s4 = (float)(1.0 / (noise * noise));
    int64_t g = (N + 255) / 256;
    const int64_t cap = 4 * (int64_t)(ctx->num_sms > 0 ? ctx->num_sms : 148);
    if (g > cap) g = cap;
    const int RB = R <= 4 ? 4 : 8;
    const dim3 grid((unsigned)g, (unsigned)((R + RB - 1) / RB));
    const size_t sh = (size_t)k * RB * sizeof(float);
    if (RB == 4)
        wb_out_kernel<4><<<grid, 256, sh, s>>>(L, N, k, W, R, u, inv_s2, inv_s4, active, Z);
    else
        wb_out_kernel<8><<<grid, 256, sh, s>>>(L, N, k, W, R, u, inv_s2, inv_s4, active, Z);
    ctx->launches++;
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
