// The backward of the kernel MVM on the tensor cores (Sec. 4.3, Eq. approx;
// Sec. 2.2, Eq. gradient): the gradient of the bilinear form
//     q = sum_c u_c^T Ktilde w_c
// with respect to (l_1..l_d, a^2, sigma^2) and X, for RBF, Matern-3/2 and
// Matern-5/2 with FP16 operands and FP32 accumulation.
//
// With H_ij = G_ij + G_ji = sum_c (u_ic w_jc + w_ic u_jc) (symmetric), the
// scaled centred inputs x^_i = (x_i - centre) / l and k' = dk/d(r^2):
//     W'_ij = a^2 k'(r_ij^2) H_ij,  rs_i = sum_j W'_ij,  (W'X^)_im = sum_j W'_ij x^_jm,
//     D_im  = sum_j W'_ij (x^_im - x^_jm) = x^_im rs_i - (W'X^)_im,
//     dq/dx_im    = (2 / l_m) D_im,
//     dq/dl_m     = -(2 / l_m) sum_i x^_im D_im,
//     dq/da^2     = 1/2 sum_ij H_ij k(r_ij^2),
//     dq/dsigma^2 = sum_c u_c^T w_c.
// (sum_ij a^2 k' G_ij (x^_im - x^_jm)^2 = 1/2 sum_ij W'_ij (x^_im - x^_jm)^2 =
// sum_i x^_im D_im, because W' is symmetric.)  So one value product
// W' [X^, 1] per row tile gives every derivative: the backward has the
// forward's shape (flash-attention backward: S and H on the tensor core, the
// elementwise W' in registers, then a second contraction).
//
// Per 128 x 128 tile, on tcgen05 with FP32 accumulators in TMEM:
//   S  = XA_i XB_j^T     (the forward's operands: s = -c^2 r^2 / 2)
//   H  = UW_i WU_j^T     UW = [a_c u | w / a_c], WU = [w / a_c | a_c u] in FP16
//                        (a_c a power of two balancing the column pair; one
//                        global power-of-two scale keeps |entries| <= 1)
//   O += W'_i Xt_j^T     W' from TMEM (.ts form), Xt = [x^ hi; 1; x^ lo; 0]
//                        rows (the ones row gives rs_i); N = 2 R_pad
// The epilogue stores W' / (a^2 k'_max) = -phi(s) H (phi = k for RBF, e^-u for
// Matern-3/2, (1 + u) e^-u for Matern-5/2) as FP16 in TMEM, and accumulates
// sum H k per thread.  Warps: 0-15 epilogue (warpgroup q: columns
// [32 q, 32 q + 32) of the tile), 16 TMA producer, 17 S / H issuer and TMEM
// owner, 18 value-product issuer.  TMEM: S [0,128), H [128,256), W' buffers
// [256,320) and [320,384), O [384, 384 + 2 R_pad).  Every wait is bounded.
#include "gpk_internal.cuh"
#include "ptx.cuh"
#include "kfun.cuh"

#include <math.h>

namespace gpk {

namespace {

constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kEpiWarps = 16;
constexpr int kThreads = (kEpiWarps + 3) * 32;
constexpr int kTmaWarp = kEpiWarps;
constexpr int kShWarp = kEpiWarps + 1;
constexpr int kOWarp = kEpiWarps + 2;
constexpr int kMaxStages = 4;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kColS = 0, kColH = 128, kColW = 256, kColO = 384;
constexpr int kMaxSmemBytes = 227 * 1024;

struct VjpParams {
    int n_it, n_jt, n_split, n_items;
    int k_pad, kh, rv;       // S contraction width, H contraction width (2 R_pad), O width (2 R_pad of Xt)
    int stages;
    int64_t N_pad;
    float* part;             // [n_split][rv][N_pad]: raw O columns
    double* hk;              // [gridDim.x]: per-CTA sum of H k
    int* err;
    uint64_t limit_ns;
};

struct VjpBarriers {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t xi_full[2];
    uint64_t xi_empty[2];
    uint64_t sh_full;
    uint64_t sh_empty;
    uint64_t w_full[2];
    uint64_t w_empty[2];
    uint64_t o_full;
    uint64_t o_empty;
    uint64_t drain[2];
};

struct VjpSmem {
    uint32_t xbytes, hbytes, vbytes, stage_bytes, xi_bytes;
    int stages;
    uint32_t total;
};

__host__ __device__ inline VjpSmem vjp_smem(int k_pad, int kh, int rv) {
    VjpSmem m;
    m.xbytes = (uint32_t)kBM * (uint32_t)k_pad * 2u;
    m.hbytes = (uint32_t)kBM * (uint32_t)kh * 2u;
    m.vbytes = 2u * (uint32_t)rv * 128u;                 // two 64-column K-blocks of rv rows
    m.stage_bytes = m.xbytes + m.hbytes + m.vbytes;
    m.xi_bytes = m.xbytes + m.hbytes;
    const uint32_t fixed = 1024u + 2u * m.xi_bytes;
    m.stages = 0;
    for (int s = kMaxStages; s >= 2; --s)
        if (fixed + (uint32_t)s * m.stage_bytes <= (uint32_t)kMaxSmemBytes - 512u) { m.stages = s; break; }
    m.total = fixed + (uint32_t)m.stages * m.stage_bytes;
    return m;
}

__device__ __forceinline__ void record_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ void item_range(const VjpParams& p, int item, int& it, int& sp, int& j0, int& j1) {
    it = item % p.n_it;
    sp = item / p.n_it;
    j0 = (int)(((int64_t)sp * p.n_jt) / p.n_split);
    j1 = (int)(((int64_t)(sp + 1) * p.n_jt) / p.n_split);
}

__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    return __all_sync(0xffffffffu, ptx::mbar_wait(bar, parity, limit_ns));
}

__device__ __forceinline__ uint32_t swz_code(uint32_t row_bytes) {
    return row_bytes == 32u ? 6u : (row_bytes == 64u ? 4u : 2u);
}

// ---- TMA producer (one thread) ------------------------------------------------
__device__ void vjp_producer(const VjpParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB,
                             const CUtensorMap* tmUW, const CUtensorMap* tmWU, const CUtensorMap* tmXt,
                             VjpBarriers& bars, uint8_t* sSt, uint8_t* sXi, const VjpSmem& m) {
    uint32_t fills = 0, xi_loads = 0;
    bool ok = true;
    int ic = 0;
    const uint32_t S = (uint32_t)p.stages;
    const uint32_t vbox = (uint32_t)p.rv * 128u;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x, ++ic) {
        int it, sp, j0, j1;
        item_range(p, item, it, sp, j0, j1);
        const int xb = ic & 1;
        if (ic >= 2 && !ptx::mbar_wait(&bars.xi_empty[xb], ((ic >> 1) - 1) & 1, p.limit_ns)) { ok = false; break; }
        uint8_t* sX = sXi + (uint32_t)xb * m.xi_bytes;
        ptx::mbar_arrive_expect_tx(&bars.xi_full[xb], m.xi_bytes);
        ptx::tma_load_2d(sX, tmA, &bars.xi_full[xb], 0, it * kBM);
        ptx::tma_load_2d(sX + m.xbytes, tmUW, &bars.xi_full[xb], 0, it * kBM);
        ++xi_loads;
        for (int jt = j0; jt < j1; ++jt) {
            const uint32_t st = fills % S, u = fills / S;
            if (u > 0 && !ptx::mbar_wait(&bars.empty[st], (u - 1) & 1, p.limit_ns)) { ok = false; break; }
            uint8_t* sx = sSt + st * m.stage_bytes;
            ptx::mbar_arrive_expect_tx(&bars.full[st], m.stage_bytes);
            ptx::tma_load_2d(sx, tmB, &bars.full[st], 0, jt * kBN);
            ptx::tma_load_2d(sx + m.xbytes, tmWU, &bars.full[st], 0, jt * kBN);
            ptx::tma_load_2d(sx + m.xbytes + m.hbytes, tmXt, &bars.full[st], jt * kBN, 0);
            ptx::tma_load_2d(sx + m.xbytes + m.hbytes + vbox, tmXt, &bars.full[st], jt * kBN + 64, 0);
            ++fills;
        }
        if (!ok) break;
    }
    if (!ok) {
        record_error(p.err, DEV_TIMEOUT);
        // every copy this thread issued lands before the CTA can exit
        const uint32_t first = fills > S ? fills - S : 0;
        for (uint32_t f = first; f < fills; ++f) ptx::mbar_wait(&bars.full[f % S], (f / S) & 1, p.limit_ns);
        for (uint32_t q = xi_loads > 2 ? xi_loads - 2 : 0; q < xi_loads; ++q)
            ptx::mbar_wait(&bars.xi_full[q & 1], (q >> 1) & 1, p.limit_ns);
    }
}

// ---- S / H issuer (one converged warp) ------------------------------------------
// For each column tile: S and H into their TMEM buffers once the epilogue has
// read the previous tile's S and H and the stage has landed.
__device__ void vjp_mma_sh(const VjpParams& p, VjpBarriers& bars, const uint8_t* sSt, const uint8_t* sXi,
                           const VjpSmem& m, uint32_t tmem) {
    const uint32_t xrow = (uint32_t)p.k_pad * 2u, hrow = (uint32_t)p.kh * 2u;
    const uint32_t hi_x = ptx::smem_desc_hi(8u * xrow, swz_code(xrow));
    const uint32_t hi_h = ptx::smem_desc_hi(8u * hrow, swz_code(hrow));
    const uint32_t id = ptx::idesc_f16(kBM, kBN, 0);
    const uint32_t S = (uint32_t)p.stages;
    const uint32_t aSt = ptx::smem_u32(sSt);
    uint32_t g = 0, st = 0, ph = 0;
    int ic = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x, ++ic) {
        int it, sp, j0, j1;
        item_range(p, item, it, sp, j0, j1);
        const uint32_t T = (uint32_t)(j1 - j0);
        const int xb = ic & 1;
        if (!warp_wait(&bars.xi_full[xb], (ic >> 1) & 1, p.limit_ns)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t aXi = ptx::smem_u32(sXi) + (uint32_t)xb * m.xi_bytes;
        for (uint32_t t = 0; t < T; ++t, ++g) {
            if (g > 0 && !warp_wait(&bars.sh_empty, (g - 1) & 1, p.limit_ns)) { ok = false; break; }
            if (!warp_wait(&bars.full[st], ph, p.limit_ns)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t aXj = aSt + st * m.stage_bytes;
            for (int kk = 0; kk < p.k_pad / 16; ++kk)
                ptx::mma_f16_ss_elect(tmem + kColS, ptx::smem_desc_at(hi_x, aXi + (uint32_t)kk * 32u),
                                      ptx::smem_desc_at(hi_x, aXj + (uint32_t)kk * 32u), id, kk > 0 ? 1u : 0u);
            for (int kk = 0; kk < p.kh / 16; ++kk)
                ptx::mma_f16_ss_elect(tmem + kColH, ptx::smem_desc_at(hi_h, aXi + m.xbytes + (uint32_t)kk * 32u),
                                      ptx::smem_desc_at(hi_h, aXj + m.xbytes + (uint32_t)kk * 32u), id,
                                      kk > 0 ? 1u : 0u);
            ptx::mma_commit_elect(&bars.sh_full);
            if (t + 1 == T) ptx::mma_commit_elect(&bars.xi_empty[xb]);   // last use of the row tile
            if (++st == S) { st = 0; ph ^= 1u; }
        }
    }
    ptx::mma_commit_elect(&bars.drain[0]);
    warp_wait(&bars.drain[0], 0, p.limit_ns);
    if (!ok && (threadIdx.x & 31) == 0) record_error(p.err, DEV_TIMEOUT);
}

// ---- value-product issuer (one converged warp) ------------------------------------
// O += W'(t) Xt_j^T with W' read from TMEM; then W' buffer t & 1 and the stage
// are released.  O is handed to the epilogue at the end of an item.
__device__ void vjp_mma_o(const VjpParams& p, VjpBarriers& bars, const uint8_t* sSt, const VjpSmem& m,
                          uint32_t tmem) {
    const uint32_t hi_v = ptx::smem_desc_hi(1024u, 2u);
    const uint32_t id = ptx::idesc_f16(kBM, p.rv, 0);
    const uint32_t S = (uint32_t)p.stages;
    const uint32_t aSt = ptx::smem_u32(sSt);
    const uint32_t vbox = (uint32_t)p.rv * 128u;
    uint32_t g = 0, st = 0, ph = 0;
    int ic = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x, ++ic) {
        int it, sp, j0, j1;
        item_range(p, item, it, sp, j0, j1);
        const uint32_t T = (uint32_t)(j1 - j0);
        for (uint32_t t = 0; t < T; ++t, ++g) {
            if (t == 0 && ic > 0 && !warp_wait(&bars.o_empty, (ic - 1) & 1, p.limit_ns)) { ok = false; break; }
            if (!warp_wait(&bars.full[st], ph, p.limit_ns)) { ok = false; break; }   // Xt_j: landed for S
            const uint32_t wb = g & 1u;
            if (!warp_wait(&bars.w_full[wb], (g >> 1) & 1, p.limit_ns)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t aV = aSt + st * m.stage_bytes + m.xbytes + m.hbytes;
#pragma unroll
            for (int kk = 0; kk < kBN / 16; ++kk) {
                const uint32_t off = (uint32_t)(kk >> 2) * vbox + (uint32_t)(kk & 3) * 32u;
                ptx::mma_f16_ts_elect(tmem + kColO, tmem + kColW + wb * 64u + (uint32_t)kk * 8u,
                                      ptx::smem_desc_at(hi_v, aV + off), id, (t > 0 || kk > 0) ? 1u : 0u);
            }
            ptx::mma_commit_elect(&bars.w_empty[wb]);   // W' buffer wb may be rewritten
            ptx::mma_commit_elect(&bars.empty[st]);     // the stage's operands are consumed
            if (++st == S) { st = 0; ph ^= 1u; }
        }
        if (!ok) break;
        ptx::mma_commit_elect(&bars.o_full);
    }
    ptx::mma_commit_elect(&bars.drain[1]);
    warp_wait(&bars.drain[1], 0, p.limit_ns);
    if (!ok && (threadIdx.x & 31) == 0) record_error(p.err, DEV_TIMEOUT);
}

// ---- epilogue: W' = -phi(s) H in FP16, sum H k --------------------------------------
template <int KIND>
__device__ __forceinline__ void wprime(float s, float h, float& w, float& hk) {
    if constexpr (KIND == GP_KERNEL_RBF) {
        const float k = ptx::ex2(s);                      // s = -log2(e) r^2 / 2
        w = -k * h;                                       // k' = -k / 2, k'_max = 1/2
        hk = h * k;
    } else {
        const float u = ptx::sqrt_approx(fmaxf(-s, 0.0f));   // u = sqrt3 r (Matern-3/2), sqrt5 r (5/2)
        const float e = ptx::ex2(-kLog2e * u);
        if constexpr (KIND == GP_KERNEL_MATERN32) {
            w = -e * h;                                   // k' = -(3/2) e^-u, k'_max = 3/2
            hk = h * fmaf(u, e, e);
        } else {
            const float pu = 1.0f + u;
            w = -pu * e * h;                              // k' = -(5/6)(1 + u) e^-u, k'_max = 5/6
            hk = h * (fmaf(u * u, 1.0f / 3.0f, pu) * e);
        }
    }
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

template <int KIND>
__device__ void vjp_epilogue(const VjpParams& p, VjpBarriers& bars, uint32_t tmem, int q, int wq, int lane,
                             double* red) {
    const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
    uint32_t g = 0;
    int ic = 0;
    bool ok = true;
    double acc = 0.0;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x, ++ic) {
        int it, sp, j0, j1;
        item_range(p, item, it, sp, j0, j1);
        const uint32_t T = (uint32_t)(j1 - j0);
        for (uint32_t t = 0; t < T; ++t, ++g) {
            if (!warp_wait(&bars.sh_full, g & 1, p.limit_ns)) { ok = false; break; }
            ptx::tc_fence_after();
            uint32_t rs[32], rh[32];
            ptx::tmem_ld32(tmem + lane_off + kColS + (uint32_t)q * 32u, rs);
            ptx::tmem_ld32(tmem + lane_off + kColH + (uint32_t)q * 32u, rh);
            ptx::tmem_wait_ld();
            ptx::tmem_reg_fence(rs);
            ptx::tmem_reg_fence(rh);
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bars.sh_empty);   // this warp's part of S and H is in registers
            uint32_t pk[16];
            float a = 0.0f;
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                float w0, w1, h0, h1;
                wprime<KIND>(__uint_as_float(rs[2 * e]), __uint_as_float(rh[2 * e]), w0, h0);
                wprime<KIND>(__uint_as_float(rs[2 * e + 1]), __uint_as_float(rh[2 * e + 1]), w1, h1);
                a += h0 + h1;
                __half2 hv = __floats2half2_rn(w0, w1);
                pk[e] = *reinterpret_cast<uint32_t*>(&hv);
            }
            acc += (double)a;
            const uint32_t wb = g & 1u;
            if (g >= 2 && !warp_wait(&bars.w_empty[wb], ((g >> 1) - 1) & 1, p.limit_ns)) { ok = false; break; }
            ptx::tmem_st16(tmem + lane_off + kColW + wb * 64u + (uint32_t)q * 16u, pk);
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bars.w_full[wb]);
        }
        if (!ok) break;
        // O read-out: this warpgroup's rv / 4 columns of its 32 rows
        if (!warp_wait(&bars.o_full, ic & 1, p.limit_ns)) { ok = false; break; }
        ptx::tc_fence_after();
        const int64_t row = (int64_t)it * kBM + wq * 32 + lane;
        const int ncol = p.rv / 4, c0 = q * ncol;
        float* dst = p.part + ((int64_t)sp * p.rv + c0) * p.N_pad + row;
        if (ncol == 16) {
            uint32_t o[16];
            ptx::tmem_ld16(tmem + lane_off + kColO + (uint32_t)c0, o);
            ptx::tmem_wait_ld();
            ptx::tmem_reg_fence(o);
#pragma unroll
            for (int c = 0; c < 16; ++c) dst[(int64_t)c * p.N_pad] = __uint_as_float(o[c]);
        } else {
            uint32_t o[8];
            tmem_ld8(tmem + lane_off + kColO + (uint32_t)c0, o);
            ptx::tmem_wait_ld();
            ptx::tmem_reg_fence(o);
#pragma unroll
            for (int c = 0; c < 8; ++c) dst[(int64_t)c * p.N_pad] = __uint_as_float(o[c]);
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&bars.o_empty);
    }
    if (!ok && lane == 0) record_error(p.err, DEV_TIMEOUT);
    // per-CTA sum of H k in a fixed order: warp shuffle tree, then the warps in order
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) red[q * 4 + wq] = acc;
}

template <int KIND>
__global__ void __launch_bounds__(kThreads, 1)
kvjp_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmUW, const __grid_constant__ CUtensorMap tmWU,
               const __grid_constant__ CUtensorMap tmXt, const VjpParams p) {
    extern __shared__ uint8_t dsm[];
    __shared__ VjpBarriers bars;
    __shared__ uint32_t tmem_slot;
    __shared__ double red[kEpiWarps];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
    const VjpSmem m = vjp_smem(p.k_pad, p.kh, p.rv);
    uint8_t* sSt = base;
    uint8_t* sXi = base + (uint32_t)p.stages * m.stage_bytes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            ptx::mbar_init(&bars.full[s], 1);
            ptx::mbar_init(&bars.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&bars.xi_full[b], 1);
            ptx::mbar_init(&bars.xi_empty[b], 1);
            ptx::mbar_init(&bars.w_full[b], kEpiWarps);   // one arrival per epilogue warp
            ptx::mbar_init(&bars.w_empty[b], 1);
            ptx::mbar_init(&bars.drain[b], 1);
        }
        ptx::mbar_init(&bars.sh_full, 1);
        ptx::mbar_init(&bars.sh_empty, kEpiWarps);
        ptx::mbar_init(&bars.o_full, 1);
        ptx::mbar_init(&bars.o_empty, kEpiWarps);
        ptx::fence_mbar_init();
    }
    if (warp == kTmaWarp && lane == 0) {
        ptx::tma_prefetch_desc(&tmA);
        ptx::tma_prefetch_desc(&tmB);
        ptx::tma_prefetch_desc(&tmUW);
        ptx::tma_prefetch_desc(&tmWU);
        ptx::tma_prefetch_desc(&tmXt);
    }
    if (warp == kShWarp) ptx::tmem_alloc(&tmem_slot, kTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_slot;
    if (warp == kTmaWarp) {
        if (lane == 0) vjp_producer(p, &tmA, &tmB, &tmUW, &tmWU, &tmXt, bars, sSt, sXi, m);
        __syncwarp();
    } else if (warp == kShWarp) {
        vjp_mma_sh(p, bars, sSt, sXi, m, tmem);
    } else if (warp == kOWarp) {
        vjp_mma_o(p, bars, sSt, m, tmem);
    } else {
        vjp_epilogue<KIND>(p, bars, tmem, warp >> 2, warp & 3, lane, red);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kEpiWarps; ++w) t += red[w];
        p.hk[blockIdx.x] = t;
    }
    if (warp == kShWarp) ptx::tmem_dealloc(tmem, kTmemCols);
}

// ---- operand preparation and the final reductions ----------------------------------
// scales[c] = a_c (power of two balancing max|u_c| and max|w_c|), scales[rp] = g:
// the power of two that brings every entry of [a u | w / a] to |.| <= 1.
__global__ void uw_scales_kernel(const unsigned* __restrict__ cmu, const unsigned* __restrict__ cmw, int R, int rp,
                                 float* __restrict__ scales, int* err) {
    __shared__ float mx[32];
    const int c = threadIdx.x;   // one warp, R <= 32
    float a = 1.0f, m = 0.0f;
    if (c < R) {
        const float mu = __uint_as_float(cmu[c]), mw = __uint_as_float(cmw[c]);
        if (!(mu <= 3.0e38f) || !(mw <= 3.0e38f)) {
            atomicCAS(err, 0, (int)DEV_NONFINITE);
        } else {
            if (mu > 0.0f && mw > 0.0f) a = exp2f(rintf(0.5f * log2f(mw / mu)));
            m = fmaxf(a * mu, mw / a);
        }
        scales[c] = a;
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (c == 0) {
        float g = 1.0f;
        if (m > 0.0f) {
            int e;
            frexpf(m, &e);            // m = f 2^e, f in [1/2, 1)
            g = ldexpf(1.0f, -e);     // m g < 1
        }
        scales[rp] = g;
    }
    (void)mx;
}

// UW[i] = g [a_c u_ic | w_ic / a_c], WU[i] = g [w_ic / a_c | a_c u_ic] in FP16 (rows i < N_pad,
// zero beyond N and beyond R in each half); U, W: R x N (column c at c * N).
__global__ void uw_prep_kernel(const float* __restrict__ U, const float* __restrict__ W, int64_t N, int64_t N_pad,
                               int R, int rp, const float* __restrict__ scales, __half* __restrict__ UW,
                               __half* __restrict__ WU) {
    const int kh = 2 * rp;
    const float g = scales[rp];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N_pad * kh;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / kh;
        const int col = (int)(e % kh);
        const int c = col < rp ? col : col - rp;
        float uw = 0.0f, wu = 0.0f;
        if (i < N && c < R) {
            const float a = scales[c];
            const float u = U[(int64_t)c * N + i] * a * g, w = W[(int64_t)c * N + i] / a * g;
            uw = col < rp ? u : w;
            wu = col < rp ? w : u;
        }
        UW[e] = __float2half_rn(uw);
        WU[e] = __float2half_rn(wu);
    }
}

__device__ __forceinline__ float decode_order(unsigned s) {
    return __uint_as_float((s & 0x80000000u) ? (s & 0x7FFFFFFFu) : ~s);
}

// Vb (d + 1 columns of N, FP32): x^_m = (x_m - centre_m) / l_m, then a column of ones.
__global__ void vb_prep_kernel(const float* __restrict__ X, int64_t N, int d, ScaleVec il,
                               const unsigned* __restrict__ bb, float* __restrict__ Vb) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * (d + 1);
         e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / N);
        const int64_t i = e % N;
        if (m < d) {
            const float centre = 0.5f * (decode_order(bb[m]) + decode_order(bb[d + m]));
            Vb[e] = (X[i * d + m] - centre) * il.v[m];
        } else {
            Vb[e] = 1.0f;
        }
    }
}

// Per row i < N: O_c = sum_s (part[s][c][i] + part[s][rx + c][i]) xs_c (hi + lo rows of Xt),
// rs_i = O_d, D_im = x^_im rs_i - O_m; gX_im = (2 / l_m) F D_im; per block sum_i x^_im D_im (FP64).
// F = a^2 k'_max / g^2 undoes the storage scale of W'.
__global__ void __launch_bounds__(256)
vjp_finish_kernel(const float* __restrict__ part, int n_split, int rv, int64_t N_pad, const float* __restrict__ xs,
                  const float* __restrict__ Vb, int64_t N, int d, ScaleVec two_over_l, float a2kp,
                  const float* __restrict__ scales, int rp, float* __restrict__ gX, double* __restrict__ lpart) {
    const int rx = rv / 2;
    const float g = scales[rp];
    const float F = a2kp / (g * g);
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double lsum[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) lsum[m] = 0.0;
    if (i < N) {
        float rs = 0.0f;
        for (int s = 0; s < n_split; ++s)
            rs += part[((int64_t)s * rv + d) * N_pad + i] + part[((int64_t)s * rv + rx + d) * N_pad + i];
        rs *= xs[d];
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            if (m < d) {
                float o = 0.0f;
                for (int s = 0; s < n_split; ++s)
                    o += part[((int64_t)s * rv + m) * N_pad + i] + part[((int64_t)s * rv + rx + m) * N_pad + i];
                const float xh = Vb[(int64_t)m * N + i];
                const float D = fmaf(xh, rs, -o * xs[m]);
                if (gX) gX[i * d + m] = two_over_l.v[m] * F * D;
                lsum[m] = (double)xh * (double)D;
            }
        }
    }
    __shared__ double red[8][32];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
        double v = lsum[m];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (l == 0) red[w][m] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
        lpart[(int64_t)blockIdx.x * 32 + threadIdx.x] = t * (double)F;
    }
}

// out[s] = sum_b part[b * stride + s] in block order (one thread per slot)
__global__ void sum_rows_kernel(const double* __restrict__ part, int nb, int stride, int ns, double* __restrict__ out) {
    const int s = threadIdx.x;
    if (s >= ns) return;
    double t = 0.0;
    for (int b = 0; b < nb; ++b) t += part[(int64_t)b * stride + s];
    out[s] = t;
}

// out[c] = u_c^T w_c in FP64, one block per column, fixed-order tree
__global__ void coldot2_kernel(const float* __restrict__ U, const float* __restrict__ W, int64_t N,
                               double* __restrict__ out) {
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
        acc = fma((double)U[(int64_t)c * N + i], (double)W[(int64_t)c * N + i], acc);
    __shared__ double r[32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) r[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += r[q];
        out[c] = t;
    }
}

float kprime_max(int kernel) {
    return kernel == GP_KERNEL_RBF ? 0.5f : (kernel == GP_KERNEL_MATERN32 ? 1.5f : 5.0f / 6.0f);
}

CUtensorMapSwizzle swz_for(uint32_t row_bytes) {
    return row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                           : (row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
}

}  // namespace

bool vjp_tc_supported(const gp_hyp_t* hyp, int R) {
    if (hyp->kernel == GP_KERNEL_MATERN12) return false;   // k' ~ 1/r: singular at coincident points
    if (hyp->d > 31 || R > 32) return false;
    const OperandLayout L = make_layout(hyp->d, GP_PREC_FP16, hyp->d > 12 ? 1 : 0, 1, 0);
    return L.k_pad != 0 && L.k_pad <= 64;
}

namespace {

struct VjpPlan {
    int n_it, n_jt, n_split, grid, rp, kh, rx, rv;
    int64_t N_pad, Nc_pad;
    int nblk_f;
};

VjpPlan vjp_plan(const Ctx* ctx, const KOp& op, int64_t N, int d, int R) {
    VjpPlan p;
    p.N_pad = op.tp.Nr_pad;
    p.Nc_pad = op.tp.Nc_pad;
    p.n_it = (int)((N + kBM - 1) / kBM);
    p.n_jt = (int)(p.Nc_pad / kBN);
    p.rp = R <= 16 ? 16 : 32;
    p.kh = 2 * p.rp;
    p.rx = (d + 1) <= 16 ? 16 : 32;
    p.rv = 2 * p.rx;
    const int G = ctx->num_sms > 0 ? ctx->num_sms : 1;
    // column split minimising the busiest CTA's tiles (+ about two tiles of per-item cost)
    int best = 1;
    double best_cost = 1e300;
    const int max_split = p.n_jt < 16 ? p.n_jt : 16;
    for (int sp = 1; sp <= max_split; ++sp) {
        const int64_t items = (int64_t)p.n_it * sp;
        const int64_t waves = (items + G - 1) / G;
        const int64_t tiles = (p.n_jt + sp - 1) / sp;
        const double cost = (double)waves * (double)(tiles + 2);
        if (cost < best_cost - 1e-9) { best_cost = cost; best = sp; }
    }
    p.n_split = best;
    const int64_t items = (int64_t)p.n_it * p.n_split;
    p.grid = (int)(items < G ? items : G);
    p.nblk_f = (int)((N + 255) / 256);
    return p;
}

template <class C>
void vjp_tc_layout(C& c, const VjpPlan& p, int64_t N, int d, int R) {
    c.template take<__half>((size_t)p.N_pad * p.kh);     // UW
    c.template take<__half>((size_t)p.N_pad * p.kh);     // WU
    c.template take<unsigned>(64);                        // column maxima of U, W, Vb
    c.template take<unsigned>(64);
    c.template take<unsigned>(64);
    c.template take<float>(64);                           // a_c, g
    c.template take<float>((size_t)N * (d + 1));          // Vb
    c.template take<__half>((size_t)p.rv * p.Nc_pad);     // Xt
    c.template take<float>(64);                           // column scales of Xt
    c.template take<float>((size_t)p.n_split * p.rv * p.N_pad);   // O partials
    c.template take<double>((size_t)p.grid);              // per-CTA sum H k
    c.template take<double>((size_t)p.nblk_f * 32);       // per-block lengthscale sums
    c.template take<double>(64);                          // sums
    c.template take<double>((size_t)R);                   // column dots
}

}  // namespace

size_t vjp_tc_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t N, int R) {
    KOp op;
    const size_t kw = kop_workspace(ctx, hyp, N, N, 1, GP_PREC_FP16, true);
    if (kw == 0) return 0;
    // the plan only needs the padded sizes, which depend on N alone
    op.tp = tp_plan(ctx, N, N, 1, 16, 1);
    const VjpPlan p = vjp_plan(ctx, op, N, hyp->d, R);
    WsCounter c;
    vjp_tc_layout(c, p, N, hyp->d, R);
    return kw + c.off;
}

int vjp_tc_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U,
               const float* W, int R, double* grad_theta_host, float* gX_dev, cudaStream_t s) {
    const int d = hyp->d;
    KOp op;
    GPK_TRY(kop_prepare(ctx, wc, op, hyp, X, N, X, N, 1, GP_PREC_FP16, s));
    if (op.tp.engine != 1 || op.lay.k_pad > 64) return GP_ERR_UNSUPPORTED;
    const VjpPlan pl = vjp_plan(ctx, op, N, d, R);
    __half* UW = wc.take<__half>((size_t)pl.N_pad * pl.kh);
    __half* WU = wc.take<__half>((size_t)pl.N_pad * pl.kh);
    unsigned* cmu = wc.take<unsigned>(64);
    unsigned* cmw = wc.take<unsigned>(64);
    unsigned* cmv = wc.take<unsigned>(64);
    float* scales = wc.take<float>(64);
    float* Vb = wc.take<float>((size_t)N * (d + 1));
    __half* Xt = wc.take<__half>((size_t)pl.rv * pl.Nc_pad);
    float* xs = wc.take<float>(64);
    float* part = wc.take<float>((size_t)pl.n_split * pl.rv * pl.N_pad);
    double* hk = wc.take<double>((size_t)pl.grid);
    double* lpart = wc.take<double>((size_t)pl.nblk_f * 32);
    double* sums = wc.take<double>(64);
    double* dots = wc.take<double>((size_t)R);
    if (!wc.ok) return GP_ERR_WORKSPACE;

    // H operands: balanced, globally scaled FP16 copies of [u | w] and [w | u]
    GPK_TRY(launch_v_colmax(ctx, U, N, R, cmu, s));
    GPK_TRY(launch_v_colmax(ctx, W, N, R, cmw, s));
    uw_scales_kernel<<<1, 32, 0, s>>>(cmu, cmw, R, pl.rp, scales, ctx->dev_err);
    int64_t g1 = (pl.N_pad * pl.kh + 255) / 256;
    if (g1 > 8192) g1 = 8192;
    uw_prep_kernel<<<(unsigned)g1, 256, 0, s>>>(U, W, N, pl.N_pad, R, pl.rp, scales, UW, WU);
    // value-product operand: [x^ (centred, / l), 1] as hi + lo FP16 rows
    ScaleVec il;
    for (int k = 0; k < 64; ++k) il.v[k] = k < d ? (float)(1.0 / (double)hyp->lengthscale[k]) : 0.0f;
    int64_t g2 = (N * (d + 1) + 255) / 256;
    if (g2 > 8192) g2 = 8192;
    vb_prep_kernel<<<(unsigned)g2, 256, 0, s>>>(X, N, d, il, op.bbox, Vb);
    ctx->launches += 3;
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    GPK_TRY(launch_v_colmax(ctx, Vb, N, d + 1, cmv, s));
    GPK_TRY(launch_v_cast(ctx, GP_PREC_FP16, 0, 1, Vb, N, pl.Nc_pad, d + 1, pl.rx, cmv, 1.0, Xt, xs, s));

    CUtensorMap tmUW, tmWU, tmXt;
    const uint32_t hrow = (uint32_t)pl.kh * 2u;
    GPK_TRY(encode_tmap_2d(&tmUW, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, UW, pl.kh, pl.N_pad, hrow, pl.kh, 128,
                           swz_for(hrow)));
    GPK_TRY(encode_tmap_2d(&tmWU, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, WU, pl.kh, pl.N_pad, hrow, pl.kh, 128,
                           swz_for(hrow)));
    GPK_TRY(encode_tmap_2d(&tmXt, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, Xt, pl.Nc_pad, pl.rv, pl.Nc_pad * 2, 64,
                           (uint32_t)pl.rv, CU_TENSOR_MAP_SWIZZLE_128B));

    VjpParams prm;
    prm.n_it = pl.n_it;
    prm.n_jt = pl.n_jt;
    prm.n_split = pl.n_split;
    prm.n_items = pl.n_it * pl.n_split;
    prm.k_pad = op.lay.k_pad;
    prm.kh = pl.kh;
    prm.rv = pl.rv;
    const VjpSmem m = vjp_smem(prm.k_pad, prm.kh, prm.rv);
    if (m.stages < 2) return GP_ERR_UNSUPPORTED;
    prm.stages = m.stages;
    prm.N_pad = pl.N_pad;
    prm.part = part;
    prm.hk = hk;
    prm.err = ctx->dev_err;
    prm.limit_ns = kWaitLimitNs;
    cudaError_t e = cudaErrorInvalidValue;
#define GPK_VJP_CASE(K)                                                                                   \
    case K: {                                                                                             \
        auto fn = kvjp_tc_kernel<K>;                                                                      \
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m.total);          \
        if (e == cudaSuccess) {                                                                           \
            fn<<<pl.grid, kThreads, m.total, s>>>(op.tmA, op.tmB, tmUW, tmWU, tmXt, prm);                  \
            e = cudaGetLastError();                                                                       \
        }                                                                                                 \
        break;                                                                                            \
    }
    prof_begin(ctx, s);
    switch (hyp->kernel) {
        GPK_VJP_CASE(GP_KERNEL_RBF)
        GPK_VJP_CASE(GP_KERNEL_MATERN32)
        GPK_VJP_CASE(GP_KERNEL_MATERN52)
        default: return GP_ERR_UNSUPPORTED;
    }
#undef GPK_VJP_CASE
    prof_end(ctx, s);
    ctx->launches++;
    if (e != cudaSuccess) return GP_ERR_CUDA;

    ScaleVec tl;
    for (int k = 0; k < 64; ++k) tl.v[k] = k < d ? (float)(2.0 / (double)hyp->lengthscale[k]) : 0.0f;
    const float a2kp = (float)hyp->outputscale * kprime_max(hyp->kernel);
    vjp_finish_kernel<<<(unsigned)pl.nblk_f, 256, 0, s>>>(part, pl.n_split, pl.rv, pl.N_pad, xs, Vb, N, d, tl, a2kp,
                                                          scales, pl.rp, gX_dev, lpart);
    sum_rows_kernel<<<1, 32, 0, s>>>(lpart, pl.nblk_f, 32, d, sums);
    sum_rows_kernel<<<1, 32, 0, s>>>(hk, pl.grid, 1, 1, sums + 32);
    coldot2_kernel<<<R, 256, 0, s>>>(U, W, N, dots);
    ctx->launches += 4;
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    double hs[64];
    double hd[32];
    float hsc[64];
    if (cudaMemcpyAsync(hs, sums, sizeof(double) * 64, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hd, dots, sizeof(double) * R, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(hsc, scales, sizeof(float) * 64, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GP_ERR_CUDA;
    const double g = (double)hsc[pl.rp];
    // dq/dl_m = -(2 / l_m) sum_i x^_im D_im (F already applied); dq/da^2 = 1/2 sum H k / g^2
    for (int k = 0; k < d; ++k) grad_theta_host[k] = -2.0 / (double)hyp->lengthscale[k] * hs[k];
    grad_theta_host[d] = 0.5 * hs[32] / (g * g);
    double sg = 0.0;
    for (int c = 0; c < R; ++c) sg += hd[c];
    grad_theta_host[d + 1] = sg;
    return GP_OK;
}

}  // namespace gpk
