// The tensor-core kernel MVM with the transposed value product
// (Eq. mvm; Sec. 4.1).
//
//   out_i = a^2 sum_j k(x_i, x_j) v_j (+ sigma^2 v_i)
//
// Same dataflow as kmvm_tc.cu (S = XA_i XB_j^T on the tensor cores with the
// norm terms folded into the contraction, the kernel function on the special
// function units, an FP32 accumulation of P V in TMEM), but the value product
// is computed transposed, for two row tiles at once:
//
//   O^T (rows r, columns i) += Vt_j (r x 128) . P_j^T      M = 128, N = 256, K = 128
//
// A tcgen05.mma occupies the issue path for about the same time whatever its
// N, so the plain orientation (M = 128 rows i, N = R_pad <= 64) spends eight
// narrow instructions per 128 x 128 tile on P V.  Transposed, one instruction
// covers 256 rows i, and the right-hand sides' hi and lo parts (rows
// [0, R_pad) and [R_pad, 2 R_pad) of Vt) share M, so carrying V as hi + lo
// costs no extra instruction.  P is the B operand and therefore lives in
// shared memory: each epilogue thread writes its row of P as 16-byte chunks in
// the 128-byte-swizzled K-major layout the MMA reads (chunk c of row n at
// physical chunk c ^ (n mod 8)), then fences to the async proxy.  With
// PSPLIT the kernel tile is carried as hi + lo (Veltkamp split in FP32 on the
// FMA pipe: hi keeps the operand format's significand, lo = k - hi exactly
// before its own rounding), and each K-block is multiplied twice.
//
// Single-term P is double-buffered per tile (two 64 KB buffers) and its value
// product issued once the whole tile is stored, so the next tile's S product,
// issued as soon as the epilogue has read S, never queues behind it.  The
// hi + lo tile needs twice the bytes: it is staged per 64-column K-block (two
// 64 KB buffers) and each K-block's product is issued as soon as it is stored.
//
// Work item = (pair of 128-row tiles, column split).  Warps: 0-15 epilogue
// (warpgroup q handles row tile q & 1, columns [64 (q >> 1), 64 (q >> 1) + 64):
// four warps per scheduler hide the TMEM and shared-memory latencies behind the
// special-function work), 16 TMA producer, 17 S issuer and TMEM owner, 18
// value-product issuer (one issuing warp serialises too many high-latency
// tcgen05 and mbarrier operations per tile pair; see tp_mma_s).  TMEM: S of
// tile 0 [0,128), S of tile 1 [128,256), O^T [256,512) (with the FP32 value
// product, which has no O^T, a second S buffer there).  The epilogue signals
// each barrier once per warp (after __syncwarp), never once per thread.
// With HS (GP_MVM_HALF_EXP) the S product accumulates in FP16 and the
// epilogue evaluates 2^s in FP16 pairs.  Shared memory: the X_j / Vt_j stage ring first, then the two
// K-block P buffers (32 KB each, 64 KB with the hi + lo split), then the
// row-tile buffers.  The A operand of the value
// product spans 128 rows of which the first rv = R_pad (1 + vsplit) hold Vt;
// the rest reads the following shared memory (the next K-block, stage or P
// buffer: always inside the allocation) and lands in accumulator rows that
// are never read.
//
// O^T rows are written raw to the partial buffer [n_split][rv][ld_part]; the
// split reduction sums the column splits and the hi / lo rows, scales by
// a^2 / s_c and adds sigma^2 v.  Every mbarrier wait is bounded; a wait that
// runs out records DEV_TIMEOUT, drains what was issued, frees TMEM and exits.
#include "gpk_internal.cuh"
#include "ptx.cuh"
#include "kfun.cuh"

namespace gpk {

namespace {

constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kPairRows = 256;
constexpr int kMaxStages = 6;
constexpr int kEpiWarps = 16;
constexpr int kThreads = (kEpiWarps + 3) * 32;
constexpr int kTmaWarp = kEpiWarps;
constexpr int kMmaWarp = kEpiWarps + 1;   // S issuer, TMEM owner
constexpr int kPvWarp = kEpiWarps + 2;    // value-product issuer
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kTmemO = 256;
constexpr uint32_t kPKBlock = (uint32_t)kPairRows * 128u;   // one 64-column K-block of P: 256 rows x 128 B
constexpr int kMaxSmemBytes = 227 * 1024;   // opt-in maximum per CTA (512 B kept for static shared memory)
constexpr uint32_t kSpvVBytes = 128u * 4u * 4u;   // FP32 value product: 128 columns x 4 rows of FP32 v

struct TpParams {
    int n_ip, n_jt, n_split, n_items;
    int k_pad, rv;        // rv: rows of Vt per tile (R_pad, or 2 R_pad with the hi + lo split)
    int stages, xi_bufs;
    int psplit;           // 1: P carried as hi + lo
    int nrhs;             // right-hand sides in use (the FP32 value product: <= 4)
    int spv;              // 1: FP32 value product; the V map is FP32, 128 columns x 4 rows per box
    int diag;             // square Matern-1/2 operator: P_ii = 0 on chip (exact diagonal added later)
    int64_t ld_part;      // n_ip * 256
    float* partial;       // [n_split][rv][ld_part]
    const uint32_t* mask; // tile skipping: bit jt of word ip * mask_words + jt / 32 set = evaluate, or null
    int mask_words;
    int* err;
    uint64_t limit_ns;
};

struct TpBarriers {
    uint64_t full[kMaxStages];
    uint64_t empty[kMaxStages];
    uint64_t s_full[4];     // [S buffer * 2 + row tile]; a second S buffer only with the FP32 value product
    uint64_t s_empty[4];
    uint64_t p_full[2];     // per P buffer: tile slot (single P) or K-block (hi + lo P)
    uint64_t p_empty[2];
    uint64_t o_full;
    uint64_t o_empty;
    uint64_t xi_full[2];
    uint64_t xi_empty[2];
    uint64_t drain[2];      // per issuing warp
};

__device__ __forceinline__ void record_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ void item_range(const TpParams& p, int item, int& ip, int& sp, int& j0, int& j1) {
    ip = item % p.n_ip;
    sp = item / p.n_ip;
    j0 = (int)(((int64_t)sp * p.n_jt) / p.n_split);
    j1 = (int)(((int64_t)(sp + 1) * p.n_jt) / p.n_split);
}

// Whether the column tile jt of row-tile pair ip is evaluated (compact support:
// a cleared bit means every kernel value of the pair rounds to zero).
__device__ __forceinline__ bool tile_on(const TpParams& p, int ip, int jt) {
    return !p.mask || ((__ldg(p.mask + (int64_t)ip * p.mask_words + (jt >> 5)) >> (jt & 31)) & 1u);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

// ---- TMA producer (one thread) ------------------------------------------------
__device__ void tp_producer(const TpParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB,
                            const CUtensorMap* tmV, TpBarriers& bars, uint8_t* sSt, uint8_t* sXi, uint32_t xbytes,
                            uint32_t vtbytes) {
    uint32_t fills = 0, xi_loads = 0;
    bool ok = true;
    int ic = 0;
    const uint32_t S = (uint32_t)p.stages;
    const uint32_t kblk = (uint32_t)p.rv * 128u;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x, ++ic) {
        int ip, sp, j0, j1;
        item_range(p, item, ip, sp, j0, j1);
        const int xb = p.xi_bufs == 2 ? (ic & 1) : 0;
        const int use = p.xi_bufs == 2 ? (ic >> 1) : ic;   // earlier uses of this buffer
        if (use >= 1 && !ptx::mbar_wait(&bars.xi_empty[xb], (use - 1) & 1, p.limit_ns)) { ok = false; break; }
        uint8_t* sX = sXi + (uint32_t)xb * 2u * xbytes;
        ptx::mbar_arrive_expect_tx(&bars.xi_full[xb], 2u * xbytes);
        ptx::tma_load_2d(sX, tmA, &bars.xi_full[xb], 0, ip * kPairRows);
        ptx::tma_load_2d(sX + xbytes, tmA, &bars.xi_full[xb], 0, ip * kPairRows + kBM);
        ++xi_loads;
        for (int jt = j0; jt < j1; ++jt) {
            if (!tile_on(p, ip, jt)) continue;
            const uint32_t st = fills % S, u = fills / S;
            if (u > 0 && !ptx::mbar_wait(&bars.empty[st], (u - 1) & 1, p.limit_ns)) { ok = false; break; }
            uint8_t* sx = sSt + st * (xbytes + vtbytes);
            ptx::mbar_arrive_expect_tx(&bars.full[st], xbytes + (p.spv ? kSpvVBytes : vtbytes));
            ptx::tma_load_2d(sx, tmB, &bars.full[st], 0, jt * kBN);
            if (p.spv) {
                ptx::tma_load_2d(sx + xbytes, tmV, &bars.full[st], jt * kBN, 0);
            } else {
                ptx::tma_load_2d(sx + xbytes, tmV, &bars.full[st], jt * kBN, 0);
                ptx::tma_load_2d(sx + xbytes + kblk, tmV, &bars.full[st], jt * kBN + 64, 0);
            }
            ++fills;
        }
        if (!ok) break;
    }
    if (!ok) {
        record_error(p.err, DEV_TIMEOUT);
        // Let every copy this thread issued land before the CTA can exit.
        const uint32_t first = fills > S ? fills - S : 0;
        for (uint32_t f = first; f < fills; ++f) ptx::mbar_wait(&bars.full[f % S], (f / S) & 1, p.limit_ns);
        const uint32_t nb = (uint32_t)p.xi_bufs;
        for (uint32_t q = xi_loads > nb ? xi_loads - nb : 0; q < xi_loads; ++q)
            ptx::mbar_wait(&bars.xi_full[q % nb], (q / nb) & 1, p.limit_ns);
    }
}

// ---- MMA issuers (two converged warps) ---------------------------------------------
// Every tcgen05 operation, mbarrier probe and index step of an issuing warp has
// a latency of the order of a hundred cycles, so one warp issuing both
// products serialises about thirty of them per tile pair; split in two, the S
// issuer re-issues S as soon as the epilogue has read it while the other warp
// is still issuing the previous tile's value product.  Both warps run their
// loops converged (every decision is warp-uniform) and issue each tcgen05.mma
// and commit from one elected lane.  The tensor pipe executes what the two
// warps issue in arrival order; S and O^T live in disjoint TMEM columns.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    return __all_sync(0xffffffffu, ptx::mbar_wait(bar, parity, limit_ns));
}

// S issuer: for each column tile, S = XA_i XB_j^T for both row tiles once both
// S buffers have been read (s_empty) and the stage has landed (full).
__device__ void tp_mma_s(const TpParams& p, TpBarriers& bars, const uint8_t* sSt, const uint8_t* sXi,
                         uint32_t xbytes, uint32_t vtbytes, uint32_t tmem, uint32_t id_s) {
    const uint32_t arow = (uint32_t)p.k_pad * 2u;                            // 32, 64 or 128 bytes
    const uint32_t swz = (arow == 32) ? 6u : (arow == 64 ? 4u : 2u);
    const int ksteps = p.k_pad / 16;
    const uint32_t S = (uint32_t)p.stages;
    const uint32_t aSt = ptx::smem_u32(sSt);
    const uint32_t stage_bytes = xbytes + vtbytes;
    const uint32_t hi_x = ptx::smem_desc_hi(8u * arow, swz);
    uint32_t g = 0, st = 0, ph = 0;   // tiles issued; stage ring slot and its fill parity
    int ic = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x, ++ic) {
        int ip, sp, j0, j1;
        item_range(p, item, ip, sp, j0, j1);
        const int xb = p.xi_bufs == 2 ? (ic & 1) : 0;
        const int use = p.xi_bufs == 2 ? (ic >> 1) : ic;
        if (!warp_wait(&bars.xi_full[xb], use & 1, p.limit_ns)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t aXi = ptx::smem_u32(sXi) + (uint32_t)xb * 2u * xbytes;
        for (int jt = j0; jt < j1; ++jt) {
            if (!tile_on(p, ip, jt)) continue;
            // S buffer of this tile (two with the FP32 value product, whose O^T columns are free)
            const uint32_t nb = p.spv ? 2u : 1u, buf = g % nb, use = g / nb;
            if (use > 0 && !(warp_wait(&bars.s_empty[2 * buf], (use - 1) & 1, p.limit_ns) &&
                             warp_wait(&bars.s_empty[2 * buf + 1], (use - 1) & 1, p.limit_ns))) { ok = false; break; }
            if (!warp_wait(&bars.full[st], ph, p.limit_ns)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t aXj = aSt + st * stage_bytes;
            for (int w = 0; w < 2; ++w) {
                for (int kk = 0; kk < ksteps; ++kk) {
                    const uint32_t koff = (uint32_t)kk * 32u;
                    ptx::mma_f16_ss_elect(tmem + buf * 256u + (uint32_t)w * 128u,
                                          ptx::smem_desc_at(hi_x, aXi + (uint32_t)w * xbytes + koff),
                                          ptx::smem_desc_at(hi_x, aXj + koff), id_s, kk > 0 ? 1u : 0u);
                }
                ptx::mma_commit_elect(&bars.s_full[2 * buf + w]);
            }
            if (++st == S) { st = 0; ph ^= 1u; }
            ++g;
        }
        if (!ok) break;
        ptx::mma_commit_elect(&bars.xi_empty[xb]);   // the row tiles' last use in this item
    }
    ptx::mma_commit_elect(&bars.drain[0]);
    warp_wait(&bars.drain[0], 0, p.limit_ns);
    if (!ok && (threadIdx.x & 31) == 0) record_error(p.err, DEV_TIMEOUT);
}

// Value-product issuer: O^T += Vt_j P_j^T for each tile (single P: the whole
// tile once both K-blocks are stored; hi + lo P: per K-block), then releases
// the P buffer and the stage; O^T is handed to the epilogue after an item.
template <int PSPLIT>
__device__ void tp_mma_pv(const TpParams& p, TpBarriers& bars, const uint8_t* sSt, const uint8_t* sP,
                          uint32_t xbytes, uint32_t vtbytes, uint32_t tmem, uint32_t id_pv) {
    const uint32_t S = (uint32_t)p.stages;
    const uint32_t aSt = ptx::smem_u32(sSt);
    const uint32_t aP = ptx::smem_u32(sP);
    const uint32_t stage_bytes = xbytes + vtbytes;
    const uint32_t kblk = (uint32_t)p.rv * 128u;
    const uint32_t hi_128 = ptx::smem_desc_hi(1024u, 2u);
    uint32_t g = 0, st = 0, ph = 0;
    int ic = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x, ++ic) {
        int ip, sp, j0, j1;
        item_range(p, item, ip, sp, j0, j1);
        if (ic > 0 && !warp_wait(&bars.o_empty, (ic - 1) & 1, p.limit_ns)) { ok = false; break; }
        uint32_t t = 0;   // evaluated tiles of this item
        for (int jt = j0; jt < j1 && ok; ++jt) {
            if (!tile_on(p, ip, jt)) continue;
            // Vt_j of this stage: landed before S of this tile was issued (already complete)
            if (!warp_wait(&bars.full[st], ph, p.limit_ns)) { ok = false; break; }
            for (uint32_t kb = 0; kb < (PSPLIT ? 2u : 1u); ++kb) {
                const uint32_t buf = PSPLIT ? kb : (g & 1u);
                const uint32_t par = PSPLIT ? (g & 1u) : ((g >> 1) & 1u);
                if (!warp_wait(&bars.p_full[buf], par, p.limit_ns)) { ok = false; break; }
                ptx::tc_fence_after();
                const uint32_t aV = aSt + st * stage_bytes + xbytes + kb * kblk;
                const uint32_t aPb = aP + buf * 2u * kPKBlock;
                // single P: K-blocks 0, 1 of the tile (8 steps); hi + lo: hi then lo of K-block kb
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const uint32_t kk = (uint32_t)(q & 3) * 32u, hq = (uint32_t)(q >> 2);
                    const uint32_t aVq = PSPLIT ? aV + kk : aV + hq * kblk + kk;
                    const uint32_t aPq = aPb + hq * kPKBlock + kk;
                    ptx::mma_f16_ss_elect(tmem + kTmemO, ptx::smem_desc_at(hi_128, aVq),
                                          ptx::smem_desc_at(hi_128, aPq), id_pv,
                                          (t > 0 || kb > 0 || q > 0) ? 1u : 0u);
                }
                ptx::mma_commit_elect(&bars.p_empty[buf]);      // this P buffer may be rewritten
            }
            if (!ok) break;
            ptx::mma_commit_elect(&bars.empty[st]);             // X_j and Vt_j of this stage are consumed
            if (++st == S) { st = 0; ph ^= 1u; }
            ++t;
            ++g;
        }
        if (!ok) break;
        ptx::mma_commit_elect(&bars.o_full);
    }
    ptx::mma_commit_elect(&bars.drain[1]);
    warp_wait(&bars.drain[1], 0, p.limit_ns);
    if (!ok && (threadIdx.x & 31) == 0) record_error(p.err, DEV_TIMEOUT);
}

template <int BF16>
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if constexpr (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}

// 32 columns [32 h, 32 h + 32) of this thread's P row: kernel values, packed
// in pairs (and, with PSPLIT, split hi + lo first), stored as four 16-byte
// chunks of the swizzled K-major layout of K-block buffer pkb.
template <int KIND, int BF16, int PSPLIT>
__device__ __forceinline__ void tp_chunk(const uint32_t (&r)[32], int h, int row, bool dtile, uint32_t pkb,
                                         uint32_t nsw) {
    // Veltkamp factor 2^(24 - t) + 1 leaves t significant bits in hi: 11 (FP16) or 8 (BF16)
    constexpr float kSplit = BF16 ? 65537.0f : 8193.0f;
    uint32_t pk[16];
    uint32_t pl[PSPLIT ? 16 : 1];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        float k0 = kernel_from_s<KIND>(__uint_as_float(r[2 * e]));
        float k1 = kernel_from_s<KIND>(__uint_as_float(r[2 * e + 1]));
        if constexpr (KIND == GP_KERNEL_MATERN12) {
            if (dtile) {
                const int col = h * 32 + 2 * e;
                if (col == row) k0 = 0.0f;
                if (col + 1 == row) k1 = 0.0f;
            }
        }
        if constexpr (PSPLIT) {
            // explicit round-to-nearest operations: no contraction into FMAs
            const float c0 = __fmul_rn(k0, kSplit), c1 = __fmul_rn(k1, kSplit);
            const float h0 = __fsub_rn(c0, __fsub_rn(c0, k0)), h1 = __fsub_rn(c1, __fsub_rn(c1, k1));
            pk[e] = pack2<BF16>(h0, h1);
            pl[e] = pack2<BF16>(__fsub_rn(k0, h0), __fsub_rn(k1, h1));
        } else {
            pk[e] = pack2<BF16>(k0, k1);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t c = (uint32_t)((h & 1) * 4 + q);
        const uint32_t off = (c ^ nsw) << 4;
        st_shared_v4(pkb + off, pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
        if constexpr (PSPLIT) st_shared_v4(pkb + kPKBlock + off, pl[4 * q], pl[4 * q + 1], pl[4 * q + 2], pl[4 * q + 3]);
    }
}

// Half-precision kernel evaluation (RBF, FP16): the S tile comes from the
// MMA as FP16 (one rounding of the exp2 argument), is loaded packed in pairs,
// and 2^s is evaluated for both halves of a register by one ex2.approx.f16x2,
// whose output is already the packed FP16 P the value product reads: no
// FP32 -> FP16 conversion, one SFU instruction per two kernel values.
// 32 columns [32 h, 32 h + 32) of this thread's P row from 16 packed S
// registers, stored as four 16-byte chunks.
__device__ __forceinline__ void tp_chunk_h(const uint32_t* r, int h, uint32_t pkb, uint32_t nsw) {
    uint32_t pk[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) pk[e] = ptx::ex2_h2(r[e]);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t c = (uint32_t)((h & 1) * 4 + q);
        st_shared_v4(pkb + ((c ^ nsw) << 4), pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
}

template <int KIND, int BF16, int PSPLIT, int HS>
__device__ void tp_epilogue(const TpParams& p, TpBarriers& bars, const uint8_t* sP, uint32_t tmem, int wg, int wq,
                            int lane) {
    const int tl = wg & 1, ch = wg >> 1;              // row tile of the pair, column half (= K-block)
    const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
    const int row = wq * 32 + lane;                   // row within the tile
    const uint32_t nrow = (uint32_t)(tl * kBM + row); // row of the P operand (0..255)
    const uint32_t nsw = nrow & 7u;
    // P buffers are 64 KB: single P: [tile slot][K-block]; hi + lo: [K-block][hi, lo]
    const uint32_t aProw = ptx::smem_u32(sP) + nrow * 128u;
    uint32_t gt = 0;
    int ic = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x, ++ic) {
        int ip, sp, j0, j1;
        item_range(p, item, ip, sp, j0, j1);
        const int it = 2 * ip + tl;   // this warpgroup's row tile
        uint32_t t = 0;               // evaluated tiles of this item
        for (int jt = j0; jt < j1; ++jt) {
            if (!tile_on(p, ip, jt)) continue;
            const uint32_t g = gt + t;
            if (!__all_sync(0xffffffffu, ptx::mbar_wait(&bars.s_full[tl], g & 1, p.limit_ns))) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t tS = tmem + lane_off + (uint32_t)tl * 128u + (uint32_t)ch * 64u;
            const bool dtile = (KIND == GP_KERNEL_MATERN12) && p.diag && (jt == it);
            uint32_t ra[32], rb[HS ? 1 : 32];
            if constexpr (HS) {
                ptx::tmem_ld32_pack16(tS, ra);     // 64 FP16 columns in 32 registers
                ptx::tmem_wait_ld();
                ptx::tmem_reg_fence(ra);
            } else {
                ptx::tmem_ld32(tS, ra);
                ptx::tmem_ld32(tS + 32u, rb);
                ptx::tmem_wait_ld();
                ptx::tmem_reg_fence(ra);
                ptx::tmem_reg_fence(rb);
            }
            ptx::tc_fence_before();
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bars.s_empty[tl]);   // this warp's part of S is in registers
            uint32_t buf;
            if constexpr (PSPLIT) {
                // K-block buffer ch is free once the previous tile's product of it is done
                buf = (uint32_t)ch;
                if (g >= 1 && !__all_sync(0xffffffffu, ptx::mbar_wait(&bars.p_empty[buf], (g - 1) & 1, p.limit_ns))) {
                    ok = false;
                    break;
                }
            } else {
                // tile slot g & 1 is free once the product of tile g - 2 is done
                buf = g & 1u;
                if (g >= 2 &&
                    !__all_sync(0xffffffffu, ptx::mbar_wait(&bars.p_empty[buf], ((g >> 1) - 1) & 1, p.limit_ns))) {
                    ok = false;
                    break;
                }
            }
            const uint32_t pkb = aProw + buf * 2u * kPKBlock + (PSPLIT ? 0u : (uint32_t)ch * kPKBlock);
            if constexpr (HS) {
                tp_chunk_h(ra, 2 * ch, pkb, nsw);
                tp_chunk_h(ra + 16, 2 * ch + 1, pkb, nsw);
            } else {
                tp_chunk<KIND, BF16, PSPLIT>(ra, 2 * ch, row, dtile, pkb, nsw);
                tp_chunk<KIND, BF16, PSPLIT>(rb, 2 * ch + 1, row, dtile, pkb, nsw);
            }
            ptx::fence_proxy_async_smem();        // P stores -> visible to the tensor core
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bars.p_full[buf]);
            ++t;
        }
        if (!ok) break;
        // O^T read-out: lanes [0, rv) are the rows of Vt; this warpgroup's 64 columns.
        if (!__all_sync(0xffffffffu, ptx::mbar_wait(&bars.o_full, ic & 1, p.limit_ns))) { ok = false; break; }
        ptx::tc_fence_after();
        if (wq * 32 < p.rv) {   // warp-uniform
            const int r = wq * 32 + lane;
            float* dst = p.partial + ((int64_t)sp * p.rv + r) * p.ld_part + (int64_t)ip * kPairRows + tl * kBM + ch * 64;
            for (int h = 0; h < 2; ++h) {
                uint32_t o[32];
                if (t > 0) {
                    ptx::tmem_ld32(tmem + lane_off + kTmemO + (uint32_t)(tl * kBM + ch * 64 + h * 32), o);
                    ptx::tmem_wait_ld();
                    ptx::tmem_reg_fence(o);
                } else {
#pragma unroll
                    for (int q = 0; q < 32; ++q) o[q] = 0u;   // every tile of the item was skipped
                }
                float4* d4 = reinterpret_cast<float4*>(dst + h * 32);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    d4[q] = make_float4(__uint_as_float(o[4 * q]), __uint_as_float(o[4 * q + 1]),
                                        __uint_as_float(o[4 * q + 2]), __uint_as_float(o[4 * q + 3]));
            }
        }
        ptx::tc_fence_before();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&bars.o_empty);
        gt += t;
    }
    if (!ok) record_error(p.err, DEV_TIMEOUT);
}

// The FP32 value product (GP_MVM_FP32_PV, 1 to 4 right-hand sides): the
// epilogue keeps its kernel values in FP32 and forms sum_j k_ij v_j itself
// with FP32 FMAs, v_j read in FP32 from the stage (TMA box of 128 columns x 4
// rows; this warpgroup's 64 columns; broadcast 16-byte reads).  No P in shared
// memory and no value-product MMAs: a tensor-core product with 1 to 4 useful
// rows of its M = 128 would cost as much as one with 64.  Each warp releases
// the stage after its reads (16 arrivals), and writes its row sums of the item
// to the partial rows ch * R_pad + r, which the split reduction adds up.
template <int KIND, int RN>
__device__ void tp_epilogue_spv(const TpParams& p, TpBarriers& bars, const uint8_t* sSt, uint32_t xbytes,
                                uint32_t vtbytes, uint32_t tmem, int wg, int wq, int lane) {
    const int tl = wg & 1, ch = wg >> 1;
    const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
    const int row = wq * 32 + lane;
    const uint32_t S = (uint32_t)p.stages;
    const uint32_t stage_bytes = xbytes + vtbytes;
    const int Rp = p.rv >> 1;
    constexpr int R = RN;   // columns 1, 2 or 4 (3 runs as 4: the fourth row of v is zero)
    uint32_t gt = 0, st = 0, ph = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x) {
        int ip, sp, j0, j1;
        item_range(p, item, ip, sp, j0, j1);
        const int it = 2 * ip + tl;
        float acc[RN];
#pragma unroll
        for (int r = 0; r < RN; ++r) acc[r] = 0.0f;
        uint32_t t = 0;
        for (int jt = j0; jt < j1; ++jt) {
            if (!tile_on(p, ip, jt)) continue;
            const uint32_t g = gt + t, buf = g & 1u;
            // hinted waits: a spinning warp would take the issue slots of the warps computing
            // beside it and of the S issuer on its scheduler (this epilogue is issue-bound)
            if (!__all_sync(0xffffffffu,
                            ptx::mbar_wait_sleep(&bars.s_full[2 * buf + tl], (g >> 1) & 1, p.limit_ns) &&
                                ptx::mbar_wait_sleep(&bars.full[st], ph, p.limit_ns))) {
                ok = false;
                break;
            }
            ptx::tc_fence_after();
            const uint32_t tS = tmem + lane_off + buf * 256u + (uint32_t)tl * 128u + (uint32_t)ch * 64u;
            const bool dtile = (KIND == GP_KERNEL_MATERN12) && p.diag && (jt == it);
            const float* vb = reinterpret_cast<const float*>(sSt + st * stage_bytes + xbytes) + ch * 64;
            // one 32-column half of S at a time (the register budget of 608 threads); the
            // buffer is released after the second load, while S of the next tile is
            // already being formed in the other one
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t rr[32];
                ptx::tmem_ld32(tS + 32u * (uint32_t)hh, rr);
                ptx::tmem_wait_ld();
                ptx::tmem_reg_fence(rr);
                if (hh == 1) {
                    ptx::tc_fence_before();
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&bars.s_empty[2 * buf + tl]);
                }
#pragma unroll
                for (int c4 = 0; c4 < 4; ++c4) {      // 16-byte chunk c: columns [8 c, 8 c + 8) of the 64
                    const int c = 4 * hh + c4;
                    float kv[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int q = 8 * c + e;
                        float k = kernel_from_s<KIND>(__uint_as_float(rr[8 * c4 + e]));
                        if constexpr (KIND == GP_KERNEL_MATERN12) {
                            if (dtile && ch * 64 + q == row) k = 0.0f;
                        }
                        kv[e] = k;
                    }
#pragma unroll
                    for (int r = 0; r < RN; ++r) {
                        {
                            const float4 va = *reinterpret_cast<const float4*>(vb + r * 128 + 8 * c);
                            const float4 vc = *reinterpret_cast<const float4*>(vb + r * 128 + 8 * c + 4);
                            acc[r] = fmaf(kv[0], va.x, acc[r]);
                            acc[r] = fmaf(kv[1], va.y, acc[r]);
                            acc[r] = fmaf(kv[2], va.z, acc[r]);
                            acc[r] = fmaf(kv[3], va.w, acc[r]);
                            acc[r] = fmaf(kv[4], vc.x, acc[r]);
                            acc[r] = fmaf(kv[5], vc.y, acc[r]);
                            acc[r] = fmaf(kv[6], vc.z, acc[r]);
                            acc[r] = fmaf(kv[7], vc.w, acc[r]);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&bars.empty[st]);   // this warp is done with the stage's Vt
            if (++st == S) { st = 0; ph ^= 1u; }
            ++t;
        }
        if (!ok) break;
#pragma unroll
        for (int r = 0; r < RN; ++r)
            p.partial[((int64_t)sp * p.rv + ch * Rp + r) * p.ld_part + (int64_t)ip * kPairRows + tl * kBM + row] =
                acc[r];
        gt += t;
    }
    if (!ok) record_error(p.err, DEV_TIMEOUT);
}

struct TpSmem {
    uint32_t xbytes, vtbytes, stage_bytes, pbuf;
    int stages, xi_bufs;
    uint32_t total;   // dynamic shared memory to request (includes 1 KB alignment slack)
};

__host__ __device__ inline TpSmem tp_smem(int k_pad, int rv, int psplit) {
    TpSmem m;
    m.xbytes = (uint32_t)kBM * (uint32_t)k_pad * 2u;
    m.vtbytes = 2u * (uint32_t)rv * 128u;
    m.stage_bytes = m.xbytes + m.vtbytes;
    m.pbuf = (uint32_t)(1 + psplit) * kPKBlock;
    const uint32_t fixed = 1024u + 4u * kPKBlock;   // two 64 KB P buffers
    m.stages = 0;
    m.xi_bufs = 2;
    for (int xb = 2; xb >= 1 && m.stages < 3; --xb) {
        const uint32_t xi = (uint32_t)xb * 2u * m.xbytes;
        int st = 0;
        for (int s = kMaxStages; s >= 2; --s)
            if (fixed + xi + (uint32_t)s * m.stage_bytes <= (uint32_t)kMaxSmemBytes - 512u) { st = s; break; }
        if (st > m.stages) { m.stages = st; m.xi_bufs = xb; }
    }
    m.total = fixed + (uint32_t)m.xi_bufs * 2u * m.xbytes + (uint32_t)m.stages * m.stage_bytes;
    return m;
}

template <int KIND, int BF16, int PSPLIT, int HS, int SPV>
__global__ void __launch_bounds__(kThreads, 1)
kmvm_tp_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmV, const TpParams p) {
    extern __shared__ uint8_t dsm[];
    __shared__ TpBarriers bars;
    __shared__ uint32_t tmem_slot;

    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
    const TpSmem m = tp_smem(p.k_pad, p.rv, PSPLIT);
    uint8_t* sSt = base;
    uint8_t* sP = base + (uint32_t)p.stages * m.stage_bytes;
    uint8_t* sXi = sP + 4u * kPKBlock;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            ptx::mbar_init(&bars.full[s], 1);
            ptx::mbar_init(&bars.empty[s], SPV ? kEpiWarps : 1);   // FP32 product: each epilogue warp
        }
        for (int b = 0; b < 4; ++b) {
            ptx::mbar_init(&bars.s_full[b], 1);
            ptx::mbar_init(&bars.s_empty[b], 8);                // the 8 warps of a row tile (one arrival each)
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&bars.xi_full[b], 1);
            ptx::mbar_init(&bars.xi_empty[b], 1);
            ptx::mbar_init(&bars.p_full[b], PSPLIT ? 8 : 16);   // K-block: 2 warpgroups; tile: all 4 (per warp)
            ptx::mbar_init(&bars.p_empty[b], 1);
        }
        ptx::mbar_init(&bars.o_full, 1);
        ptx::mbar_init(&bars.o_empty, kEpiWarps);
        ptx::mbar_init(&bars.drain[0], 1);
        ptx::mbar_init(&bars.drain[1], 1);
        ptx::fence_mbar_init();
    }
    if (warp == kTmaWarp && lane == 0) {
        ptx::tma_prefetch_desc(&tmA);
        ptx::tma_prefetch_desc(&tmB);
        ptx::tma_prefetch_desc(&tmV);
    }
    if (warp == kMmaWarp) ptx::tmem_alloc(&tmem_slot, kTmemCols);
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == kTmaWarp) {
        if (lane == 0) tp_producer(p, &tmA, &tmB, &tmV, bars, sSt, sXi, m.xbytes, m.vtbytes);
        __syncwarp();
    } else if (warp == kMmaWarp) {
        tp_mma_s(p, bars, sSt, sXi, m.xbytes, m.vtbytes, tmem,
                 HS ? ptx::idesc_f16_dh(kBM, kBN) : ptx::idesc_f16(kBM, kBN, BF16));
    } else if (warp == kPvWarp) {
        if constexpr (!SPV)
            tp_mma_pv<PSPLIT>(p, bars, sSt, sP, m.xbytes, m.vtbytes, tmem, ptx::idesc_f16(kBM, kPairRows, BF16));
    } else {
        if constexpr (SPV > 0)
            tp_epilogue_spv<KIND, SPV>(p, bars, sSt, m.xbytes, m.vtbytes, tmem, warp >> 2, warp & 3, lane);
        else
            tp_epilogue<KIND, BF16, PSPLIT, HS>(p, bars, sP, tmem, warp >> 2, warp & 3, lane);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == kMmaWarp) ptx::tmem_dealloc(tmem, kTmemCols);
}

template <int KIND, int BF16, int PSPLIT, int HS = 0, int SPV = 0>
cudaError_t launch_tp_typed(const TcPlan& plan, const TpParams& prm, const CUtensorMap& a, const CUtensorMap& b,
                            const CUtensorMap& v, cudaStream_t s) {
    const TpSmem m = tp_smem(prm.k_pad, prm.rv, PSPLIT);
    auto kfn = kmvm_tp_kernel<KIND, BF16, PSPLIT, HS, SPV>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)m.total);
    if (e != cudaSuccess) return e;
    kfn<<<plan.grid, kThreads, m.total, s>>>(a, b, v, prm);
    return cudaGetLastError();
}

}  // namespace

bool tp_supported(int k_pad, int R_pad, int vsplit, int psplit) {
    const int rv = R_pad * (1 + vsplit);
    return k_pad <= 64 && rv <= 128 && rv % 32 == 0 && tp_smem(k_pad, rv, psplit).stages >= 2;
}

TcPlan tp_plan(const Ctx* ctx, int64_t Nr, int64_t Nc, int R, int k_pad, int vsplit) {
    TcPlan p;
    p.engine = 1;
    p.k_pad = k_pad;
    p.R_pad = ((R + 15) / 16) * 16;
    p.rv = p.R_pad * (1 + vsplit);
    const int n_it = (int)((Nr + kBM - 1) / kBM);
    p.n_it = (n_it + 1) / 2;                  // pairs of row tiles
    p.n_jt = (int)((Nc + kBN - 1) / kBN);
    p.Nr_pad = (int64_t)p.n_it * kPairRows;
    p.Nc_pad = (int64_t)p.n_jt * kBN;
    const int G = ctx->num_sms > 0 ? ctx->num_sms : 1;
    // Column split minimising the busiest CTA's work (waves x tiles per item
    // plus about two tiles of per-item cost) plus the reduction, which always
    // runs here (it also sums the hi and lo rows).
    int best = 1;
    double best_cost = 1e300;
    const int max_split = p.n_jt < 16 ? p.n_jt : 16;
    for (int sp = 1; sp <= max_split; ++sp) {
        const int64_t items = (int64_t)p.n_it * sp;
        const int64_t waves = (items + G - 1) / G;
        const int64_t tiles = (p.n_jt + sp - 1) / sp;
        double cost = (double)waves * (double)(tiles + 2);
        cost += 0.05 * (double)sp * (double)p.n_it * 2.0 * (double)p.rv / (double)G / 64.0;
        if (cost < best_cost - 1e-9) { best_cost = cost; best = sp; }
    }
    p.n_split = best;
    const int64_t items = (int64_t)p.n_it * p.n_split;
    p.grid = (int)(items < G ? items : G);
    return p;
}

size_t tp_partial_floats(const TcPlan& p) { return (size_t)p.n_split * p.rv * p.Nr_pad; }

int launch_kmvm_tp(Ctx* ctx, const TcPlan& plan, const OperandLayout& L, const MvmArgs& a, const CUtensorMap& tmA,
                   const CUtensorMap& tmB, const CUtensorMap& tmV, const float* outscale, float* partial,
                   const uint32_t* mask, cudaStream_t s) {
    TpParams prm;
    prm.n_ip = plan.n_it;
    prm.n_jt = plan.n_jt;
    prm.n_split = plan.n_split;
    prm.n_items = plan.n_it * plan.n_split;
    prm.k_pad = plan.k_pad;
    prm.rv = plan.rv;
    prm.psplit = L.psplit;
    prm.nrhs = a.R;
    prm.spv = L.fp32_pv ? 1 : 0;
    const TpSmem m = tp_smem(plan.k_pad, plan.rv, L.psplit);
    prm.stages = m.stages;
    prm.xi_bufs = m.xi_bufs;
    if (!tp_supported(plan.k_pad, plan.R_pad, plan.rv / plan.R_pad - 1, L.psplit)) return GP_ERR_UNSUPPORTED;
    prm.diag = a.diag_coef != 0.0f ? 1 : 0;
    prm.ld_part = plan.Nr_pad;
    prm.partial = partial;
    prm.mask = mask;
    prm.mask_words = (plan.n_jt + 31) / 32;
    prm.err = ctx->dev_err;
    prm.limit_ns = kWaitLimitNs;
    const int bf = (L.prec == GP_PREC_BF16) ? 1 : 0;
    cudaError_t e = cudaErrorInvalidValue;
    const bool hs = L.half_exp != 0;
    if (hs && !(a.kernel == GP_KERNEL_RBF && !bf && !L.psplit && plan.k_pad == 16)) return GP_ERR_UNSUPPORTED;
    prof_begin(ctx, s);
#define GPK_TP_CASE(K)                                                                              \
    case K:                                                                                         \
        if (bf)                                                                                     \
            e = L.psplit ? launch_tp_typed<K, 1, 1>(plan, prm, tmA, tmB, tmV, s)                     \
                         : launch_tp_typed<K, 1, 0>(plan, prm, tmA, tmB, tmV, s);                    \
        else                                                                                        \
            e = L.psplit ? launch_tp_typed<K, 0, 1>(plan, prm, tmA, tmB, tmV, s)                     \
                         : launch_tp_typed<K, 0, 0>(plan, prm, tmA, tmB, tmV, s);                    \
        break;
    const bool spv = L.fp32_pv != 0;
    if (spv && (bf || L.psplit || hs || a.R > 4 || plan.rv != 2 * plan.R_pad)) return GP_ERR_UNSUPPORTED;
    if (hs) {
        e = launch_tp_typed<GP_KERNEL_RBF, 0, 0, 1>(plan, prm, tmA, tmB, tmV, s);
    } else if (spv) {
        // accumulators for 1, 2 or 4 columns (3 runs as 4 on a zero fourth row of v)
#define GPK_TP_SPV(K)                                                                            \
    case K:                                                                                      \
        e = a.R == 1 ? launch_tp_typed<K, 0, 0, 0, 1>(plan, prm, tmA, tmB, tmV, s)               \
          : a.R == 2 ? launch_tp_typed<K, 0, 0, 0, 2>(plan, prm, tmA, tmB, tmV, s)               \
                     : launch_tp_typed<K, 0, 0, 0, 4>(plan, prm, tmA, tmB, tmV, s);              \
        break;
        switch (a.kernel) {
            GPK_TP_SPV(GP_KERNEL_RBF)
            GPK_TP_SPV(GP_KERNEL_MATERN32)
            GPK_TP_SPV(GP_KERNEL_MATERN12)
            GPK_TP_SPV(GP_KERNEL_MATERN52)
            default: return GP_ERR_INVALID;
        }
#undef GPK_TP_SPV
    } else switch (a.kernel) {
        GPK_TP_CASE(GP_KERNEL_RBF)
        GPK_TP_CASE(GP_KERNEL_MATERN32)
        GPK_TP_CASE(GP_KERNEL_MATERN12)
        GPK_TP_CASE(GP_KERNEL_MATERN52)
        default: return GP_ERR_INVALID;
    }
#undef GPK_TP_CASE
    prof_end(ctx, s);
    ctx->launches++;
    if (e != cudaSuccess) return GP_ERR_CUDA;
    // splits x {hi, lo} rows: partial[s][part * R_pad + c] = partial'[s * parts + part][c]
    const int parts = plan.rv / plan.R_pad;
    return launch_split_reduce(ctx, partial, plan.n_split * parts, plan.Nr_pad, a.Nr, a.R, plan.R_pad, outscale,
                               0.0f, a.noise + a.diag_coef, a.Vnoise, a.Nc, a.out, a.ld_out, s);
}

}  // namespace gpk
