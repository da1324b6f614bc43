// The tensor-core kernel MVM (Eq. mvm; Sec. 4.1), one-row-tile engine.
//
//   out_i = a^2 sum_j k(x_i, x_j) v_j (+ sigma^2 v_i)
//
// One CTA owns a 128-row tile of the output and streams 128-column tiles of
// the kernel matrix, which never leaves the chip ("matrix-free"):
//   1. TMA brings the column tile's operand rows XB_j (128 x K) and the cast
//      right-hand sides Vt_j (R_pad x 128) into a 4-stage shared-memory ring.
//   2. One thread issues S = XA_i XB_j^T (tcgen05.mma kind::f16, M=N=128,
//      K = 16/32/64) into a TMEM buffer; with the norm terms folded into the
//      contraction dimension S is already s_ij = -c^2 r_ij^2 / 2.
//   3. An epilogue warpgroup loads its whole S tile from TMEM (one row per
//      thread, 4 loads in flight), releases the S buffer at once so the next
//      S product can start, evaluates the kernel function on the special
//      function units, rounds to FP16/BF16 and stores P into its own TMEM
//      buffer.
//   4. The MMA thread issues O += P Vt_j^T with P taken from TMEM
//      (M = 128, N = R_pad, K = 128), accumulating in FP32 in TMEM.  This is
//      the paper's block summation in higher precision, with 128 x 128 blocks.
// Tiles alternate between two epilogue warpgroups and two P buffers; the S
// product of tile t+2 runs while the epilogue of tile t is still computing,
// so the special function units (the roofline of this kernel) see no bubble
// from the tensor-core round trip.  After the last column tile, warpgroup 0
// reads O and writes a^2 O / s_c (+ sigma^2 v) -- or the raw partial when the
// column range is split across CTAs -- straight to global memory.
//
// TMEM columns: S buffers [0, 128 nsb), P buffers of 64 (hi) or 128 (hi, lo)
// columns after them, then O (R_pad <= 64).  FP16: 2 S + 2 x 64 P + O = 448;
// BF16 hi+lo: 1 S + 2 x 128 P + O = 448 (one S buffer, released early).
//
// Warp roles (320 threads): warps 0-3 epilogue WG0, 4-7 epilogue WG1,
// warp 8 TMA producer, warp 9 MMA issuer + TMEM owner.  Persistent CTAs walk
// the (row tile, column split) work items round-robin.  Every mbarrier wait is
// bounded; a wait that runs out records DEV_TIMEOUT in the device error word,
// drains the asynchronous copies / MMAs it issued, frees TMEM and exits.
#include "gpk_internal.cuh"
#include "ptx.cuh"
#include "kfun.cuh"

namespace gpk {

namespace {

constexpr int kBM = 128;
constexpr int kBN = 128;
constexpr int kStages = 8;
constexpr int kThreads = 320;
constexpr int kTmaWarp = 8;
constexpr int kMmaWarp = 9;
constexpr uint32_t kTmemCols = 512;

constexpr int kMinSmemBytes = 120 * 1024; // keeps one CTA per SM (TMEM is taken whole)
constexpr int kMaxSmemBytes = 227 * 1024; // opt-in maximum per CTA

struct TcParams {
    int n_it, n_jt, n_split, n_items;
    int k_pad, R_pad, R;
    int vsplit;                  // 1: Vt carries hi rows then lo rows
    int psplit;                  // 1: the kernel tile is carried as hi + lo (two P column blocks)
    int stages;                  // shared-memory ring depth (<= kStages)
    int diag;                    // square operator: P_ii is set to 0 on chip and the exact
                                 // a^2 v_i is added with the noise term (k(x, x) = 1)
    int64_t Nr;
    float noise;                 // sigma^2, 0 = no noise term
    const float* Vnoise;         // FP32 V (ld = ld_v) for the noise term
    int64_t ld_v;
    const float* outscale;       // [R_pad] a^2 / s_c
    float* out;                  // Nr x R col-major (ld_out)
    int64_t ld_out;
    float* partial;              // [n_split][R_pad][ld_part] when n_split > 1
    int64_t ld_part;
    int* err;
    uint64_t limit_ns;
};

struct TcBarriers {
    uint64_t full[kStages];
    uint64_t empty[kStages];
    uint64_t s_full[2];
    uint64_t s_empty[2];
    uint64_t p_full[2];
    uint64_t pv_done[2];
    uint64_t o_full;
    uint64_t o_empty;
    uint64_t xi_full[2];      // row tile of item ic lives in buffer ic & 1
    uint64_t xi_empty[2];
    uint64_t drain;
};

__device__ __forceinline__ void record_error(int* err, int code) { atomicCAS(err, 0, code); }

// TMEM column layout (see the header comment).
struct TmemCols {
    uint32_t nsb;     // S buffers (2, or 1 with the hi + lo kernel tile)
    uint32_t pw;      // columns of one P buffer (64 or 128)
    __device__ __forceinline__ uint32_t s(uint32_t b) const { return b * 128u; }
    __device__ __forceinline__ uint32_t p(uint32_t b) const { return nsb * 128u + b * pw; }
    __device__ __forceinline__ uint32_t o() const { return nsb * 128u + 2u * pw; }
};
__device__ __forceinline__ TmemCols tmem_cols(int psplit) {
    TmemCols c;
    c.nsb = psplit ? 1u : 2u;
    c.pw = psplit ? 128u : 64u;
    return c;
}

__device__ __forceinline__ void item_range(const TcParams& p, int item, int& it, int& j0, int& j1) {
    it = item % p.n_it;
    const int sp = item / p.n_it;
    j0 = (int)(((int64_t)sp * p.n_jt) / p.n_split);
    j1 = (int)(((int64_t)(sp + 1) * p.n_jt) / p.n_split);
}

// ---- TMA producer (one thread) ------------------------------------------------
__device__ void tc_producer(const TcParams& p, const CUtensorMap* tmA, const CUtensorMap* tmB,
                            const CUtensorMap* tmV, TcBarriers& bars, uint8_t* sXi, uint8_t* sSt,
                            uint32_t xbytes, uint32_t vbytes) {
    uint32_t fills = 0, xi_loads = 0;
    bool ok = true;
    int ic = 0;
    const uint32_t S = (uint32_t)p.stages;
    const int natoms = p.k_pad > 64 ? p.k_pad / 64 : 1;
    const uint32_t abytes = xbytes / natoms;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x, ++ic) {
        int it, j0, j1;
        item_range(p, item, it, j0, j1);
        const int xb = ic & 1;
        if (ic >= 2 && !ptx::mbar_wait(&bars.xi_empty[xb], ((ic >> 1) - 1) & 1, p.limit_ns)) { ok = false; break; }
        uint8_t* sX = sXi + xb * xbytes;
        ptx::mbar_arrive_expect_tx(&bars.xi_full[xb], xbytes);
        for (int a = 0; a < natoms; ++a)
            ptx::tma_load_2d(sX + a * abytes, tmA, &bars.xi_full[xb], a * 64, it * kBM);
        ++xi_loads;
        for (int jt = j0; jt < j1; ++jt) {
            const uint32_t st = fills % S, u = fills / S;
            if (u > 0 && !ptx::mbar_wait(&bars.empty[st], (u - 1) & 1, p.limit_ns)) { ok = false; break; }
            uint8_t* sx = sSt + st * (xbytes + vbytes);
            ptx::mbar_arrive_expect_tx(&bars.full[st], xbytes + vbytes);
            for (int a = 0; a < natoms; ++a) ptx::tma_load_2d(sx + a * abytes, tmB, &bars.full[st], a * 64, jt * kBN);
            const uint32_t vbox = (uint32_t)p.R_pad * 128u;   // one 64-column box of R_pad rows
            for (int part = 0; part <= p.vsplit; ++part) {
                uint8_t* sv = sx + xbytes + part * 2u * vbox;
                ptx::tma_load_2d(sv, tmV, &bars.full[st], jt * kBN, part * p.R_pad);
                ptx::tma_load_2d(sv + vbox, tmV, &bars.full[st], jt * kBN + 64, part * p.R_pad);
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
        for (uint32_t q = xi_loads > 2 ? xi_loads - 2 : 0; q < xi_loads; ++q)
            ptx::mbar_wait(&bars.xi_full[q & 1], (q >> 1) & 1, p.limit_ns);
    }
}

// ---- MMA issuer (one thread) ----------------------------------------------------
// Event driven: the thread polls (non-blocking) and issues whichever product
// is ready -- S(g) into S buffer g % nsb once the epilogue has loaded
// S(g - nsb) from it and the operands have landed, P.V(g) once P(g) is
// stored -- so neither kind of product waits behind the other.
__device__ void tc_mma(const TcParams& p, TcBarriers& bars, const uint8_t* sXi, const uint8_t* sSt,
                       uint32_t xbytes, uint32_t vbytes, uint32_t tmem, uint32_t id_s, uint32_t id_pv) {
    const uint32_t arow = p.k_pad * 2 < 128 ? (uint32_t)p.k_pad * 2u : 128u;  // bytes per row of one atom
    const uint32_t swz = (arow == 32) ? 6u : (arow == 64 ? 4u : 2u);         // 32B / 64B / 128B swizzle
    const uint32_t sbo_x = 8u * arow;                                        // 8 rows of the swizzle atom
    const uint32_t abytes = (uint32_t)kBM * arow;                            // one atom of a 128-row tile
    const int ksteps = p.k_pad / 16;
    const uint32_t S = (uint32_t)p.stages;
    const TmemCols tc = tmem_cols(p.psplit);
    const uint32_t aSt = ptx::smem_u32(sSt);
    const uint32_t stage_bytes = xbytes + vbytes;
    const uint32_t vbox = (uint32_t)p.R_pad * 128u;
    const int nprod = 1 + p.vsplit + p.psplit;
    const long long limit = (long long)(p.limit_ns * 2ull);
    const uint32_t hi_x = ptx::smem_desc_hi(sbo_x, swz);   // row tiles: swizzle by row width
    const uint32_t hi_v = ptx::smem_desc_hi(1024u, 2u);     // right-hand sides: 128-byte swizzle
    uint32_t n = 0, gt = 0;
    int ic = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items && ok; item += gridDim.x, ++ic) {
        int it, j0, j1;
        item_range(p, item, it, j0, j1);
        const uint32_t T = (uint32_t)(j1 - j0);
        const int xb = ic & 1;
        if (!ptx::mbar_wait(&bars.xi_full[xb], (ic >> 1) & 1, p.limit_ns)) { ok = false; break; }
        ptx::tc_fence_after();
        const uint32_t aXi = ptx::smem_u32(sXi) + (uint32_t)xb * xbytes;
        uint32_t ts = 0, tp = 0;            // next tile for S, next tile for P.V
        long long idle_since = clock64();
        while (tp < T) {
            bool progressed = false;
            // ---- S(ts): needs its S buffer released and its operands landed
            if (ts < T) {
                const uint32_t g = gt + ts, b = g % tc.nsb, f = n + ts, st = f % S;
                const bool buf_free = (g < tc.nsb) || ptx::mbar_test(&bars.s_empty[b], (g / tc.nsb - 1) & 1);
                if (buf_free && ptx::mbar_test(&bars.full[st], (f / S) & 1)) {
                    ptx::tc_fence_after();
                    const uint32_t aXj = aSt + st * stage_bytes;
                    const uint32_t dS = tmem + tc.s(b);
                    for (int kk = 0; kk < ksteps; ++kk) {
                        const uint32_t koff = ((uint32_t)kk * 32u / arow) * abytes + ((uint32_t)kk * 32u) % arow;
                        ptx::mma_f16_ss(dS, ptx::smem_desc_at(hi_x, aXi + koff), ptx::smem_desc_at(hi_x, aXj + koff),
                                        id_s, kk > 0 ? 1u : 0u);
                    }
                    ptx::mma_commit(&bars.s_full[g & 1]);   // one barrier per epilogue warpgroup
                    if (ts + 1 == T) ptx::mma_commit(&bars.xi_empty[xb]);   // last use of this row tile
                    ++ts;
                    progressed = true;
                }
            }
            // ---- P.V(tp): needs P(tp) stored (and, first in an item, O read out)
            if (tp < ts) {
                const uint32_t g = gt + tp, pb = g & 1;
                const bool o_free = (tp > 0) || (ic == 0) || ptx::mbar_test(&bars.o_empty, (ic - 1) & 1);
                if (o_free && ptx::mbar_test(&bars.p_full[pb], (g >> 1) & 1)) {
                    ptx::tc_fence_after();
                    const uint32_t f = n + tp, st = f % S;
                    const uint32_t aV = aSt + st * stage_bytes + xbytes;
                    // Products accumulated into O: P_hi V_hi, then P_hi V_lo (vsplit), then P_lo V_hi (psplit).
                    const uint32_t dO = tmem + tc.o();
                    for (int q = 0; q < nprod; ++q) {
                        const uint32_t vpart = (q == 1 && p.vsplit) ? 1u : 0u;
                        const uint32_t aP = tmem + tc.p(pb) + ((q == nprod - 1 && p.psplit && q > 0) ? 64u : 0u);
                        const uint32_t aVq = aV + 2u * vpart * vbox;
                        const uint32_t acc0 = (tp > 0 || q > 0) ? 1u : 0u;
#pragma unroll
                        for (int kk = 0; kk < kBN / 16; ++kk) {
                            const uint32_t off = (uint32_t)(kk >> 2) * vbox + (uint32_t)(kk & 3) * 32u;
                            ptx::mma_f16_ts(dO, aP + (uint32_t)kk * 8u, ptx::smem_desc_at(hi_v, aVq + off), id_pv,
                                            kk > 0 ? 1u : acc0);
                        }
                    }
                    ptx::mma_commit(&bars.empty[st]);     // X_j and V_j of this stage are consumed
                    ptx::mma_commit(&bars.pv_done[pb]);   // P buffer pb may be rewritten
                    ++tp;
                    progressed = true;
                }
            }
            if (progressed) {
                idle_since = clock64();
            } else {
                // Back off: this warp shares its scheduler with two epilogue warps,
                // and a tight poll loop would take their issue slots.
                __nanosleep(64);
                if (clock64() - idle_since > limit) {
                    ok = false;
                    break;
                }
            }
        }
        if (!ok) break;
        ptx::mma_commit(&bars.o_full);
        n += T;
        gt += T;
    }
    // No MMA may be in flight when TMEM is released.
    ptx::mma_commit(&bars.drain);
    ptx::mbar_wait(&bars.drain, 0, p.limit_ns);
    if (!ok) record_error(p.err, DEV_TIMEOUT);
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

// ---- epilogue warpgroups ------------------------------------------------------------
template <int BF16>
__device__ __forceinline__ float unpack_lo(uint32_t v) {
    if constexpr (BF16) return __uint_as_float(v << 16);
    else return __half2float(__ushort_as_half((unsigned short)(v & 0xFFFFu)));
}
template <int BF16>
__device__ __forceinline__ float unpack_hi(uint32_t v) {
    if constexpr (BF16) return __uint_as_float(v & 0xFFFF0000u);
    else return __half2float(__ushort_as_half((unsigned short)(v >> 16)));
}

template <int KIND, int BF16, int PSPLIT>
__device__ __forceinline__ void tc_chunk(const uint32_t (&r)[32], int h, int row, bool dtile, uint32_t tP,
                                         uint32_t tPlo) {
    uint32_t pk[16];
    uint32_t pl[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        float k0 = kernel_from_s<KIND>(__uint_as_float(r[2 * e]));
        float k1 = kernel_from_s<KIND>(__uint_as_float(r[2 * e + 1]));
        if constexpr (KIND == GP_KERNEL_MATERN12) {
            // exp(-r) has a kink at r = 0: the on-chip diagonal is skipped and the
            // exact a^2 v_i is added with the noise term instead.
            if (dtile) {
                const int col = h * 32 + 2 * e;
                if (col == row) k0 = 0.0f;
                if (col + 1 == row) k1 = 0.0f;
            }
        }
        pk[e] = pack2<BF16>(k0, k1);
        if constexpr (PSPLIT) pl[e] = pack2<BF16>(k0 - unpack_lo<BF16>(pk[e]), k1 - unpack_hi<BF16>(pk[e]));
    }
    ptx::tmem_st16(tP + (uint32_t)h * 16u, pk);
    if constexpr (PSPLIT) ptx::tmem_st16(tPlo + (uint32_t)h * 16u, pl);
}

template <int KIND, int BF16, int PSPLIT>
__device__ void tc_epilogue(const TcParams& p, TcBarriers& bars, uint32_t tmem, int wg, int wq, int lane) {
    const uint32_t lane_off = (uint32_t)(wq * 32) << 16;
    const int row = wq * 32 + lane;
    const TmemCols tc = tmem_cols(PSPLIT);
    uint32_t gt = 0;
    int ic = 0;
    bool ok = true;
    for (int item = blockIdx.x; item < p.n_items; item += gridDim.x, ++ic) {
        int it, j0, j1;
        item_range(p, item, it, j0, j1);
        const uint32_t T = (uint32_t)(j1 - j0);
        for (uint32_t t = 0; t < T; ++t) {
            const uint32_t g = gt + t, pb = g & 1;
            if ((int)pb != wg) continue;
            const uint32_t sb = g % tc.nsb;
            // s_full[pb] completes once per tile of this warpgroup (tiles g = pb, pb + 2, ...),
            // so a waiter is never more than one phase behind (parity waits stay exact)
            if (!ptx::mbar_wait(&bars.s_full[pb], (g >> 1) & 1, p.limit_ns)) { ok = false; break; }
            ptx::tc_fence_after();
            const uint32_t tS = tmem + lane_off + tc.s(sb);
            const bool dtile = (KIND == GP_KERNEL_MATERN12) && p.diag && (j0 + (int)t == it);
            const uint32_t tP = tmem + lane_off + tc.p(pb);
            const uint32_t tPlo = tP + 64u;
            // The tile is processed in two 64-column halves (about 110 live registers,
            // no spills under the 168-register budget of 320 threads).
            uint32_t ra[32], rb[32];
            ptx::tmem_ld32(tS, ra);
            ptx::tmem_ld32(tS + 32u, rb);
            ptx::tmem_wait_ld();
            ptx::tmem_reg_fence(ra);
            ptx::tmem_reg_fence(rb);
            if (g >= 2) {                            // P.V of the buffer's previous tile is done
                if (!ptx::mbar_wait(&bars.pv_done[pb], ((g >> 1) - 1) & 1, p.limit_ns)) { ok = false; break; }
                ptx::tc_fence_after();
            }
            tc_chunk<KIND, BF16, PSPLIT>(ra, 0, row, dtile, tP, tPlo);
            tc_chunk<KIND, BF16, PSPLIT>(rb, 1, row, dtile, tP, tPlo);
            ptx::tmem_ld32(tS + 64u, ra);
            ptx::tmem_ld32(tS + 96u, rb);
            ptx::tmem_wait_ld();
            ptx::tmem_reg_fence(ra);
            ptx::tmem_reg_fence(rb);
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.s_empty[sb]);     // the MMA may overwrite this S buffer now
            tc_chunk<KIND, BF16, PSPLIT>(ra, 2, row, dtile, tP, tPlo);
            tc_chunk<KIND, BF16, PSPLIT>(rb, 3, row, dtile, tP, tPlo);
            ptx::tmem_wait_st();
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.p_full[pb]);
        }
        if (!ok) break;
        if (wg == 0) {
            if (!ptx::mbar_wait(&bars.o_full, ic & 1, p.limit_ns)) { ok = false; break; }
            ptx::tc_fence_after();
            const int64_t i = (int64_t)it * kBM + row;
            const int sp = item / p.n_it;
            for (int c0 = 0; c0 < p.R_pad; c0 += 16) {
                uint32_t o[16];
                ptx::tmem_ld16(tmem + lane_off + tc.o() + (uint32_t)c0, o);
                ptx::tmem_wait_ld();
                ptx::tmem_reg_fence(o);
                if (i < p.Nr) {
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int c = c0 + e;
                        if (c < p.R) {
                            const float acc = __uint_as_float(o[e]);
                            if (p.n_split == 1) {
                                float val = acc * p.outscale[c];
                                if (p.noise != 0.0f) val = fmaf(p.noise, p.Vnoise[c * p.ld_v + i], val);
                                p.out[c * p.ld_out + i] = val;
                            } else {
                                p.partial[((int64_t)sp * p.R_pad + c) * p.ld_part + i] = acc;
                            }
                        }
                    }
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&bars.o_empty);
        }
        gt += T;
    }
    if (!ok) record_error(p.err, DEV_TIMEOUT);
}

template <int KIND, int BF16, int PSPLIT>
__global__ void __launch_bounds__(kThreads, 1)
kmvm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmV, const TcParams p) {
    extern __shared__ uint8_t dsm[];
    __shared__ TcBarriers bars;
    __shared__ uint32_t tmem_slot;

    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(dsm) + 1023) & ~uintptr_t(1023));
    const uint32_t xbytes = (uint32_t)kBM * (uint32_t)p.k_pad * 2u;
    const uint32_t vbytes = (uint32_t)(1 + p.vsplit) * (uint32_t)p.R_pad * (uint32_t)kBN * 2u;
    uint8_t* sXi = base;                 // two row-tile buffers
    uint8_t* sSt = base + 2 * xbytes;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            ptx::mbar_init(&bars.full[s], 1);
            ptx::mbar_init(&bars.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&bars.s_full[b], 1);
            ptx::mbar_init(&bars.s_empty[b], 128);
            ptx::mbar_init(&bars.p_full[b], 128);
            ptx::mbar_init(&bars.pv_done[b], 1);
        }
        ptx::mbar_init(&bars.o_full, 1);
        ptx::mbar_init(&bars.o_empty, 128);
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&bars.xi_full[b], 1);
            ptx::mbar_init(&bars.xi_empty[b], 1);
        }
        ptx::mbar_init(&bars.drain, 1);
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
        if (lane == 0) tc_producer(p, &tmA, &tmB, &tmV, bars, sXi, sSt, xbytes, vbytes);
        __syncwarp();
    } else if (warp == kMmaWarp) {
        if (lane == 0)
            tc_mma(p, bars, sXi, sSt, xbytes, vbytes, tmem, ptx::idesc_f16(kBM, kBN, BF16),
                   ptx::idesc_f16(kBM, p.R_pad, BF16));
        __syncwarp();
    } else {
        tc_epilogue<KIND, BF16, PSPLIT>(p, bars, tmem, warp >> 2, warp & 3, lane);
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    if (warp == kMmaWarp) ptx::tmem_dealloc(tmem, kTmemCols);
}

template <int KIND, int BF16, int PSPLIT>
cudaError_t launch_tc_typed(const TcPlan& plan, const TcParams& prm, const CUtensorMap& a, const CUtensorMap& b,
                            const CUtensorMap& v, cudaStream_t s) {
    const int smem = tc_smem_bytes(plan.k_pad, plan.R_pad, prm.vsplit);
    auto kfn = kmvm_tc_kernel<KIND, BF16, PSPLIT>;
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kfn<<<plan.grid, kThreads, smem, s>>>(a, b, v, prm);
    return cudaGetLastError();
}

}  // namespace

int tc_stages(int k_pad, int R_pad, int vsplit) {
    const int xbytes = kBM * k_pad * 2;
    const int vbytes = (1 + vsplit) * R_pad * kBN * 2;
    for (int st = kStages; st >= 2; --st)
        if (1024 + 2 * xbytes + st * (xbytes + vbytes) <= kMaxSmemBytes) return st;
    return 0;
}

int tc_smem_bytes(int k_pad, int R_pad, int vsplit) {
    const int xbytes = kBM * k_pad * 2;
    const int vbytes = (1 + vsplit) * R_pad * kBN * 2;
    int need = 1024 + 2 * xbytes + tc_stages(k_pad, R_pad, vsplit) * (xbytes + vbytes);
    return need < kMinSmemBytes ? kMinSmemBytes : need;
}

TcPlan tc_plan(const Ctx* ctx, int64_t Nr, int64_t Nc, int R, int k_pad) {
    TcPlan p;
    p.k_pad = k_pad;
    p.R_pad = ((R + 15) / 16) * 16;
    p.n_it = (int)((Nr + kBM - 1) / kBM);
    p.n_jt = (int)((Nc + kBN - 1) / kBN);
    p.Nr_pad = (int64_t)p.n_it * kBM;
    p.Nc_pad = (int64_t)p.n_jt * kBN;
    const int G = ctx->num_sms > 0 ? ctx->num_sms : 1;
    // Pick the column split minimising the busiest CTA's work: waves x tiles
    // per item, plus a fixed per-item cost (pipeline fill, O read-out) of about
    // two tiles, plus the partial-sum reduction when split.
    int best = 1;
    double best_cost = 1e300;
    const int max_split = p.n_jt < 16 ? p.n_jt : 16;
    for (int sp = 1; sp <= max_split; ++sp) {
        const int64_t items = (int64_t)p.n_it * sp;
        const int64_t waves = (items + G - 1) / G;
        const int64_t tiles = (p.n_jt + sp - 1) / sp;
        double cost = (double)waves * (double)(tiles + 2);
        if (sp > 1) cost += 0.05 * (double)sp * (double)p.n_it * (double)p.R_pad / (double)G / 64.0;
        if (cost < best_cost - 1e-9) { best_cost = cost; best = sp; }
    }
    p.n_split = best;
    const int64_t items = (int64_t)p.n_it * p.n_split;
    p.grid = (int)(items < G ? items : G);
    return p;
}

size_t tc_partial_floats(const TcPlan& p) {
    return p.n_split > 1 ? (size_t)p.n_split * p.R_pad * p.Nr_pad : 0;
}

int launch_kmvm_tc(Ctx* ctx, const TcPlan& plan, const OperandLayout& L, const MvmArgs& a, const CUtensorMap& tmA,
                   const CUtensorMap& tmB, const CUtensorMap& tmV, const float* outscale, float* partial,
                   cudaStream_t s) {
    TcParams prm;
    prm.n_it = plan.n_it;
    prm.n_jt = plan.n_jt;
    prm.n_split = plan.n_split;
    prm.n_items = plan.n_it * plan.n_split;
    prm.k_pad = plan.k_pad;
    prm.R_pad = plan.R_pad;
    prm.R = a.R;
    prm.vsplit = L.vsplit;
    prm.psplit = L.psplit;
    prm.stages = tc_stages(plan.k_pad, plan.R_pad, L.vsplit);
    if (prm.stages < 2) return GP_ERR_UNSUPPORTED;
    prm.Nr = a.Nr;
    prm.noise = a.noise + a.diag_coef;
    prm.diag = a.diag_coef != 0.0f ? 1 : 0;
    prm.Vnoise = a.Vnoise;
    prm.ld_v = a.Nc;
    prm.outscale = outscale;
    prm.out = a.out;
    prm.ld_out = a.ld_out;
    prm.partial = partial;
    prm.ld_part = plan.Nr_pad;
    prm.err = ctx->dev_err;
    prm.limit_ns = kWaitLimitNs;
    const int bf = (L.prec == GP_PREC_BF16) ? 1 : 0;
    cudaError_t e = cudaErrorInvalidValue;
    prof_begin(ctx, s);
#define GPK_TC_CASE(K)                                                                  \
    case K:                                                                             \
        e = bf ? (L.psplit ? launch_tc_typed<K, 1, 1>(plan, prm, tmA, tmB, tmV, s)      \
                           : launch_tc_typed<K, 1, 0>(plan, prm, tmA, tmB, tmV, s))     \
               : launch_tc_typed<K, 0, 0>(plan, prm, tmA, tmB, tmV, s);                 \
        break;
    switch (a.kernel) {
        GPK_TC_CASE(GP_KERNEL_RBF)
        GPK_TC_CASE(GP_KERNEL_MATERN32)
        GPK_TC_CASE(GP_KERNEL_MATERN12)
        GPK_TC_CASE(GP_KERNEL_MATERN52)
        default: return GP_ERR_INVALID;
    }
#undef GPK_TC_CASE
    prof_end(ctx, s);
    ctx->launches++;
    if (e != cudaSuccess) return GP_ERR_CUDA;
    if (plan.n_split > 1)
        return launch_split_reduce(ctx, partial, plan.n_split, plan.Nr_pad, a.Nr, a.R, plan.R_pad, outscale, 0.0f,
                                   prm.noise, a.Vnoise, a.Nc, a.out, a.ld_out, s);
    return GP_OK;
}

}  // namespace gpk
