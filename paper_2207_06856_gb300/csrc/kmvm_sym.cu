// The symmetric half-work kernel MVM (an extension in the direction of
// the Conclusion's future work: K = K^T lets an MVM evaluate N (N + 1) / 2
// kernel values instead of N^2).
//
// FP32 on the CUDA cores, square operators only (GP_MVM_SYMMETRIC with
// GP_PREC_FP32).  The points are cut into 256-row blocks I and 64-column tiles
// J; a thread block takes one row block and the column tiles at or after its
// diagonal, evaluates k_ij once for every pair with j > i and uses it twice:
//   row pass:     out_i += a^2 sum_j k_ij v_j   (two rows per thread, packed
//                                               FP32x2 arithmetic as in the
//                                               SIMT engine; the 256 x 64 tile
//                                               of k kept in shared memory)
//   column pass:  out_j += a^2 sum_i k_ij v_i   (two columns per lane, the rows
//                                               split over the four warps)
// and the diagonal adds (a^2 k(0) + sigma^2) v_i = (a^2 + sigma^2) v_i.  The
// column sums of a tile and the row sums of a block are added to the output
// with FP32 atomics, so the order of the additions (and the last bits of the
// result) varies from run to run; the MVM tolerance of the FP32 engines (1e-5)
// is unaffected.  Every kernel value is evaluated once, against twice in the
// other engines; the shared-memory broadcasts of v (the SIMT engine's bound)
// are not saved, since each pair still needs v_j for its row and v_i for its
// column.
#include "gpk_internal.cuh"
#include "kfun.cuh"

namespace gpk {

namespace {

constexpr int kSymT = 128;        // threads per block
constexpr int kSymRows = 256;     // rows per block: two per thread
constexpr int kSymCols = 64;      // columns per tile
constexpr int kKtLd = kSymRows + 1;
constexpr int kSymMaxDp = 32;
constexpr int kSymMaxR = 24;

template <int DPM, int RPM>
constexpr size_t sym_smem_floats() {
    return (size_t)kSymCols * kKtLd + (size_t)kSymCols * (DPM + 4) + (size_t)kSymCols * (RPM + 4) +
           (size_t)kSymRows * (RPM + 4);
}

template <int KIND, int DPM, int RPM>
__global__ void __launch_bounds__(kSymT)
kmvm_sym_kernel(const float* __restrict__ Xs, int64_t N, int dp, const float* __restrict__ V, int R, int n_jt,
                float a2, float noise, float* __restrict__ out, int64_t ld_out) {
    extern __shared__ __align__(16) float smem[];
    float* kt = smem;                                       // [kSymCols][kKtLd]   k_ij, column j = row of kt
    float* red = smem;                                      // [kSymRows][RPM + 1] after the column pass
    float(*sx)[DPM + 4] = reinterpret_cast<float(*)[DPM + 4]>(smem + kSymCols * kKtLd);         // -x_j
    float(*svj)[RPM + 4] = reinterpret_cast<float(*)[RPM + 4]>(smem + kSymCols * kKtLd + kSymCols * (DPM + 4));
    float(*svi)[RPM + 4] = reinterpret_cast<float(*)[RPM + 4]>(smem + kSymCols * kKtLd + kSymCols * (DPM + 4) +
                                                               kSymCols * (RPM + 4));
    const int I = blockIdx.x, G = gridDim.y;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int64_t ib = (int64_t)I * kSymRows;
    const int64_t i0 = ib + t, i1 = i0 + kSymT;
    for (int e = t; e < kSymRows * RPM; e += kSymT) {
        const int c = e / kSymRows, ii = e % kSymRows;
        svi[ii][c] = (c < R && ib + ii < N) ? V[(int64_t)c * N + ib + ii] : 0.0f;
    }
    float2 x0[DPM / 2], x1[DPM / 2], acc0[RPM / 2], acc1[RPM / 2];
#pragma unroll
    for (int h = 0; h < DPM / 2; ++h) {
        const int k = 2 * h;   // dp is a multiple of 4
        x0[h] = (i0 < N && k < dp) ? make_float2(Xs[i0 * dp + k], Xs[i0 * dp + k + 1]) : make_float2(0.0f, 0.0f);
        x1[h] = (i1 < N && k < dp) ? make_float2(Xs[i1 * dp + k], Xs[i1 * dp + k + 1]) : make_float2(0.0f, 0.0f);
    }
#pragma unroll
    for (int h = 0; h < RPM / 2; ++h) { acc0[h] = make_float2(0.0f, 0.0f); acc1[h] = make_float2(0.0f, 0.0f); }

    const int jt0 = I * (kSymRows / kSymCols);   // the first column tile that meets row block I
    for (int jt = jt0 + (int)blockIdx.y; jt < n_jt; jt += G) {
        const int64_t jb = (int64_t)jt * kSymCols;
        __syncthreads();   // the previous tile is done with sx, svj and kt / red
        for (int e = t; e < kSymCols * DPM; e += kSymT) {
            const int jj = e / DPM, k = e % DPM;
            sx[jj][k] = (jb + jj < N && k < dp) ? -Xs[(jb + jj) * dp + k] : 0.0f;
        }
        for (int e = t; e < kSymCols * RPM; e += kSymT) {
            const int c = e / kSymCols, jj = e % kSymCols;
            svj[jj][c] = (c < R && jb + jj < N) ? V[(int64_t)c * N + jb + jj] : 0.0f;
        }
        __syncthreads();
        // row pass; in the tiles that meet the block's own rows only j > i counts
        const bool diag = jb < ib + kSymRows;
        for (int jj = 0; jj < kSymCols; ++jj) {
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
            float k0 = kernel_from_s<KIND>(-(q0.x + q0.y));
            float k1 = kernel_from_s<KIND>(-(q1.x + q1.y));
            if (diag) {
                const int64_t j = jb + jj;
                if (j <= i0) k0 = 0.0f;
                if (j <= i1) k1 = 0.0f;
            }
            kt[jj * kKtLd + t] = k0;
            kt[jj * kKtLd + t + kSymT] = k1;
            const float2 kk0 = make_float2(k0, k0), kk1 = make_float2(k1, k1);
#pragma unroll
            for (int c = 0; c < RPM; c += 4) {
                if (c < R) {
                    const float4 v4 = *reinterpret_cast<const float4*>(&svj[jj][c]);   // broadcast
                    const float2 va = make_float2(v4.x, v4.y), vb = make_float2(v4.z, v4.w);
                    acc0[c / 2] = __ffma2_rn(kk0, va, acc0[c / 2]);
                    acc1[c / 2] = __ffma2_rn(kk1, va, acc1[c / 2]);
                    acc0[c / 2 + 1] = __ffma2_rn(kk0, vb, acc0[c / 2 + 1]);
                    acc1[c / 2 + 1] = __ffma2_rn(kk1, vb, acc1[c / 2 + 1]);
                }
            }
        }
        __syncthreads();
        // column pass: warp w takes rows [64 w, 64 w + 64) of the block, the lane
        // columns lane and lane + 32 of the tile
        float2 ca[RPM / 2], cb[RPM / 2];
#pragma unroll
        for (int h = 0; h < RPM / 2; ++h) { ca[h] = make_float2(0.0f, 0.0f); cb[h] = make_float2(0.0f, 0.0f); }
        for (int ii = w * 64; ii < w * 64 + 64; ++ii) {
            const float ka = kt[lane * kKtLd + ii], kb = kt[(lane + 32) * kKtLd + ii];
            const float2 kka = make_float2(ka, ka), kkb = make_float2(kb, kb);
#pragma unroll
            for (int c = 0; c < RPM; c += 4) {
                if (c < R) {
                    const float4 v4 = *reinterpret_cast<const float4*>(&svi[ii][c]);   // broadcast
                    const float2 va = make_float2(v4.x, v4.y), vb = make_float2(v4.z, v4.w);
                    ca[c / 2] = __ffma2_rn(kka, va, ca[c / 2]);
                    cb[c / 2] = __ffma2_rn(kkb, va, cb[c / 2]);
                    ca[c / 2 + 1] = __ffma2_rn(kka, vb, ca[c / 2 + 1]);
                    cb[c / 2 + 1] = __ffma2_rn(kkb, vb, cb[c / 2 + 1]);
                }
            }
        }
        __syncthreads();   // kt is read: its space takes the four warps' column sums
#pragma unroll
        for (int c = 0; c < RPM; ++c) {
            if (c < R) {
                red[(w * kSymCols + lane) * (RPM + 1) + c] = (c & 1) ? ca[c / 2].y : ca[c / 2].x;
                red[(w * kSymCols + lane + 32) * (RPM + 1) + c] = (c & 1) ? cb[c / 2].y : cb[c / 2].x;
            }
        }
        __syncthreads();
        for (int e = t; e < kSymCols * R; e += kSymT) {
            const int col = e % kSymCols, c = e / kSymCols;
            const int64_t j = jb + col;
            if (j < N) {
                float sum = 0.0f;
#pragma unroll
                for (int q = 0; q < kSymT / 32; ++q) sum += red[(q * kSymCols + col) * (RPM + 1) + c];
                atomicAdd(out + (int64_t)c * ld_out + j, a2 * sum);
            }
        }
    }
    if (jt0 + (int)blockIdx.y >= n_jt) return;   // took no column tile
    // rows of the block; the block with the diagonal tile adds (a^2 + sigma^2) v_i
    const bool own_diag = blockIdx.y == 0;
#pragma unroll
    for (int c = 0; c < RPM; ++c) {
        if (c < R) {
            const float s0 = (c & 1) ? acc0[c / 2].y : acc0[c / 2].x;
            const float s1 = (c & 1) ? acc1[c / 2].y : acc1[c / 2].x;
            if (i0 < N) {
                float o = a2 * s0;
                if (own_diag) o = fmaf(a2 + noise, svi[t][c], o);
                atomicAdd(out + (int64_t)c * ld_out + i0, o);
            }
            if (i1 < N) {
                float o = a2 * s1;
                if (own_diag) o = fmaf(a2 + noise, svi[t + kSymT][c], o);
                atomicAdd(out + (int64_t)c * ld_out + i1, o);
            }
        }
    }
}

template <int KIND, int DPM, int RPM>
cudaError_t launch_sym_typed(dim3 grid, cudaStream_t s, const float* Xs, int64_t N, int dp, const float* V, int R,
                             int n_jt, float a2, float noise, float* out, int64_t ld_out) {
    auto fn = kmvm_sym_kernel<KIND, DPM, RPM>;
    const size_t smem = sizeof(float) * sym_smem_floats<DPM, RPM>();
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<grid, kSymT, smem, s>>>(Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
    return cudaGetLastError();
}

template <int KIND, int DPM>
cudaError_t launch_sym_r(int RPM, dim3 grid, cudaStream_t s, const float* Xs, int64_t N, int dp, const float* V,
                         int R, int n_jt, float a2, float noise, float* out, int64_t ld_out) {
    switch (RPM) {
        case 4: return launch_sym_typed<KIND, DPM, 4>(grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
        case 8: return launch_sym_typed<KIND, DPM, 8>(grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
        case 12: return launch_sym_typed<KIND, DPM, 12>(grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
        case 16: return launch_sym_typed<KIND, DPM, 16>(grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
        case 20: return launch_sym_typed<KIND, DPM, 20>(grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
        default: return launch_sym_typed<KIND, DPM, 24>(grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
    }
}

template <int KIND>
cudaError_t launch_sym_kind(int DPM, int RPM, dim3 grid, cudaStream_t s, const float* Xs, int64_t N, int dp,
                            const float* V, int R, int n_jt, float a2, float noise, float* out, int64_t ld_out) {
    switch (DPM) {
        case 8: return launch_sym_r<KIND, 8>(RPM, grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
        case 16: return launch_sym_r<KIND, 16>(RPM, grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
        default: return launch_sym_r<KIND, 32>(RPM, grid, s, Xs, N, dp, V, R, n_jt, a2, noise, out, ld_out);
    }
}

}  // namespace

// out (N x R, ld_out) = a^2 K V + noise V for the square operator of the scaled
// inputs Xs (N x dp, dp a multiple of 4, as the SIMT engine's); R <= 24.
int launch_kmvm_sym(Ctx* ctx, const MvmArgs& a, float outputscale, const float* Xs, int dp, const float* V,
                    cudaStream_t s) {
    if (a.R > kSymMaxR || dp > kSymMaxDp || (dp & 3) || a.Nr != a.Nc) return GP_ERR_UNSUPPORTED;
    const int RPM = ((a.R + 3) / 4) * 4;
    const int DPM = dp <= 8 ? 8 : dp <= 16 ? 16 : 32;
    const int64_t nb = (a.Nr + kSymRows - 1) / kSymRows;
    const int64_t n_jt = (a.Nr + kSymCols - 1) / kSymCols;
    if (nb > 0x7fffffff || n_jt > 0x7fffffff) return GP_ERR_UNSUPPORTED;
    for (int r = 0; r < a.R; ++r)
        if (cudaMemsetAsync(a.out + (int64_t)r * a.ld_out, 0, sizeof(float) * a.Nr, s) != cudaSuccess)
            return GP_ERR_CUDA;
    // G column-tile groups per row block: thread blocks to fill the SMs many
    // times over (the blocks of the first row blocks carry the most tiles and
    // start first), few enough that each keeps its row sums over several tiles
    const int64_t G = n_jt < 32 ? n_jt : 32;
    const dim3 grid((unsigned)nb, (unsigned)G);
    const int n = (int)n_jt;
    cudaError_t e;
    prof_begin(ctx, s);
    switch (a.kernel) {
        case GP_KERNEL_RBF:
            e = launch_sym_kind<GP_KERNEL_RBF>(DPM, RPM, grid, s, Xs, a.Nr, dp, V, a.R, n, outputscale, a.noise, a.out, a.ld_out);
            break;
        case GP_KERNEL_MATERN32:
            e = launch_sym_kind<GP_KERNEL_MATERN32>(DPM, RPM, grid, s, Xs, a.Nr, dp, V, a.R, n, outputscale, a.noise, a.out, a.ld_out);
            break;
        case GP_KERNEL_MATERN12:
            e = launch_sym_kind<GP_KERNEL_MATERN12>(DPM, RPM, grid, s, Xs, a.Nr, dp, V, a.R, n, outputscale, a.noise, a.out, a.ld_out);
            break;
        default:
            e = launch_sym_kind<GP_KERNEL_MATERN52>(DPM, RPM, grid, s, Xs, a.Nr, dp, V, a.R, n, outputscale, a.noise, a.out, a.ld_out);
            break;
    }
    prof_end(ctx, s);
    ctx->launches++;
    return e == cudaSuccess ? GP_OK : GP_ERR_CUDA;
}

}  // namespace gpk
