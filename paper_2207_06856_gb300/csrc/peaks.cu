// Measurement support: throughput micro-benchmarks of the units that bound
// the kernel MVM (special-function ex2 and sqrt, FP32 FMA), and CUDA-event
// timing of the tensor-core MVM launches inside real solves.
#include "gpk_internal.cuh"
#include "ptx.cuh"

namespace gpk {

namespace {

constexpr int kChains = 8;
constexpr int kIters = 2048;

template <int OP>
__global__ void __launch_bounds__(256) peak_kernel(float seed, float* sink) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = 0.5f + 0.01f * (float)c + seed * (float)threadIdx.x;
    for (int it = 0; it < kIters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            if constexpr (OP == 0) v[c] = ptx::ex2(-v[c]);              // stays in (0.5, 1)
            else if constexpr (OP == 1) v[c] = ptx::sqrt_approx(v[c] + 0.25f) ;
            else if constexpr (OP == 2) v[c] = fmaf(v[c], 0.999f, 0.0005f);
        }
        if constexpr (OP == 3) {
            // FP32 pair -> packed FP16x2 and back (one conversion each way per pair)
#pragma unroll
            for (int c = 0; c < kChains; c += 2) {
                __half2 h = __floats2half2_rn(v[c], v[c + 1]);
                float2 f = __half22float2(h);
                v[c] = f.x * 0.999f;
                v[c + 1] = f.y * 0.999f;
            }
        }
        if constexpr (OP == 4) {
            // the FP16 epilogue per pair of kernel values: 2 ex2 + 1 pack
#pragma unroll
            for (int c = 0; c < kChains; c += 2) {
                const float a = ptx::ex2(-v[c]), b = ptx::ex2(-v[c + 1]);
                __half2 h = __floats2half2_rn(a, b);
                unsigned u = *reinterpret_cast<unsigned*>(&h);
                v[c] = __uint_as_float((u & 0x3ff) | 0x3f000000u);
                v[c + 1] = __uint_as_float(((u >> 16) & 0x3ff) | 0x3f000000u);
            }
        }
    }
    float acc = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c];
    if (acc == 12345.678f) sink[0] = acc;   // keeps the chains alive
}

template <int OP>
double time_peak(const Ctx* ctx, float* sink, cudaStream_t s) {
    const int blocks = (ctx->num_sms > 0 ? ctx->num_sms : 148) * 8;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    peak_kernel<OP><<<blocks, 256, 0, s>>>(1e-6f, sink);   // warm-up
    double best = 0.0;
    for (int rep = 0; rep < 5; ++rep) {
        cudaEventRecord(a, s);
        peak_kernel<OP><<<blocks, 256, 0, s>>>(1e-6f, sink);
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, a, b);
        const double ops = (double)blocks * 256.0 * kIters * kChains;
        const double rate = ops / (ms * 1e-3);
        if (rate > best) best = rate;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

}  // namespace

void prof_begin(Ctx* ctx, cudaStream_t s) {
    if (!ctx->prof || ctx->prof_n >= Ctx::kProfMax) return;
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n], s);
}
void prof_end(Ctx* ctx, cudaStream_t s) {
    if (!ctx->prof || ctx->prof_n >= Ctx::kProfMax) return;
    cudaEventRecord(ctx->prof_ev[2 * ctx->prof_n + 1], s);
    ctx->prof_n++;
}

}  // namespace gpk

extern "C" {

int gp_measure_peaks(gp_ctx* ctx, double* ex2_per_s, double* sqrt_per_s, double* ffma_per_s, void* stream) {
    return gp_measure_peaks2(ctx, ex2_per_s, sqrt_per_s, ffma_per_s, nullptr, nullptr, stream);
}

int gp_measure_peaks2(gp_ctx* ctx, double* ex2_per_s, double* sqrt_per_s, double* ffma_per_s, double* pack_per_s,
                      double* ex2pack_per_s, void* stream) {
    if (!ctx) return GP_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    float* sink = nullptr;
    if (cudaMalloc(&sink, 256) != cudaSuccess) return GP_ERR_OOM;
    const double e = gpk::time_peak<0>(ctx, sink, s);
    const double q = gpk::time_peak<1>(ctx, sink, s);
    const double f = gpk::time_peak<2>(ctx, sink, s);
    const double k = gpk::time_peak<3>(ctx, sink, s);   // counted per chain element: one pair = 2
    const double m = gpk::time_peak<4>(ctx, sink, s);   // kernel values per second (ex2 + half a pack each)
    cudaFree(sink);
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    if (ex2_per_s) *ex2_per_s = e;
    if (sqrt_per_s) *sqrt_per_s = q;
    if (ffma_per_s) *ffma_per_s = f;
    if (pack_per_s) *pack_per_s = k / 2.0;
    if (ex2pack_per_s) *ex2pack_per_s = m;
    return GP_OK;
}

int gp_ctx_profile(gp_ctx* ctx, int enable) {
    if (!ctx) return GP_ERR_INVALID;
    if (enable && !ctx->prof_ev_ready) {
        for (int i = 0; i < 2 * gpk::Ctx::kProfMax; ++i)
            if (cudaEventCreate(&ctx->prof_ev[i]) != cudaSuccess) return GP_ERR_CUDA;
        ctx->prof_ev_ready = true;
    }
    ctx->prof = enable != 0;
    ctx->prof_n = 0;
    return GP_OK;
}

int gp_ctx_profile_read(gp_ctx* ctx, double* total_ms, int64_t* launches) {
    if (!ctx) return GP_ERR_INVALID;
    double t = 0.0;
    for (int i = 0; i < ctx->prof_n; ++i) {
        if (cudaEventSynchronize(ctx->prof_ev[2 * i + 1]) != cudaSuccess) return GP_ERR_CUDA;
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, ctx->prof_ev[2 * i], ctx->prof_ev[2 * i + 1]) != cudaSuccess) return GP_ERR_CUDA;
        t += ms;
    }
    if (total_ms) *total_ms = t;
    if (launches) *launches = ctx->prof_n;
    ctx->prof_n = 0;
    return GP_OK;
}

}  // extern "C"
