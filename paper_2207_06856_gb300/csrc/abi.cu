// C ABI: context management, status strings, argument validation and gp_kmvm.
#include "gpk_internal.cuh"
#include "ptx.cuh"

#include <math.h>
#include <new>

using namespace gpk;


namespace {

// Makes the context's device current for the duration of a call and restores
// the caller's device afterwards.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = (prev == dev) || (cudaSetDevice(dev) == cudaSuccess);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// The bounded-wait path of the kernels, exercised on a wait that nothing
// completes: an mbarrier expecting one arrival that never comes.  Every lane
// waits with the helper the MVM kernels use (spin or hinted), gives up after
// the limit and lane 0 records DEV_TIMEOUT in the error word.
__global__ void wait_check_kernel(uint64_t limit_ns, int sleep, int* err, long long* waited_cycles) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    __syncwarp();
    const long long t0 = clock64();
    const bool ok = sleep ? ptx::mbar_wait_sleep(&bar, 0, limit_ns) : ptx::mbar_wait(&bar, 0, limit_ns);
    const long long t1 = clock64();
    if (threadIdx.x == 0) {
        if (!ok) atomicCAS(err, DEV_OK, DEV_TIMEOUT);
        if (waited_cycles) *waited_cycles = t1 - t0;
    }
}

}  // namespace

namespace gpk {

int check_hyp(const gp_hyp_t* hyp) {
    if (!hyp || !hyp->lengthscale) return GP_ERR_INVALID;
    if (hyp->kernel < GP_KERNEL_RBF || hyp->kernel > GP_KERNEL_MATERN52) return GP_ERR_INVALID;
    if (hyp->d < 1 || hyp->d > 64) return GP_ERR_INVALID;
    for (int k = 0; k < hyp->d; ++k) {
        const float l = hyp->lengthscale[k];
        if (!(l > 0.0f) || !isfinite(l)) return GP_ERR_INVALID;
    }
    if (!(hyp->outputscale > 0.0) || !isfinite(hyp->outputscale)) return GP_ERR_INVALID;
    if (!(hyp->noise >= 0.0) || !isfinite(hyp->noise)) return GP_ERR_INVALID;
    return GP_OK;
}

}  // namespace gpk

extern "C" {

const char* gp_strerror(int status) {
    switch (status) {
        case GP_OK: return "success";
        case GP_ERR_INVALID: return "invalid argument";
        case GP_ERR_CUDA: return "CUDA runtime or driver error";
        case GP_ERR_WORKSPACE: return "context workspace too small";
        case GP_ERR_BREAKDOWN: return "CG breakdown: an LSE sum was not positive";
        case GP_ERR_NONFINITE: return "non-finite value in an input or iterate";
        case GP_ERR_NOT_CONVERGED: return "CG did not reach the tolerance within max_iter";
        case GP_ERR_TIMEOUT: return "a bounded device-side wait ran out";
        case GP_ERR_OOM: return "device allocation failed";
        case GP_ERR_UNSUPPORTED: return "unsupported shape or option";
    }
    return "unknown status";
}

int gp_ctx_create(int device, size_t workspace_bytes, gp_ctx** out) {
    if (!out) return GP_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return GP_ERR_INVALID;
    DeviceGuard g(device);
    if (!g.ok) return GP_ERR_CUDA;
    gp_ctx* c = new (std::nothrow) gp_ctx();
    if (!c) return GP_ERR_OOM;
    c->device = device;
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        delete c;
        return GP_ERR_CUDA;
    }
    if (cudaMalloc((void**)&c->dev_err, 256) != cudaSuccess || cudaMemset(c->dev_err, 0, 256) != cudaSuccess ||
        cudaMallocHost((void**)&c->host_pinned, 4096) != cudaSuccess) {
        gp_ctx_destroy(c);
        return GP_ERR_OOM;
    }
    if (workspace_bytes > 0) {
        if (cudaMalloc(&c->ws, workspace_bytes) != cudaSuccess) {
            c->ws = nullptr;
            gp_ctx_destroy(c);
            return GP_ERR_OOM;
        }
        c->ws_bytes = workspace_bytes;
    }
    *out = c;
    return GP_OK;
}

void gp_ctx_destroy(gp_ctx* ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->dev_err) cudaFree(ctx->dev_err);
    if (ctx->prof_ev_ready)
        for (int i = 0; i < 2 * gpk::Ctx::kProfMax; ++i) cudaEventDestroy(ctx->prof_ev[i]);
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    delete ctx;
}

int gp_ctx_reserve(gp_ctx* ctx, size_t workspace_bytes) {
    if (!ctx) return GP_ERR_INVALID;
    if (workspace_bytes <= ctx->ws_bytes) return GP_OK;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GP_ERR_CUDA;
    if (cudaDeviceSynchronize() != cudaSuccess) return GP_ERR_CUDA;
    void* p = nullptr;
    if (cudaMalloc(&p, workspace_bytes) != cudaSuccess) return GP_ERR_OOM;
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = p;
    ctx->ws_bytes = workspace_bytes;
    return GP_OK;
}

size_t gp_ctx_workspace_bytes(const gp_ctx* ctx) { return ctx ? ctx->ws_bytes : 0; }

int64_t gp_ctx_launch_count(const gp_ctx* ctx) { return ctx ? ctx->launches : 0; }

int gp_wait_check(gp_ctx* ctx, double limit_ms, int sleep, long long* waited_cycles, void* stream) {
    if (!ctx || !(limit_ms > 0.0) || limit_ms > 1000.0) return GP_ERR_INVALID;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    long long* dw = nullptr;
    if (waited_cycles) {
        if (ctx->ws_bytes < 256) return GP_ERR_WORKSPACE;
        dw = (long long*)ctx->ws;
    }
    wait_check_kernel<<<1, 32, 0, s>>>((uint64_t)(limit_ms * 1e6), sleep ? 1 : 0, ctx->dev_err, dw);
    ctx->launches++;
    if (cudaGetLastError() != cudaSuccess) return GP_ERR_CUDA;
    if (waited_cycles) {
        if (cudaMemcpyAsync(waited_cycles, dw, sizeof(long long), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GP_ERR_CUDA;
    }
    return GP_OK;
}

int gp_ctx_check(gp_ctx* ctx, void* stream) {
    if (!ctx) return GP_ERR_INVALID;
    DeviceGuard g(ctx->device);
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaStreamSynchronize(s) != cudaSuccess) return GP_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GP_ERR_CUDA;
    if (v == DEV_OK) return GP_OK;
    if (cudaMemset(ctx->dev_err, 0, sizeof(int)) != cudaSuccess) return GP_ERR_CUDA;
    switch (v) {
        case DEV_TIMEOUT: return GP_ERR_TIMEOUT;
        case DEV_NONFINITE: return GP_ERR_NONFINITE;
        case DEV_BREAKDOWN: return GP_ERR_BREAKDOWN;
    }
    return GP_ERR_CUDA;
}

static int check_kmvm_args(const gp_hyp_t* hyp, int64_t Nr, int64_t Nc, int R, int flags) {
    GPK_TRY(check_hyp(hyp));
    if (Nr < 1 || Nc < 1 || Nr > (int64_t(1) << 31) - 256 || Nc > (int64_t(1) << 31) - 256) return GP_ERR_INVALID;
    if (R < 1 || R > 64) return GP_ERR_INVALID;
    return check_mvm_flags(flags, true);
}

size_t gp_kmvm_workspace_size(const gp_hyp_t* hyp, int64_t Nr, int64_t Nc, int R, int flags) {
    if (check_kmvm_args(hyp, Nr, Nc, R, flags) != GP_OK) return 0;
    gpk::Ctx probe;
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&probe.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) probe.num_sms = 148;
    // Worst case for the square flag (non-square needs the most).
    return kop_workspace(&probe, hyp, Nr, Nc, R, flags, false);
}

int gp_kmvm(gp_ctx* ctx, const gp_hyp_t* hyp, const float* Xr, int64_t Nr, const float* Xc, int64_t Nc,
            const float* V, int R, float* out, int flags, void* stream) {
    if (!ctx || !Xr || !Xc || !V || !out) return GP_ERR_INVALID;
    GPK_TRY(check_kmvm_args(hyp, Nr, Nc, R, flags));
    const bool add_noise = (flags & GP_MVM_ADD_NOISE) != 0;
    if (add_noise && (Xr != Xc || Nr != Nc)) return GP_ERR_INVALID;
    // out must not overlap V
    const char* vb = (const char*)V;
    const char* ve = vb + (size_t)Nc * R * sizeof(float);
    const char* ob = (const char*)out;
    const char* oe = ob + (size_t)Nr * R * sizeof(float);
    if (ob < ve && vb < oe) return GP_ERR_INVALID;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    WsCarver wc(ctx->ws, ctx->ws_bytes);
    KOp op;
    GPK_TRY(kop_prepare(ctx, wc, op, hyp, Xr, Nr, Xc, Nc, R, flags & ~GP_MVM_ADD_NOISE, s));
    return kop_apply(ctx, op, V, R, out, Nr, add_noise, s);
}

int gp_kmvm_tile_count(gp_ctx* ctx, const gp_hyp_t* hyp, const float* Xr, int64_t Nr, const float* Xc, int64_t Nc,
                       int flags, int64_t* evaluated, int64_t* total, void* stream) {
    if (!ctx || !Xr || !Xc || !evaluated || !total) return GP_ERR_INVALID;
    GPK_TRY(check_kmvm_args(hyp, Nr, Nc, 1, flags));
    if ((flags & 0xff) == GP_PREC_FP32) return GP_ERR_UNSUPPORTED;
    DeviceGuard g(ctx->device);
    if (!g.ok) return GP_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    WsCarver wc(ctx->ws, ctx->ws_bytes);
    KOp op;
    GPK_TRY(kop_prepare(ctx, wc, op, hyp, Xr, Nr, Xc, Nc, 1, flags & ~GP_MVM_ADD_NOISE, s));
    if (op.tp.engine != 1) return GP_ERR_UNSUPPORTED;
    *total = (int64_t)op.tp.n_it * op.tp.n_jt;
    if (!op.skip) {
        *evaluated = *total;
        return GP_OK;
    }
    unsigned long long c = 0;
    if (cudaMemcpyAsync(&c, op.skip_count, sizeof(c), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GP_ERR_CUDA;
    *evaluated = (int64_t)c;
    return GP_OK;
}

}  // extern "C"
