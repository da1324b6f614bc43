// gp_kmvm_noalloc: the kernel MVM of gp_kmvm for callers that cannot allocate
// device memory.
//
// Who needs this: code that runs where cudaMalloc is unavailable or not
// allowed -- inside a host application that owns the device memory through its
// own pool allocator and forbids side allocations, in latency-critical loops
// where an allocation (and the device synchronisation it may imply) is not
// acceptable, or in plugins that are handed device pointers but no context to
// allocate with.  Such callers cannot create a gp_ctx (which allocates its
// workspace), so this entry point takes no context and allocates nothing: its
// scratch (operand arrays, cast right-hand sides, split partial sums and the
// device error word) lives in one file-scope __device__ array of fixed size,
// which every GPU that loads the library holds until the process exits.
//
// The device address of that array is looked up once per device with
// cudaGetSymbolAddress (host code only holds a stand-in for the symbol).  That
// set-up happens during the first call on each device, so the first call on a
// device should come before any stream capture.  Every call shares the array:
// two calls whose work overlaps on the GPU (different streams, no ordering)
// race on it and corrupt each other's results.
#include "gpk_internal.cuh"

#include <mutex>

static __device__ __align__(256) unsigned char g_kmvm_noalloc_scratch[GPK_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 128;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set up once).
int scratch_address(int dev, void** out) {
    if (dev < 0 || dev >= kMaxDevices) return GP_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_kmvm_noalloc_scratch) != cudaSuccess || !p) return GP_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return GP_OK;
}

int check_args(const gp_hyp_t* hyp, const float* Xr, int64_t Nr, const float* Xc, int64_t Nc, const float* V,
               int R, const float* out, int flags) {
    if (!Xr || !Xc || !V || !out) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_hyp(hyp));
    if (Nr < 1 || Nc < 1 || Nr > (int64_t(1) << 31) - 256 || Nc > (int64_t(1) << 31) - 256) return GP_ERR_INVALID;
    if (R < 1 || R > 64) return GP_ERR_INVALID;
    GPK_TRY(gpk::check_mvm_flags(flags, true));   // the same flags as gp_kmvm
    if ((flags & GP_MVM_ADD_NOISE) && (Xr != Xc || Nr != Nc)) return GP_ERR_INVALID;
    const char* vb = (const char*)V;
    const char* ve = vb + (size_t)Nc * R * sizeof(float);
    const char* ob = (const char*)out;
    const char* oe = ob + (size_t)Nr * R * sizeof(float);
    if (ob < ve && vb < oe) return GP_ERR_INVALID;
    return GP_OK;
}

}  // namespace

extern "C" int gp_kmvm_noalloc(const gp_hyp_t* hyp, const float* Xr, int64_t Nr, const float* Xc, int64_t Nc,
                               const float* V, int R, float* out, int flags, void* stream) {
    GPK_TRY(check_args(hyp, Xr, Nr, Xc, Nc, V, R, out, flags));
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GP_ERR_CUDA;
    void* base = nullptr;
    GPK_TRY(scratch_address(dev, &base));
    cudaStream_t s = (cudaStream_t)stream;

    // A context on the stack: no device allocation, its workspace is the array.
    gpk::Ctx c;
    c.device = dev;
    if (cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GP_ERR_CUDA;
    c.dev_err = reinterpret_cast<int*>(base);                      // first 256 bytes: error word
    c.ws = static_cast<unsigned char*>(base) + 256;
    c.ws_bytes = GPK_NOALLOC_SCRATCH_BYTES - 256;

    const bool square = (Xr == Xc && Nr == Nc);
    const int mvm_flags = flags & ~GP_MVM_ADD_NOISE;
    if (gpk::kop_workspace(&c, hyp, Nr, Nc, R, mvm_flags, square) > c.ws_bytes) return GP_ERR_WORKSPACE;

    // The array keeps the previous call's contents: the error word must start at 0.
    if (cudaMemsetAsync(c.dev_err, 0, sizeof(int), s) != cudaSuccess) return GP_ERR_CUDA;
    gpk::WsCarver wc(c.ws, c.ws_bytes);
    gpk::KOp op;
    GPK_TRY(gpk::kop_prepare(&c, wc, op, hyp, Xr, Nr, Xc, Nc, R, mvm_flags, s));
    return gpk::kop_apply(&c, op, V, R, out, Nr, (flags & GP_MVM_ADD_NOISE) != 0, s);
}

extern "C" int gp_kmvm_noalloc_check(void* stream) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GP_ERR_CUDA;
    void* base = nullptr;
    GPK_TRY(scratch_address(dev, &base));
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return GP_ERR_CUDA;
    int v = 0;
    if (cudaMemcpy(&v, base, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GP_ERR_CUDA;
    if (v == gpk::DEV_OK) return GP_OK;
    if (cudaMemset(base, 0, sizeof(int)) != cudaSuccess) return GP_ERR_CUDA;
    switch (v) {
        case gpk::DEV_TIMEOUT: return GP_ERR_TIMEOUT;
        case gpk::DEV_NONFINITE: return GP_ERR_NONFINITE;
        case gpk::DEV_BREAKDOWN: return GP_ERR_BREAKDOWN;
    }
    return GP_ERR_CUDA;
}
