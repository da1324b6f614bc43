// Internal declarations shared by the translation units of libgpk.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/gpk.h"

namespace gpk {

// ----------------------------------------------------------------------------
// Host-side context
// ----------------------------------------------------------------------------
struct Ctx {
    int device = 0;
    int num_sms = 0;
    void* ws = nullptr;           // device workspace
    size_t ws_bytes = 0;
    int* dev_err = nullptr;       // device error word (own allocation, 64 B)
    int* host_pinned = nullptr;   // pinned host scratch (flags, small readbacks), 4 KB
    int64_t launches = 0;         // kernels launched through this context
    // CUDA-event timing of the tensor-core MVM launches (gp_ctx_profile)
    static constexpr int kProfMax = 8192;
    bool prof = false;
    bool prof_ev_ready = false;
    int prof_n = 0;
    cudaEvent_t prof_ev[2 * kProfMax];
};
void prof_begin(Ctx* ctx, cudaStream_t s);
void prof_end(Ctx* ctx, cudaStream_t s);

// Bump allocator over the context workspace (alignment 256 B).
struct WsCarver {
    uint8_t* base;
    size_t cap;
    size_t off = 0;
    bool ok = true;
    WsCarver(void* b, size_t c) : base((uint8_t*)b), cap(c) {}
    template <class T> T* take(size_t count) {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (off + bytes > cap) { ok = false; return nullptr; }
        T* p = (T*)(base + off);
        off += bytes;
        return p;
    }
};
// Size-only variant of the carver (for *_workspace_size queries).
struct WsCounter {
    size_t off = 0;
    template <class T> void take(size_t count) { off += (count * sizeof(T) + 255) & ~size_t(255); }
};

#define GPK_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e__ = (expr);                            \
        if (e__ != cudaSuccess) return GP_ERR_CUDA;          \
    } while (0)

#define GPK_TRY(expr)                                        \
    do {                                                     \
        int s__ = (expr);                                    \
        if (s__ != GP_OK) return s__;                        \
    } while (0)

// Device error word codes (written by kernels with atomicCAS from 0).
enum DevErr : int {
    DEV_OK = 0,
    DEV_TIMEOUT = 1,      // bounded mbarrier wait ran out
    DEV_NONFINITE = 2,    // non-finite operand scale
    DEV_BREAKDOWN = 3,
};

// Wait limit for device-side spins (nanoseconds; counted in SM clock cycles).
constexpr uint64_t kWaitLimitNs = 1000000000ull;   // 1 s

// ----------------------------------------------------------------------------
// Operand preparation: scaled inputs, norms, V scaling / casting.
// ----------------------------------------------------------------------------
struct OperandLayout {
    int prec = 0;    // GP_PREC_FP16 / GP_PREC_BF16
    int xsplit = 0;  // 1: inputs carried as hi + lo
    int nt = 0;      // number of terms carrying t = -|x|^2/2
    int kdim = 0;    // used columns of the contraction dimension
    int k_pad = 0;   // 16, 32 or 64 (0: does not fit)
    int vsplit = 0;  // 1: right-hand sides carried as hi + lo (extra P.V product)
    int psplit = 0;  // 1: kernel tile carried as hi + lo (extra P.V product; BF16)
    int half_exp = 0;  // 1: S rounded to FP16 by the MMA, 2^s in FP16 (RBF, FP16, k_pad 16)
    int fp32_pv = 0;   // 1: value product in FP32 on the epilogue threads (FP16, pair engine, R <= 4)
};
OperandLayout make_layout(int d, int prec, int xsplit, int vsplit, int psplit);
float kernel_input_scale(int kernel);   // c such that x_hat = c x / l

// Per-dimension input scales c / l_k, passed to kernels by value.
struct ScaleVec {
    float v[64];
};

// Launchers (return GP_OK or GP_ERR_CUDA).  All on `stream`.
// XA / XB may be null (that side is not written).
// bb: bounding box from launch_bbox (the inputs are centred on its midpoint,
// which leaves a stationary kernel unchanged and keeps |x^| small).
int launch_prep_x(Ctx* ctx, const OperandLayout& L, const float* X, int64_t N, int64_t N_pad, int d,
                  const ScaleVec& inv, const unsigned* bb, void* XA, void* XB, cudaStream_t s);
// Per-dimension min / max of X (N x d) as order-preserving integer codes:
// bb[k] = min, bb[d + k] = max.  Deterministic (atomic min / max).
int launch_bbox(Ctx* ctx, const float* X, int64_t N, int d, unsigned* bb, cudaStream_t s);
int launch_prep_x_f32(Ctx* ctx, const float* X, int64_t N, int64_t N_pad, int d, int dp, const ScaleVec& inv,
                      float* Xs, cudaStream_t s);
int launch_v_colmax(Ctx* ctx, const float* V, int64_t N, int R, unsigned* cmax_bits, cudaStream_t s);
int launch_v_pack32(Ctx* ctx, const float* V, int64_t N, int64_t N_pad, int R, const unsigned* cmax_bits,
                    double outputscale, float* V32, float* outscale, cudaStream_t s);
// Vt rows: [0, R_pad) the (hi) cast, [R_pad, 2 R_pad) the lo parts when vsplit.
int launch_v_cast(Ctx* ctx, int prec, int scale_mode, int vsplit, const float* V, int64_t N, int64_t N_pad, int R,
                  int R_pad, const unsigned* cmax_bits, double outputscale, void* Vt, float* outscale,
                  cudaStream_t s);

// ----------------------------------------------------------------------------
// MVM engines
// ----------------------------------------------------------------------------
struct MvmArgs {
    int kernel;
    int64_t Nr, Nc;
    int R;
    float noise;               // sigma^2 added as noise * Vnoise (0: none)
    const float* Vnoise;       // FP32 V for the noise term (Nc x R col-major) or null
    float* out;                // Nr x R col-major
    int64_t ld_out;
    float diag_coef = 0.0f;    // square operator: the exact a^2 v_i of the diagonal is
                               // added here and the on-chip diagonal is skipped
};

// Tensor-core engine (kmvm_tc.cu).
struct TcPlan {
    int n_it = 0, n_jt = 0, n_split = 1, grid = 0, R_pad = 0, k_pad = 0;
    int64_t Nr_pad = 0, Nc_pad = 0;
    int engine = 0;   // 0: one row tile per item (kmvm_tc.cu); 1: row-tile pairs, transposed P.V (kmvm_tp.cu)
    int rv = 0;       // engine 1: rows of Vt per tile (R_pad, or 2 R_pad with the hi + lo split)
};
TcPlan tc_plan(const Ctx* ctx, int64_t Nr, int64_t Nc, int R, int k_pad);
int tc_smem_bytes(int k_pad, int R_pad, int vsplit);
int tc_stages(int k_pad, int R_pad, int vsplit);
size_t tc_partial_floats(const TcPlan& p);
int launch_kmvm_tc(Ctx* ctx, const TcPlan& plan, const OperandLayout& L, const MvmArgs& a, const CUtensorMap& tmA,
                   const CUtensorMap& tmB, const CUtensorMap& tmV, const float* outscale, float* partial,
                   cudaStream_t s);

// Tensor-core engine with the transposed value product (kmvm_tp.cu).  n_it
// counts pairs of 128-row tiles; the partial buffer is always used.
bool tp_supported(int k_pad, int R_pad, int vsplit, int psplit);
TcPlan tp_plan(const Ctx* ctx, int64_t Nr, int64_t Nc, int R, int k_pad, int vsplit);
size_t tp_partial_floats(const TcPlan& p);
int launch_kmvm_tp(Ctx* ctx, const TcPlan& plan, const OperandLayout& L, const MvmArgs& a, const CUtensorMap& tmA,
                   const CUtensorMap& tmB, const CUtensorMap& tmV, const float* outscale, float* partial,
                   const uint32_t* mask, cudaStream_t s);

// SIMT FP32 engine (kmvm_simt.cu).  Scaled FP32 inputs with row stride dp.
struct SimtPlan {
    int dp = 0, R_pad = 0, n_rowblk = 0, n_split = 1;
};
SimtPlan simt_plan(const Ctx* ctx, int64_t Nr, int64_t Nc, int d, int R);
size_t simt_partial_floats(const SimtPlan& p, int64_t Nr);
int launch_kmvm_simt(Ctx* ctx, const SimtPlan& plan, const MvmArgs& a, float outputscale, const float* Xrs,
                     const float* Xcs, const float* V, float* partial, cudaStream_t s);

// Symmetric half-work FP32 engine (kmvm_sym.cu): square operator, R <= 24.
int launch_kmvm_sym(Ctx* ctx, const MvmArgs& a, float outputscale, const float* Xs, int dp, const float* V,
                    cudaStream_t s);

// Summation-variant study engine (kmvm_sum.cu): CUDA-core FP16 products,
// accumulation scheme 1..4 (GP_MVM_SUM), R <= 8, scaled inputs as the SIMT engine's.
int launch_kmvm_sum(Ctx* ctx, int scheme, const MvmArgs& a, float outputscale, const float* Xrs, const float* Xcs,
                    int dp, const float* V, const unsigned* cmax_bits, cudaStream_t s);

// out[c][i] = scale_c * sum_s partial[s][c][i] + noise * Vnoise[c][i], with
// partial laid out [n_split][RP][ld_part]; scale_c = outscale[c] or outscale_const.
int launch_split_reduce(Ctx* ctx, const float* partial, int n_split, int64_t ld_part, int64_t Nr, int R, int RP,
                        const float* outscale, float outscale_const, float noise, const float* Vnoise,
                        int64_t ld_v, float* out, int64_t ld_out, cudaStream_t s);

// Prepared kernel-MVM operator (mvm.cu): the input side is prepared once,
// every apply casts V and runs the engine.
struct KOp {
    int kernel = 0, prec = 0, flags = 0, d = 0, R_max = 0;
    bool square = false;
    int64_t Nr = 0, Nc = 0;
    float a2 = 1.0f, noise = 0.0f;
    OperandLayout lay;
    TcPlan tp;
    SimtPlan sp;
    void* XA = nullptr;
    void* XB = nullptr;
    float* Xs_r = nullptr;
    float* Xs_c = nullptr;
    void* Vt = nullptr;
    float* outscale = nullptr;
    unsigned* cmax = nullptr;
    unsigned* bbox = nullptr;
    float* partial = nullptr;
    CUtensorMap tmA, tmB, tmV;
    int sum = 0;   // summation-variant study scheme (GP_MVM_SUM), 0 = none
    bool sym = false;   // symmetric half-work FP32 MVM (GP_MVM_SYMMETRIC)
    // compact-support tile skipping (GP_MVM_SKIP_TILES, pair engine)
    bool skip = false;
    uint32_t* mask = nullptr;
    float* rbox = nullptr;
    float* cbox = nullptr;
    unsigned long long* skip_count = nullptr;
};
size_t kop_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t Nr, int64_t Nc, int R, int flags, bool square);
int kop_prepare(Ctx* ctx, WsCarver& wc, KOp& op, const gp_hyp_t* hyp, const float* Xr, int64_t Nr,
                const float* Xc, int64_t Nc, int R, int flags, cudaStream_t s);
// out = K(Xr, Xc) V (+ sigma^2 V if add_noise); V: Nc x R (ld Nc), out: Nr x R (ld ld_out).
int kop_apply(Ctx* ctx, KOp& op, const float* V, int R, float* out, int64_t ld_out, bool add_noise, cudaStream_t s);

// Tensor-map helper (driver entry point fetched through the runtime).
int encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                   uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz);

// Tile skipping (skip.cu): -s*, the mask's size in words, and its preparation
// (bounding boxes of the operand tiles, then the mask and its popcount).
double skip_threshold(int kernel, int prec);
size_t skip_words(const TcPlan& p);
int prepare_skip(Ctx* ctx, KOp& op, cudaStream_t s);

// Hyperparameter validation shared by the entry points.
int check_hyp(const gp_hyp_t* hyp);
// MVM precision / option flags (GP_PREC_* | GP_MVM_*) accepted by every entry
// point that takes them; GP_MVM_ADD_NOISE only where allow_noise.
int check_mvm_flags(int flags, bool allow_noise);

// ---- preconditioner (precond.cu) ----
size_t pivchol_workspace(const Ctx* ctx, int64_t N, int d, int rank);
// rank_out_host null: asynchronous form (no host sync; L zeroed first and the
// core built at the full width `rank`).
int pivchol_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, int rank, float* L,
                int32_t* piv, double* core, int* rank_out_host, cudaStream_t s);
size_t woodbury_workspace(const Ctx* ctx, int64_t N, int k, int R);
// cinv (k x k FP64) = C^{-1} from the core factor, once per preconditioner use.
int woodbury_prepare(Ctx* ctx, const double* core, int k, double* cinv, cudaStream_t s);
// Z = P^{-1} W on the active columns (active may be null = all).  cinv from
// woodbury_prepare, or null to form it in the call's own scratch.
int woodbury_apply(Ctx* ctx, WsCarver& wc, const float* L, const double* core, const double* cinv, int k,
                   double noise, int64_t N, const float* W, int R, const int* active, float* Z, cudaStream_t s);

// ---- solver (cg.cu), backward (vjp.cu), loss (mll.cu) ----
size_t cg_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t N, int R, int rank, const gp_cg_opts_t* o);

// Per-column state of the solver (device memory).
struct ColState {
    double gamma_s;     // r^T z = gamma_s 2^gamma_e (the LSE form: log r^T z = log gamma_s + gamma_e log 2)
    double gamma;       // r^T z (Alg. 1)
    double alpha, beta;
    double bnorm, rnorm, relres;
    double gamma0;      // r_0^T z_0 (the SLQ quadrature weight ||P^{-1/2} r_0||^2)
    int active;
    int iters;
    int breakdown;
    int gamma_e;
};

struct CgBufs {
    float *r, *z, *d, *Kd, *rho, *zeta;
    double *dpart, *gpart, *coef, *ahist, *bhist, *rhist;
    ColState* st;
    int* nact;
    int* aflags;
    int* len0;   // per-column iterations of the first (unrestarted) run
    double* cinv;  // C^{-1} of the Woodbury core (rank > 0)
    int nb_max, nblk_dot;
};

// Step-able solver.  setup() enqueues the set-up phase; every phase ends with
// an asynchronous copy of the number of still-active columns to *flag_host
// and, when ev is given, an event record.  Once that phase has completed
// (wait() or an event query), step() reads the flag and enqueues the next
// phase or reports the solve done.  No call blocks except wait() and finish().
struct CgSolver {
    Ctx* ctx = nullptr;
    cudaStream_t s = nullptr;
    gp_hyp_t hyp{};
    const float* X = nullptr;
    const float* B = nullptr;
    float* U = nullptr;
    int64_t N = 0;
    int R = 0;
    gp_cg_opts_t o{};
    gp_precond_t pc{};
    int rank = 0, stable = 0, reorth = 0, passes = 1, vg = 1;
    CgBufs b{};
    KOp op, op_chk_own, op_ref_own;
    KOp* op_chk = nullptr;
    KOp* op_ref = nullptr;   // iterations after the first true-residual check (refine_precision)
    WsCarver wc_rest{nullptr, 0};
    int* flag_host = nullptr;
    cudaEvent_t ev = nullptr;
    int k = 0, nb0 = 0, restarts = 0, iters = 0;
    bool last_check = false, len_recorded = false, escalated = false, refined = false;
    bool relax_off = false;   // the relaxed MVM stalled and was given up for this solve
    int k_sw = 0;             // iteration of the switch to the refine MVM
    float r_sw = 0.0f;        // largest active residual at the switch

    int setup(Ctx* c, WsCarver& wc, const gp_hyp_t* h, const float* X, int64_t N, const float* B, int R, float* U,
              const gp_precond_t* pc, const gp_cg_opts_t* o, cudaStream_t s, int* flag_host, cudaEvent_t ev);
    int wait();                   // block until the last enqueued phase has completed
    int step(bool* done);         // enqueue the next phase (or report done)
    int enqueue_state(ColState* host_st);   // asynchronous D2H of the per-column states
    // Summary from states copied by enqueue_state; returns the solve's status.
    int summarize(const ColState* hs, gp_cg_stats_t* stats) const;
    int finish(gp_cg_stats_t* stats);        // blocking: copy back, summarize

  private:
    int launched(int n);
    int flag_copy();
    int precond(const float* W, float* Z, bool masked);
    int dots(const float* A, const float* Bv, bool masked);
    int scalar(int mode, int kk);
    int start(bool from_x, int k0);
    int iterate();
};

int cg_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, const float* B, int R,
           float* U, const gp_precond_t* pc, const gp_cg_opts_t* o, gp_cg_stats_t* stats, cudaStream_t s);
size_t vjp_workspace(int64_t N, int d, int R);
int vjp_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U, const float* W,
            int R, double* grad_theta_host, float* gX_dev, cudaStream_t s);
int launch_scale_cols(Ctx* ctx, const float* src, int64_t N, int dp, int d, const float* ls_host, float* dst,
                      cudaStream_t s);
// Tensor-core backward (vjp_tc.cu): RBF / Matern-3/2 / Matern-5/2, d <= 31, R <= 32,
// FP16 operands with FP32 accumulation.
bool vjp_tc_supported(const gp_hyp_t* hyp, int R);
size_t vjp_tc_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t N, int R);
int vjp_tc_run(Ctx* ctx, WsCarver& wc, const gp_hyp_t* hyp, const float* X, int64_t N, const float* U,
               const float* W, int R, double* grad_theta_host, float* gX_dev, cudaStream_t s);
int slq_quadrature_host(const double* alpha, const double* beta, int J, double gamma0, double* out);

}  // namespace gpk

// The opaque handle of the C ABI is the context itself.
struct gp_ctx : public gpk::Ctx {};
