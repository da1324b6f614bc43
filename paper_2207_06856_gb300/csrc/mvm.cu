// Kernel-MVM operator: prepares the input-side operands once and applies
// K(Xr, Xc) V (+ sigma^2 V) any number of times.  Used by gp_kmvm and by
// every solver, so the MVM inside CG is exactly the MVM that gp_kmvm exposes.
#include "gpk_internal.cuh"

#include <math.h>
#include <string.h>

namespace gpk {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

CUtensorMapSwizzle swizzle_for_row_bytes(uint32_t row_bytes) {
    return row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                           : (row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
}
// Rows wider than 128 bytes are loaded as several 128-byte swizzle atoms.
uint32_t atom_row_bytes(int k_pad) { return (uint32_t)(k_pad * 2 < 128 ? k_pad * 2 : 128); }

}  // namespace

int encode_tmap_2d(CUtensorMap* map, CUtensorMapDataType dt, const void* base, uint64_t inner, uint64_t outer,
                   uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return GP_ERR_CUDA;
    cuuint64_t dims[2] = {inner, outer};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_outer};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? GP_OK : GP_ERR_CUDA;
}

// Allocation plan of a KOp, shared by the size query and the real carve so the
// two can never disagree.
template <class A>
static void kop_layout(A& a, KOp& op, int64_t Nr, int64_t Nc, int R_max, bool square) {
    if (op.sum) {
        a.template take<float>((size_t)Nr * op.sp.dp);
        if (!square) a.template take<float>((size_t)Nc * op.sp.dp);
        a.template take<unsigned>(64);
    } else if (op.prec == GP_PREC_FP32) {
        a.template take<float>((size_t)Nr * op.sp.dp);
        if (!square) a.template take<float>((size_t)Nc * op.sp.dp);
        a.template take<float>(simt_partial_floats(op.sp, Nr));
    } else {
        a.template take<uint16_t>((size_t)op.tp.Nr_pad * op.lay.k_pad);
        a.template take<uint16_t>((size_t)op.tp.Nc_pad * op.lay.k_pad);
        const int rp = ((R_max + 15) / 16) * 16;
        a.template take<uint16_t>((size_t)(op.lay.vsplit ? 2 : 1) * rp * op.tp.Nc_pad);
        a.template take<float>(64);
        a.template take<unsigned>(64);
        a.template take<unsigned>(128);
        a.template take<float>(op.tp.engine == 1 ? tp_partial_floats(op.tp)
                                                  : (size_t)op.tp.n_split * rp * op.tp.Nr_pad);
        if (op.skip) {
            a.template take<uint32_t>(skip_words(op.tp));
            a.template take<float>((size_t)((Nr + 127) / 128) * 2 * op.d);
            a.template take<float>((size_t)op.tp.n_jt * 2 * op.d);
            a.template take<unsigned long long>(1);
        }
    }
}

int check_mvm_flags(int flags, bool allow_noise) {
    const int prec = flags & 0xff;
    if (prec != GP_PREC_FP32 && prec != GP_PREC_FP16 && prec != GP_PREC_BF16) return GP_ERR_INVALID;
    const int known = 0xff | GP_MVM_ADD_NOISE | GP_MVM_XSPLIT | GP_MVM_NO_XSPLIT | GP_MVM_SCALE_SQRT_N |
                      GP_MVM_VSPLIT | GP_MVM_BF16_SINGLE | GP_MVM_ONE_TILE | GP_MVM_PSPLIT | GP_MVM_HALF_EXP |
                      GP_MVM_SKIP_TILES | GP_MVM_SUM_MASK | GP_MVM_SYMMETRIC | GP_MVM_FP32_PV;
    if ((flags & GP_MVM_SYMMETRIC) && prec != GP_PREC_FP32) return GP_ERR_INVALID;
    if ((flags & GP_MVM_FP32_PV) && prec != GP_PREC_FP16) return GP_ERR_INVALID;
    const int sum = (flags & GP_MVM_SUM_MASK) >> 18;
    if (sum > 4 || (sum && prec != GP_PREC_FP16)) return GP_ERR_INVALID;
    if (flags & ~known) return GP_ERR_INVALID;
    if (!allow_noise && (flags & GP_MVM_ADD_NOISE)) return GP_ERR_INVALID;
    if ((flags & GP_MVM_XSPLIT) && (flags & GP_MVM_NO_XSPLIT)) return GP_ERR_INVALID;
    return GP_OK;
}

static int kop_plan(const Ctx* ctx, KOp& op, const gp_hyp_t* hyp, int64_t Nr, int64_t Nc, int R, int flags) {
    op.kernel = hyp->kernel;
    op.d = hyp->d;
    op.prec = flags & 0xff;
    op.flags = flags;
    op.Nr = Nr;
    op.Nc = Nc;
    op.a2 = (float)hyp->outputscale;
    op.noise = (float)hyp->noise;
    op.R_max = R;
    op.sum = (flags & GP_MVM_SUM_MASK) >> 18;
    if (op.sum) {
        // summation-variant study: the CUDA-core FP16 engine on the SIMT engine's scaled inputs
        if (R > 8 || (flags & (GP_MVM_SKIP_TILES | GP_MVM_HALF_EXP | GP_MVM_PSPLIT | GP_MVM_ONE_TILE | GP_MVM_FP32_PV)))
            return GP_ERR_UNSUPPORTED;
        op.sp = simt_plan(ctx, Nr, Nc, hyp->d, R);
        if (op.sp.dp > 32) return GP_ERR_UNSUPPORTED;
    } else if (op.prec == GP_PREC_FP32) {
        // the FP32 engine has no kernel tile to round: these options do not apply
        if (flags & (GP_MVM_SKIP_TILES | GP_MVM_HALF_EXP)) return GP_ERR_UNSUPPORTED;
        op.sp = simt_plan(ctx, Nr, Nc, hyp->d, R < 32 ? R : 32);
        if (flags & GP_MVM_SYMMETRIC) {
            if (Nr != Nc || R > 24 || op.sp.dp > 32) return GP_ERR_UNSUPPORTED;
            op.sym = true;
        }
    } else if (op.prec == GP_PREC_FP16 || op.prec == GP_PREC_BF16) {
        const bool bf = op.prec == GP_PREC_BF16;
        // Inputs carried as hi + lo by default for BF16 (8-bit significand), for
        // FP16 beyond 12 dimensions, where one rounding of |x^| ~ sqrt(d)
        // moves the distances by a relative 2^-12 sqrt(d), and for FP16
        // whenever the split fits in the same contraction width (d <= 4: the
        // S product costs the same, and close pairs keep their distances).
        int xsplit = (flags & GP_MVM_XSPLIT) ? 1 : 0;
        const bool free_split = make_layout(hyp->d, op.prec, 1, 0, 0).k_pad == make_layout(hyp->d, op.prec, 0, 0, 0).k_pad;
        if (!(flags & GP_MVM_NO_XSPLIT) && (bf || hyp->d > 12 || free_split)) xsplit = 1;
        if (flags & GP_MVM_NO_XSPLIT) xsplit = 0;
        if (xsplit && make_layout(hyp->d, op.prec, 1, 0, 0).k_pad == 0) xsplit = 0;   // does not fit
        const int single = (flags & GP_MVM_BF16_SINGLE) ? 1 : 0;
        int vsplit = bf ? !single : ((flags & GP_MVM_VSPLIT) ? 1 : 0);
        int psplit = bf ? !single : 0;
        const int Rc = R < 64 ? R : 64;
        const int Rp = ((Rc + 15) / 16) * 16;
        const OperandLayout probe = make_layout(hyp->d, op.prec, xsplit, 1, psplit);
        // Pair engine (transposed value product) unless asked otherwise or the
        // operands do not fit its shared-memory plan.  There FP16 carries v as
        // hi + lo (the lo rows share the MMA's M dimension) and, with
        // GP_MVM_PSPLIT, the kernel tile as hi + lo too.
        const int want_psplit = bf ? psplit : ((flags & GP_MVM_PSPLIT) ? 1 : 0);
        const bool pair = !(flags & GP_MVM_ONE_TILE) && probe.k_pad != 0 &&
                          tp_supported(probe.k_pad, Rp, bf ? vsplit : 1, want_psplit);
        if (pair && !bf) {
            vsplit = 1;
            psplit = want_psplit;
        }
        op.lay = make_layout(hyp->d, op.prec, xsplit, vsplit, psplit);
        if (op.lay.k_pad == 0) return GP_ERR_UNSUPPORTED;
        if (flags & GP_MVM_SKIP_TILES) {
            if (!pair) return GP_ERR_UNSUPPORTED;
            op.skip = true;
        }
        if (flags & GP_MVM_HALF_EXP) {
            if (bf || !pair || psplit || op.lay.k_pad != 16 || hyp->kernel != GP_KERNEL_RBF) return GP_ERR_UNSUPPORTED;
            op.lay.half_exp = 1;
        }
        if (flags & GP_MVM_FP32_PV) {
            if (bf || !pair || psplit || op.lay.half_exp || R > 4) return GP_ERR_UNSUPPORTED;
            op.lay.fp32_pv = 1;
        }
        op.tp = pair ? tp_plan(ctx, Nr, Nc, Rc, op.lay.k_pad, vsplit) : tc_plan(ctx, Nr, Nc, Rc, op.lay.k_pad);
    } else {
        return GP_ERR_INVALID;
    }
    return GP_OK;
}

size_t kop_workspace(const Ctx* ctx, const gp_hyp_t* hyp, int64_t Nr, int64_t Nc, int R, int flags, bool square) {
    KOp op;
    if (kop_plan(ctx, op, hyp, Nr, Nc, R, flags) != GP_OK) return 0;
    WsCounter c;
    kop_layout(c, op, Nr, Nc, R, square);
    return c.off;
}

int kop_prepare(Ctx* ctx, WsCarver& wc, KOp& op, const gp_hyp_t* hyp, const float* Xr, int64_t Nr,
                const float* Xc, int64_t Nc, int R, int flags, cudaStream_t s) {
    GPK_TRY(kop_plan(ctx, op, hyp, Nr, Nc, R, flags));
    const bool square = (Xr == Xc && Nr == Nc);
    op.square = square;
    ScaleVec inv;
    memset(&inv, 0, sizeof(inv));
    const float c = kernel_input_scale(hyp->kernel);
    if (op.sum) {
        for (int k = 0; k < hyp->d; ++k) inv.v[k] = (float)((double)c / sqrt(2.0) / (double)hyp->lengthscale[k]);
        op.Xs_r = wc.take<float>((size_t)Nr * op.sp.dp);
        op.Xs_c = square ? op.Xs_r : wc.take<float>((size_t)Nc * op.sp.dp);
        op.cmax = wc.take<unsigned>(64);
        if (!wc.ok) return GP_ERR_WORKSPACE;
        GPK_TRY(launch_prep_x_f32(ctx, Xr, Nr, Nr, hyp->d, op.sp.dp, inv, op.Xs_r, s));
        if (!square) GPK_TRY(launch_prep_x_f32(ctx, Xc, Nc, Nc, hyp->d, op.sp.dp, inv, op.Xs_c, s));
        return GP_OK;
    }
    if (op.prec == GP_PREC_FP32) {
        // SIMT engine: q = |x^_i - x^_j|^2 with x^ = (c / sqrt2) x / l, so s = -q.
        for (int k = 0; k < hyp->d; ++k) inv.v[k] = (float)((double)c / sqrt(2.0) / (double)hyp->lengthscale[k]);
        op.Xs_r = wc.take<float>((size_t)Nr * op.sp.dp);
        op.Xs_c = square ? op.Xs_r : wc.take<float>((size_t)Nc * op.sp.dp);
        op.partial = wc.take<float>(simt_partial_floats(op.sp, Nr));
        if (!wc.ok) return GP_ERR_WORKSPACE;
        GPK_TRY(launch_prep_x_f32(ctx, Xr, Nr, Nr, hyp->d, op.sp.dp, inv, op.Xs_r, s));
        if (!square) GPK_TRY(launch_prep_x_f32(ctx, Xc, Nc, Nc, hyp->d, op.sp.dp, inv, op.Xs_c, s));
        return GP_OK;
    }
    for (int k = 0; k < hyp->d; ++k) inv.v[k] = (float)((double)c / (double)hyp->lengthscale[k]);
    op.XA = wc.take<uint16_t>((size_t)op.tp.Nr_pad * op.lay.k_pad);
    op.XB = wc.take<uint16_t>((size_t)op.tp.Nc_pad * op.lay.k_pad);
    const int rp = ((op.R_max + 15) / 16) * 16;
    op.Vt = wc.take<uint16_t>((size_t)(op.lay.vsplit ? 2 : 1) * rp * op.tp.Nc_pad);
    op.outscale = wc.take<float>(64);
    op.cmax = wc.take<unsigned>(64);
    op.bbox = wc.take<unsigned>(128);
    op.partial = wc.take<float>(op.tp.engine == 1 ? tp_partial_floats(op.tp)
                                                  : (size_t)op.tp.n_split * rp * op.tp.Nr_pad);
    if (op.skip) {
        op.mask = wc.take<uint32_t>(skip_words(op.tp));
        op.rbox = wc.take<float>((size_t)((Nr + 127) / 128) * 2 * op.d);
        op.cbox = wc.take<float>((size_t)op.tp.n_jt * 2 * op.d);
        op.skip_count = wc.take<unsigned long long>(1);
    }
    if (!wc.ok) return GP_ERR_WORKSPACE;
    GPK_TRY(launch_bbox(ctx, Xc, Nc, hyp->d, op.bbox, s));
    if (square) {
        GPK_TRY(launch_prep_x(ctx, op.lay, Xr, Nr, op.tp.Nr_pad, hyp->d, inv, op.bbox, op.XA, op.XB, s));
    } else {
        GPK_TRY(launch_prep_x(ctx, op.lay, Xr, Nr, op.tp.Nr_pad, hyp->d, inv, op.bbox, op.XA, nullptr, s));
        GPK_TRY(launch_prep_x(ctx, op.lay, Xc, Nc, op.tp.Nc_pad, hyp->d, inv, op.bbox, nullptr, op.XB, s));
    }
    const CUtensorMapDataType dt =
        op.prec == GP_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    const uint32_t rowb = (uint32_t)op.lay.k_pad * 2u;
    const uint32_t arb = atom_row_bytes(op.lay.k_pad);
    GPK_TRY(encode_tmap_2d(&op.tmA, dt, op.XA, op.lay.k_pad, op.tp.Nr_pad, rowb, arb / 2, 128,
                           swizzle_for_row_bytes(arb)));
    GPK_TRY(encode_tmap_2d(&op.tmB, dt, op.XB, op.lay.k_pad, op.tp.Nc_pad, rowb, arb / 2, 128,
                           swizzle_for_row_bytes(arb)));
    if (op.skip) GPK_TRY(prepare_skip(ctx, op, s));
    return GP_OK;
}

int kop_apply(Ctx* ctx, KOp& op, const float* V, int R, float* out, int64_t ld_out, bool add_noise, cudaStream_t s) {
    if (R > op.R_max) return GP_ERR_INVALID;
    const int maxc = op.prec == GP_PREC_FP32 ? 32 : 64;
    for (int c0 = 0; c0 < R; c0 += maxc) {
        const int rc = (R - c0) < maxc ? (R - c0) : maxc;
        MvmArgs a;
        a.kernel = op.kernel;
        a.Nr = op.Nr;
        a.Nc = op.Nc;
        a.R = rc;
        a.noise = add_noise ? op.noise : 0.0f;
        a.Vnoise = V + (int64_t)c0 * op.Nc;
        a.out = out + (int64_t)c0 * ld_out;
        a.ld_out = ld_out;
        // exp(-r) (Matern-1/2) is not smooth at r = 0, where the rounding of the
        // on-chip distance would show; its diagonal is added exactly instead.
        a.diag_coef = (op.square && op.prec != GP_PREC_FP32 && op.kernel == GP_KERNEL_MATERN12) ? op.a2 : 0.0f;
        const float* Vc = V + (int64_t)c0 * op.Nc;
        if (op.sum) {
            GPK_TRY(launch_v_colmax(ctx, Vc, op.Nc, rc, op.cmax, s));
            GPK_TRY(launch_kmvm_sum(ctx, op.sum, a, op.a2, op.Xs_r, op.Xs_c, op.sp.dp, Vc, op.cmax, s));
        } else if (op.sym) {
            if (!op.square) return GP_ERR_UNSUPPORTED;
            GPK_TRY(launch_kmvm_sym(ctx, a, op.a2, op.Xs_r, op.sp.dp, Vc, s));
        } else if (op.prec == GP_PREC_FP32) {
            SimtPlan pl = op.sp;
            pl.R_pad = ((rc + 3) / 4) * 4;   // <= the plan's, which sized the partial buffer
            GPK_TRY(launch_kmvm_simt(ctx, pl, a, op.a2, op.Xs_r, op.Xs_c, Vc, op.partial, s));
        } else {
            TcPlan pl = op.tp;
            pl.R_pad = ((rc + 15) / 16) * 16;
            if (pl.engine == 1) pl.rv = pl.R_pad * (op.lay.vsplit ? 2 : 1);
            GPK_TRY(launch_v_colmax(ctx, Vc, op.Nc, rc, op.cmax, s));
            if (pl.engine == 1 && op.lay.fp32_pv) {
                // FP32 value product: v in FP32 (4 rows, in the FP16 Vt buffer's space, which
                // holds 2 x 16 FP16 rows), one TMA box of 128 columns x 4 rows per stage
                GPK_TRY(launch_v_pack32(ctx, Vc, op.Nc, pl.Nc_pad, rc, op.cmax, op.a2, (float*)op.Vt, op.outscale,
                                        s));
                GPK_TRY(encode_tmap_2d(&op.tmV, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, op.Vt, pl.Nc_pad, 4, pl.Nc_pad * 4,
                                       128, 4, CU_TENSOR_MAP_SWIZZLE_NONE));
                GPK_TRY(launch_kmvm_tp(ctx, pl, op.lay, a, op.tmA, op.tmB, op.tmV, op.outscale, op.partial,
                                       op.skip ? op.mask : nullptr, s));
                continue;
            }
            GPK_TRY(launch_v_cast(ctx, op.prec, (op.flags & GP_MVM_SCALE_SQRT_N) ? 1 : 0, op.lay.vsplit, Vc, op.Nc,
                                  pl.Nc_pad, rc, pl.R_pad, op.cmax, op.a2, op.Vt, op.outscale, s));
            const CUtensorMapDataType dt =
                op.prec == GP_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
            const uint64_t vrows = (uint64_t)(op.lay.vsplit ? 2 : 1) * pl.R_pad;
            if (pl.engine == 1) {
                // one box carries the hi and lo rows of a 64-column K-block
                GPK_TRY(encode_tmap_2d(&op.tmV, dt, op.Vt, pl.Nc_pad, vrows, pl.Nc_pad * 2, 64, (uint32_t)pl.rv,
                                       CU_TENSOR_MAP_SWIZZLE_128B));
                GPK_TRY(launch_kmvm_tp(ctx, pl, op.lay, a, op.tmA, op.tmB, op.tmV, op.outscale, op.partial,
                                       op.skip ? op.mask : nullptr, s));
            } else {
                GPK_TRY(encode_tmap_2d(&op.tmV, dt, op.Vt, pl.Nc_pad, vrows, pl.Nc_pad * 2, 64, pl.R_pad,
                                       CU_TENSOR_MAP_SWIZZLE_128B));
                GPK_TRY(launch_kmvm_tc(ctx, pl, op.lay, a, op.tmA, op.tmB, op.tmV, op.outscale, op.partial, s));
            }
        }
    }
    return GP_OK;
}

}  // namespace gpk
