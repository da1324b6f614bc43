"""Parity of the CUDA kernel MVM (gp_kmvm, Eq. mvm) with the FP64 oracle.

Tolerances (relative Frobenius error per right-hand side, max over columns):
FP16 / BF16 tensor-core operands with FP32 accumulation <= 2e-3; FP32 SIMT
<= 1e-5.  Both follow from the arithmetic: one rounding of the kernel value
and of v to 11 (FP16) or 8 (BF16) significant bits, errors that average over
the row sum, and FP32 accumulation (2^-24 per add)."""

import numpy as np
import pytest

import oracle as O
from paper_2207_06856_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 2e-3}
KNAME = {0: "rbf", 1: "matern32", 2: "matern12", 3: "matern52"}


@pytest.fixture(scope="module")
def ctx():
    from paper_2207_06856_gb300 import gpk
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = gpk.Context(0)
    yield c
    c.close()


def _run(ctx, X, V, kern, ls, a2, s2, prec, Xc=None, add_noise=True, flags=0, guard=64):
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    hyp = gpk.Hyper(kern, ls, a2, s2)
    Xd = torch.from_numpy(X).to(dev)
    Xcd = Xd if Xc is None else torch.from_numpy(Xc).to(dev)
    Vd = torch.from_numpy(V).to(dev)
    R, Nr = V.shape[0], X.shape[0]
    buf = torch.full((R * Nr + 2 * guard,), float("nan"), device=dev)
    out = buf[guard:guard + R * Nr].view(R, Nr)
    gpk.kmvm(ctx, hyp, Xd, Vd, Xc=Xcd, precision=prec, add_noise=add_noise, flags=flags, out=out)
    ctx.check()
    b = buf.cpu().numpy()
    assert np.all(np.isnan(b[:guard])) and np.all(np.isnan(b[-guard:])), "write outside the output"
    return out.cpu().numpy().astype(np.float64)


def _ref(X, V, kern, ls, a2, s2, Xc=None, add_noise=True):
    Xc = X if Xc is None else Xc
    return O.kmvm(X, Xc, V.T.astype(np.float64), O.Hyp(KNAME[kern], ls, a2, s2), add_noise=add_noise).T


def _colerr(got, ref):
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


SHAPES = [(1, 1, 1), (100, 3, 1), (129, 4, 16), (700, 8, 17), (1000, 11, 5), (333, 18, 17), (2048, 8, 17),
          (257, 16, 33), (4097, 2, 2), (640, 30, 3)]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("kern", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", SHAPES)
def test_kmvm_matches_oracle(ctx, prec, kern, shape):
    N, d, R = shape
    X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=N + d + R, kernel=kern, lengthscale=1.0,
                                                   outputscale=1.3, noise=0.05)
    got = _run(ctx, X, V, kern, ls, a2, s2, prec)
    assert _colerr(got, _ref(X, V, kern, ls, a2, s2)) <= TOL[prec]


@pytest.mark.parametrize("kern", [0, 1])
@pytest.mark.parametrize("R", [3, 7, 10, 14, 19, 23, 27, 31, 45])
def test_kmvm_fp32_every_column_padding(ctx, kern, R):
    """The FP32 engine keeps accumulators for the columns in use rounded up to a
    multiple of 4 (and chunks of 32 beyond that): every padding, and a second
    chunk narrower than the first, against the oracle."""
    N, d = 517, 5
    X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=7 * R + kern, kernel=kern)
    got = _run(ctx, X, V, kern, ls, a2, s2, "fp32")
    assert _colerr(got, _ref(X, V, kern, ls, a2, s2)) <= TOL["fp32"]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("kern", [0, 1, 2])
@pytest.mark.parametrize("shape", [(129, 4, 16), (700, 8, 17), (333, 18, 17), (257, 16, 33), (2048, 8, 64)])
def test_kmvm_engines_agree_with_oracle(ctx, prec, kern, shape):
    """Both tensor-core engines (row-tile pairs with the transposed value
    product, the default; one row tile with P V) meet the tolerance, FP16 (the
    pair engine with single-term P, the default, and with the tile as hi + lo)
    and single-term BF16 (which both engines run)."""
    from paper_2207_06856_gb300 import gpk
    N, d, R = shape
    X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=3 * N + d, kernel=kern)
    ref = _ref(X, V, kern, ls, a2, s2)
    base = gpk.MVM_BF16_SINGLE if prec == "bf16" else 0
    tol = 8e-3 if prec == "bf16" else TOL[prec]
    for fl in (0, gpk.MVM_ONE_TILE, gpk.MVM_PSPLIT):
        got = _run(ctx, X, V, kern, ls, a2, s2, prec, flags=base | fl)
        assert _colerr(got, ref) <= tol, (fl, _colerr(got, ref))


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_kmvm_rectangular_without_noise(ctx, prec):
    """Predictive-mean shape K(X*, X) v (Sec. 3.1): different row and column sets."""
    X, V, kern, ls, a2, s2 = workloads.random_problem(1500, 8, 3, seed=5)
    Xs = np.random.default_rng(6).standard_normal((300, 8)).astype(np.float32)
    got = _run(ctx, Xs, V, kern, ls, a2, s2, prec, Xc=X, add_noise=False)
    assert _colerr(got, _ref(Xs, V, kern, ls, a2, s2, Xc=X, add_noise=False)) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("kern", [0, 1])
def test_kmvm_rank_one_limit(ctx, prec, kern):
    """l -> infinity: K = a^2 1 1^T, so out = a^2 (1^T v) 1 + sigma^2 v.  v has a
    nonzero mean so 1^T v does not cancel (cancellation is covered below)."""
    X, V, _, _, _, _ = workloads.random_problem(900, 5, 4, seed=7)
    V = V + 1.0
    ls = np.full(5, 1e6, np.float32)
    got = _run(ctx, X, V, kern, ls, 1.7, 0.1, prec)
    ref = 1.7 * np.ones((4, 900)) * V.astype(np.float64).sum(axis=1, keepdims=True) + 0.1 * V
    assert _colerr(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec,flags_name", [("fp16", "vsplit"), ("bf16", "default"), ("fp32", "default")])
def test_kmvm_rank_one_limit_with_cancellation(ctx, prec, flags_name):
    """1^T v of 900 standard normals can be ~1 while |v| ~ 30: a single FP16
    rounding of v then gives ~1e-2 relative error (the half-precision MVM of
    the paper has the same property).  Carrying v as hi + lo removes it."""
    from paper_2207_06856_gb300 import gpk
    X, V, _, _, _, _ = workloads.random_problem(900, 5, 4, seed=7)
    ls = np.full(5, 1e6, np.float32)
    fl = gpk.MVM_VSPLIT if flags_name == "vsplit" else 0
    got = _run(ctx, X, V, 0, ls, 1.7, 0.1, prec, flags=fl)
    ref = 1.7 * np.ones((4, 900)) * V.astype(np.float64).sum(axis=1, keepdims=True) + 0.1 * V
    assert _colerr(got, ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
def test_kmvm_far_apart_limit(ctx, prec):
    """Points ten lengthscales apart (an 8 x 8 x 8 grid, offset far from the
    origin): the kernel matrix is a^2 I to within exp(-50), out = (a^2 + sigma^2) v."""
    g = np.arange(8, dtype=np.float32)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) + 100.0
    N = X.shape[0]
    V = np.random.default_rng(8).standard_normal((3, N)).astype(np.float32)
    ls = np.full(3, 0.1, np.float32)
    got = _run(ctx, X, V, 0, ls, 0.9, 0.2, prec)
    assert _colerr(got, 1.1 * V.astype(np.float64)) <= TOL[prec]


def test_kmvm_bf16_single_term(ctx):
    """Single-term BF16 (flag): each kernel value and v rounded once to 8
    significant bits; for random-sign v the relative error is about
    2^-8/sqrt(3) per source, so the bound here is 8e-3, not 2e-3."""
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(3000, 8, 17, seed=13)
    got = _run(ctx, X, V, kern, ls, a2, s2, "bf16", flags=gpk.MVM_BF16_SINGLE)
    err = _colerr(got, _ref(X, V, kern, ls, a2, s2))
    assert err <= 8e-3


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_kmvm_symmetry(ctx, prec):
    """u^T (Ktilde v) = v^T (Ktilde u)."""
    X, V, kern, ls, a2, s2 = workloads.random_problem(3000, 6, 2, seed=9, kernel=1)
    got = _run(ctx, X, V, kern, ls, a2, s2, prec)
    u, v = V[0].astype(np.float64), V[1].astype(np.float64)
    lhs, rhs = u @ got[1], v @ got[0]
    assert abs(lhs - rhs) <= 4 * TOL[prec] * max(abs(lhs), np.linalg.norm(u) * np.linalg.norm(got[1]) * 1e-2)


@pytest.mark.parametrize("flags_name", ["xsplit", "sqrtn"])
def test_kmvm_options(ctx, flags_name):
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(1200, 8, 5, seed=10)
    fl = gpk.MVM_XSPLIT if flags_name == "xsplit" else gpk.MVM_SCALE_SQRT_N
    got = _run(ctx, X, V, kern, ls, a2, s2, "fp16", flags=fl)
    assert _colerr(got, _ref(X, V, kern, ls, a2, s2)) <= TOL["fp16"]


@pytest.mark.parametrize("prec", ["fp16", "bf16", "fp32"])
def test_kmvm_precision_workload_sampled_rows(ctx, prec):
    """The benchmark's MVM shape (N = 65,536, d = 8, 1 + 16 right-hand sides,
    standardised Gaussian inputs, l = 1): 256 sampled rows against exact FP64 rows."""
    w = workloads.precision()
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    B = w.rhs()
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    out = gpk.kmvm(ctx, hyp, torch.from_numpy(w.X).to(dev), torch.from_numpy(B).to(dev), precision=prec,
                   add_noise=True)
    ctx.check()
    got = out.cpu().numpy().astype(np.float64)
    rows = np.sort(np.random.default_rng(11).choice(w.N, 256, replace=False))
    ref = O.kmvm_rows(w.X, rows, B.T.astype(np.float64), O.Hyp("rbf", w.lengthscale, w.outputscale, w.noise)).T
    assert _colerr(got[:, rows], ref) <= TOL[prec]


def test_kmvm_scale_workload_sampled_rows(ctx):
    """The scale workload's MVM (N = 1,843,200, d = 11, Matern-3/2, FP16): 48 sampled rows."""
    w = workloads.scale()
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    B = w.rhs()[:5]
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    out = gpk.kmvm(ctx, hyp, torch.from_numpy(w.X).to(dev), torch.from_numpy(B).to(dev), precision="fp16",
                   add_noise=True)
    ctx.check()
    rows = np.sort(np.random.default_rng(12).choice(w.N, 48, replace=False))
    got = out[:, torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64)
    ref = O.kmvm_rows(w.X, rows, B.T.astype(np.float64), O.Hyp("matern32", w.lengthscale, w.outputscale, w.noise)).T
    assert _colerr(got, ref) <= TOL["fp16"]


def test_kmvm_rejects_bad_arguments(ctx):
    from paper_2207_06856_gb300 import gpk
    dev = torch.device("cuda:0")
    X = torch.randn(10, 3, device=dev)
    V = torch.randn(2, 10, device=dev)
    with pytest.raises(gpk.GPKError):
        gpk.kmvm(ctx, gpk.Hyper(0, np.array([1.0, -1.0, 1.0]), 1.0, 0.1), X, V)
    with pytest.raises(gpk.GPKError):
        gpk.kmvm(ctx, gpk.Hyper(0, np.ones(3), 1.0, 0.1), X, V, Xc=torch.randn(12, 3, device=dev)[:10],
                 add_noise=True)
    with pytest.raises(gpk.GPKError):
        gpk.kmvm(ctx, gpk.Hyper(0, np.ones(3), 1.0, 0.1), X, torch.randn(65, 10, device=dev))



HALF_SHAPES = [(1, 1, 1), (100, 3, 1), (129, 4, 16), (700, 8, 17), (1000, 11, 5), (2048, 8, 17), (4097, 2, 2),
               (2048, 8, 64), (3001, 12, 9)]


@pytest.mark.parametrize("shape", HALF_SHAPES)
def test_kmvm_half_exp_matches_oracle(ctx, shape):
    """Half-precision kernel evaluation (GP_MVM_HALF_EXP, RBF, FP16): the exp2
    argument is rounded once to FP16 by the tensor core (11 significant bits,
    round to nearest) and 2^s is evaluated in FP16.  Per value that adds a
    relative error of at most 2^-11 |s| ln 2 for the argument and one FP16
    ulp for the exponential; over a row sum these average like the FP16
    rounding of the kernel value itself, so the 2e-3 bound of the FP16 MVM
    holds."""
    from paper_2207_06856_gb300 import gpk
    N, d, R = shape
    X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=5 * N + d + R, kernel=0, lengthscale=1.0,
                                                   outputscale=1.3, noise=0.05)
    got = _run(ctx, X, V, 0, ls, a2, s2, "fp16", flags=gpk.MVM_HALF_EXP)
    assert _colerr(got, _ref(X, V, 0, ls, a2, s2)) <= TOL["fp16"]


def test_kmvm_half_exp_limits(ctx):
    """Rank-one (l -> infinity: every argument rounds to 0, 2^0 = 1 exactly) and
    far-apart (arguments below -2^4: the FP16 exponential underflows to 0)
    limits of the half-precision evaluation."""
    from paper_2207_06856_gb300 import gpk
    X, V, _, _, _, _ = workloads.random_problem(900, 5, 4, seed=7)
    V = V + 1.0
    got = _run(ctx, X, V, 0, np.full(5, 1e6, np.float32), 1.7, 0.1, "fp16", flags=gpk.MVM_HALF_EXP)
    ref = 1.7 * np.ones((4, 900)) * V.astype(np.float64).sum(axis=1, keepdims=True) + 0.1 * V
    assert _colerr(got, ref) <= TOL["fp16"]
    g = np.arange(8, dtype=np.float32)
    Xg = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3) + 100.0
    Vg = np.random.default_rng(8).standard_normal((3, Xg.shape[0])).astype(np.float32)
    got = _run(ctx, Xg, Vg, 0, np.full(3, 0.1, np.float32), 0.9, 0.2, "fp16", flags=gpk.MVM_HALF_EXP)
    assert _colerr(got, 1.1 * Vg.astype(np.float64)) <= TOL["fp16"]


def test_kmvm_half_exp_precision_workload_sampled_rows(ctx):
    """The benchmark's MVM shape with the half-precision evaluation: 256
    sampled rows against exact FP64 rows."""
    from paper_2207_06856_gb300 import gpk
    w = workloads.precision()
    dev = torch.device("cuda:0")
    B = w.rhs()
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    out = gpk.kmvm(ctx, hyp, torch.from_numpy(w.X).to(dev), torch.from_numpy(B).to(dev), precision="fp16",
                   add_noise=True, flags=gpk.MVM_HALF_EXP)
    ctx.check()
    got = out.cpu().numpy().astype(np.float64)
    rows = np.sort(np.random.default_rng(11).choice(w.N, 256, replace=False))
    ref = O.kmvm_rows(w.X, rows, B.T.astype(np.float64), O.Hyp("rbf", w.lengthscale, w.outputscale, w.noise)).T
    assert _colerr(got[:, rows], ref) <= TOL["fp16"]


@pytest.mark.parametrize("case", ["matern32", "bf16", "d18", "psplit", "one_tile"])
def test_kmvm_half_exp_unsupported(ctx, case):
    """The half-precision evaluation exists for RBF, FP16, a contraction width
    of 16 and the pair engine with a single-term tile; anything else is
    refused (GP_ERR_UNSUPPORTED), never silently run another way."""
    from paper_2207_06856_gb300 import gpk
    kern, prec, d, fl = 0, "fp16", 8, gpk.MVM_HALF_EXP
    if case == "matern32":
        kern = 1
    elif case == "bf16":
        prec = "bf16"
    elif case == "d18":
        d = 18
    elif case == "psplit":
        fl |= gpk.MVM_PSPLIT
    else:
        fl |= gpk.MVM_ONE_TILE
    X, V, _, ls, a2, s2 = workloads.random_problem(300, d, 3, seed=2, kernel=kern)
    with pytest.raises(gpk.GPKError):
        _run(ctx, X, V, kern, ls, a2, s2, prec, flags=fl)


@pytest.mark.parametrize("where", ["V", "X"])
def test_kmvm_nonfinite_input_is_reported(ctx, where):
    """A NaN in the right-hand sides (their column scale) or in the inputs
    (their FP16 norm terms) is recorded on the device and reported as
    GP_ERR_NONFINITE by the context check, not returned as a silent result."""
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(500, 6, 3, seed=41)
    if where == "V":
        V[1, 17] = np.nan
    else:
        X[33, 2] = np.nan
    dev = torch.device("cuda:0")
    gpk.kmvm(ctx, gpk.Hyper(kern, ls, a2, s2), torch.from_numpy(X).to(dev), torch.from_numpy(V).to(dev),
             precision="fp16", add_noise=True)
    with pytest.raises(gpk.GPKError) as ei:
        ctx.check()
    assert ei.value.status == gpk.GP_ERR_NONFINITE
    ctx.check()   # the word was cleared


def _clusters(n_per, centres, spread, seed, ragged=0):
    """Points in tight clusters, written cluster by cluster (so 128-row tiles
    are compact), with the last `ragged` points dropped."""
    rng = np.random.default_rng(seed)
    X = np.concatenate([c + spread * rng.standard_normal((n_per, len(c))) for c in centres])
    return X[:len(X) - ragged].astype(np.float32)


@pytest.mark.parametrize("prec,flags_name,kern", [("fp16", "", 0), ("fp16", "", 1), ("fp16", "MVM_PSPLIT", 0),
                                                  ("fp16", "MVM_HALF_EXP", 0), ("bf16", "", 0), ("fp16", "", 3)])
def test_skip_tiles_bit_identical_clustered(ctx, prec, flags_name, kern):
    """Compact support (Sec. 3.1, Fig. 2c): 16 clusters 40 lengthscales apart
    (within +-90 lengthscales of the origin, where the FP16 norm terms fit),
    stored cluster by cluster, plus a pair of clusters just beyond the FP16
    underflow distance of the RBF kernel (6.3 lengthscales, the adversarial
    case for the margin).  Skipping the tiles whose kernel values all round to
    zero leaves the result bit-identical, while most entries are skipped."""
    from paper_2207_06856_gb300 import gpk
    d = 3
    g = (np.arange(4) - 1.5) * 40.0
    centres = [np.array([a, b, 0.0]) for a in g for b in g] + [np.array([0.0, 90.0, 0]), np.array([6.3, 90.0, 0])]
    X = _clusters(700, centres, 0.05, seed=44, ragged=37)
    N = X.shape[0]
    V = np.random.default_rng(45).standard_normal((17, N)).astype(np.float32)
    ls = np.ones(d, np.float32)
    base = getattr(gpk, flags_name) if flags_name else 0
    a = _run(ctx, X, V, kern, ls, 1.0, 0.05, prec, flags=base)
    b = _run(ctx, X, V, kern, ls, 1.0, 0.05, prec, flags=base | gpk.MVM_SKIP_TILES)
    assert np.array_equal(a, b)
    hyp = gpk.Hyper(kern, ls, 1.0, 0.05)
    ev, tot = gpk.kmvm_tile_count(ctx, hyp, torch.from_numpy(X).to("cuda:0"), precision=prec,
                                  flags=base | gpk.MVM_SKIP_TILES)
    assert ev < 0.35 * tot, (ev, tot)


def test_skip_tiles_bit_identical_precision_workload(ctx):
    """The benchmark's MVM (N = 65,536, d = 8 standard normal, l = 1): the bound
    skips nothing there (the data has no far-apart tiles) and the result is
    bit-identical."""
    from paper_2207_06856_gb300 import gpk
    w = workloads.precision()
    dev = torch.device("cuda:0")
    hyp = gpk.Hyper(w.kernel, w.lengthscale, w.outputscale, w.noise)
    X = torch.from_numpy(w.X).to(dev)
    B = torch.from_numpy(w.rhs()).to(dev)
    a = gpk.kmvm(ctx, hyp, X, B, precision="fp16", add_noise=True).cpu().numpy()
    b = gpk.kmvm(ctx, hyp, X, B, precision="fp16", add_noise=True, flags=gpk.MVM_SKIP_TILES).cpu().numpy()
    ctx.check()
    assert np.array_equal(a, b)
    ev, tot = gpk.kmvm_tile_count(ctx, hyp, X, flags=gpk.MVM_SKIP_TILES)
    assert 0 < ev <= tot


@pytest.mark.parametrize("case", ["fp32", "one_tile"])
def test_skip_tiles_unsupported(ctx, case):
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(300, 3, 2, seed=46)
    prec, fl = ("fp32", gpk.MVM_SKIP_TILES) if case == "fp32" else ("fp16", gpk.MVM_SKIP_TILES | gpk.MVM_ONE_TILE)
    with pytest.raises(gpk.GPKError):
        _run(ctx, X, V, kern, ls, a2, s2, prec, flags=fl)


def test_summation_variants_ordering(ctx):
    """Summation-variant study (Sec. 4.1, Fig. 4b; App. B, Fig. A.1a) on inputs
    shaped like the scale workload (d = 11, Matern-3/2, anisotropic mixture):
    with FP16 kernel values and FP16 products, accumulating in FP32 meets the
    FP16 MVM tolerance; one running FP16 sum is far worse; FP16 block sums and
    Kahan-compensated FP16 sums recover most of the loss."""
    from paper_2207_06856_gb300 import gpk
    w = workloads.scale(N=6000)
    X = w.X
    V = np.stack([w.y, np.random.default_rng(47).standard_normal(X.shape[0])]).astype(np.float32)
    ls = w.lengthscale
    ref = _ref(X, V, w.kernel, ls, w.outputscale, w.noise)
    err = {}
    for s in (1, 2, 3, 4):
        got = _run(ctx, X, V, w.kernel, ls, w.outputscale, w.noise, "fp16", flags=gpk.MVM_SUM(s))
        err[s] = _colerr(got, ref)
    assert err[1] <= TOL["fp16"], err
    assert err[2] > 3 * err[1], err
    assert err[3] < err[2] and err[4] < err[2], err


def test_summation_variants_refuse_other_shapes(ctx):
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(300, 3, 9, seed=48)
    with pytest.raises(gpk.GPKError):     # more than 8 right-hand sides
        _run(ctx, X, V, kern, ls, a2, s2, "fp16", flags=gpk.MVM_SUM(2))
    with pytest.raises(gpk.GPKError):     # FP16 only
        _run(ctx, X, V[:2], kern, ls, a2, s2, "bf16", flags=gpk.MVM_SUM(2))


@pytest.mark.parametrize("kern", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 2, 1), (129, 4, 5), (700, 8, 17), (1000, 11, 24), (4097, 3, 2), (600, 29, 12)])
def test_symmetric_half_work_mvm_matches_oracle(ctx, kern, shape):
    """The symmetric half-work MVM (GP_MVM_SYMMETRIC, FP32): each kernel value
    evaluated once for both row blocks; the FP32 tolerance (1e-5) against the
    FP64 oracle, including ragged block counts and the diagonal blocks."""
    from paper_2207_06856_gb300 import gpk
    N, d, R = shape
    X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=N + 11 * d + R, kernel=kern)
    got = _run(ctx, X, V, kern, ls, a2, s2, "fp32", flags=gpk.MVM_SYMMETRIC)
    assert _colerr(got, _ref(X, V, kern, ls, a2, s2)) <= TOL["fp32"]
    got0 = _run(ctx, X, V, kern, ls, a2, s2, "fp32", flags=gpk.MVM_SYMMETRIC, add_noise=False)
    assert _colerr(got0, _ref(X, V, kern, ls, a2, s2, add_noise=False)) <= TOL["fp32"]


def test_symmetric_half_work_mvm_refuses_other_shapes(ctx):
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(300, 3, 25, seed=49)
    with pytest.raises(gpk.GPKError):       # more than 24 right-hand sides
        _run(ctx, X, V, kern, ls, a2, s2, "fp32", flags=gpk.MVM_SYMMETRIC)
    Xs = np.random.default_rng(50).standard_normal((300, 3)).astype(np.float32)
    with pytest.raises(gpk.GPKError):       # not a square operator
        _run(ctx, Xs, V[:3], kern, ls, a2, s2, "fp32", Xc=X, add_noise=False, flags=gpk.MVM_SYMMETRIC)
    with pytest.raises(gpk.GPKError):       # FP32 only
        _run(ctx, X, V[:3], kern, ls, a2, s2, "fp16", flags=gpk.MVM_SYMMETRIC)


@pytest.mark.parametrize("sleep", [False, True])
def test_device_wait_runs_out_and_context_stays_usable(ctx, sleep):
    """Failure detection without a fault: a bounded mbarrier wait that nothing
    completes (the wait helpers of the MVM kernels) gives up after its limit,
    the error word reads GP_ERR_TIMEOUT once, and the context then computes a
    correct MVM."""
    import time
    from paper_2207_06856_gb300 import gpk
    ctx.check()
    t0 = time.perf_counter()
    cyc = ctx.wait_check(5.0, sleep=sleep)
    assert time.perf_counter() - t0 < 10.0
    assert cyc >= 2 * 5_000_000          # the limit counts 2 SM cycles per ns
    with pytest.raises(gpk.GPKError) as e:
        ctx.check()
    assert e.value.status == gpk.GP_ERR_TIMEOUT
    ctx.check()                           # read once, then cleared
    X, V, kern, ls, a2, s2 = workloads.random_problem(700, 8, 17, seed=3)
    got = _run(ctx, X, V, kern, ls, a2, s2, "fp16")
    assert _colerr(got, _ref(X, V, kern, ls, a2, s2)) <= TOL["fp16"]


@pytest.mark.parametrize("kern", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 2, 1), (300, 3, 1), (1000, 8, 2), (4097, 4, 4), (2500, 16, 3)])
@pytest.mark.parametrize("xsplit", [False, True])
def test_fp32_value_product_matches_oracle(ctx, kern, shape, xsplit):
    """GP_MVM_FP32_PV (1 to 4 right-hand sides): the kernel values stay FP32 and
    the products are FP32 FMAs, so only the FP16 rounding of the inputs remains
    (the FP16 tolerance); with the inputs as hi + lo the MVM is FP32-accurate
    up to the two-term norm representation (1e-4)."""
    from paper_2207_06856_gb300 import gpk
    N, d, R = shape
    X, V, _, ls, a2, s2 = workloads.random_problem(N, d, R, seed=N + 7 * d + R, kernel=kern)
    fl = gpk.MVM_FP32_PV | (gpk.MVM_XSPLIT if xsplit else 0)   # without: the engine's default input split
    got = _run(ctx, X, V, kern, ls, a2, s2, "fp16", flags=fl)
    err = _colerr(got, _ref(X, V, kern, ls, a2, s2))
    assert err <= (1e-4 if xsplit else TOL["fp16"]), err
    if N > 1:   # rectangular operator (the predictive-mean shape), rows at new points: coincident
        # points would put Matern-1/2's kink at r = 0 under the distance's rounding
        Xr = np.random.default_rng(N).standard_normal((N // 2 + 1, d)).astype(np.float32)
        got = _run(ctx, Xr, V, kern, ls, a2, s2, "fp16", Xc=X, add_noise=False, flags=fl)
        assert _colerr(got, _ref(Xr, V, kern, ls, a2, s2, Xc=X, add_noise=False)) <= (1e-4 if xsplit else TOL["fp16"])


def test_fp32_value_product_refusals(ctx):
    from paper_2207_06856_gb300 import gpk
    X, V, kern, ls, a2, s2 = workloads.random_problem(500, 4, 5, seed=3)
    with pytest.raises(gpk.GPKError):       # more than 4 right-hand sides
        _run(ctx, X, V, kern, ls, a2, s2, "fp16", flags=gpk.MVM_FP32_PV)
    with pytest.raises(gpk.GPKError):       # FP16 only
        _run(ctx, X, V[:2], kern, ls, a2, s2, "bf16", flags=gpk.MVM_FP32_PV)
    with pytest.raises(gpk.GPKError):       # not with the hi + lo kernel tile
        _run(ctx, X, V[:2], kern, ls, a2, s2, "fp16", flags=gpk.MVM_FP32_PV | gpk.MVM_PSPLIT)
