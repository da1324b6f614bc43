"""Seeded synthetic workloads for the GP solve (inputs only, no method arithmetic).

The paper measures on UCI regression sets (Kin40K, Elevators, HouseElectric,
...; Sec. 5, Table 1) that are not available here.  These generators stand in
for them with the shapes, sizes and value distributions of the workloads the
library is measured on.  They are the only code that both the CUDA path's
tests and the FP64 oracle's tests share, and they hold none of the method's
arithmetic: they only draw X, y, probes and hyperparameters.

Every generator uses numpy's PCG64 (``np.random.default_rng(seed)``), which
gives the same stream on x86_64 and aarch64.  Arrays are float32 in the
library's caller layout: X is N x d row-major, right-hand sides are N x R
column-major (one contiguous vector per column, i.e. a (R, N) C array).

Kernel codes follow the C ABI: 0 RBF, 1 Matern-3/2, 2 Matern-1/2, 3 Matern-5/2.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

RBF, MATERN32, MATERN12, MATERN52 = 0, 1, 2, 3
KERNEL_NAMES = {RBF: "rbf", MATERN32: "matern32", MATERN12: "matern12", MATERN52: "matern52"}


@dataclass
class Workload:
    """One synthetic GP problem.

    X: (N, d) float32 inputs; y: (N,) float32 targets; Z: (M, N) float32 probe
    vectors (row c is probe c); hyperparameters theta = (lengthscale[d],
    outputscale a^2, noise sigma^2); rank: pivoted-Cholesky rank; tol: CG
    relative-residual tolerance.
    """
    name: str
    X: np.ndarray
    y: np.ndarray
    Z: np.ndarray
    kernel: int
    lengthscale: np.ndarray
    outputscale: float
    noise: float
    rank: int
    tol: float
    max_iter: int = 50
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    def rhs(self) -> np.ndarray:
        """B = [y, z_1..z_M] as an (R, N) float32 array (column-major N x R)."""
        return np.ascontiguousarray(np.vstack([self.y[None, :], self.Z]).astype(np.float32))


def _standardize(A: np.ndarray) -> np.ndarray:
    return (A - A.mean(axis=0)) / A.std(axis=0)


def rademacher(rng: np.random.Generator, M: int, N: int) -> np.ndarray:
    return (rng.integers(0, 2, size=(M, N)) * 2 - 1).astype(np.float32)


def plain(N: int = 2048, seed: int = 0) -> Workload:
    """Plain method: N=2048, d=8, X ~ U[0,1]^8, y = sin(2 pi mean(x)) + N(0, 0.1^2),
    RBF l=0.5, a^2=1, sigma^2=0.01, rank-20 preconditioner, tol 1e-4, one RHS."""
    rng = np.random.default_rng(seed)
    d = 8
    X = rng.uniform(0.0, 1.0, size=(N, d))
    y = np.sin(2.0 * math.pi * X.mean(axis=1)) + 0.1 * rng.standard_normal(N)
    return Workload("plain", X.astype(np.float32), y.astype(np.float32),
                    np.zeros((0, N), np.float32), RBF, np.full(d, 0.5, np.float32),
                    1.0, 0.01, 20, 1e-4, max_iter=500)


def precision(N: int = 65536, seed: int = 0, kernel: int = RBF, M: int = 16) -> Workload:
    """Precision study: N=65,536, d=8, X ~ N(0, I) standardised, y as in
    `plain` on the standardised inputs, l=1.0, a^2=1, sigma^2=0.05,
    1 + 16 right-hand sides (y and Rademacher probes), rank 100, tol 1e-2.
    Stands in for Kin40K (36K x 8) and the residual study of Fig. 5."""
    rng = np.random.default_rng(seed)
    d = 8
    X = _standardize(rng.standard_normal((N, d)))
    y = np.sin(2.0 * math.pi * X.mean(axis=1)) + 0.1 * rng.standard_normal(N)
    Z = rademacher(rng, M, N)
    return Workload("precision", X.astype(np.float32), y.astype(np.float32), Z, kernel,
                    np.full(d, 1.0, np.float32), 1.0, 0.05, 100, 1e-2, max_iter=1000)


def _gmm(rng: np.random.Generator, N: int, d: int, comps: int, mean_scale: float,
         std_lo: float, std_hi: float) -> np.ndarray:
    means = mean_scale * rng.standard_normal((comps, d))
    stds = rng.uniform(std_lo, std_hi, size=(comps, d))
    lab = rng.integers(0, comps, size=N)
    return means[lab] + stds[lab] * rng.standard_normal((N, d))


def differentiation(N: int = 262144, seed: int = 0, M: int = 16, n_features: int = 2048) -> Workload:
    """Differentiation study: N=262,144, d=18, X from an 8-component Gaussian
    mixture (means ~ N(0, 4I), per-component diagonal std ~ U[0.3, 1]);
    y = a random-Fourier-feature draw from an ARD RBF GP (2048 features,
    generating lengthscales ~ U[0.5, 2]^18, a^2 = 1) + N(0, 0.1^2).
    Model initialisation l = 1, a^2 = 1, sigma^2 = 0.01.  Stands in for
    Elevators (d = 18) at larger N and the trajectories of Fig. 6."""
    rng = np.random.default_rng(seed)
    d = 18
    X = _gmm(rng, N, d, 8, 2.0, 0.3, 1.0)
    gen_ls = rng.uniform(0.5, 2.0, size=d)
    omega = rng.standard_normal((n_features, d)) / gen_ls
    phase = rng.uniform(0.0, 2.0 * math.pi, size=n_features)
    w = rng.standard_normal(n_features)
    f = np.empty(N)
    for i0 in range(0, N, 16384):
        i1 = min(N, i0 + 16384)
        f[i0:i1] = math.sqrt(2.0 / n_features) * (np.cos(X[i0:i1] @ omega.T + phase) @ w)
    y = f + 0.1 * rng.standard_normal(N)
    Z = rng.standard_normal((M, N))  # the solver may redraw P-distributed probes from these
    return Workload("differentiation", X.astype(np.float32), y.astype(np.float32),
                    Z.astype(np.float32), RBF, np.full(d, 1.0, np.float32), 1.0, 0.01,
                    100, 1.0, max_iter=50, extra={"generating_lengthscale": gen_ls})


def scale(N: int = 1843200, seed: int = 0, M: int = 16) -> Workload:
    """Scale study: N=1,843,200, d=11, standardised 16-component anisotropic
    Gaussian mixture; y = standardised sum of 8 random-direction sinusoids
    + N(0, 0.1^2); Matern-3/2 ARD (l = 1), a^2 = 1, sigma^2 = 0.05, rank 100,
    CG tolerance 1.0, 1 + 16 right-hand sides.  Stands in for HouseElectric
    (1,844.3K points; Table 1)."""
    rng = np.random.default_rng(seed)
    d = 11
    X = _standardize(_gmm(rng, N, d, 16, 2.0, 0.2, 1.5))
    dirs = rng.standard_normal((8, d))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    freq = rng.uniform(0.5, 2.0, size=8)
    phase = rng.uniform(0.0, 2.0 * math.pi, size=8)
    g = np.sin((X @ dirs.T) * freq + phase).sum(axis=1)
    y = (g - g.mean()) / g.std() + 0.1 * rng.standard_normal(N)
    Z = rademacher(rng, M, N)
    return Workload("scale", X.astype(np.float32), y.astype(np.float32), Z, MATERN32,
                    np.full(d, 1.0, np.float32), 1.0, 0.05, 100, 1.0, max_iter=50)


@dataclass
class Request:
    """One posterior-mean request of the serving workload."""
    rid: int
    arrival_s: float
    X: np.ndarray          # (N, d) float32 training inputs
    y: np.ndarray          # (N,) float32 targets
    Xstar: np.ndarray      # (1024, d) float32 test inputs
    kernel: int
    lengthscale: np.ndarray
    outputscale: float
    noise: float


def serving(n_requests: int = 512, rate_per_s: float = 1.0, seed: int = 1,
            n_min: int = 1000, n_max: int = 200000, n_test: int = 1024) -> list:
    """Serving: Poisson arrivals at `rate_per_s`, N log-uniform in
    [n_min, n_max], d in {4, 8, 16}, kernel in {RBF, Matern-3/2},
    l ~ U[0.5, 2], a^2 ~ U[0.5, 2], sigma^2 ~ U[0.01, 0.1], X ~ N(0, I),
    y = sin(2 pi mean(x)) + N(0, 0.1^2), 1024 test points ~ N(0, I)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        N = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        d = int(rng.choice([4, 8, 16]))
        kern = int(rng.choice([RBF, MATERN32]))
        ls = float(rng.uniform(0.5, 2.0))
        X = rng.standard_normal((N, d))
        y = np.sin(2.0 * math.pi * X.mean(axis=1)) + 0.1 * rng.standard_normal(N)
        Xs = rng.standard_normal((n_test, d))
        out.append(Request(rid, t, X.astype(np.float32), y.astype(np.float32),
                           Xs.astype(np.float32), kern, np.full(d, ls, np.float32),
                           float(rng.uniform(0.5, 2.0)), float(rng.uniform(0.01, 0.1))))
    return out


def random_problem(N: int, d: int, R: int, seed: int = 0, kernel: int = RBF,
                   lengthscale: float = 1.0, outputscale: float = 1.0, noise: float = 0.05,
                   dist: str = "normal") -> tuple:
    """Small generic problem for kernel tests: (X (N,d), V (R,N), hyperparameters)."""
    rng = np.random.default_rng(seed)
    if dist == "normal":
        X = rng.standard_normal((N, d))
    else:
        X = rng.uniform(0.0, 1.0, size=(N, d))
    V = rng.standard_normal((R, N))
    ls = np.full(d, lengthscale) * rng.uniform(0.8, 1.25, size=d)
    return (X.astype(np.float32), V.astype(np.float32), kernel,
            ls.astype(np.float32), float(outputscale), float(noise))
