"""torch.autograd wrapper of gp_mll_and_grad and a hyperparameter-fitting loop.

The loss is the negative log marginal likelihood (Eq. loss); its gradient is
the pseudo-loss gradient of Eq. approx computed by the CUDA library (solves of
Eq. cg with the stable CG of Alg. 2, then the hand-written backward of the
kernel MVM).  Only argument marshalling happens here.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import gpk


class MarginalLikelihood(torch.autograd.Function):
    """mll = MarginalLikelihood.apply(lengthscale, outputscale, noise, X, y, Z, E, cfg)

    lengthscale (d,), outputscale (), noise () are float tensors (any device);
    X (N, d), y (N,), Z (M, N) [, E (M, rank)] float32 CUDA tensors; cfg is a
    FitConfig.  Returns the loss (a 0-dim float64 tensor on the CPU; NaN when
    no log-determinant was requested).  backward() returns the library's
    gradient for l, a^2, sigma^2 and X."""

    @staticmethod
    def forward(fctx, lengthscale, outputscale, noise, X, y, Z, E, cfg):
        hyp = gpk.Hyper(cfg.kernel, lengthscale.detach().float().cpu().numpy(), float(outputscale.detach()),
                        float(noise.detach()))
        pc = gpk.pivchol(cfg.ctx, hyp, X, cfg.rank) if cfg.rank > 0 else None
        mll, g, gX, _, info = gpk.mll_and_grad(
            cfg.ctx, hyp, X, y, Z, precond=pc, E=E if cfg.precond_probes else None,
            precond_probes=cfg.precond_probes, want_logdet=cfg.want_logdet, tol=cfg.tol, max_iter=cfg.max_iter,
            min_iter=cfg.min_iter, precision=cfg.precision, want_X=X.requires_grad, loss_depth=cfg.loss_depth)
        cfg.last_info = info
        d = hyp.d
        fctx.grads = (torch.tensor(g[:d], dtype=lengthscale.dtype, device=lengthscale.device),
                      torch.tensor(g[d], dtype=outputscale.dtype, device=outputscale.device),
                      torch.tensor(g[d + 1], dtype=noise.dtype, device=noise.device), gX)
        return torch.tensor(mll, dtype=torch.float64)

    @staticmethod
    def backward(fctx, grad_out):
        gl, ga, gs, gX = fctx.grads
        s = grad_out.to(torch.float32).item() if grad_out.numel() == 1 else 1.0
        return (gl * s, ga * s, gs * s, None if gX is None else gX * s, None, None, None, None)


@dataclass
class FitConfig:
    ctx: object
    kernel: int
    rank: int = 100
    tol: float = 1.0
    max_iter: int = 50
    min_iter: int = 10
    precision: object = "fp16"
    precond_probes: bool = True
    want_logdet: bool = True
    loss_depth: int = 0
    last_info: dict | None = None


def softplus_inv(x: float) -> float:
    return float(x + math.log(-math.expm1(-x)))


def fit(ctx, X, y, kernel: int, init_lengthscale, init_outputscale: float, init_noise: float, steps: int = 20,
        lr: float = 0.05, M: int = 16, rank: int = 100, tol: float = 1.0, max_iter: int = 50,
        precision="fp16", seed: int = 0, min_noise: float = 1e-4, callback=None, min_iter: int = 10,
        loss_depth: int = 0):
    """Adam on softplus-raw (l, a^2, sigma^2) for `steps` steps (the paper's
    training loop: Adam, CG tolerance 1.0 with an iteration floor by default).
    Probes are redrawn every step from a seeded generator (standard normals z~
    and e, used as z = L e + sigma z~).  Returns the history
    [(loss, l, a^2, sigma^2, info)]."""
    dev = X.device
    d = X.shape[1]
    raw_l = torch.tensor([softplus_inv(float(v)) for v in np.atleast_1d(init_lengthscale)], dtype=torch.float64,
                         requires_grad=True)
    raw_a = torch.tensor(softplus_inv(init_outputscale), dtype=torch.float64, requires_grad=True)
    raw_s = torch.tensor(softplus_inv(max(init_noise - min_noise, 1e-6)), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([raw_l, raw_a, raw_s], lr=lr)
    cfg = FitConfig(ctx=ctx, kernel=kernel, rank=rank, tol=tol, max_iter=max_iter, min_iter=min_iter,
                    precision=precision, loss_depth=loss_depth)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    for step in range(steps):
        Z = torch.randn((M, X.shape[0]), generator=gen).to(dev)
        E = torch.randn((M, rank), generator=gen).to(dev)
        opt.zero_grad()
        l = torch.nn.functional.softplus(raw_l)
        a2 = torch.nn.functional.softplus(raw_a)
        s2 = torch.nn.functional.softplus(raw_s) + min_noise
        loss = MarginalLikelihood.apply(l, a2, s2, X, y, Z, E, cfg)
        loss.backward()
        opt.step()
        rec = (float(loss.detach()), l.detach().numpy().copy(), float(a2.detach()), float(s2.detach()), cfg.last_info)
        hist.append(rec)
        if callback:
            callback(step, rec)
    return hist
