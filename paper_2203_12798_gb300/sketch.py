"""Learned test matrix for the stage-1 range finder.

Alg. 1 sketches every slice with a Gaussian test matrix Omega (J x l).  Here
Omega is a trainable parameter instead, fitted to slices drawn like the ones
it will compress by minimising the part of each slice that the sketch misses,

    L(Omega) = (1/K) sum_k ||X_k - Y_k Y_k^+ X_k||_F^2 / ||X_k||_F^2,   Y_k = X_k Omega,

with the library's forward and backward kernels (``dpar2_sketch_loss_fwd`` /
``dpar2_sketch_loss_bwd``) behind a ``torch.autograd.Function``.  For 16-bit X
the kernels use Omega rounded to X's type (as ``dpar2_compress`` does); the
gradient at the rounded point is returned for the FP32 parameter.

L is invariant under Omega -> Omega T for any invertible T (the sketch only
fixes a column space), so training may re-orthonormalise Omega between steps
without changing the loss; ``train_sketch`` rescales the orthonormal basis by
sqrt(J) to keep the entry scale of a standard Gaussian matrix.
"""
from __future__ import annotations

import math

import torch


class SketchLoss(torch.autograd.Function):
    """loss = SketchLoss.apply(omega, X, offsets, ctx): a 0-dim float64 tensor
    on omega's device.  One backward per forward, in order: a second forward on
    the same library context before the first one's backward makes that
    backward raise."""

    @staticmethod
    def forward(fctx, omega, X, offsets, ctx):
        loss = ctx.sketch_loss_fwd(X, offsets, omega.detach().contiguous())
        fctx.lib_ctx = ctx
        fctx.gen = ctx._sk_gen
        return torch.tensor(loss, dtype=torch.float64, device=omega.device)

    @staticmethod
    def backward(fctx, g):
        ctx = fctx.lib_ctx
        if ctx._sk_gen != fctx.gen:
            raise RuntimeError("SketchLoss: another forward ran on this context before this backward")
        return ctx.sketch_loss_bwd(float(g)), None, None, None


def gaussian_omega(ctx, J: int, ell: int, seed: int = 0) -> torch.Tensor:
    """The Gaussian test matrix dpar2_compress draws for `seed` (J x l)."""
    return ctx.gaussian(seed, 0, J * ell, round16=True).view(J, ell).clone()


def train_sketch(ctx, X: torch.Tensor, offsets, J: int, ell: int, steps: int = 100, lr: float = 0.02,
                 seed: int = 0, batch: int = 0, omega0: torch.Tensor | None = None, orthonormalize_every: int = 0,
                 generator_seed: int = 1, log=None) -> torch.Tensor:
    """Fit Omega (J x l) to the slices of X (first J columns) with Adam on
    SketchLoss, starting from omega0 or from the Gaussian matrix of `seed`.

    batch > 0 draws that many consecutive slices per step (a fixed seeded
    sequence of slice ranges); 0 uses every slice each step.  Returns the
    trained Omega (float32, X's device)."""
    off = torch.as_tensor(offsets, dtype=torch.int64).cpu()
    K = off.numel() - 1
    om = (gaussian_omega(ctx, J, ell, seed) if omega0 is None else omega0.clone()).requires_grad_(True)
    opt = torch.optim.Adam([om], lr=lr)
    g = torch.Generator().manual_seed(generator_seed)
    scale = math.sqrt(J)
    for it in range(steps):
        if batch and batch < K:
            k0 = int(torch.randint(0, K - batch + 1, (1,), generator=g))
            r0, r1 = int(off[k0]), int(off[k0 + batch])
            Xb, ob = X[r0:r1], off[k0:k0 + batch + 1] - r0
        else:
            Xb, ob = X, off
        opt.zero_grad(set_to_none=True)
        loss = SketchLoss.apply(om, Xb, ob, ctx)
        loss.backward()
        opt.step()
        if log is not None:
            log(it, float(loss))
        if orthonormalize_every and (it + 1) % orthonormalize_every == 0:
            # a change of basis of the column space: the loss is unchanged, the
            # optimiser's moments refer to the old basis and start afresh
            with torch.no_grad():
                ctx.orthonormalize(om.data)
                om.data.mul_(scale)
            opt = torch.optim.Adam([om], lr=lr)
    return om.detach()


__all__ = ["SketchLoss", "gaussian_omega", "train_sketch"]
