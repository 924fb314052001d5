"""Learned sketch through the C ABI: the range-finder loss and its gradient
against the FP64 oracle on the same (16-bit representable) X and Omega, the
loss against the stage-1 compression's own residual, the autograd wrapper,
and what a trained test matrix gains over the Gaussian one on held-out slices
drawn from the same generator instance.

Tolerances: loss 1e-5 relative (FP32 accumulation of O(1e-7) per product,
the residual ratios here are 0.2-0.6 so cancellation costs < 10x).  Gradient,
relative in the Frobenius norm: the backward pass forms (I - Q Q^T) X X^T Q
as the difference X (X^T Q) - Q (Q^T X X^T Q) of two terms of size sigma_1^2
whose difference is of size sigma_1 sigma_{l+1}, each term accumulated in
FP32 over J columns, so the gradient carries a relative error of about
sqrt(J) u sigma_1 / sigma_{l+1} (u = 2^-24); the bound is 8 times that, at
least 1e-4."""
import numpy as np
import pytest
import torch

import synth
from oracle import dpar2 as od

from _gpu import api_or_skip, padded, slices_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return api_or_skip()


@pytest.fixture(scope="module")
def ctx(api):
    return api.Context(0)


def _data(K, Imin, Imax, J, R, seed):
    d = synth.spectrogram_like(K=K, Imin=Imin, Imax=Imax, J=J, R=R, seed=seed)
    X = synth.bf16_representable(d["X"])  # exact in fp32, bf16 and fp16
    return X, d["offsets"]


# (K, Imin, Imax, J, R, l, dtype): generic FP32 path; tensor-core path with
# several 128-row tiles and ragged row / column tails, both MMA widths; FP16;
# the full spectrogram width
CASES = [
    (10, 30, 90, 70, 6, 12, torch.float32),
    (9, 100, 300, 200, 10, 20, torch.bfloat16),
    (6, 60, 200, 130, 20, 40, torch.bfloat16),
    (5, 64, 200, 96, 8, 16, torch.float16),
    (7, 129, 257, 72, 10, 30, torch.bfloat16),
    # the learned-sketch workload's shape: J = 2049, l = 30, I_k in [100, 704]
    (6, 100, 704, 2049, 20, 30, torch.bfloat16),
]


@pytest.mark.parametrize("K,Imin,Imax,J,R,ell,dtype", CASES)
def test_loss_and_gradient_match_oracle(api, ctx, K, Imin, Imax, J, R, ell, dtype):
    X, off = _data(K, Imin, Imax, J, R, seed=2100 + K)
    om = synth.gaussian_matrix(J, ell, seed=K + ell)  # representable in every dtype
    Xd = padded(X.cuda(), J, dtype)
    loss = ctx.sketch_loss_fwd(Xd, off, om.cuda().contiguous())
    grad = ctx.sketch_loss_bwd(1.0).double().cpu().numpy()
    Xs = slices_np(X, off, J)
    Om = om.double().numpy()
    ref = od.sketch_loss(Xs, Om)
    gref = od.sketch_loss_grad(Xs, Om)
    assert abs(loss - ref) <= 1e-5 * ref
    ell_ = Om.shape[1]
    kappa = max(s[0] / s[ell_] if s.size > ell_ else 1.0 for s in (np.linalg.svd(x, compute_uv=False) for x in Xs))
    tol = max(1e-4, 8.0 * np.sqrt(J) * 2.0 ** -24 * kappa)
    err = np.linalg.norm(grad - gref) / np.linalg.norm(gref)
    print(f"\ngradient relative error {err:.2e} (bound {tol:.2e}, sigma_1 / sigma_l+1 = {kappa:.1f})")
    assert err <= tol


def test_gradient_scale_and_repeat(api, ctx):
    X, off = _data(6, 100, 200, 96, 8, seed=2200)
    om = synth.gaussian_matrix(96, 16, seed=3).cuda().contiguous()
    Xd = padded(X.cuda(), 96, torch.bfloat16)
    l1 = ctx.sketch_loss_fwd(Xd, off, om)
    g1 = ctx.sketch_loss_bwd(1.0).clone()
    g3 = ctx.sketch_loss_bwd(-3.0)  # the saved state serves several backward calls
    # (W is split into 16-bit parts after scaling: equal up to FP32 rounding)
    assert float((g3 + 3.0 * g1).norm()) <= 1e-5 * float((3.0 * g1).norm())
    assert ctx.sketch_loss_fwd(Xd, off, om) == l1  # deterministic


def test_loss_equals_stage1_residual_of_compress(api, ctx):
    # with R = l and p = 0 the stage-1 approximation A_k B_k C_k^T is Q_k Q_k^T X_k,
    # so (||X_k||^2 - ||B_k||^2) / ||X_k||^2 averaged over k is the sketch loss
    J, ell = 160, 20
    X, off = _data(12, 80, 260, J, 10, seed=2300)
    Xd = padded(X.cuda(), J, torch.bfloat16)
    om = synth.gaussian_matrix(J, ell, seed=11).cuda().contiguous()
    loss = ctx.sketch_loss_fwd(Xd, off, om)
    comp = ctx.compress(Xd, off, R=ell, p=0, omega=om, J=J)
    t = comp.tensors()
    xn = t["xnorm2"].cpu()
    bk = (t["Bk"].double().cpu() ** 2).sum(1)
    stage1 = float(((xn - bk) / xn).mean())
    assert abs(loss - stage1) <= 1e-5 * loss


def test_autograd_function_and_orthonormalize(api, ctx):
    from paper_2203_12798_gb300.sketch import SketchLoss

    J, ell = 96, 12
    X, off = _data(6, 60, 150, J, 6, seed=2400)
    Xd = padded(X.cuda(), J, torch.float32)
    om = synth.gaussian_matrix(J, ell, seed=5).cuda().requires_grad_(True)
    loss = SketchLoss.apply(om, Xd, off, ctx)
    (2.5 * loss).backward()
    ref = od.sketch_loss_grad(slices_np(X, off, J), om.detach().double().cpu().numpy())
    g = om.grad.double().cpu().numpy()
    assert np.linalg.norm(g - 2.5 * ref) <= 1e-4 * 2.5 * np.linalg.norm(ref)
    # orthonormalising the test matrix keeps its column space, hence the loss
    Q = om.detach().clone()
    ctx.orthonormalize(Q)
    Qn = Q.double().cpu()
    assert torch.allclose(Qn.T @ Qn, torch.eye(ell, dtype=torch.float64), atol=1e-5)
    l0 = ctx.sketch_loss_fwd(Xd, off, om.detach().contiguous())
    l1 = ctx.sketch_loss_fwd(Xd, off, Q)
    assert abs(l1 - l0) <= 1e-5 * l0
    # a backward whose forward was superseded raises instead of using stale state
    a = SketchLoss.apply(om, Xd, off, ctx)
    SketchLoss.apply(om, Xd, off, ctx)
    with pytest.raises(RuntimeError):
        a.backward()


def test_trained_sketch_beats_gaussian_on_held_out_slices(api, ctx):
    from paper_2203_12798_gb300.sketch import gaussian_omega, train_sketch

    J, R, ell = 256, 8, 12
    d = synth.spectrogram_like(K=160, Imin=100, Imax=300, J=J, R=R, seed=2000)
    off = d["offsets"]
    Xd = padded(d["X"].cuda(), J, torch.bfloat16)
    ktr = 100
    r = int(off[ktr])
    Xtr, otr = Xd[:r], off[:ktr + 1]
    Xhe, ohe = Xd[r:], off[ktr:] - r
    om_g = gaussian_omega(ctx, J, ell, seed=0)
    lg = ctx.sketch_loss_fwd(Xhe, ohe, om_g)
    om = train_sketch(ctx, Xtr, otr, J, ell, steps=60, lr=0.05, seed=0)
    lt = ctx.sketch_loss_fwd(Xhe, ohe, om)
    # the best any l-column sketch can do per slice: the tail of its spectrum
    Xs = slices_np(Xhe.float(), ohe, J)
    lopt = float(np.mean([np.sum(s[ell:] ** 2) / np.sum(s ** 2)
                          for s in (np.linalg.svd(x, compute_uv=False) for x in Xs)]))
    assert lopt < lt < lg
    assert lg - lt >= 0.4 * (lg - lopt)
