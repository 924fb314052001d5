"""Pins of the oracle's learned-sketch loss and gradient: the projection
definition computed through an independent QR route, exactness when the
sketch spans the row space, invariance to Omega -> Omega T, and central
finite differences of the analytic gradient."""
import numpy as np
import pytest

from oracle import dpar2 as od


def _slices(rng, K=4, J=12, n=(15, 25)):
    return [rng.standard_normal((rng.integers(*n), J)) @ np.diag(np.linspace(2, 0.1, J)) for _ in range(K)]


def test_loss_equals_projection_residual_via_qr():
    rng = np.random.default_rng(0)
    Xs = _slices(rng)
    Om = rng.standard_normal((12, 5))
    ref = 0.0
    for X in Xs:
        Q, _ = np.linalg.qr(X @ Om)
        ref += np.sum((X - Q @ (Q.T @ X)) ** 2) / np.sum(X * X)
    assert od.sketch_loss(Xs, Om) == pytest.approx(ref / len(Xs), rel=1e-10)


def test_loss_zero_when_sketch_spans_row_space_and_invariant():
    rng = np.random.default_rng(1)
    Xs = [rng.standard_normal((20, 3)) @ rng.standard_normal((3, 10)) for _ in range(3)]
    assert od.sketch_loss(Xs, rng.standard_normal((10, 4))) == pytest.approx(0.0, abs=1e-12)
    Xs = _slices(rng)
    Om = rng.standard_normal((12, 5))
    T = rng.standard_normal((5, 5))
    assert od.sketch_loss(Xs, Om @ T) == pytest.approx(od.sketch_loss(Xs, Om), rel=1e-9)


def test_gradient_matches_central_finite_differences():
    rng = np.random.default_rng(2)
    Xs = _slices(rng)
    Om = rng.standard_normal((12, 5))
    g = od.sketch_loss_grad(Xs, Om)
    h = 1e-6
    fd = np.zeros_like(Om)
    for i in range(Om.shape[0]):
        for j in range(Om.shape[1]):
            E = np.zeros_like(Om)
            E[i, j] = h
            fd[i, j] = (od.sketch_loss(Xs, Om + E) - od.sketch_loss(Xs, Om - E)) / (2 * h)
    # central differences carry ~eps |L| / h ~ 2e-10 of roundoff on every entry
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)
    # the gradient is orthogonal to the invariance directions Omega -> Omega T
    assert abs(np.sum(g * (Om @ rng.standard_normal((5, 5))))) < 1e-9 * np.linalg.norm(g) * np.linalg.norm(Om) * 5


def test_loss_is_the_rank_l_randomized_svd_residual():
    # Alg. 1 at target rank R = l keeps all of Q^T X, so its residual is the loss
    rng = np.random.default_rng(3)
    Xs = _slices(rng, K=3, J=12)
    Om = rng.standard_normal((12, 5))
    res = []
    for X in Xs:
        U, S, V = od.randomized_svd(X, 5, Om)
        res.append(np.sum((X - U @ np.diag(S) @ V.T) ** 2) / np.sum(X * X))
    assert od.sketch_loss(Xs, Om) == pytest.approx(np.mean(res), rel=1e-10)
