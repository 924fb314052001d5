"""Pins of the oracle's Algorithm 1 (randomized SVD) and the two-stage
compression (Sec. III-B): exact recovery of matrices whose SVD is known by
construction, the Eckart-Young closed form, the Halko-Martinsson-Tropp error
bound, orthonormality and ordering invariants, and the stage-2 identity."""
import numpy as np
import pytest

from oracle import dpar2 as od


def _orth(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    return q


def _with_spectrum(rng, I, J, s):
    """A = U diag(s) V^T with known singular values s (descending)."""
    r = len(s)
    return _orth(rng, I, r) @ np.diag(s) @ _orth(rng, J, r).T


@pytest.mark.parametrize("I,J,r,R,ell,q", [(120, 40, 6, 10, 20, 0), (90, 64, 10, 10, 20, 0),
                                            (60, 30, 8, 8, 12, 1), (200, 50, 5, 10, 20, 2)])
def test_exact_recovery_when_rank_le_sketch(I, J, r, R, ell, q):
    rng = np.random.default_rng(I + J + r)
    s = np.sort(rng.uniform(1.0, 10.0, r))[::-1]
    A = _with_spectrum(rng, I, J, s)
    U, S, V = od.randomized_svd(A, R, rng.standard_normal((J, ell)), q)
    rec = U @ np.diag(S) @ V.T
    assert np.sum((A - rec) ** 2) / np.sum(A ** 2) <= 1e-24
    # singular values equal the constructed ones, padded with zeros
    np.testing.assert_allclose(S[:r], s[:min(r, R)], rtol=1e-12)
    assert np.all(S[r:] == 0)
    kept = S > 0
    np.testing.assert_allclose(U[:, kept].T @ U[:, kept], np.eye(kept.sum()), atol=1e-13)
    np.testing.assert_allclose(V[:, kept].T @ V[:, kept], np.eye(kept.sum()), atol=1e-13)
    assert np.all(np.diff(S[kept]) <= 0)


def test_truncation_is_eckart_young_when_sketch_spans_range():
    rng = np.random.default_rng(3)
    s = np.array([9.0, 7.0, 5.0, 3.0, 2.0, 1.0, 0.5, 0.25])
    A = _with_spectrum(rng, 80, 30, s)
    U, S, V = od.randomized_svd(A, 4, rng.standard_normal((30, 12)))
    err = np.sum((A - U @ np.diag(S) @ V.T) ** 2)
    assert err == pytest.approx(np.sum(s[4:] ** 2), rel=1e-10)
    np.testing.assert_allclose(S, s[:4], rtol=1e-12)


def test_short_slice_fewer_rows_than_sketch_columns():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((7, 40))  # I_k < l and I_k < R
    U, S, V = od.randomized_svd(A, 10, rng.standard_normal((40, 20)))
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, A, atol=1e-12)
    assert np.all(S[7:] == 0) and np.all(U[:, 7:] == 0)


def test_halko_martinsson_tropp_expected_error_bound():
    """E||A - Q Q^T A||_F <= (1 + k/(p-1))^(1/2) (sum_{j>k} s_j^2)^(1/2)
    (Halko et al. 2011, Thm. 10.5) for a Gaussian sketch of k + p columns;
    the mean over 200 sketches must satisfy it."""
    rng = np.random.default_rng(11)
    s = 1.0 / (1.0 + np.arange(40)) ** 1.5
    A = _with_spectrum(rng, 100, 60, s)
    k, p = 6, 6
    errs = []
    for t in range(200):
        Y = A @ rng.standard_normal((60, k + p))
        Q, _ = np.linalg.qr(Y)
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A)))
    bound = np.sqrt(1 + k / (p - 1)) * np.sqrt(np.sum(s[k:] ** 2))
    assert np.mean(errs) <= bound
    # and the oracle's rank-(k+p) reconstruction reaches the same range error
    U, S, V = od.randomized_svd(A, k + p, rng.standard_normal((60, k + p)))
    assert np.linalg.norm(A - U @ np.diag(S) @ V.T) <= 3 * bound


def _lowrank_slices(rng, K, J, R, Imin=30, Imax=60):
    H = rng.standard_normal((R, R))
    V = rng.standard_normal((J, R))
    W = np.abs(1 + 0.3 * rng.standard_normal((K, R)))
    Xs = []
    for k in range(K):
        I = rng.integers(Imin, Imax + 1)
        Xs.append(_orth(rng, I, R) @ H @ np.diag(W[k]) @ V.T)
    return Xs, H, V, W


def test_stage2_identity_and_compressed_slices_exact_on_lowrank():
    rng = np.random.default_rng(21)
    R, J = 5, 24
    Xs, H, V, W = _lowrank_slices(rng, 12, J, R)
    comp = od.compress(Xs, R, rng.standard_normal((J, 2 * R)), rng.standard_normal((12 * R, 2 * R)))
    D, E, F = comp["D"], comp["E"], comp["F"]
    np.testing.assert_allclose(D.T @ D, np.eye(R), atol=1e-12)
    np.testing.assert_allclose(F.T @ F, np.eye(R), atol=1e-12)
    # F^(k) E = (C_k B_k)^T D exactly when M has rank <= R
    for k in range(12):
        CB = comp["C"][k] * comp["B"][k]
        np.testing.assert_allclose(comp["Fk"][k] @ np.diag(E), CB.T @ D, atol=1e-10)
    # X_k = A_k F^(k) E D^T on noiseless rank-R data
    for X, Xt in zip(Xs, od.compressed_slices(comp)):
        np.testing.assert_allclose(Xt, X, atol=1e-10 * np.abs(X).max())


def test_preprocessed_size_theorem_count():
    assert od.preprocessed_size([3, 4, 5], 7, 3, 2) == 12 * 2 + 3 * 4 + 7 * 2 + 2
    # compression ratio of Sec. IV-B: ~ 1/(R/J + R^2/(IJ) + R/(IK)) for equal I
    I, J, K, R = 700, 2049, 8000, 10
    ratio = I * J * K / od.preprocessed_size([I] * K, J, K, R)
    assert ratio == pytest.approx(1.0 / (R / J + R * R / (I * J) + R / (I * K)), rel=1e-3)
