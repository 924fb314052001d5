"""Pins of the post-fit analyses' oracle (Sec. IV-E): each function checked
against something other than itself -- a library routine computing the same
quantity another way, python loops over the definition, a closed form, or an
invariant -- chosen so that a dropped term, a transposed operand or a wrong
order fails one of them."""
import numpy as np
import pytest

from oracle import analytics as oa


def _slices(K, I, R, seed):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal((I, R)) for _ in range(K)]


# ------------------------------------------------------------ feature PCC --

def test_feature_pcc_equals_numpy_corrcoef():
    V = np.random.default_rng(0).standard_normal((17, 6))
    np.testing.assert_allclose(oa.feature_pcc(V), np.corrcoef(V), rtol=0, atol=1e-13)


def test_feature_pcc_affine_rows_and_invariance():
    rng = np.random.default_rng(1)
    v = rng.standard_normal(8)
    V = np.stack([v, 3.0 * v + 2.0, -0.5 * v + 7.0, rng.standard_normal(8)])
    C = oa.feature_pcc(V)
    assert C[0, 1] == pytest.approx(1.0, abs=1e-14)
    assert C[0, 2] == pytest.approx(-1.0, abs=1e-14)
    np.testing.assert_allclose(np.diag(C), 1.0, atol=1e-14)
    # a positive affine map of every row leaves every coefficient unchanged
    a = rng.uniform(0.5, 2.0, size=(4, 1))
    b = rng.standard_normal((4, 1))
    np.testing.assert_allclose(oa.feature_pcc(a * V + b), C, atol=1e-13)


# ------------------------------------------------------------- similarity --

def test_similarity_matches_loops_over_the_definition():
    U = _slices(5, 4, 3, 2)
    gamma = 0.01
    S = oa.similarity(U, gamma)
    for i in range(5):
        for j in range(5):
            d2 = 0.0
            for a in range(4):
                for b in range(3):
                    d2 += (U[i][a, b] - U[j][a, b]) ** 2
            assert S[i, j] == pytest.approx(np.exp(-gamma * d2), rel=1e-14)


def test_similarity_symmetry_unit_diagonal_and_two_slice_closed_form():
    U = _slices(6, 5, 2, 3)
    S = oa.similarity(U, 0.3)
    np.testing.assert_allclose(S, S.T, rtol=0, atol=0)
    np.testing.assert_allclose(np.diag(S), 1.0, rtol=0, atol=0)
    # U_1 = U_0 + t E with ||E||_F = 1: sim = exp(-gamma t^2)
    E = np.zeros((5, 2))
    E[2, 1] = 1.0
    S2 = oa.similarity([U[0], U[0] + 1.5 * E], 0.3)
    assert S2[0, 1] == pytest.approx(np.exp(-0.3 * 2.25), rel=1e-14)
    # gamma = 0: every pair is fully similar
    np.testing.assert_allclose(oa.similarity(U, 0.0), 1.0, rtol=0, atol=0)


# -------------------------------------------------------------------- kNN --

def test_knn_matches_python_sort_and_leaves_out_the_target():
    S = oa.similarity(_slices(40, 6, 3, 4), 0.05)
    t = 7
    idx, val = oa.knn(S, t, 10)
    order = sorted((j for j in range(40) if j != t), key=lambda j: S[t, j], reverse=True)
    assert list(idx) == order[:10]
    assert t not in idx
    assert np.all(np.diff(val) <= 0)
    np.testing.assert_array_equal(val, S[t, idx])


def test_knn_equal_scores_ordered_by_index():
    S = np.full((6, 6), 0.5)
    S[2, 4] = 0.9
    idx, _ = oa.knn(S, 2, 3)
    assert list(idx) == [4, 0, 1]


# -------------------------------------------------------------------- RWR --

def _walk_matrix(S):
    """Row-normalised adjacency written out entry by entry (independent of the
    oracle's helpers): A~(i, j) = S(i, j) / sum_{m != i} S(i, m), A~(i, i) = 0."""
    K = S.shape[0]
    At = np.zeros((K, K))
    for i in range(K):
        tot = sum(S[i, m] for m in range(K) if m != i)
        for j in range(K):
            if j != i:
                At[i, j] = S[i, j] / tot
    return At


def test_rwr_equals_closed_form_fixed_point():
    S = oa.similarity(_slices(30, 5, 3, 5), 0.05)
    c, t = 0.15, 3
    r = oa.rwr(S, t, c=c, iters=100)
    At = _walk_matrix(S)
    q = np.zeros(30)
    q[t] = 1.0
    r_star = c * np.linalg.solve(np.eye(30) - (1.0 - c) * At.T, q)
    # the iteration contracts by (1 - c) per step in the 1-norm: 0.85^100 ~ 9e-8
    assert np.abs(r - r_star).sum() <= 2.0 * (1.0 - c) ** 100
    np.testing.assert_allclose(oa.rwr(S, t, c=c, iters=400), r_star, rtol=0, atol=1e-13)


def test_rwr_conserves_mass_and_row_normalisation_is_stochastic():
    S = oa.similarity(_slices(25, 4, 2, 6), 0.1)
    At = oa.row_normalize(oa.adjacency(S))
    np.testing.assert_allclose(At, _walk_matrix(S), rtol=1e-14, atol=0)
    np.testing.assert_allclose(At.sum(axis=1), 1.0, atol=1e-14)
    np.testing.assert_array_equal(np.diag(At), 0.0)
    for iters in (1, 5, 100):
        assert oa.rwr(S, 0, iters=iters).sum() == pytest.approx(1.0, abs=1e-13)


def test_rwr_topk_ranks_the_scores():
    S = oa.similarity(_slices(30, 5, 3, 7), 0.05)
    r = oa.rwr(S, 11)
    idx, val = oa.rwr_topk(S, 11, 10)
    order = sorted((j for j in range(30) if j != 11), key=lambda j: r[j], reverse=True)
    assert list(idx) == order[:10]
    np.testing.assert_array_equal(val, r[idx])


def test_planted_transposition_in_rwr_caught(monkeypatch):
    # walking along A~ instead of A~^T: A~ is not symmetric (its rows are
    # scaled by different sums), so the closed-form pin must fail
    orig = oa.row_normalize
    monkeypatch.setattr(oa, "row_normalize", lambda A: orig(A).T.copy())
    with pytest.raises(AssertionError):
        test_rwr_equals_closed_form_fixed_point()


def test_planted_missing_self_loop_removal_caught(monkeypatch):
    monkeypatch.setattr(oa, "adjacency", lambda S: np.array(S, dtype=np.float64, copy=True))
    with pytest.raises(AssertionError):
        test_rwr_equals_closed_form_fixed_point()
