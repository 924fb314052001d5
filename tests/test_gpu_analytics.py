"""Post-fit analyses (Sec. IV-E) on the GPU against the FP64 oracle: the
similarity matrix (tensor-core Gram of the flattened U_k), top-k selection,
random walks with restarts and the feature correlation of V.  Rankings are
integer results decided by floating point, so both sides rank the same FP32
scores (the GPU's) and must agree exactly; the scores themselves are compared
with the oracle's FP64 values within the FP32 level."""
import numpy as np
import pytest
import torch

import synth
from _gpu import api_or_skip
from oracle import analytics as oa

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return api_or_skip()


@pytest.fixture(scope="module")
def ctx(api):
    c = api.Context(0)
    yield c
    c.close()


def _U(K, I, R, seed, clusters=8):
    d = synth.stock_factors(K=K, I=I, R=R, clusters=clusters, seed=seed)
    return d["U"]


EPS32 = 2.0 ** -24


def _sim_tol(S_ref, U, gamma):
    """Elementwise bound on |S_gpu - S_ref|: the Gram entry <U_i, U_j> is an
    FP32 sum of L products (tensor-core accumulation), off by about
    sqrt(L) eps32 (n_i + n_j) with n_i = ||U_i||^2 (a factor 4 of margin), and
    d^2 = n_i + n_j - 2 G_ij inherits twice that; S = exp(-gamma d^2) moves by
    gamma S |d(d^2)|, plus FP32 rounding of the exponential."""
    L = U[0].numel()
    n = (U.double() ** 2).sum(dim=(1, 2)).numpy()
    dd2 = 2 * 4 * np.sqrt(L) * EPS32 * (n[:, None] + n[None, :])
    return S_ref * (gamma * dd2 + 4 * EPS32)


# (K, I, R): several 128-row blocks with a ragged last one and L = I R past a
# 64-column step; one block with L < 64; K one past a block boundary.
SIM_CASES = [(300, 50, 10), (130, 7, 3), (129, 64, 10), (17, 324, 10)]


@pytest.mark.parametrize("K,I,R", SIM_CASES)
@pytest.mark.parametrize("gamma", [0.01, 0.2])
def test_similarity_matches_oracle(ctx, K, I, R, gamma):
    U = _U(K, I, R, seed=K + I)
    S = ctx.similarity(U.reshape(K, I * R).cuda(), gamma)
    torch.cuda.synchronize()
    ref = oa.similarity([u.double().numpy() for u in U], gamma)
    got = S.double().cpu().numpy()
    assert np.all(np.abs(got - ref) <= _sim_tol(ref, U, gamma))
    np.testing.assert_array_equal(got, got.T)
    np.testing.assert_array_equal(np.diag(got), 1.0)


def test_similarity_of_equal_slices_is_one(ctx):
    # the definition gives exactly 1; the Gram identity cancels n_3 + n_7 - 2 G_37
    # at FP32 accuracy, so S is 1 within the bound of _sim_tol
    U = _U(40, 30, 5, seed=3)
    U[7] = U[3]
    S = ctx.similarity(U.reshape(40, 150).cuda(), 0.5).cpu()
    assert abs(float(S[3, 7]) - 1.0) <= _sim_tol(np.ones((40, 40)), U, 0.5)[3, 7]


@pytest.mark.parametrize("K,k", [(300, 10), (1000, 16), (12, 10), (5, 10)])
def test_topk_ranks_like_the_oracle(ctx, K, k):
    U = _U(K, 20, 6, seed=K)
    S = ctx.similarity(U.reshape(K, 120).cuda(), 0.05)
    targets = list(range(0, K, max(1, K // 7)))
    idx, val = ctx.topk(S[targets].contiguous(), k, exclude=targets)
    Sn = S.double().cpu().numpy()
    for row, t in enumerate(targets):
        ri, rv = oa.knn(Sn, t, k)
        got_i = idx[row].cpu().numpy()
        n_avail = K - 1
        assert list(got_i[:min(k, n_avail)]) == list(ri)
        if k > n_avail:
            assert np.all(got_i[n_avail:] == -1)
        np.testing.assert_array_equal(val[row, :len(rv)].double().cpu().numpy(), rv)


def test_topk_ties_ordered_by_index(ctx):
    sc = torch.full((3, 40), 0.5, dtype=torch.float32)
    sc[1, 33] = 0.9
    sc[2, 5] = 0.7
    idx, _ = ctx.topk(sc.cuda(), 5, exclude=[-1, 2, 5])
    idx = idx.cpu().tolist()
    assert idx[0] == [0, 1, 2, 3, 4]
    assert idx[1] == [33, 0, 1, 3, 4]
    assert idx[2] == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("K,nq", [(300, 3), (1000, 16), (129, 1)])
def test_rwr_matches_oracle(ctx, K, nq):
    U = _U(K, 24, 8, seed=K + 5)
    S = ctx.similarity(U.reshape(K, 192).cuda(), 0.01)
    targets = [int(t) for t in np.linspace(0, K - 1, nq).round()]
    r = ctx.rwr(S, targets, c=0.15, iters=100).double().cpu().numpy()
    Sn = S.double().cpu().numpy()
    for q, t in enumerate(targets):
        ref = oa.rwr(Sn, t, c=0.15, iters=100)
        # FP32 sums of K terms per step; the iteration contracts by 0.85 per step
        assert np.max(np.abs(r[q] - ref)) <= 2e-7 + 1e-5 * np.max(np.abs(ref))
        assert abs(r[q].sum() - 1.0) <= 1e-4
    # the RWR ranking of the GPU's scores
    idx, _ = ctx.topk(torch.from_numpy(r).float().cuda(), 10, exclude=targets)
    for q, t in enumerate(targets):
        order = sorted((j for j in range(K) if j != t), key=lambda j: (-np.float32(r[q][j]), j))
        assert idx[q].cpu().tolist() == order[:10]


def test_rwr_zero_steps_is_the_query(ctx):
    U = _U(50, 10, 4, seed=9)
    S = ctx.similarity(U.reshape(50, 40).cuda(), 0.1)
    r = ctx.rwr(S, [4, 9], iters=0).cpu().numpy()
    e = np.zeros((2, 50))
    e[0, 4] = e[1, 9] = 1.0
    np.testing.assert_array_equal(r, e)


@pytest.mark.parametrize("J,R", [(88, 10), (2049, 10), (5, 3)])
def test_feature_pcc_matches_oracle(ctx, J, R):
    V = synth.gaussian_matrix(J, R, seed=J, representable16=False)
    V[min(2, J - 1)] = 3.0 * V[0] + 1.0  # a perfectly correlated pair
    C = ctx.feature_pcc(V.contiguous().cuda()).double().cpu().numpy()
    ref = oa.feature_pcc(V.double().numpy())
    assert np.max(np.abs(C - ref)) <= 2e-6


def test_feature_pcc_constant_row_is_nan(ctx):
    V = synth.gaussian_matrix(6, 4, seed=2, representable16=False)
    V[3] = 2.5
    C = ctx.feature_pcc(V.contiguous().cuda()).cpu().numpy()
    assert np.all(np.isnan(C[3])) and np.all(np.isnan(C[:, 3]))
    assert not np.any(np.isnan(np.delete(np.delete(C, 3, 0), 3, 1)))


def test_analyses_reject_bad_arguments(api, ctx):
    U = torch.zeros(4, 8, device="cuda")
    with pytest.raises(api.Dpar2Error):
        ctx.similarity(U, -1.0)
    S = torch.eye(4, device="cuda")
    with pytest.raises(api.Dpar2Error):
        ctx.rwr(S, [7])
    with pytest.raises(api.Dpar2Error):
        ctx.topk(S, 17)


def test_stock_sized_similarity_and_rwr_on_samples(ctx):
    """The workload's size (K = 4742 stocks over I = 324 days, R = 10): the
    oracle recomputes sampled rows of S from the definition, and the RWR of
    one query from the GPU's S."""
    K, I, R = 4742, 324, 10
    U = _U(K, I, R, seed=1007, clusters=40)
    S = ctx.similarity(U.reshape(K, I * R).cuda(), 0.01)
    torch.cuda.synchronize()
    Un = U.double().numpy()
    rows = [0, 1, 777, 2048, K - 1]
    for i in rows:
        d2 = ((Un - Un[i][None]) ** 2).sum(axis=(1, 2))
        ref = np.exp(-0.01 * d2)
        tol = _sim_tol(ref[None, :], U, 0.01)[i]
        assert np.all(np.abs(S[i].double().cpu().numpy() - ref) <= tol)
    Sn = S.double().cpu().numpy()
    np.testing.assert_array_equal(Sn, Sn.T)
    r = ctx.rwr(S, [11], c=0.15, iters=100).double().cpu().numpy()[0]
    ref = oa.rwr(Sn, 11, c=0.15, iters=100)
    assert np.max(np.abs(r - ref)) <= 1e-5 * np.max(np.abs(ref))
