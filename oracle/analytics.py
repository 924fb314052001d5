"""Plain FP64 oracle of the post-fit analyses of DPar2's discovery section
(Sec. IV-E of Jang & Kang, arXiv 2203.12798).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Float64 numpy, each
quantity computed from its definition in the paper, one step at a time:

  feature_pcc   Pearson correlation coefficients between the latent feature
                vectors V(i, :) (Sec. IV-E, feature similarity on the stock
                data);
  similarity    sim(s_i, s_j) = exp(-gamma ||U_i - U_j||_F^2) between slices
                of equal length (Eq. similarity), differences taken entry by
                entry;
  knn           the k slices most similar to a target by that measure
                (Sec. IV-E, k-nearest neighbours);
  rwr           random walks with restarts on the similarity graph (Sec. IV-E):
                adjacency A(i, j) = sim(s_i, s_j) off the diagonal and 0 on it,
                A~ its row-normalised form, and the power iteration
                r <- (1 - c) A~^T r + c q from r = q, q one-hot at the target.

Readings of points the paper leaves open:
  * the starting vector of the RWR power iteration is the query vector q;
  * a row of A that sums to zero (a slice whose similarity to every other
    slice underflows) is left as zeros in A~ (the walk restarts from there);
  * k-NN and RWR rankings leave the target itself out; equal scores are
    ordered by slice index (any order of equal scores is a valid ranking).

Pins (tests/test_oracle_analytics.py): feature_pcc against numpy.corrcoef,
+-1 for affinely related rows and invariance under per-row affine maps;
similarity against python loops over the definition, symmetry, unit
diagonal, a two-slice closed form; knn against a python sort; rwr against
the closed form c (I - (1 - c) A~^T)^-1 q of its fixed point, mass
conservation sum(r) = 1, and a planted transposition caught.
"""
from __future__ import annotations

import numpy as np


def feature_pcc(V):
    """J x J Pearson correlation coefficients between the rows of V (J x R).
    Rows of zero variance give NaN, as the coefficient is undefined there."""
    V = np.asarray(V, dtype=np.float64)
    C = V - V.mean(axis=1, keepdims=True)
    cov = C @ C.T
    sd = np.sqrt(np.diag(cov))
    with np.errstate(invalid="ignore", divide="ignore"):
        return cov / np.outer(sd, sd)


def similarity(U_slices, gamma):
    """K x K matrix of exp(-gamma ||U_i - U_j||_F^2) for K slices U_i of one
    shape (I x R); the squared distance is summed from the entry differences."""
    U = [np.asarray(u, dtype=np.float64) for u in U_slices]
    K = len(U)
    S = np.empty((K, K))
    for i in range(K):
        for j in range(K):
            d = U[i] - U[j]
            S[i, j] = np.exp(-gamma * np.sum(d * d))
    return S


def knn(S, target, k):
    """Indices and scores of the k slices j != target with the largest
    S[target, j], largest first, equal scores by index."""
    row = np.asarray(S[target], dtype=np.float64)
    cand = [j for j in range(row.size) if j != target]
    cand.sort(key=lambda j: (-row[j], j))
    idx = np.array(cand[:k], dtype=np.int64)
    return idx, row[idx]


def adjacency(S):
    """The similarity graph's adjacency: S with a zero diagonal (no self loops)."""
    A = np.array(S, dtype=np.float64, copy=True)
    np.fill_diagonal(A, 0.0)
    return A


def row_normalize(A):
    """A~ = D^-1 A, D the diagonal of row sums (zero rows stay zero)."""
    d = A.sum(axis=1)
    inv = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    return A * inv[:, None]


def rwr(S, target, c=0.15, iters=100):
    """RWR scores of every slice for a query at `target`: `iters` steps of
    r <- (1 - c) A~^T r + c q from r = q."""
    At = row_normalize(adjacency(S))
    K = At.shape[0]
    q = np.zeros(K)
    q[target] = 1.0
    r = q.copy()
    for _ in range(iters):
        r = (1.0 - c) * (At.T @ r) + c * q
    return r


def rwr_topk(S, target, k, c=0.15, iters=100):
    """The k slices j != target with the highest RWR scores, highest first."""
    r = rwr(S, target, c, iters)
    cand = [j for j in range(r.size) if j != target]
    cand.sort(key=lambda j: (-r[j], j))
    idx = np.array(cand[:k], dtype=np.int64)
    return idx, r[idx]
