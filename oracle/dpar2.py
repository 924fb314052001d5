"""Plain FP64 oracle of DPar2 (Jang & Kang, arXiv 2203.12798).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Everything is float64
numpy; library primitives (matmul, LAPACK QR / SVD, pinv) serve as single
steps, with no blocking, fusion or reordering beyond the paper's formulas.

Notation follows the paper: slices X_k (I_k x J), target rank R, test matrix
Omega (J x (R+s)), stage-1 factors A_k B_k C_k^T, stage-2 factors D E F^T with
R x R blocks F^(k), PARAFAC2 factors Q_k, H, S_k = diag(W(k,:)), V.

Readings of points the paper leaves open:
  * randomized SVD keeps min(R, rank) components; singular values of B at or
    below max(I,J) * eps * sigma_1 count as zero, and their columns of A, C
    and entries of B are set to zero (A stays column-orthonormal on the rest);
  * sign convention: every right singular vector gets a non-negative entry
    sum (the stage-2 sketch sees the signs of the columns of M, so the CUDA
    path applies the same rule);
  * power iterations (q >= 1) re-orthonormalise between the products with A
    and A^T (Halko et al.'s subspace iteration); in exact arithmetic this is
    Alg. 1's (A A^T)^q A Omega;
  * initialisation: H = I_R, W = ones(K, R) (S_k = I), V given by the caller;
  * "Normalize H / V": every column scaled to unit 2-norm right after its
    update (columns of norm <= 1e-300 left alone); W absorbs the scale;
  * pseudoinverse: SVD-based, singular values <= max(m,n) * eps * sigma_1
    treated as zero (MATLAB's default tolerance);
  * the Q-step's R x R SVD keeps directions with sigma > R * eps * sigma_max;
  * convergence value e = sum_k ||Y_k - H S_k V^T||_F^2 evaluated after the W
    update of each iteration; the loop stops after max_iter iterations or
    when e_prev - e <= tol * e_prev (tol < 0 never stops early).
"""
from __future__ import annotations

import numpy as np

EPS = np.finfo(np.float64).eps


# ---------------------------------------------------------------- helpers --

def _sign_fix(U, V):
    """Flip (u_i, v_i) pairs so that every right singular vector v_i has a
    non-negative entry sum.  The SVD fixes singular vectors only up to sign
    (Sec. II-B); the two-stage compression is sensitive to the choice because
    M's columns meet the stage-2 test matrix, so both implementations use
    this one rule."""
    if U.size == 0:
        return U, V
    s = np.where(V.sum(axis=0) < 0, -1.0, 1.0)
    return U * s, V * s


def pinv(A):
    """Moore-Penrose pseudoinverse with MATLAB's default tolerance."""
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    tol = max(A.shape) * EPS * (s[0] if s.size else 0.0)
    sinv = np.where(s > tol, 1.0 / np.where(s > tol, s, 1.0), 0.0)
    return (Vt.T * sinv) @ U.T


def khatri_rao(A, B):
    """Column-wise Kronecker product, (A ⊙ B)[i*IB + j, r] = A[i, r] B[j, r]."""
    I, R = A.shape
    J = B.shape[0]
    return (A[:, None, :] * B[None, :, :]).reshape(I * J, R)


def unfold(T, mode):
    """Mode-n matricization (Kolda & Bader): for an I1 x I2 x I3 tensor the
    column index of element (i1,i2,i3) runs over the other modes with the
    lowest remaining mode fastest."""
    return np.moveaxis(T, mode, 0).reshape(T.shape[mode], -1, order="F")


# ------------------------------------------------------- Algorithm 1 -------

def randomized_svd(A, R, Omega, q=0):
    """Algorithm 1 (randomized SVD of A, I x J) at target rank R.

    Y = (A A^T)^q A Omega; Q R <- Y (Householder QR, LAPACK); B = Q^T A;
    truncated SVD B = U~ Sigma V^T at rank R; returns (U = Q U~, sigma, V)
    with shapes (I x R, R, J x R), zero-padded past the numerical rank."""
    A = np.asarray(A, dtype=np.float64)
    I, J = A.shape
    Y = A @ Omega
    Q, _ = np.linalg.qr(Y)
    for _ in range(q):
        Z, _ = np.linalg.qr(A.T @ Q)
        Q, _ = np.linalg.qr(A @ Z)
    B = Q.T @ A
    Ut, s, Vt = np.linalg.svd(B, full_matrices=False)
    r = min(R, s.size)
    tol = max(I, J) * EPS * (s[0] if s.size else 0.0)
    keep = (s[:r] > tol).astype(np.float64)
    U = np.zeros((I, R))
    S = np.zeros(R)
    V = np.zeros((J, R))
    U[:, :r] = (Q @ Ut[:, :r]) * keep
    S[:r] = s[:r] * keep
    V[:, :r] = Vt[:r].T * keep
    U, V = _sign_fix(U, V)
    return U, S, V


# ------------------------------------------- two-stage compression ---------

def compress(X_slices, R, Omega, Omega2, q=0):
    """Stage 1 (Eq. fstage_svd) and stage 2 (Eq. matricization_svd) of
    Sec. III-B / Alg. 3: X_k ~ A_k B_k C_k^T for every k, then the randomized
    SVD M = ||_k (C_k B_k) ~ D E F^T of the J x KR concatenation.

    Returns dict(A=[I_k x R], B=[R], C=[J x R], M (J x KR), D (J x R),
    E (R), F (KR x R), Fk=[R x R blocks of F])."""
    A, Bs, C = [], [], []
    for X in X_slices:
        a, b, c = randomized_svd(X, R, Omega, q)
        A.append(a)
        Bs.append(b)
        C.append(c)
    M = np.concatenate([c * b for b, c in zip(Bs, C)], axis=1)
    D, E, F = randomized_svd(M, R, Omega2, q)
    K = len(X_slices)
    Fk = [F[k * R:(k + 1) * R] for k in range(K)]
    return dict(A=A, B=Bs, C=C, M=M, D=D, E=E, F=F, Fk=Fk)


def compressed_slices(comp):
    """X~_k = A_k F^(k) E D^T (Eq. Xk_final)."""
    D, E = comp["D"], comp["E"]
    return [a @ f @ np.diag(E) @ D.T for a, f in zip(comp["A"], comp["Fk"])]


def preprocessed_size(I, J, K, R):
    """Theorem 2 count of stored numbers: sum_k I_k R (A_k) + K R^2 (F^(k))
    + J R (D) + R (E)."""
    return int(np.sum(I)) * R + K * R * R + J * R + R


# ------------------------------------------------------------ CP-ALS -------

def mttkrp(Yt, mode, A1, A2):
    """Y_(n) (A1 ⊙ A2) with the unfolding above (mode 0: W⊙V, 1: W⊙H, 2: V⊙H)."""
    return unfold(Yt, mode) @ khatri_rao(A1, A2)


def _normalize_columns(M):
    n = np.linalg.norm(M, axis=0)
    return M / np.where(n > 1e-300, n, 1.0)


def cp_als_sweep(Yt, H, V, W):
    """One CP-ALS iteration on the R x J x K tensor Y (Alg. 2 / Alg. 3, the
    H, V, W updates with normalisation of H and V)."""
    H = mttkrp(Yt, 0, W, V) @ pinv((W.T @ W) * (V.T @ V))
    H = _normalize_columns(H)
    V = mttkrp(Yt, 1, W, H) @ pinv((W.T @ W) * (H.T @ H))
    V = _normalize_columns(V)
    W = mttkrp(Yt, 2, V, H) @ pinv((V.T @ V) * (H.T @ H))
    return H, V, W


def _polar_from_svd(T):
    """Z P^T from the SVD T = Z Sigma P^T, keeping sigma > n eps sigma_max."""
    Z, s, Pt = np.linalg.svd(T, full_matrices=False)
    tol = max(T.shape) * EPS * (s[0] if s.size else 0.0)
    keep = s > tol
    return (Z[:, keep] @ Pt[keep])


def _y_loss(Ys, H, V, W):
    return float(sum(np.sum((Y - H @ np.diag(W[k]) @ V.T) ** 2) for k, Y in enumerate(Ys)))


# ------------------------------------------------------- Algorithm 2 -------

def parafac2_als(X_slices, V0, max_iter=32, tol=-1.0, H0=None, W0=None):
    """Algorithm 2 (PARAFAC2-ALS, Kiers et al.) on the raw slices.

    Returns dict(H, V, W, Q=[I_k x R], U=[Q_k H], losses=[e_Y per iteration],
    iters) where e_Y = sum_k ||Q_k^T X_k - H S_k V^T||^2."""
    K = len(X_slices)
    R = V0.shape[1]
    H = np.eye(R) if H0 is None else np.array(H0, dtype=np.float64)
    W = np.ones((K, R)) if W0 is None else np.array(W0, dtype=np.float64)
    V = np.array(V0, dtype=np.float64)
    losses = []
    Qs = None
    for it in range(max_iter):
        Qs = [_polar_from_svd(X @ V @ np.diag(W[k]) @ H.T) for k, X in enumerate(X_slices)]
        Ys = [Q.T @ X for Q, X in zip(Qs, X_slices)]
        Yt = np.stack(Ys, axis=2)
        H, V, W = cp_als_sweep(Yt, H, V, W)
        e = _y_loss(Ys, H, V, W)
        losses.append(e)
        if tol >= 0 and len(losses) > 1 and losses[-2] - e <= tol * losses[-2]:
            break
    U = [Q @ H for Q in Qs]
    return dict(H=H, V=V, W=W, Q=Qs, U=U, losses=losses, iters=len(losses))


# ------------------------------------------------------- Algorithm 3 -------

def dpar2_als(comp, V0, max_iter=32, tol=-1.0, H0=None, W0=None):
    """The iteration part of Algorithm 3 on the compressed slices, written
    with the plain definitions: Z_k Sigma_k P_k^T = SVD(F^(k) E D^T V S_k H^T)
    (Eq. q_k), Y_k = P_k Z_k^T F^(k) E D^T materialised (Sec. III-D), the
    tensor Y built from the Y_k and one CP-ALS sweep on it.

    Returns dict(H, V, W, Zp=[Z_k P_k^T], U=[A_k Z_k P_k^T H], losses, iters)."""
    D, E, Fk, A = comp["D"], comp["E"], comp["Fk"], comp["A"]
    K = len(Fk)
    R = D.shape[1]
    H = np.eye(R) if H0 is None else np.array(H0, dtype=np.float64)
    W = np.ones((K, R)) if W0 is None else np.array(W0, dtype=np.float64)
    V = np.array(V0, dtype=np.float64)
    EDt = np.diag(E) @ D.T
    losses = []
    Zp = None
    for it in range(max_iter):
        Zp = [_polar_from_svd(Fk[k] @ EDt @ V @ np.diag(W[k]) @ H.T) for k in range(K)]
        Ys = [zp.T @ Fk[k] @ EDt for k, zp in enumerate(Zp)]
        Yt = np.stack(Ys, axis=2)
        H, V, W = cp_als_sweep(Yt, H, V, W)
        e = _y_loss(Ys, H, V, W)
        losses.append(e)
        if tol >= 0 and len(losses) > 1 and losses[-2] - e <= tol * losses[-2]:
            break
    U = [a @ zp @ H for a, zp in zip(A, Zp)]
    return dict(H=H, V=V, W=W, Zp=Zp, U=U, losses=losses, iters=len(losses))


def dpar2(X_slices, R, Omega, Omega2, V0, max_iter=32, tol=-1.0, q=0):
    """Algorithm 3 end to end: compression, then the compressed iterations."""
    comp = compress(X_slices, R, Omega, Omega2, q)
    fit = dpar2_als(comp, V0, max_iter, tol)
    fit["comp"] = comp
    return fit


# ------------------------------------------------------------ fitness ------

def squared_error(X_slices, U, W, V):
    """sum_k ||X_k - U_k S_k V^T||_F^2 computed directly from the slices."""
    return float(sum(np.sum((X - U[k] @ np.diag(W[k]) @ V.T) ** 2) for k, X in enumerate(X_slices)))


def fitness(X_slices, U, W, V):
    """Sec. IV-A: 1 - sum_k ||X_k - X^_k||^2 / sum_k ||X_k||^2."""
    tot = float(sum(np.sum(X ** 2) for X in X_slices))
    return 1.0 - squared_error(X_slices, U, W, V) / tot


# ----------------------------------------------------- learned sketch ------

def sketch_loss(X_slices, Omega):
    """Range-finder loss of a sketch matrix Omega (J x l):
    L = (1/K) sum_k ||X_k - Y_k Y_k^+ X_k||_F^2 / ||X_k||_F^2, Y_k = X_k Omega.
    Uses Y Y^+ X = Y G^+ Y^T X with G = Y^T Y."""
    tot = 0.0
    for X in X_slices:
        Y = X @ Omega
        P = X.T @ Y  # J x l  (= A Omega with A = X^T X)
        G = Y.T @ Y
        nx = float(np.sum(X * X))
        f = nx - float(np.trace(pinv(G) @ (P.T @ P)))
        tot += f / nx
    return tot / len(X_slices)


def sketch_loss_grad(X_slices, Omega):
    """Analytic gradient of sketch_loss with respect to Omega:
    d/dOmega [ -tr(G^-1 N) ] = -2 [A^2 Omega G^-1 - A Omega G^-1 N G^-1],
    A = X^T X, G = Omega^T A Omega, N = Omega^T A^2 Omega (per slice,
    divided by ||X_k||^2 and averaged over slices)."""
    g = np.zeros_like(Omega, dtype=np.float64)
    for X in X_slices:
        Y = X @ Omega
        P = X.T @ Y  # A Omega
        Z = X @ P
        A2O = X.T @ Z  # A^2 Omega
        Gi = pinv(Y.T @ Y)
        N = P.T @ P
        nx = float(np.sum(X * X))
        g += -2.0 * (A2O @ Gi - P @ Gi @ N @ Gi) / nx
    return g / len(X_slices)
