"""The stopping rule of the library's one-sided Jacobi solvers, checked in FP64
on the cyclic round-robin ordering they use: a pair is rotated when the cosine
of its columns |g| / sqrt(a b) exceeds tol, and the iteration ends after a
sweep whose largest cosine r is at most rstop = sqrt(tol / sqrt(n)), without
the sweep that would only confirm convergence (rotations perturb the other
inner products of their columns by about the angle times those products, so
such a sweep leaves cosines of about sqrt(n) r^2 <= tol).  The polar factor
Z P^T of the final columns must then equal the one from a full SVD to about
tol, as it does when the iteration runs until a sweep rotates nothing
(singular values spread geometrically over condition numbers 1e2 - 1e4)."""
import numpy as np
import pytest


def round_robin_pairs(n):
    """The kernels' cyclic round-robin rounds over m = n (+1 when odd) players."""
    m = n + (n & 1)
    for rr in range(m - 1):
        pairs = []
        for c in range(m):
            if c == 0:
                p = 1 + rr
            else:
                x = c - 1
                p = 0 if x == rr else 1 + ((2 * rr - x + 2 * (m - 1)) % (m - 1))
            if c < p < n:
                pairs.append((c, p))
        yield pairs


def jacobi(T, tol, rstop, cap=60):
    t = T.copy()
    v = np.eye(T.shape[1])
    n = T.shape[1]
    for sweep in range(1, cap + 1):
        rmax = 0.0
        for pairs in round_robin_pairs(n):
            for c, p in pairs:
                a, b, g = t[:, c] @ t[:, c], t[:, p] @ t[:, p], t[:, c] @ t[:, p]
                rel = abs(g) / np.sqrt(a * b) if a > 0 and b > 0 else 0.0
                rmax = max(rmax, rel)
                if rel > tol:
                    zeta = (b - a) / (2 * g)
                    tt = np.sign(zeta) / (abs(zeta) + np.sqrt(1 + zeta * zeta))
                    cs = 1 / np.sqrt(1 + tt * tt)
                    sn = cs * tt
                    t[:, [c, p]] = np.stack([cs * t[:, c] - sn * t[:, p], sn * t[:, c] + cs * t[:, p]], 1)
                    v[:, [c, p]] = np.stack([cs * v[:, c] - sn * v[:, p], sn * v[:, c] + cs * v[:, p]], 1)
        if rmax <= rstop:
            return t, v, sweep
    return t, v, cap


def off_cosine(t):
    z = t / np.linalg.norm(t, axis=0)
    g = z.T @ z
    return np.abs(g - np.diag(np.diag(g))).max()


@pytest.mark.parametrize("n,cond", [(10, 1e2), (16, 1e3), (24, 1e4)])
def test_early_stop_leaves_cosines_at_tol_and_the_same_polar_factor(n, cond):
    rng = np.random.default_rng(n)
    tol = max(1e-6, n * 1.2e-7)
    rstop = np.sqrt(tol / np.sqrt(n))
    for trial in range(3):
        U, _ = np.linalg.qr(rng.standard_normal((n, n)))
        W, _ = np.linalg.qr(rng.standard_normal((n, n)))
        T = U @ np.diag(np.geomspace(1.0, 1.0 / cond, n)) @ W.T
        exact = U @ W.T
        t1, v1, s1 = jacobi(T, tol, tol)    # until a sweep rotates nothing above tol
        t2, v2, s2 = jacobi(T, tol, rstop)  # the library's rule
        assert s2 <= s1
        assert off_cosine(t2) <= 2 * tol
        p1 = (t1 / np.linalg.norm(t1, axis=0)) @ v1.T
        p2 = (t2 / np.linalg.norm(t2, axis=0)) @ v2.T
        # both at the tolerance (measured 0.3 - 0.8 tol here), and the early
        # stop changes the polar factor by less than that
        assert np.abs(p1 - exact).max() <= 2 * tol
        assert np.abs(p2 - exact).max() <= 2 * tol
        assert np.abs(p2 - p1).max() <= tol


def test_round_robin_rounds_cover_every_pair_once():
    for n in (7, 10, 16, 25, 32):
        seen = set()
        for pairs in round_robin_pairs(n):
            cols = [c for pr in pairs for c in pr]
            assert len(cols) == len(set(cols))  # disjoint within a round
            for pr in pairs:
                assert pr not in seen
                seen.add(pr)
        assert len(seen) == n * (n - 1) // 2
