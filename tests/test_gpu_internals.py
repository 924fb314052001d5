"""Stage-1 intermediates of the CUDA path checked one by one against their
definitions (Alg. 1 steps), through the context's scratch-inspection hook:
  Q = Q1 M2 spans the sketch X Omega and is column-orthonormal (CholeskyQR2),
  B1 = Q1^T X_k (projection pass), GB = B1 B1^T (Gram of the small SVD),
  T = M2 U~_R with U~_R the top eigenvectors of M2^T GB M2."""
import numpy as np
import pytest
import torch

import synth
from oracle import dpar2 as od

from _gpu import api_or_skip, padded, slices_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype,K,J,R,p", [(torch.float32, 12, 80, 6, 10), (torch.bfloat16, 12, 80, 6, 10),
                                           (torch.float32, 12, 64, 10, 10), (torch.float32, 64, 64, 10, 10),
                                           (torch.float32, 10, 300, 20, 10), (torch.bfloat16, 10, 130, 30, 20),
                                           (torch.float16, 12, 257, 10, 10), (torch.bfloat16, 6, 200, 30, 20),
                                           (torch.bfloat16, 40, 2049, 10, 10)])
def test_stage1_intermediates(dtype, K, J, R, p):
    api = api_or_skip()
    ctx = api.Context(0)
    ell = R + p
    LP, Jp = (ell + 7) // 8 * 8, (J + 3) // 4 * 4
    d = synth.plain_parafac2(K=K, Imin=40, Imax=150, J=J, R=R, seed=31)
    X = padded(d["X"].cuda().float(), J, dtype)
    off = d["offsets"]
    om = synth.gaussian_matrix(J, ell, seed=32).cuda()
    om2 = synth.gaussian_matrix(K * R, ell, seed=33).cuda()
    comp = ctx.compress(X, off, R=R, p=p, omega=om, omega2=om2, J=J)
    N = int(off[-1])
    Q1 = ctx.scratch("Y", (N, LP)).double().cpu().numpy()
    M2 = ctx.scratch("M2", (K, LP, LP)).double().cpu().numpy()
    B1 = ctx.scratch("B1", (K, LP, Jp)).double().cpu().numpy()
    GB = ctx.scratch("GB", (K, LP, LP), torch.float64).cpu().numpy()
    T = ctx.scratch("T", (K, LP, R)).double().cpu().numpy()
    tt = {key: v.double().cpu().numpy() for key, v in comp.tensors().items() if v is not None}
    Xs = slices_np(X, off, J)
    Om = om.double().cpu().numpy()
    o = [int(v) for v in off]
    for k in range(K):
        x = Xs[k]
        q1 = Q1[o[k]:o[k + 1]]
        Q = q1 @ M2[k]
        np.testing.assert_allclose(Q.T @ Q, np.eye(LP)[:, :LP] * (np.linalg.norm(Q, axis=0) > 0.5), atol=2e-5,
                                   err_msg=f"Q orthonormal, slice {k}")
        Y = x @ Om
        resid = Y - Q @ (Q.T @ Y)
        assert np.linalg.norm(resid) <= 1e-5 * np.linalg.norm(Y), f"sketch span, slice {k}"
        np.testing.assert_allclose(B1[k][:, :J], q1.T @ x, atol=2e-5 * np.abs(q1.T @ x).max(),
                                   err_msg=f"B1, slice {k}")
        g = B1[k][:, :J] @ B1[k][:, :J].T
        np.testing.assert_allclose(GB[k][:ell, :ell], g[:ell, :ell], atol=1e-5 * np.abs(g).max(),
                                   err_msg=f"GB, slice {k}")
        m2 = M2[k][:ell, :ell]
        Gt = m2.T @ g[:ell, :ell] @ m2
        lam, U = np.linalg.eigh(Gt)
        Ur = U[:, np.argsort(-lam)[:R]]
        Tk = T[k][:ell]
        # same column space as M2 U~_R (columns are unique up to sign)
        Tref = m2 @ Ur
        for r in range(R):
            c = abs(Tk[:, r] @ Tref[:, r]) / (np.linalg.norm(Tk[:, r]) * np.linalg.norm(Tref[:, r]))
            assert c >= 1 - 1e-4, f"T column {r}, slice {k}: cos {c}"
        # M_k = B1^T T (block C_k B_k of M) and A_k = Q1 T
        Mk = tt["M"][k]
        np.testing.assert_allclose(Mk, B1[k][:, :J].T @ T[k], atol=2e-5 * np.abs(Mk).max(),
                                   err_msg=f"M block, slice {k}")
        np.testing.assert_allclose(tt["A"][o[k]:o[k + 1]], q1 @ T[k], atol=2e-5, err_msg=f"A, slice {k}")
        np.testing.assert_allclose(tt["Bk"][k], np.linalg.norm(Mk, axis=0), rtol=1e-5)
        # and the stage-1 reconstruction error equals the oracle's randomized SVD's
        a, b, c = od.randomized_svd(x, R, Om)
        e_o = np.sum((x - a @ np.diag(b) @ c.T) ** 2)
        e_g = np.sum((x - tt["A"][o[k]:o[k + 1]] @ Mk.T) ** 2)
        assert abs(e_g - e_o) <= 1e-5 * np.sum(x * x), f"stage-1 error, slice {k}: {e_g} vs {e_o}"
    comp.free()
    ctx.close()
