"""Helpers shared by the GPU tests: library loading and oracle-side views of
GPU results (no numerical method code here; the oracle computes, these only
reshape)."""
import numpy as np
import pytest
import torch

import synth


def api_or_skip():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2203_12798_gb300 as pkg

    pkg.build()
    return pkg.load()


def slices_np(X, offsets, J):
    """float64 numpy slices of the stored X (first J columns)."""
    Xn = X[:, :J].double().cpu().numpy()
    off = [int(v) for v in offsets]
    return [Xn[off[k]:off[k + 1]] for k in range(len(off) - 1)]


def padded(X, J, dtype, mult=16):
    """Copy X (N x J) into a row-padded (N x ld) tensor of `dtype` (ld * size % mult == 0)."""
    es = torch.empty((), dtype=dtype).element_size()
    step = mult // es
    ld = (J + step - 1) // step * step
    out = torch.zeros(X.shape[0], ld, dtype=dtype, device=X.device)
    out[:, :J] = X.to(dtype)
    return out


def problem(K=64, Imin=50, Imax=200, J=64, R=10, seed=1001, snr_db=20.0, device="cuda"):
    d = synth.plain_parafac2(K=K, Imin=Imin, Imax=Imax, J=J, R=R, seed=seed, snr_db=snr_db)
    return d


def rel_sq_err(Xs, recs):
    num = sum(float(np.sum((x - r) ** 2)) for x, r in zip(Xs, recs))
    den = sum(float(np.sum(x * x)) for x in Xs)
    return num / den
