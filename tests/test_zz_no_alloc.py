"""The allocation-free identity-mode error entry point
(dpar2_reconstruct_error_noalloc) against dpar2_reconstruct_error, through the
C ABI.  The file name puts it last in collection, so in a full run it also
executes after every other GPU test of the same process; it passes alone too."""
import numpy as np
import pytest
import torch

import synth

from _gpu import api_or_skip, padded

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return api_or_skip()


@pytest.fixture(scope="module")
def ctx(api):
    return api.Context(0)


def test_noalloc_equals_reconstruct_error_on_consecutive_calls(api, ctx):
    d = synth.plain_parafac2(K=64, Imin=50, Imax=200, J=64, R=10, seed=1001)
    X = padded(d["X"].cuda().float(), 64, torch.float32)
    comp = ctx.compress(X, d["offsets"], R=10, p=10, J=64)
    res = ctx.fit(comp, max_iter=12)
    sq, fit = ctx.reconstruct_error(comp, res.H, res.V, res.W, Upol=res.Upol)
    tot = float((X.double() ** 2).sum())
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        sq2, fit2 = ctx.reconstruct_error_noalloc(comp, res.H, res.V, res.W, res.Upol)
        # the same kernels on the same inputs: equal up to summation order
        assert abs(sq2 - sq) <= 1e-9 * tot
        assert abs(fit2 - fit) <= 1e-9
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0  # no device memory taken


def test_noalloc_rejects_problems_beyond_its_scratch(api, ctx):
    # K R^2 = 4.2e6 > 4,194,304: rejected before anything is launched
    K, J, R = 42000, 24, 10
    off = torch.arange(K + 1, dtype=torch.int64)  # one row per slice
    X = torch.rand(K, J, device="cuda")
    comp = ctx.compress(X, off, R=R, p=10, J=J)
    H = torch.zeros(R, R, device="cuda")
    V = torch.zeros(J, R, device="cuda")
    W = torch.zeros(K, R, device="cuda")
    Up = torch.zeros(K, R, R, device="cuda")
    with pytest.raises(api.Dpar2Error) as e:
        ctx.reconstruct_error_noalloc(comp, H, V, W, Up)
    assert api.STATUS[e.value.code] == "INVALID_ARG" and "scratch" in str(e.value)
    # the entry point stays usable after a rejection
    d = synth.plain_parafac2(K=16, Imin=30, Imax=60, J=32, R=4, seed=3)
    X2 = padded(d["X"].cuda().float(), 32, torch.float32)
    c2 = ctx.compress(X2, d["offsets"], R=4, p=4, J=32)
    r2 = ctx.fit(c2, max_iter=4)
    sq_a, _ = ctx.reconstruct_error(c2, r2.H, r2.V, r2.W, Upol=r2.Upol)
    sq_b, _ = ctx.reconstruct_error_noalloc(c2, r2.H, r2.V, r2.W, r2.Upol)
    assert abs(sq_a - sq_b) <= 1e-9 * float((X2.double() ** 2).sum())
