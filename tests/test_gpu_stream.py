"""Compression from host memory (dpar2_compress_host) against dpar2_compress
on the same X: stage 1 is per slice (Alg. 1), so compressing chunk by chunk
must give the compression of the whole tensor; the library's launch counter.

Tolerances: the chunks run the same kernels per slice, but a chunk of fewer
than 256 slices sums its CholeskyQR Grams in a different order, so results
agree to FP32 rounding (relative 1e-5 on the reconstructions), not bit for
bit; the copy of X that X_dev receives is exact."""
import numpy as np
import pytest
import torch

import synth

from _gpu import api_or_skip, padded, rel_sq_err, slices_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    return api_or_skip()


@pytest.fixture(scope="module")
def ctx(api):
    return api.Context(0)


def _recs(t, off):
    A = t["A"].double().cpu().numpy()
    D = t["D"].double().cpu().numpy()
    Ft = t["Ft"].double().cpu().numpy()
    o = [int(v) for v in off]
    return [A[o[k]:o[k + 1]] @ Ft[k] @ D.T for k in range(len(o) - 1)]


# (J, dtype, keep X on the device, chunk bytes): J = 77 pads rows (staged
# copies re-pitched on the device), J = 64 FP32 has the device pitch (direct
# copies); chunks of a few slices up to the whole tensor
CASES = [(77, torch.bfloat16, True, 40_000), (77, torch.bfloat16, False, 200_000), (64, torch.float32, False, 60_000),
         (64, torch.float32, True, 0), (301, torch.float16, False, 150_000)]


@pytest.mark.parametrize("J,dtype,keep,chunk", CASES)
def test_compress_host_equals_compress(api, ctx, J, dtype, keep, chunk):
    d = synth.plain_parafac2(K=90, Imin=20, Imax=300, J=J, R=10, seed=41)
    off = d["offsets"]
    om = synth.gaussian_matrix(J, 20, seed=4).cuda()
    om2 = synth.gaussian_matrix(90 * 10, 20, seed=5).cuda()
    Xd = padded(d["X"].cuda().float(), J, dtype)
    Xh = Xd[:, :J].cpu().contiguous().pin_memory()
    ref = ctx.compress(Xd, off, R=10, p=10, omega=om, omega2=om2, J=J)
    Xkeep = torch.full_like(Xd, 3.0) if keep else None
    got = ctx.compress_host(Xh, off, R=10, p=10, omega=om, omega2=om2, X_dev=Xkeep, chunk_bytes=chunk)
    a, b = ref.tensors(), got.tensors()
    Xs = slices_np(Xd, off, J)
    tot = sum(float(np.sum(x * x)) for x in Xs)
    ra, rb = _recs(a, off), _recs(b, off)
    assert abs(rel_sq_err(Xs, ra) - rel_sq_err(Xs, rb)) <= 1e-6
    assert np.sqrt(sum(np.sum((x - y) ** 2) for x, y in zip(ra, rb)) / tot) <= 1e-5
    np.testing.assert_allclose(b["xnorm2"].cpu().numpy(), a["xnorm2"].cpu().numpy(), rtol=1e-9)
    assert torch.equal(a["rank1"], b["rank1"])
    # the per-slice stage-1 factors: the same reconstructions A_k M_k^T
    A1, A2 = a["A"].double().cpu().numpy(), b["A"].double().cpu().numpy()
    M1, M2 = a["M"].double().cpu().numpy(), b["M"].double().cpu().numpy()
    o = [int(v) for v in off]
    for k in range(0, 90, 11):
        x1 = A1[o[k]:o[k + 1]] @ M1[k].T
        x2 = A2[o[k]:o[k + 1]] @ M2[k].T
        assert np.linalg.norm(x1 - x2) <= 1e-5 * max(np.linalg.norm(x1), 1e-30)
    if keep:
        assert torch.equal(Xkeep, Xd)  # X rows copied, pad columns zeroed
    # the fit on either compression reaches the same fitness
    fa = ctx.fit(ref, max_iter=8).fitness
    fb = ctx.fit(got, max_iter=8).fitness
    assert abs(fa - fb) <= 1e-5


def test_compress_host_rejects_bad_arguments(api, ctx):
    d = synth.plain_parafac2(K=4, Imin=30, Imax=40, J=32, R=4, seed=1)
    Xh = d["X"].float().contiguous()
    bad = d["offsets"].clone()
    bad[2] = bad[1]
    with pytest.raises(api.Dpar2Error) as e:
        ctx.compress_host(Xh, bad, R=4, p=4)
    assert e.value.code == 2
    Xu = torch.zeros(Xh.shape[0], 33, device="cuda")  # 33 floats = 132 bytes per row
    with pytest.raises(api.Dpar2Error) as e:
        ctx.compress_host(Xh, d["offsets"], R=4, p=4, X_dev=Xu)
    assert e.value.code in (1, 2)


def test_kernel_launch_counter_counts_graph_launches(api, ctx):
    # the per-iteration ALS loop runs as one CUDA graph by default and as
    # separate launches with FLAG_NO_GRAPH: the same kernels, so the same
    # count (at least three launches per iteration); the persistent form runs
    # the whole loop in one launch
    d = synth.plain_parafac2(K=30, Imin=50, Imax=150, J=64, R=10, seed=23)
    X = padded(d["X"].cuda().float(), 64, torch.float32)
    comp = ctx.compress(X, d["offsets"], R=10, p=10, J=64)
    torch.cuda.synchronize()
    n0 = api.kernel_launches()
    ctx.fit(comp, max_iter=6, flags=api.FLAG_NO_PERSIST)
    n1 = api.kernel_launches()
    ctx.fit(comp, max_iter=6, flags=api.FLAG_NO_PERSIST | api.FLAG_NO_GRAPH)
    n2 = api.kernel_launches()
    ctx.fit(comp, max_iter=6)
    n3 = api.kernel_launches()
    assert n1 - n0 == n2 - n1 >= 6 * 3
    assert n3 - n2 < 6 * 3
