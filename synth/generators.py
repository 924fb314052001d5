"""Seeded generators of irregular dense tensors {X_k} (I_k x J slices).

Every generator is deterministic given (seed, device).  X is returned as one
row-major matrix of sum(I_k) rows with ``offsets`` (int64, K+1) delimiting
the slices, which is the layout the library consumes.

Workload shapes follow the dataset statistics of the paper's Table
"Description" (max I_k, J, K of FMA / Urban / US Stock); the data itself is
synthetic: a PARAFAC2 model X_k = U_k H S_k V^T (Def. 1, Sec. II-C) plus
noise, with the per-workload post-processing stated in each function.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch


@dataclass(frozen=True)
class Workload:
    name: str
    K: int
    Imin: int
    Imax: int
    J: int
    R: int
    p: int
    lengths: str  # "uniform" | "loguniform"
    kind: str  # "plain" | "spectrogram" | "series"

    @property
    def ell(self) -> int:
        return self.R + self.p


WORKLOADS = {
    # K=64, I_k in U{50..200}, J=64, R=10; noisy (20 dB) PARAFAC2 model.
    "plain": Workload("plain", 64, 50, 200, 64, 10, 10, "uniform", "plain"),
    # FMA-shaped: K=8000, I_k in U{100..704}, J=2049, R=10, nonnegative magnitudes.
    "spectrogram": Workload("spectrogram", 8000, 100, 704, 2049, 10, 10, "uniform", "spectrogram"),
    # US-Stock-shaped: K=4742, I_k log-uniform in [100,7883], J=88, R=20.
    "skewed": Workload("skewed", 4742, 100, 7883, 88, 20, 10, "loguniform", "series"),
    # Urban-shaped rank sweep: K=8455, I_k in U{32..174}, J=2049 (R set per run).
    "ranksweep": Workload("ranksweep", 8455, 32, 174, 2049, 10, 10, "uniform", "spectrogram"),
    # learned-sketch training set: 2000 FMA-shaped slices, R=20.
    "learned": Workload("learned", 2000, 100, 704, 2049, 20, 10, "uniform", "spectrogram"),
    # the paper's synthetic scalability tensors (Sec. IV-A/IV-C): regular I x J x K,
    # uniform on [0, 1); sizes from 1000^3 to 2000 x 2000 x 4000.
    "tenrand": Workload("tenrand", 4000, 2000, 2000, 2000, 10, 10, "uniform", "tenrand"),
}


def workload(name: str, **overrides) -> Workload:
    w = WORKLOADS[name]
    if overrides:
        d = dict(w.__dict__)
        d.update(overrides)
        w = Workload(**d)
    return w


def _gen(device, seed: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def make_row_offsets(K: int, Imin: int, Imax: int, seed: int, lengths: str = "uniform") -> torch.Tensor:
    """Slice lengths I_k drawn on the CPU; returns int64 offsets (K+1)."""
    g = _gen("cpu", seed)
    if lengths == "uniform":
        I = torch.randint(Imin, Imax + 1, (K,), generator=g, dtype=torch.int64)
    elif lengths == "loguniform":
        u = torch.rand(K, generator=g, dtype=torch.float64)
        I = torch.exp(math.log(Imin) + u * (math.log(Imax) - math.log(Imin)))
        I = I.round().clamp(Imin, Imax).to(torch.int64)
    else:
        raise ValueError(lengths)
    off = torch.zeros(K + 1, dtype=torch.int64)
    off[1:] = torch.cumsum(I, 0)
    return off


def bf16_representable(x: torch.Tensor) -> torch.Tensor:
    """Round to the nearest bf16 value and flush magnitudes below 2^-14 to 0,
    so the result is exactly representable in fp32, bf16 and fp16 alike."""
    y = x.to(torch.float32).to(torch.bfloat16).to(torch.float32)
    return torch.where(y.abs() < 2.0 ** -14, torch.zeros_like(y), y)


def gaussian_matrix(rows: int, cols: int, seed: int, device="cpu", representable16: bool = True) -> torch.Tensor:
    """Seeded standard Gaussian rows x cols matrix (float32)."""
    g = _gen(device, seed)
    x = torch.randn(rows, cols, generator=g, device=device, dtype=torch.float32)
    return bf16_representable(x) if representable16 else x


def _model_energy(H, V, W, offsets) -> float:
    """sum_k ||H diag(W_k) V^T||_F^2 (the model's energy when every U_k has
    orthonormal columns)."""
    G = (H.T @ H) * (V.T @ V)
    I = (offsets[1:] - offsets[:-1]).to(W.device)
    cnt = (I >= H.shape[0]).to(W.dtype)  # slices with I_k < R have orthonormal rows: approximate
    return float(((W @ G) * W).sum(1).mul(cnt).sum())


def _orthonormal(n: int, r: int, g, device, dtype) -> torch.Tensor:
    """n x r with orthonormal columns (n >= r) or orthonormal rows (n < r)."""
    if n >= r:
        q, _ = torch.linalg.qr(torch.randn(n, r, generator=g, device=device, dtype=dtype).cpu())
        return q.to(device)
    q, _ = torch.linalg.qr(torch.randn(r, n, generator=g, device=device, dtype=dtype).cpu())
    return q.T.contiguous().to(device)


def _parafac2_slices(offsets, J, R, seed, device, dtype, s_std=0.3):
    """Yields (k, r0, r1, signal_k) for the PARAFAC2 model U_k H S_k V^T."""
    g = _gen(device, seed)
    K = offsets.numel() - 1
    H = torch.randn(R, R, generator=g, device=device, dtype=dtype)
    V = torch.randn(J, R, generator=g, device=device, dtype=dtype)
    W = (1.0 + s_std * torch.randn(K, R, generator=g, device=device, dtype=dtype)).abs()
    off = offsets.tolist()
    for k in range(K):
        n = off[k + 1] - off[k]
        U = _orthonormal(n, R, g, device, dtype)
        yield k, off[k], off[k + 1], U, H, V, W


def plain_parafac2(K=64, Imin=50, Imax=200, J=64, R=10, seed=1001, snr_db=20.0,
                   device="cpu", dtype=torch.float64, offsets=None):
    """X_k = U_k H S_k V^T + noise, U_k orthonormal (QR of a Gaussian), H and V
    Gaussian, S_k = diag|N(1, 0.3)|; noise variance set globally for the given
    SNR (sigma^2 = ||signal||_F^2 / (10^(snr/10) N)); snr_db=None -> noiseless.

    Returns dict(X, offsets, U (list), H, V, W)."""
    if offsets is None:
        offsets = make_row_offsets(K, Imin, Imax, seed)
    N = int(offsets[-1])
    X = torch.empty(N, J, device=device, dtype=dtype)
    Us = []
    H = V = W = None
    for k, r0, r1, U, H, V, W in _parafac2_slices(offsets, J, R, seed + 7, device, dtype):
        X[r0:r1] = U @ (H * W[k]) @ V.T
        Us.append(U)
    if snr_db is not None:
        g = _gen(device, seed + 13)
        sig2 = float((X * X).sum()) / (10.0 ** (snr_db / 10.0) * X.numel())
        X += math.sqrt(sig2) * torch.randn(X.shape, generator=g, device=device, dtype=dtype)
    return dict(X=X, offsets=offsets, U=Us, H=H, V=V, W=W)


def spectrogram_like(K=8000, Imin=100, Imax=704, J=2049, R=10, seed=1002, snr_db=20.0,
                     device="cpu", out_dtype=torch.float32, ld=None, chunk_rows=1 << 20):
    """|PARAFAC2 model + noise|: nonnegative magnitudes shaped like log-power
    spectrogram slices (time x frequency).  Generated in float32 chunk by
    chunk directly into an (sum I_k) x ld buffer of ``out_dtype`` (ld >= J;
    columns >= J are zero).  Returns dict(X, offsets, ld)."""
    offsets = make_row_offsets(K, Imin, Imax, seed)
    N = int(offsets[-1])
    ld = J if ld is None else ld
    X = torch.zeros(N, ld, device=device, dtype=out_dtype)
    g = _gen(device, seed + 7)
    H = torch.randn(R, R, generator=g, device=device)
    V = torch.randn(J, R, generator=g, device=device)
    Wt = (1.0 + 0.3 * torch.randn(K, R, generator=g, device=device)).abs()
    # ||U_k H S_k V^T||_F^2 = ||H S_k V^T||_F^2 (U_k orthonormal columns), so the
    # global signal energy per entry is known before any slice is formed.
    e_sig = _model_energy(H, V, Wt, offsets) / N
    sigma = math.sqrt(e_sig / 10.0 ** (snr_db / 10.0))
    off = offsets.tolist()
    # group slices by length so the orthonormal U_k are made by batched QR
    lengths = torch.tensor([off[k + 1] - off[k] for k in range(K)])
    gu = _gen(device, seed + 11)
    gq = _gen("cpu", seed + 17)
    for n in torch.unique(lengths).tolist():
        ks = (lengths == n).nonzero().flatten().tolist()
        for b0 in range(0, len(ks), 256):
            kb = ks[b0:b0 + 256]
            # orthonormal U_k from batched QR on the host (small n x R matrices)
            A = torch.randn(len(kb), n, R, generator=gq)
            if n >= R:
                U, _ = torch.linalg.qr(A)
            else:
                Qt, _ = torch.linalg.qr(A.transpose(1, 2))
                U = Qt.transpose(1, 2)
            U = U.to(device)
            HS = H.unsqueeze(0) * Wt[kb].unsqueeze(1)  # B x R x R
            sl = U @ (HS @ V.T.unsqueeze(0))  # B x n x J
            sl += sigma * torch.randn(sl.shape, generator=gu, device=device)
            sl = sl.abs_()
            for i, k in enumerate(kb):
                X[off[k]:off[k + 1], :J] = sl[i].to(out_dtype)
    return dict(X=X, offsets=offsets, ld=ld)


def _ar1_rows(T, J, phi, g, device):
    """T x J AR(1) along rows with unit stationary variance."""
    e = torch.empty(T, J, device=device)
    c = math.sqrt(1.0 - phi * phi)
    B = 64
    L = torch.tril(torch.tensor([[phi ** (i - j) if i >= j else 0.0 for j in range(B)] for i in range(B)],
                                device=device, dtype=torch.float32))
    state = torch.randn(J, generator=g, device=device)
    for t0 in range(0, T, B):
        n = min(B, T - t0)
        xi = c * torch.randn(n, J, generator=g, device=device)
        pw1 = phi ** torch.arange(1, n + 1, device=device, dtype=torch.float32)
        blk = L[:n, :n] @ xi + pw1.view(n, 1) * state.view(1, J)
        e[t0:t0 + n] = blk
        state = blk[-1]
    return e


def skewed_series(K=4742, Imin=100, Imax=7883, J=88, R=20, seed=1003, phi=0.95, ar_scale=0.3,
                  device="cpu", out_dtype=torch.float32, ld=None):
    """Stock-like series: low-rank PARAFAC2 signal scaled to unit entry
    variance, plus ar_scale * AR(1) noise along rows (phi, innovations
    N(0, 1 - phi^2)), then every slice's columns z-scored (a column with zero
    variance is only centred).  I_k log-uniform in [Imin, Imax]."""
    offsets = make_row_offsets(K, Imin, Imax, seed, "loguniform")
    N = int(offsets[-1])
    ld = J if ld is None else ld
    X = torch.zeros(N, ld, device=device, dtype=out_dtype)
    g = _gen(device, seed + 7)
    H = torch.randn(R, R, generator=g, device=device)
    V = torch.randn(J, R, generator=g, device=device)
    Wt = (1.0 + 0.3 * torch.randn(K, R, generator=g, device=device)).abs()
    scale = 1.0 / math.sqrt(_model_energy(H, V, Wt, offsets) / N)
    off = offsets.tolist()
    for k in range(K):
        n = off[k + 1] - off[k]
        U = _orthonormal(n, R, g, device, torch.float32)
        s = scale * (U @ (H * Wt[k]) @ V.T)
        s += ar_scale * _ar1_rows(n, J, phi, g, device)
        mu = s.mean(0, keepdim=True)
        sd = s.std(0, keepdim=True)
        s = (s - mu) / torch.where(sd > 0, sd, torch.ones_like(sd))
        X[off[k]:off[k + 1], :J] = s.to(out_dtype)
    return dict(X=X, offsets=offsets, ld=ld)


def tenrand(I=2000, J=2000, K=4000, seed=1006, device="cpu", out_dtype=torch.float32, ld=None,
            chunk_rows=1 << 20):
    """The synthetic tensors of the paper's scalability experiments (Sec. IV-A,
    "Synthetic Data"; Tensor Toolbox's tenrand(I, J, K)): entries drawn
    independently and uniformly from [0, 1), slice k = X(:, :, k), every slice
    I x J.  Written chunk by chunk into a (K I) x ld buffer of ``out_dtype``
    (ld >= J, columns >= J zero) straight from the device generator, so a
    32 GB BF16 tensor needs no FP32 copy.  Returns dict(X, offsets, ld)."""
    offsets = torch.arange(K + 1, dtype=torch.int64) * I
    N = K * I
    ld = J if ld is None else ld
    X = torch.zeros(N, ld, device=device, dtype=out_dtype)
    g = _gen(device, seed)
    for r0 in range(0, N, chunk_rows):
        r1 = min(N, r0 + chunk_rows)
        X[r0:r1, :J] = torch.rand(r1 - r0, J, generator=g, device=device).to(out_dtype)
    return dict(X=X, offsets=offsets, ld=ld)


def stock_factors(K=4742, I=324, R=10, clusters=40, spread=0.6, seed=1007, device="cpu"):
    """Fitted-factor-like inputs for the post-fit analyses (Sec. IV-E): K
    slices of one length I (stocks over a common date range), U_k = Q_k H
    with Q_k = the orthonormal factor of (C_c + spread * N(0, 1)) for the
    slice's cluster c (clusters of similar stocks), C_c standard Gaussian
    I x R, and H with unit-norm columns, so that ||U_k||_F^2 = R as for the
    U_k = Q_k H of a fit.  Returns dict(U (K, I, R) float32, labels (K,))."""
    g = _gen(device, seed)
    H = torch.randn(R, R, generator=g, device=device)
    H = H / H.norm(dim=0, keepdim=True)
    C = torch.randn(clusters, I, R, generator=g, device=device)
    labels = torch.randint(0, clusters, (K,), generator=g, device=device)
    A = C[labels] + spread * torch.randn(K, I, R, generator=g, device=device)
    Q, _ = torch.linalg.qr(A.cpu())
    U = (Q.to(device) @ H).float().contiguous()
    return dict(U=U, labels=labels)
