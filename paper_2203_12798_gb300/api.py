"""Python binding of libdpar2 (ctypes over the C ABI of include/dpar2.h).

Argument marshalling only: tensors are passed as raw device pointers together
with the current torch CUDA stream; every numerical step runs in the
library's kernels.  The library must be built (``build.build()``); importing
this module on a machine without it raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from .build import LIB

F32, BF16, F16 = 0, 1, 2
_DT = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
FLAG_PER_SLICE, FLAG_NO_GRAPH, FLAG_GENERIC, FLAG_DROP_M, FLAG_COLD_QSTEP = 0x1, 0x2, 0x4, 0x8, 0x10
FLAG_FIVE_LAUNCH = 0x20
FLAG_NO_PERSIST = 0x40

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "SHAPE", 3: "CUDA", 4: "NUMERICAL", 5: "TIMEOUT", 6: "OOM",
          7: "UNSUPPORTED"}


class Dpar2Error(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"dpar2 {STATUS.get(code, code)}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int), ("p", ctypes.c_int), ("q", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("max_iter", ctypes.c_int), ("tol", ctypes.c_double), ("schedule", ctypes.c_int),
                ("flags", ctypes.c_uint), ("proj_cols", ctypes.c_int)]


class CompView(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("J", ctypes.c_int), ("R", ctypes.c_int), ("ell", ctypes.c_int),
                ("Jq", ctypes.c_int), ("N", ctypes.c_int64), ("offsets", ctypes.c_void_p), ("A", ctypes.c_void_p),
                ("Bk", ctypes.c_void_p), ("Ms", ctypes.c_void_p), ("D", ctypes.c_void_p), ("E", ctypes.c_void_p),
                ("Ft", ctypes.c_void_p), ("xnorm2", ctypes.c_void_p), ("rank1", ctypes.c_void_p)]


_lib = None
VP, I64, DP = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)

# name -> (restype, argtypes); mirrors include/dpar2.h
SIGNATURES = {
    "dpar2_options_default": (ctypes.c_int, [ctypes.POINTER(Options)]),
    "dpar2_create": (ctypes.c_int, [ctypes.POINTER(VP), ctypes.c_int]),
    "dpar2_destroy": (None, [VP]),
    "dpar2_last_error": (ctypes.c_char_p, [VP]),
    "dpar2_gaussian": (ctypes.c_int, [VP, ctypes.c_uint64, ctypes.c_uint32, I64, VP, ctypes.c_int, VP]),
    "dpar2_philox_words": (ctypes.c_int, [VP, ctypes.c_uint64, ctypes.c_uint32, I64, VP, VP]),
    "dpar2_compress": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), VP, I64,
                                      ctypes.c_int, ctypes.POINTER(Options), VP, VP, ctypes.POINTER(VP), VP]),
    "dpar2_compress_host": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), VP,
                                           ctypes.c_int, ctypes.POINTER(Options), VP, VP, VP, I64, ctypes.c_size_t,
                                           ctypes.POINTER(VP), VP]),
    "dpar2_kernel_launches": (ctypes.c_longlong, []),
    "dpar2_fit": (ctypes.c_int, [VP, VP, ctypes.POINTER(Options), VP, VP, VP, VP, VP, VP, DP,
                                 ctypes.POINTER(ctypes.c_int), DP, VP]),
    "dpar2_reconstruct_error": (ctypes.c_int, [VP, VP, VP, I64, ctypes.c_int, VP, VP, VP, VP, DP, DP, VP]),
    "dpar2_reconstruct_error_noalloc": (ctypes.c_int, [VP, VP, VP, VP, VP, VP, DP, DP, VP]),
    "dpar2_last_info": (ctypes.c_int, [VP]),
    "dpar2_comp_bytes": (ctypes.c_size_t, [VP]),
    "dpar2_comp_device_bytes": (ctypes.c_size_t, [VP]),
    "dpar2_comp_view_get": (ctypes.c_int, [VP, ctypes.POINTER(CompView)]),
    "dpar2_projection_config": (ctypes.c_int, [VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "dpar2_comp_m": (ctypes.c_int, [VP, VP, VP, VP]),
    "dpar2_comp_free": (None, [VP]),
    "dpar2_sketch_loss_fwd": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), VP,
                                             I64, ctypes.c_int, VP, ctypes.c_int, DP, VP]),
    "dpar2_sketch_loss_bwd": (ctypes.c_int, [VP, ctypes.c_double, VP, VP]),
    "dpar2_orthonormalize": (ctypes.c_int, [VP, I64, ctypes.c_int, VP, VP]),
    "dpar2_upload_rows": (ctypes.c_int, [VP, VP, I64, ctypes.c_int, ctypes.c_int, VP, I64, VP]),
    "dpar2_scratch": (ctypes.c_int, [VP, ctypes.c_char_p, ctypes.POINTER(VP), ctypes.POINTER(ctypes.c_size_t)]),
    "dpar2_set_timing": (ctypes.c_int, [VP, ctypes.c_int]),
    "dpar2_last_timings": (ctypes.c_int, [VP, DP, ctypes.c_int]),
    "dpar2_similarity": (ctypes.c_int, [VP, ctypes.c_int, I64, VP, I64, ctypes.c_double, VP, I64, VP]),
    "dpar2_topk": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int, VP, I64, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                  VP, VP, VP]),
    "dpar2_rwr": (ctypes.c_int, [VP, ctypes.c_int, VP, I64, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                 ctypes.c_double, ctypes.c_int, VP, VP]),
    "dpar2_feature_pcc": (ctypes.c_int, [VP, ctypes.c_int, ctypes.c_int, VP, VP, VP]),
}

PHASES = ["sketch", "qr", "project", "small", "stage2", "compress", "als", "output"]


def lib():
    """Load libdpar2.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_2203_12798_gb300.build.build()")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def kernel_launches() -> int:
    """Kernels the library has launched since it was loaded (all contexts)."""
    return int(lib().dpar2_kernel_launches())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Context:
    """A library context bound to one CUDA device (owns reusable scratch)."""

    def __init__(self, device: int = 0):
        self.device = device
        self._h = ctypes.c_void_p()
        self._check(lib().dpar2_create(ctypes.byref(self._h), device), "dpar2_create")

    def _check(self, code, what=""):
        if code != 0:
            msg = lib().dpar2_last_error(self._h).decode() if self._h else what
            raise Dpar2Error(code, msg or what)

    def close(self):
        if self._h:
            lib().dpar2_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, Xh: torch.Tensor, Xd: torch.Tensor):
        """Host rows (rows x J, packed; pinned for async) -> device rows with row stride Xd.stride(0)."""
        assert Xh.dim() == 2 and Xh.is_contiguous() and Xd.dim() == 2 and Xd.stride(1) == 1
        self._check(lib().dpar2_upload_rows(self._h, _ptr(Xh), Xh.shape[0], Xh.shape[1], _DT[Xh.dtype], _ptr(Xd),
                                            Xd.stride(0), _stream()))

    def scratch(self, name: str, shape, dtype=torch.float32) -> torch.Tensor:
        """Copy of the named scratch buffer of the last call (inspection only)."""
        p = ctypes.c_void_p()
        nb = ctypes.c_size_t()
        self._check(lib().dpar2_scratch(self._h, name.encode(), ctypes.byref(p), ctypes.byref(nb)))
        out = torch.empty(shape, dtype=dtype, device=f"cuda:{self.device}")
        need = out.numel() * out.element_size()
        assert need <= nb.value, (name, need, nb.value)
        out.view(-1).view(torch.uint8).copy_(_DevPtr(p.value, need).as_tensor(f"cuda:{self.device}"))
        return out

    # ------------------------------------------------------------- timing
    def set_timing(self, on: bool = True):
        self._check(lib().dpar2_set_timing(self._h, int(on)))

    def last_info(self) -> dict:
        """Information bits of the last call (dropped pivots, Jacobi sweep cap, pinv fallback)."""
        v = lib().dpar2_last_info(self._h)
        return {"rank_drop": bool(v & 4), "sweep_cap": bool(v & 8), "pinv": bool(v & 16)}

    def timings(self) -> dict:
        """Milliseconds of each phase of the last compress / fit (CUDA events
        recorded on the library's work stream)."""
        buf = (ctypes.c_double * len(PHASES))()
        n = lib().dpar2_last_timings(self._h, buf, len(PHASES))
        return {PHASES[i]: buf[i] for i in range(n)}

    # ------------------------------------------------------------- RNG
    def gaussian(self, seed: int, stream_id: int, n: int, round16: bool = True, out=None):
        out = torch.empty(n, dtype=torch.float32, device=f"cuda:{self.device}") if out is None else out
        self._check(lib().dpar2_gaussian(self._h, seed, stream_id, n, _ptr(out), int(round16), _stream()))
        return out

    def philox_words(self, seed: int, stream_id: int, n: int):
        out = torch.empty(n, dtype=torch.int32, device=f"cuda:{self.device}")
        self._check(lib().dpar2_philox_words(self._h, seed, stream_id, n, _ptr(out), _stream()))
        return out

    # ------------------------------------------------------------- method
    def compress(self, X: torch.Tensor, offsets, R=10, p=10, q=0, seed=0, omega=None, omega2=None, flags=0,
                 J=None, schedule=-1, proj_cols=0) -> "Compressed":
        """X: CUDA tensor (sum I_k) x ldx of float32/bfloat16/float16 (columns >= J ignored)."""
        assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        J = X.shape[1] if J is None else J
        off = torch.as_tensor(offsets, dtype=torch.int64).cpu().contiguous()
        K = off.numel() - 1
        opt = Options()
        lib().dpar2_options_default(ctypes.byref(opt))
        opt.R, opt.p, opt.q, opt.seed, opt.flags, opt.schedule = R, p, q, seed, flags, schedule
        opt.proj_cols = proj_cols
        h = ctypes.c_void_p()
        offp = ctypes.cast(off.data_ptr(), ctypes.POINTER(ctypes.c_int64))
        self._check(lib().dpar2_compress(self._h, K, J, offp, _ptr(X), X.stride(0), _DT[X.dtype],
                                         ctypes.byref(opt), _ptr(omega), _ptr(omega2), ctypes.byref(h),
                                         _stream()))
        return Compressed(self, h, off)

    def compress_host(self, Xh: torch.Tensor, offsets, R=10, p=10, q=0, seed=0, omega=None, omega2=None, flags=0,
                      X_dev=None, chunk_bytes=0, schedule=-1, proj_cols=0) -> "Compressed":
        """Xh: host tensor (sum I_k) x J of float32/bfloat16/float16, packed rows
        (pin_memory() for asynchronous copies); X_dev: optional CUDA tensor
        (sum I_k) x ldx receiving X."""
        assert not Xh.is_cuda and Xh.dim() == 2 and Xh.is_contiguous()
        J = Xh.shape[1]
        off = torch.as_tensor(offsets, dtype=torch.int64).cpu().contiguous()
        K = off.numel() - 1
        opt = Options()
        lib().dpar2_options_default(ctypes.byref(opt))
        opt.R, opt.p, opt.q, opt.seed, opt.flags, opt.schedule = R, p, q, seed, flags, schedule
        opt.proj_cols = proj_cols
        h = ctypes.c_void_p()
        offp = ctypes.cast(off.data_ptr(), ctypes.POINTER(ctypes.c_int64))
        ldx = X_dev.stride(0) if X_dev is not None else 0
        self._check(lib().dpar2_compress_host(self._h, K, J, offp, ctypes.c_void_p(Xh.data_ptr()), _DT[Xh.dtype],
                                              ctypes.byref(opt), _ptr(omega), _ptr(omega2), _ptr(X_dev), ldx,
                                              chunk_bytes, ctypes.byref(h), _stream()))
        return Compressed(self, h, off)

    def projection_config(self):
        """(schedule, columns per work item) of the last compression's tensor-core
        projection; (-1, 0) if none ran."""
        sch, cols = ctypes.c_int(-1), ctypes.c_int(0)
        self._check(lib().dpar2_projection_config(self._h, ctypes.byref(sch), ctypes.byref(cols)))
        return sch.value, cols.value

    def fit(self, comp: "Compressed", max_iter=32, tol=-1.0, seed=0, V0=None, want_U=False, want_upol=True,
            fitness=True, flags=0):
        v = comp.view()
        dev = f"cuda:{self.device}"
        H = torch.empty(v.R, v.R, device=dev)
        V = torch.empty(v.J, v.R, device=dev)
        W = torch.empty(v.K, v.R, device=dev)
        Up = torch.empty(v.K, v.R, v.R, device=dev) if want_upol else None
        U = torch.empty(v.N, v.R, device=dev) if want_U else None
        hist = (ctypes.c_double * max_iter)()
        iters = ctypes.c_int(0)
        fit = ctypes.c_double(0.0)
        opt = Options()
        lib().dpar2_options_default(ctypes.byref(opt))
        opt.R, opt.max_iter, opt.tol, opt.seed, opt.flags = v.R, max_iter, tol, seed, flags
        self._check(lib().dpar2_fit(self._h, comp._h, ctypes.byref(opt), _ptr(V0), _ptr(H), _ptr(V), _ptr(W),
                                    _ptr(Up), _ptr(U), hist, ctypes.byref(iters),
                                    ctypes.byref(fit) if fitness else None, _stream()))
        return FitResult(H=H, V=V, W=W, Upol=Up, U=U, losses=list(hist)[:iters.value], iters=iters.value,
                         fitness=fit.value if fitness else None)

    def reconstruct_error(self, comp: "Compressed", H, V, W, Upol=None, X=None):
        sq = ctypes.c_double()
        fit = ctypes.c_double()
        ldx = X.stride(0) if X is not None else 0
        dt = _DT[X.dtype] if X is not None else 0
        self._check(lib().dpar2_reconstruct_error(self._h, comp._h, _ptr(X), ldx, dt, _ptr(H), _ptr(V), _ptr(W),
                                                  _ptr(Upol), ctypes.byref(sq), ctypes.byref(fit), _stream()))
        return sq.value, fit.value

    # ------------------------------------------------------------- learned sketch
    def sketch_loss_fwd(self, X: torch.Tensor, offsets, omega: torch.Tensor) -> float:
        """Range-finder loss (1/K) sum_k ||X_k - Y_k Y_k^+ X_k||^2 / ||X_k||^2 of
        omega (J x l, float32, CUDA; X's first J columns are the slices' columns);
        keeps what the backward pass needs."""
        assert X.is_cuda and X.dim() == 2 and X.stride(1) == 1
        assert omega.is_cuda and omega.dtype == torch.float32 and omega.is_contiguous()
        J = omega.shape[0]
        assert X.shape[1] >= J
        off = torch.as_tensor(offsets, dtype=torch.int64).cpu().contiguous()
        offp = ctypes.cast(off.data_ptr(), ctypes.POINTER(ctypes.c_int64))
        loss = ctypes.c_double()
        self._check(lib().dpar2_sketch_loss_fwd(self._h, off.numel() - 1, J, offp, _ptr(X), X.stride(0),
                                                _DT[X.dtype], _ptr(omega), omega.shape[1], ctypes.byref(loss),
                                                _stream()))
        self._sk_gen = getattr(self, "_sk_gen", 0) + 1
        self._sk_shape = tuple(omega.shape)
        return loss.value

    def sketch_loss_bwd(self, grad_scale: float = 1.0, out=None) -> torch.Tensor:
        """grad_scale * dL/dOmega for the X and omega of the last sketch_loss_fwd."""
        shape = getattr(self, "_sk_shape", None)
        if shape is None:
            raise RuntimeError("sketch_loss_bwd needs a sketch_loss_fwd first")
        out = torch.empty(shape, dtype=torch.float32, device=f"cuda:{self.device}") if out is None else out
        self._check(lib().dpar2_sketch_loss_bwd(self._h, float(grad_scale), _ptr(out), _stream()))
        return out

    def orthonormalize(self, A: torch.Tensor) -> torch.Tensor:
        """In place: A (rows x cols, float32, CUDA) <- an orthonormal basis of
        its column space (CholeskyQR2, A = Q R with R upper triangular)."""
        assert A.is_cuda and A.dtype == torch.float32 and A.is_contiguous() and A.dim() == 2
        self._check(lib().dpar2_orthonormalize(self._h, A.shape[0], A.shape[1], _ptr(A), _stream()))
        return A

    # ------------------------------------------------------------- post-fit analyses
    def similarity(self, U: torch.Tensor, gamma: float, out=None) -> torch.Tensor:
        """S (K x K) = exp(-gamma ||U_i - U_j||_F^2) for the rows of U (K x L,
        float32, CUDA: each row one slice's U_k flattened)."""
        assert U.is_cuda and U.dtype == torch.float32 and U.dim() == 2 and U.stride(1) == 1
        K, L = U.shape
        S = torch.empty(K, K, dtype=torch.float32, device=U.device) if out is None else out
        self._check(lib().dpar2_similarity(self._h, K, L, _ptr(U), U.stride(0), float(gamma), _ptr(S), S.stride(0),
                                           _stream()))
        return S

    def topk(self, scores: torch.Tensor, k: int, exclude=None):
        """(idx, val): the k largest entries of each row of scores (float32,
        CUDA), largest first, ties by lower index, column exclude[row] left out."""
        assert scores.is_cuda and scores.dtype == torch.float32 and scores.dim() == 2 and scores.stride(1) == 1
        n_rows, n = scores.shape
        idx = torch.empty(n_rows, k, dtype=torch.int32, device=scores.device)
        val = torch.empty(n_rows, k, dtype=torch.float32, device=scores.device)
        ex = None
        if exclude is not None:
            ex = (ctypes.c_int * n_rows)(*[int(v) for v in exclude])
        self._check(lib().dpar2_topk(self._h, n_rows, n, _ptr(scores), scores.stride(0), ex, k, _ptr(idx), _ptr(val),
                                     _stream()))
        return idx, val

    def rwr(self, S: torch.Tensor, targets, c: float = 0.15, iters: int = 100) -> torch.Tensor:
        """RWR scores (len(targets) x K) on the similarity graph of S."""
        assert S.is_cuda and S.dtype == torch.float32 and S.dim() == 2 and S.stride(1) == 1
        K = S.shape[0]
        t = [int(v) for v in targets]
        r = torch.empty(len(t), K, dtype=torch.float32, device=S.device)
        self._check(lib().dpar2_rwr(self._h, K, _ptr(S), S.stride(0), len(t), (ctypes.c_int * len(t))(*t), float(c),
                                    int(iters), _ptr(r), _stream()))
        return r

    def feature_pcc(self, V: torch.Tensor) -> torch.Tensor:
        """Pearson correlation coefficients (J x J) between the rows of V (J x R)."""
        assert V.is_cuda and V.dtype == torch.float32 and V.is_contiguous() and V.dim() == 2
        J, R = V.shape
        C = torch.empty(J, J, dtype=torch.float32, device=V.device)
        self._check(lib().dpar2_feature_pcc(self._h, J, R, _ptr(V), _ptr(C), _stream()))
        return C

    def reconstruct_error_noalloc(self, comp: "Compressed", H, V, W, Upol):
        """Identity-mode error with the library's fixed device scratch (no device
        allocation; calls must not overlap in time)."""
        sq = ctypes.c_double()
        fit = ctypes.c_double()
        self._check(lib().dpar2_reconstruct_error_noalloc(self._h, comp._h, _ptr(H), _ptr(V), _ptr(W), _ptr(Upol),
                                                          ctypes.byref(sq), ctypes.byref(fit), _stream()))
        return sq.value, fit.value


@dataclass
class FitResult:
    H: torch.Tensor
    V: torch.Tensor
    W: torch.Tensor
    Upol: torch.Tensor
    U: torch.Tensor
    losses: list
    iters: int
    fitness: float


class Compressed:
    """Library-owned compressed representation (A_k, B_k, M, D, E, F^(k)E)."""

    def __init__(self, ctx: Context, h, offsets):
        self.ctx = ctx
        self._h = h
        self.offsets = offsets

    def view(self) -> CompView:
        v = CompView()
        self.ctx._check(lib().dpar2_comp_view_get(self._h, ctypes.byref(v)))
        return v

    def nbytes(self) -> int:
        return int(lib().dpar2_comp_bytes(self._h))

    def device_nbytes(self) -> int:
        return int(lib().dpar2_comp_device_bytes(self._h))

    def tensors(self):
        """Copies of the compressed factors as torch tensors (for inspection)."""
        v = self.view()
        dev = f"cuda:{self.ctx.device}"

        def cp(ptr, shape, dtype=torch.float32):
            out = torch.empty(shape, dtype=dtype, device=dev)
            if ptr:
                nb = out.numel() * out.element_size()
                src = _DevPtr(ptr, nb)
                out.view(-1).view(torch.uint8).copy_(src.as_tensor(dev))
            return out

        R, K, J, N = v.R, v.K, v.J, v.N
        M = None
        if v.Ms:
            M = torch.empty((K, J, R), dtype=torch.float32, device=dev)
            self.ctx._check(lib().dpar2_comp_m(self.ctx._h, self._h, _ptr(M), _stream()))
        return dict(A=cp(v.A, (N, R)), Bk=cp(v.Bk, (K, R)), M=M,
                    D=cp(v.D, (J, R)), E=cp(v.E, (R,)), Ft=cp(v.Ft, (K, R, R)),
                    xnorm2=cp(v.xnorm2, (K,), torch.float64), rank1=cp(v.rank1, (K,), torch.int32))

    def free(self):
        if self._h:
            lib().dpar2_comp_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class _DevPtr:
    """Wraps a raw device pointer as a uint8 torch tensor through __cuda_array_interface__."""

    def __init__(self, ptr, nbytes):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (int(ptr), False),
                                         "version": 3, "strides": None}

    def as_tensor(self, dev):
        return torch.as_tensor(self, device=dev)
