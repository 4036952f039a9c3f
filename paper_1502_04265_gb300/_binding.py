"""Thin ctypes binding of libgbkm.so (include/gbkm.h).

Argument marshalling only: every function takes torch CUDA tensors, passes
their device pointers and the current torch stream to the C ABI call of the
same name, and returns the output tensors.  There is no CPU path: if the
library is not built, or a tensor is not on the GPU, the call raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import torch

from . import build as _build

GBKM_OK, GBKM_EINVAL, GBKM_ENOMEM, GBKM_ECUDA, GBKM_ETIMEOUT, GBKM_EUNSUPPORTED, GBKM_EDEGENERATE = (
    0, -1, -2, -3, -4, -5, -6)
GBKM_ETOOBIG = -7
NOALLOC_SCRATCH_BYTES = 64 << 20
DTYPES = {"f32": 0, "bf16": 1, "fp8": 2}
ENGINES = {"auto": 0, "simt": 1, "tcgen05": 2}
STATUS_NAMES = {0: "GBKM_OK", -1: "GBKM_EINVAL", -2: "GBKM_ENOMEM", -3: "GBKM_ECUDA",
                -4: "GBKM_ETIMEOUT", -5: "GBKM_EUNSUPPORTED", -6: "GBKM_EDEGENERATE", -7: "GBKM_ETOOBIG"}


class GbkmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class Problem(ct.Structure):
    _fields_ = [("X", ct.c_void_p), ("n", ct.c_int64), ("d", ct.c_int64), ("k", ct.c_int64),
                ("u", ct.c_void_p), ("C_out", ct.c_void_p), ("labels_out", ct.c_void_p),
                ("cost_out", ct.c_void_p)]


class MLP(ct.Structure):
    _fields_ = [("d_in", ct.c_int64), ("hidden", ct.c_int64), ("k", ct.c_int64), ("params", ct.c_void_p),
                ("params_bf16", ct.c_void_p), ("adam_m", ct.c_void_p), ("adam_v", ct.c_void_p),
                ("wd_mask", ct.c_void_p), ("step", ct.c_int64)]


class AssignOpts(ct.Structure):
    _fields_ = [("compute", ct.c_int32), ("engine", ct.c_int32), ("recheck", ct.c_int32),
                ("center_terms", ct.c_int32)]


_vp, _i64, _i32 = ct.c_void_p, ct.c_int64, ct.c_int32
_SIGS = {
    "gbkm_create": (ct.c_int, [ct.POINTER(ct.c_void_p), ct.c_int, _vp]),
    "gbkm_destroy": (ct.c_int, [_vp]),
    "gbkm_set_stream": (ct.c_int, [_vp, _vp]),
    "gbkm_last_error": (ct.c_char_p, [_vp]),
    "gbkm_sync": (ct.c_int, [_vp]),
    "gbkm_launch_count": (ct.c_int64, [_vp]),
    "gbkm_version": (ct.c_int, []),
    "gbkm_profile_enable": (ct.c_int, [_vp, ct.c_int]),
    "gbkm_profile_read": (ct.c_int, [_vp, ct.c_char_p, _i64]),
    "gbkm_debug_set_wait_limit": (ct.c_int, [_vp, ct.c_uint64]),
    "gbkm_debug_fail_alloc": (ct.c_int, [_vp, ct.c_int]),
    "gbkm_debug_stall_loads": (ct.c_int, [_vp, ct.c_int]),
    "gbkm_probe_peak": (ct.c_int, [_vp, _i32, ct.POINTER(ct.c_double)]),
    "kmeans_row_norms": (ct.c_int, [_vp, _vp, _i64, _i64, _vp]),
    "gbkm_host_alloc": (ct.c_int, [ct.c_size_t, ct.POINTER(ct.c_void_p)]),
    "gbkm_host_free": (ct.c_int, [_vp]),
    "kmeans_ingest": (ct.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "kmeans_quantize": (ct.c_int, [_vp, _vp, _i64, _i64, _i32, _vp, _vp]),
    "kmeans_project_block": (ct.c_int, [_vp, _vp, _i32, _i64, _i64, _vp, _i64, _vp, _vp]),
    "kmeans_rsvd": (ct.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _i64, _i64, _vp, _vp, _vp]),
    "kmeans_seed_pp": (ct.c_int, [_vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp, _vp]),
    "kmeans_seed_pp_q": (ct.c_int, [_vp, _vp, _vp, _vp, _i64, _i64, _vp, _i64, _vp, _vp, _vp]),
    "kmeans_assign": (ct.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, _i64, _vp, _i64,
                                 ct.POINTER(AssignOpts), _vp, _vp, _vp]),
    "kmeans_update": (ct.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp]),
    "kmeans_cost": (ct.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp]),
    "kmeans_update_noalloc": (ct.c_int, [_vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                                         _vp, _vp]),
    "kmeans_update_scratch_bytes": (ct.c_int64, [_i64, _i64, _i64]),
    "kmeans_piecy_lift": (ct.c_int, [_vp, _vp, _i64, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _vp, _vp, _vp]),
    "kmeans_bico_query": (ct.c_int, [_vp, _vp, _vp, _vp, _vp, _i64, _i64, _vp, _vp, _i64, _vp, _vp, _vp,
                                     ct.c_double, ct.POINTER(AssignOpts), _vp, _vp, _vp]),
    "kmeans_batch_run": (ct.c_int, [_vp, ct.POINTER(Problem), _i64, _i64, _i64, _i32, _i32]),
    "kmeans_batch_replay": (ct.c_int, [_vp]),
    "kmeans_autotune": (ct.c_int, [_vp, _i32, _i64, _i64, ct.POINTER(ct.c_int32)]),
    "kmeans_autotune_assign": (ct.c_int, [_vp, _i32, _i64, _i64, ct.POINTER(ct.c_int32), ct.POINTER(ct.c_int32),
                                          ct.POINTER(ct.c_int32)]),
    "kmeans_mlp_param_count": (ct.c_int64, [_i64, _i64, _i64]),
    "kmeans_gemm_bf16": (ct.c_int, [_vp, _vp, _vp, _i64, _i64, _i64, _vp, _i32, _i32, _vp, _i64]),
    "kmeans_mlp_forward": (ct.c_int, [_vp, ct.POINTER(MLP), _vp, _i64, _vp, _vp, _i32, _i32]),
    "kmeans_mlp_train_step": (ct.c_int, [_vp, ct.POINTER(MLP), _vp, _vp, _i64, ct.c_float, ct.c_float, _vp, _vp]),
    "kmeans_center_separation": (ct.c_int, [_vp, _vp, _i64, _i64, _vp]),
    "kmeans_learned_assign": (ct.c_int, [_vp, ct.POINTER(MLP), _vp, _vp, _i64, _i64, _vp, _i64, _vp, _i32, _vp,
                                         _vp, _vp]),
}

_lib = None
_lock = threading.Lock()


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libgbkm.so (building it first if asked).  Raises if it is not there."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing:
            path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libgbkm.so is not built ({path}); run paper_1502_04265_gb300.build.build()")
        L = ct.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _ptr(t):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("libgbkm takes CUDA tensors only (no CPU path)")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous (row-major)")
    return ct.c_void_p(t.data_ptr())


def _req(t, dtype, shape=None, name="tensor"):
    if t is None:
        raise ValueError(f"{name} is required")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return t


def _same_device(ref, **tensors):
    """Every given tensor (None skipped) must live on ref's device: the library reads them all
    through one device's address space."""
    for name, t in tensors.items():
        if t is not None and t.device != ref.device:
            raise ValueError(f"{name} is on {t.device}, but the input is on {ref.device}")


def _update_args(X, labels, C_old, w, C_new, counts, cost_old, cost_new, n_empty):
    """Checks and default outputs shared by kmeans_update and kmeans_update_noalloc: a C_old that is
    not k x d, or an output of the wrong shape, would make the kernels read or write past it."""
    _req(X, torch.float32, name="X")
    if X.dim() != 2:
        raise ValueError("X must be n x d")
    n, d = X.shape
    _req(labels, torch.int32, (n,), "labels")
    _req(C_old, torch.float32, name="C_old")
    if C_old.dim() != 2 or C_old.shape[1] != d:
        raise ValueError(f"C_old must be k x {d}, got {tuple(C_old.shape)}")
    k = C_old.shape[0]
    if w is not None:
        _req(w, torch.float32, (n,), "w")
    dev = X.device
    C_new = C_new if C_new is not None else torch.empty_like(C_old)
    counts = counts if counts is not None else torch.empty(k, dtype=torch.float64, device=dev)
    cost_old = cost_old if cost_old is not None else torch.empty(1, dtype=torch.float64, device=dev)
    cost_new = cost_new if cost_new is not None else torch.empty(1, dtype=torch.float64, device=dev)
    n_empty = n_empty if n_empty is not None else torch.empty(1, dtype=torch.int64, device=dev)
    _req(C_new, torch.float32, (k, d), "C_new")
    _req(counts, torch.float64, (k,), "counts")
    _req(cost_old, torch.float64, (1,), "cost_old")
    _req(cost_new, torch.float64, (1,), "cost_new")
    _req(n_empty, torch.int64, (1,), "n_empty")
    _same_device(X, labels=labels, C_old=C_old, w=w, C_new=C_new, counts=counts, cost_old=cost_old,
                 cost_new=cost_new, n_empty=n_empty)
    return n, d, k, C_new, counts, cost_old, cost_new, n_empty


class Context:
    """Owns one gbkm_ctx on a device; every call binds it to torch's current stream."""

    def __init__(self, device=None):
        L = load()
        dev = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.device = dev
        h = ct.c_void_p()
        with torch.cuda.device(dev):
            stream = torch.cuda.current_stream(dev).cuda_stream
            rc = L.gbkm_create(ct.byref(h), dev.index, ct.c_void_p(stream))
        if rc != GBKM_OK:
            raise GbkmError(rc, "gbkm_create failed")
        self._h = h

    @property
    def handle(self):
        return self._h

    def bind_stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        load().gbkm_set_stream(self._h, ct.c_void_p(s))

    def check(self, rc):
        if rc != GBKM_OK:
            msg = load().gbkm_last_error(self._h).decode()
            raise GbkmError(rc, msg)

    def sync(self):
        """Wait for the stream and raise on a device-reported status."""
        self.bind_stream()
        self.check(load().gbkm_sync(self._h))

    def launch_count(self) -> int:
        return int(load().gbkm_launch_count(self._h))

    def profile(self, enable: bool = True):
        """Turn on per-kernel CUDA-event timing on this context's stream."""
        self.check(load().gbkm_profile_enable(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """{kernel name: (launches, total ms)} since the last read; synchronises the stream."""
        self.bind_stream()
        buf = ct.create_string_buffer(1 << 14)
        rc = load().gbkm_profile_read(self._h, buf, len(buf))
        if rc < 0:
            self.check(rc)
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms = line.split()
            out[name] = (int(n), float(ms))
        return out

    def set_wait_limit(self, ns: int):
        """Limit of every bounded device wait of later tensor-core launches (0: the 2 s default)."""
        self.check(load().gbkm_debug_set_wait_limit(self._h, int(ns)))

    PROBE_UNITS = {"bf16": 0, "tf32": 1, "fp8": 2, "ffma": 3, "fp64": 4}

    def probe_peak(self, unit: str) -> float:
        """Measured TFLOP/s of one arithmetic unit ("bf16", "tf32", "fp8" tensor-core MMAs at the
        engine's shape; "ffma", "fp64" CUDA-core FMAs).  Synchronises."""
        self.bind_stream()
        out = ct.c_double()
        self.check(load().gbkm_probe_peak(self._h, self.PROBE_UNITS[unit], ct.byref(out)))
        return float(out.value)

    def stall_loads(self, on: bool):
        """Make later tensor-core launches issue no copies, so that their bounded waits run out."""
        self.check(load().gbkm_debug_stall_loads(self._h, 1 if on else 0))

    def fail_next_allocs(self, count: int):
        """Make the next `count` workspace growths fail as out of memory (host-side injection)."""
        self.check(load().gbkm_debug_fail_alloc(self._h, int(count)))

    def close(self):
        if getattr(self, "_h", None):
            load().gbkm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx = {}


def default_context(device=None) -> Context:
    idx = torch.cuda.current_device() if device is None else torch.device(device).index
    if idx not in _default_ctx:
        _default_ctx[idx] = Context(idx)
    return _default_ctx[idx]


def _ctx(ctx, ref):
    c = ctx or default_context(ref.device)
    c.bind_stream()
    return c


def gbkm_sync(ctx=None):
    (ctx or default_context()).sync()


def gbkm_version() -> int:
    return int(load().gbkm_version())


# ------------------------------------------------------------------ A1
def kmeans_row_norms(X, xnorm=None, ctx=None):
    _req(X, torch.float32, name="X")
    n, d = X.shape
    if xnorm is None:
        xnorm = torch.empty(n, dtype=torch.float32, device=X.device)
    _req(xnorm, torch.float32, (n,), "xnorm")
    _same_device(X, xnorm=xnorm)
    c = _ctx(ctx, X)
    c.check(load().kmeans_row_norms(c.handle, _ptr(X), n, d, _ptr(xnorm)))
    return xnorm


# ------------------------------------------------------------------ A0
def kmeans_quantize(X, dtype="bf16", Xq=None, scales=None, residuals=True, ctx=None):
    """(Xq, scales): for "fp8" the per-block scales; for "bf16" the rows' rounding residuals
    (n FP32, the side data kmeans_assign takes as Xop_scales), or None with residuals=False."""
    _req(X, torch.float32, name="X")
    n, d = X.shape
    if dtype == "bf16":
        Xq = Xq if Xq is not None else torch.empty((n, d), dtype=torch.bfloat16, device=X.device)
        if scales is None and residuals:
            scales = torch.empty(n, dtype=torch.float32, device=X.device)
    elif dtype == "fp8":
        Xq = Xq if Xq is not None else torch.empty((n, d), dtype=torch.uint8, device=X.device)
        nb = (d + 127) // 128
        scales = scales if scales is not None else torch.empty((n, nb), dtype=torch.float32, device=X.device)
    else:
        raise ValueError("dtype must be 'bf16' or 'fp8'")
    _req(Xq, torch.bfloat16 if dtype == "bf16" else torch.uint8, (n, d), "Xq")
    if scales is not None:
        _req(scales, torch.float32, (n,) if dtype == "bf16" else (n, (d + 127) // 128), "scales")
    _same_device(X, Xq=Xq, scales=scales)
    c = _ctx(ctx, X)
    c.check(load().kmeans_quantize(c.handle, _ptr(X), n, d, DTYPES[dtype], _ptr(Xq), _ptr(scales)))
    return Xq, scales


# ------------------------------------------------------------------ A0 + A1 from host memory
class HostBlock:
    """A page-locked, device-mapped host block from gbkm_host_alloc, viewed as a CPU tensor
    (`.tensor`); kmeans_ingest reads such blocks directly.  Freed by close() or on collection."""

    def __init__(self, shape, dtype=torch.float32):
        import numpy as np

        shape = tuple(int(s) for s in shape)
        itemsize = torch.empty((), dtype=dtype).element_size()
        nbytes = max(1, itemsize * int(np.prod(shape)))
        p = ct.c_void_p()
        rc = load().gbkm_host_alloc(nbytes, ct.byref(p))
        if rc != GBKM_OK:
            raise GbkmError(rc, f"gbkm_host_alloc of {nbytes} bytes failed")
        self._p = p.value
        raw = (ct.c_uint8 * nbytes).from_address(self._p)
        flat = torch.frombuffer(raw, dtype=torch.uint8)
        self.tensor = flat[:itemsize * int(np.prod(shape))].view(dtype).view(shape)

    def close(self):
        if getattr(self, "_p", None):
            self.tensor = None
            load().gbkm_host_free(ct.c_void_p(self._p))
            self._p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kmeans_ingest(X_src, X_dev=None, xnorm=None, Xq=None, resid=None, copy=True, quantize=True, device=None,
                  ctx=None):
    """One read of X_src (a CUDA tensor, or a CPU tensor inside a HostBlock): returns (X_dev, xnorm,
    Xq, resid) with X_dev the device copy (None with copy=False), xnorm the squared row norms, and
    the BF16 copy with the rows' rounding residuals (None with quantize=False)."""
    _req(X_src, torch.float32, name="X_src")
    if not X_src.is_contiguous():
        raise ValueError("X_src must be contiguous (row-major)")
    n, d = X_src.shape
    dev = X_src.device if X_src.is_cuda else torch.device(device if device is not None else "cuda")
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())
    if copy and X_dev is None:
        X_dev = torch.empty((n, d), dtype=torch.float32, device=dev)
    if xnorm is None:
        xnorm = torch.empty(n, dtype=torch.float32, device=dev)
    if quantize:
        Xq = Xq if Xq is not None else torch.empty((n, d), dtype=torch.bfloat16, device=dev)
        resid = resid if resid is not None else torch.empty(n, dtype=torch.float32, device=dev)
        _req(Xq, torch.bfloat16, (n, d), "Xq")
        _req(resid, torch.float32, (n,), "resid")
    if copy:
        _req(X_dev, torch.float32, (n, d), "X_dev")
    _req(xnorm, torch.float32, (n,), "xnorm")
    _same_device(xnorm, X_dev=X_dev if copy else None, Xq=Xq if quantize else None,
                 resid=resid if quantize else None, X_src=X_src if X_src.is_cuda else None)
    c = _ctx(ctx, xnorm)
    c.check(load().kmeans_ingest(c.handle, ct.c_void_p(X_src.data_ptr()), n, d, _ptr(X_dev) if copy else None,
                                 _ptr(xnorm), _ptr(Xq) if quantize else None, _ptr(resid) if quantize else None))
    return (X_dev if copy else None), xnorm, (Xq if quantize else None), (resid if quantize else None)


# ------------------------------------------------------------------ A2: the basis
def kmeans_rsvd(A, Omega, ell, w=None, V=None, sigma=None, info=None, ctx=None):
    """Top-ell right singular vectors (d x ell, sign-normalised) and singular values of
    diag(sqrt(w)) A by the randomised scheme with the d x s random matrix Omega."""
    _req(A, torch.float32, name="A")
    _req(Omega, torch.float32, name="Omega")
    n, d = A.shape
    s = Omega.shape[1]
    if Omega.shape[0] != d:
        raise ValueError("Omega must be d x s")
    if w is not None:
        _req(w, torch.float32, (n,), "w")
    V = V if V is not None else torch.empty((d, ell), dtype=torch.float32, device=A.device)
    sigma = sigma if sigma is not None else torch.empty(ell, dtype=torch.float32, device=A.device)
    info = info if info is not None else torch.zeros(1, dtype=torch.int32, device=A.device)
    _req(V, torch.float32, (d, ell), "V")
    _req(sigma, torch.float32, (ell,), "sigma")
    _req(info, torch.int32, (1,), "info")
    _same_device(A, Omega=Omega, w=w, V=V, sigma=sigma, info=info)
    c = _ctx(ctx, A)
    c.check(load().kmeans_rsvd(c.handle, _ptr(A), n, d, _ptr(w), _ptr(Omega), s, ell, _ptr(V), _ptr(sigma),
                               _ptr(info)))
    return V, sigma, info


# ------------------------------------------------------------------ A2
def kmeans_project_block(X, V, Y=None, X_lift=None, lift=False, ctx=None):
    if X.dtype == torch.float32:
        xt = 0
    elif X.dtype == torch.bfloat16:
        xt = 1
    else:
        raise TypeError("X must be float32 or bfloat16")
    n, d = X.shape
    _req(V, torch.float32, name="V")
    r = V.shape[1]
    if V.shape[0] != d:
        raise ValueError("V must be d x r")
    if Y is None:
        Y = torch.empty((n, r), dtype=torch.float32, device=X.device)
    if lift and X_lift is None:
        X_lift = torch.empty((n, d), dtype=torch.float32, device=X.device)
    _req(Y, torch.float32, (n, r), "Y")
    if X_lift is not None:
        _req(X_lift, torch.float32, (n, d), "X_lift")
    _same_device(X, V=V, Y=Y, X_lift=X_lift)
    c = _ctx(ctx, X)
    c.check(load().kmeans_project_block(c.handle, _ptr(X), xt, n, d, _ptr(V), r, _ptr(Y), _ptr(X_lift)))
    return (Y, X_lift) if X_lift is not None else Y


def kmeans_piecy_lift(X, piece_rows, Omegas, ell, w=None, X_lift=None, ctx=None):
    """Per-piece bases (randomised SVD with Omegas[q] for piece q) and the d-dimensional lift of every
    piece onto its own basis.  Returns (X_lift n x d, V pieces x d x ell, sigma pieces x ell, info)."""
    _req(X, torch.float32, name="X")
    n, d = X.shape
    pieces = (n + piece_rows - 1) // piece_rows
    _req(Omegas, torch.float32, name="Omegas")
    if Omegas.dim() != 3 or Omegas.shape[0] != pieces or Omegas.shape[1] != d:
        raise ValueError(f"Omegas must be {pieces} x {d} x s")
    s = Omegas.shape[2]
    if w is not None:
        _req(w, torch.float32, (n,), "w")
    dev = X.device
    X_lift = X_lift if X_lift is not None else torch.empty((n, d), dtype=torch.float32, device=dev)
    _req(X_lift, torch.float32, (n, d), "X_lift")
    V = torch.empty((pieces, d, ell), dtype=torch.float32, device=dev)
    sigma = torch.empty((pieces, ell), dtype=torch.float32, device=dev)
    info = torch.zeros(pieces, dtype=torch.int32, device=dev)
    _same_device(X, Omegas=Omegas, w=w, X_lift=X_lift)
    c = _ctx(ctx, X)
    c.check(load().kmeans_piecy_lift(c.handle, _ptr(X), n, d, _ptr(w), piece_rows, _ptr(Omegas), s, ell, _ptr(X_lift),
                                     _ptr(V), _ptr(sigma), _ptr(info)))
    return X_lift, V, sigma, info


# ------------------------------------------------------------------ A3
def kmeans_seed_pp(X, k, u, w=None, idx_out=None, C_out=None, Xq=None, xresid=None, ctx=None):
    """k-means++ seeding; with Xq (the BF16 copy) and xresid (its rows' residuals) the rounds filter
    rows through the copy first (kmeans_seed_pp_q), with the same picks."""
    _req(X, torch.float32, name="X")
    n, d = X.shape
    _req(u, torch.float64, name="u")
    if u.numel() < k:
        raise ValueError("u needs k uniforms")
    if w is not None:
        _req(w, torch.float32, (n,), "w")
    if (Xq is None) != (xresid is None):
        raise ValueError("Xq and xresid go together")
    if Xq is not None:
        _req(Xq, torch.bfloat16, (n, d), "Xq")
        _req(xresid, torch.float32, (n,), "xresid")
    idx_out = idx_out if idx_out is not None else torch.empty(k, dtype=torch.int64, device=X.device)
    C_out = C_out if C_out is not None else torch.empty((k, d), dtype=torch.float32, device=X.device)
    _req(idx_out, torch.int64, (k,), "idx_out")
    _req(C_out, torch.float32, (k, d), "C_out")
    _same_device(X, u=u, w=w, Xq=Xq, xresid=xresid, idx_out=idx_out, C_out=C_out)
    c = _ctx(ctx, X)
    if Xq is None:
        c.check(load().kmeans_seed_pp(c.handle, _ptr(X), n, d, _ptr(w), k, _ptr(u), _ptr(idx_out), _ptr(C_out)))
    else:
        c.check(load().kmeans_seed_pp_q(c.handle, _ptr(X), _ptr(Xq), _ptr(xresid), n, d, _ptr(w), k, _ptr(u),
                                        _ptr(idx_out), _ptr(C_out)))
    return idx_out, C_out


# ------------------------------------------------------------------ A4 + A5
def kmeans_assign(X, C, Xop=None, Xop_scales=None, xnorm=None, compute="f32", engine="auto",
                  recheck=True, labels=None, min_d2=None, n_rechecked=None, center_terms=1, ctx=None):
    _req(X, torch.float32, name="X")
    n, d = X.shape
    _req(C, torch.float32, name="C")
    k = C.shape[0]
    if C.shape[1] != d:
        raise ValueError("C must be k x d")
    if compute == "bf16":
        _req(Xop, torch.bfloat16, (n, d), "Xop")
    elif compute == "fp8":
        _req(Xop, torch.uint8, (n, d), "Xop")
    if xnorm is not None:
        _req(xnorm, torch.float32, (n,), "xnorm")
    labels = labels if labels is not None else torch.empty(n, dtype=torch.int32, device=X.device)
    _req(labels, torch.int32, (n,), "labels")
    if min_d2 is not None:
        _req(min_d2, torch.float32, (n,), "min_d2")
    if compute == "fp8":
        _req(Xop_scales, torch.float32, (n, (d + 127) // 128), "Xop_scales")
    elif Xop_scales is not None:
        _req(Xop_scales, torch.float32, (n,), "Xop_scales")
    _same_device(X, C=C, Xop=Xop, Xop_scales=Xop_scales, xnorm=xnorm, labels=labels, min_d2=min_d2,
                 n_rechecked=n_rechecked)
    opts = AssignOpts(DTYPES[compute], ENGINES[engine], 1 if recheck else 0, int(center_terms))
    c = _ctx(ctx, X)
    c.check(load().kmeans_assign(c.handle, _ptr(Xop), _ptr(Xop_scales), _ptr(X), _ptr(xnorm), n, d,
                                 _ptr(C), k, ct.byref(opts), _ptr(labels), _ptr(min_d2),
                                 _ptr(n_rechecked)))
    return labels


# ------------------------------------------------------------------ A6 + A7
def kmeans_update(X, labels, C_old, w=None, C_new=None, counts=None, cost_old=None, cost_new=None,
                  n_empty=None, ctx=None):
    n, d, k, C_new, counts, cost_old, cost_new, n_empty = _update_args(
        X, labels, C_old, w, C_new, counts, cost_old, cost_new, n_empty)
    c = _ctx(ctx, X)
    c.check(load().kmeans_update(c.handle, _ptr(X), n, d, _ptr(w), _ptr(labels), k, _ptr(C_old),
                                 _ptr(C_new), _ptr(counts), _ptr(cost_old), _ptr(cost_new),
                                 _ptr(n_empty)))
    return {"C_new": C_new, "counts": counts, "cost_old": cost_old, "cost_new": cost_new,
            "n_empty": n_empty}


def kmeans_cost(X, C, w=None, cost=None, ctx=None):
    _req(X, torch.float32, name="X")
    n, d = X.shape
    _req(C, torch.float32, name="C")
    if C.dim() != 2 or C.shape[1] != d:
        raise ValueError(f"C must be k x {d}")
    if w is not None:
        _req(w, torch.float32, (n,), "w")
    cost = cost if cost is not None else torch.empty(1, dtype=torch.float64, device=X.device)
    _req(cost, torch.float64, (1,), "cost")
    _same_device(X, C=C, w=w, cost=cost)
    c = _ctx(ctx, X)
    c.check(load().kmeans_cost(c.handle, _ptr(X), n, d, _ptr(w), _ptr(C), C.shape[0], _ptr(cost)))
    return cost


def kmeans_update_noalloc(X, labels, C_old, w=None, C_new=None, counts=None, cost_old=None,
                          cost_new=None, n_empty=None):
    """kmeans_update without a context and without any device allocation by the library.

    For callers that must not allocate device memory (a locked caching allocator, a
    memory-capped serving process, a loop where an allocation is not allowed): the library
    uses a fixed scratch block compiled into it, shared by every call on the device, so calls
    that overlap on the GPU race.  Output tensors left as None are created here by torch,
    before the call; pass them in to allocate nothing at all.  Work is queued on torch's
    current stream of X's device, which must be the current device.
    """
    n, d, k, C_new, counts, cost_old, cost_new, n_empty = _update_args(
        X, labels, C_old, w, C_new, counts, cost_old, cost_new, n_empty)
    dev = X.device
    if dev.index != torch.cuda.current_device():
        raise ValueError("X must live on the current CUDA device")
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = load().kmeans_update_noalloc(ct.c_void_p(stream), _ptr(X), n, d, _ptr(w), _ptr(labels), k,
                                      _ptr(C_old), _ptr(C_new), _ptr(counts), _ptr(cost_old),
                                      _ptr(cost_new), _ptr(n_empty))
    if rc != GBKM_OK:
        raise GbkmError(rc, "kmeans_update_noalloc failed" +
                        (" (problem exceeds the fixed scratch block)" if rc == GBKM_ETOOBIG else ""))
    return {"C_new": C_new, "counts": counts, "cost_old": cost_old, "cost_new": cost_new,
            "n_empty": n_empty}


def kmeans_update_scratch_bytes(n, d, k):
    """Bytes of the fixed scratch block that kmeans_update_noalloc needs for an n x d, k-cluster
    update (host arithmetic only; -1 for sizes the update does not take)."""
    return int(load().kmeans_update_scratch_bytes(n, d, k))


# ------------------------------------------------------------------ A8
def kmeans_batch_run(problems, seeds, iters, compute="bf16", graph=True, autotune=False, ctx=None):
    """Run k-means++ and `iters` Lloyd iterations for many problems x `seeds` seeds in one call.

    problems: list of dicts with X (n x d float32), k, u (seeds x k float64); optional C_out
    (seeds x k x d), labels_out (seeds x n int32), cost_out (seeds x 2 float64) are created if absent.
    Returns the list of dicts with the outputs filled (asynchronously, on the current stream).
    """
    arr = (Problem * len(problems))()
    keep = []
    for i, pr in enumerate(problems):
        X = _req(pr["X"], torch.float32, name="X")
        n, d = X.shape
        k = int(pr["k"])
        u = _req(pr["u"], torch.float64, (seeds, k), "u")
        dev = X.device
        pr.setdefault("C_out", torch.empty((seeds, k, d), dtype=torch.float32, device=dev))
        pr.setdefault("labels_out", torch.empty((seeds, n), dtype=torch.int32, device=dev))
        pr.setdefault("cost_out", torch.empty((seeds, 2), dtype=torch.float64, device=dev))
        _req(pr["C_out"], torch.float32, (seeds, k, d), "C_out")
        _req(pr["labels_out"], torch.int32, (seeds, n), "labels_out")
        _req(pr["cost_out"], torch.float64, (seeds, 2), "cost_out")
        _same_device(problems[0]["X"], X=X, u=u, C_out=pr["C_out"], labels_out=pr["labels_out"],
                     cost_out=pr["cost_out"])
        arr[i] = Problem(X.data_ptr(), n, d, k, u.data_ptr(), _ptr(pr["C_out"]).value,
                         _ptr(pr["labels_out"]).value, _ptr(pr["cost_out"]).value)
        keep.append(pr)
    flags = (1 if graph else 0) | (2 if autotune else 0)
    c = _ctx(ctx, problems[0]["X"])
    c.check(load().kmeans_batch_run(c.handle, arr, len(problems), seeds, iters, DTYPES[compute], flags))
    return keep


def kmeans_batch_replay(ctx=None):
    """Relaunch the graph recorded by the last graph-mode kmeans_batch_run on this context."""
    c = ctx or default_context()
    c.bind_stream()
    c.check(load().kmeans_batch_replay(c.handle))


def kmeans_autotune(d, ncols, compute="bf16", ctx=None):
    """Center-chunk width (64, 128 or 256) the autotuner picks for this shape (synchronises)."""
    c = ctx or default_context()
    c.bind_stream()
    out = ct.c_int32()
    c.check(load().kmeans_autotune(c.handle, DTYPES[compute], d, ncols, ct.byref(out)))
    return int(out.value)


def kmeans_autotune_assign(d, k, compute="f32", ctx=None):
    """Tune the single-problem assignment for this shape (engine, chunk width, stage ring); later
    kmeans_assign calls with engine="auto" on the shape use the choice.  Returns a dict."""
    c = ctx or default_context()
    c.bind_stream()
    eng, bn, st = ct.c_int32(), ct.c_int32(), ct.c_int32()
    c.check(load().kmeans_autotune_assign(c.handle, DTYPES[compute], d, k, ct.byref(eng), ct.byref(bn), ct.byref(st)))
    names = {v: k_ for k_, v in ENGINES.items()}
    return {"engine": names.get(int(eng.value), int(eng.value)), "bn": int(bn.value), "stages": int(st.value)}


# ------------------------------------------------------------------ A9
def kmeans_mlp_param_count(d_in, hidden, k):
    return int(load().kmeans_mlp_param_count(d_in, hidden, k))


def kmeans_gemm_bf16(A, B, bias=None, act=0, out_bf16=False, Y=None, ctx=None):
    """Y = act(A B^T + bias) on the tensor cores (A: M x K, B: N x K, BF16)."""
    _req(A, torch.bfloat16, name="A")
    _req(B, torch.bfloat16, name="B")
    M, K = A.shape
    if B.dim() != 2 or B.shape[1] != K:
        raise ValueError(f"B must be N x {K}")
    N = B.shape[0]
    if Y is None:
        Y = torch.empty((M, N), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=A.device)
    _req(Y, torch.bfloat16 if out_bf16 else torch.float32, name="Y")
    if Y.dim() != 2 or Y.shape[0] != M or Y.shape[1] < N:
        raise ValueError(f"Y must be {M} x (at least {N})")
    if bias is not None:
        _req(bias, torch.float32, (N,), "bias")
    _same_device(A, B=B, bias=bias, Y=Y)
    c = _ctx(ctx, A)
    c.check(load().kmeans_gemm_bf16(c.handle, _ptr(A), _ptr(B), M, N, K, _ptr(bias), act, 1 if out_bf16 else 0,
                                    _ptr(Y), Y.shape[1]))
    return Y


def _mlp_struct(net):
    return MLP(net.d_in, net.hidden, net.k, _ptr(net.params).value, _ptr(net.params_bf16).value,
               _ptr(net.adam_m).value if net.adam_m is not None else None,
               _ptr(net.adam_v).value if net.adam_v is not None else None,
               _ptr(net.wd_mask).value if net.wd_mask is not None else None, net.step)


def kmeans_mlp_forward(net, Xh, logits=None, top_idx=None, topm=32, group=1, ctx=None):
    _req(Xh, torch.bfloat16, name="Xh")
    if Xh.dim() != 2 or Xh.shape[1] != net.d_in:
        raise ValueError(f"Xh must be n x {net.d_in}")
    n = Xh.shape[0]
    if logits is not None:
        _req(logits, torch.float32, (n, net.k), "logits")
    if top_idx is not None:
        _req(top_idx, torch.int32, (n, topm), "top_idx")
    _same_device(Xh, params=net.params, logits=logits, top_idx=top_idx)
    m = _mlp_struct(net)
    c = _ctx(ctx, Xh)
    c.check(load().kmeans_mlp_forward(c.handle, ct.byref(m), _ptr(Xh), n, _ptr(logits), _ptr(top_idx), topm, int(group)))
    return logits, top_idx


def kmeans_mlp_train_step(net, Xh, labels, lr, wd=0.0, loss_rows=None, grad_out=None, ctx=None):
    _req(Xh, torch.bfloat16, name="Xh")
    if Xh.dim() != 2 or Xh.shape[1] != net.d_in:
        raise ValueError(f"Xh must be B x {net.d_in}")
    B = Xh.shape[0]
    _req(labels, torch.int32, (B,), "labels")
    if loss_rows is not None:
        _req(loss_rows, torch.float32, (B,), "loss_rows")
    if grad_out is not None:
        _req(grad_out, torch.float32, (net.params.numel(),), "grad_out")
    _same_device(Xh, params=net.params, labels=labels, loss_rows=loss_rows, grad_out=grad_out)
    m = _mlp_struct(net)
    c = _ctx(ctx, Xh)
    c.check(load().kmeans_mlp_train_step(c.handle, ct.byref(m), _ptr(Xh), _ptr(labels), B, lr, wd,
                                         _ptr(loss_rows), _ptr(grad_out)))
    net.step = int(m.step)


def kmeans_center_separation(C, s2=None, ctx=None):
    _req(C, torch.float32, name="C")
    k, d = C.shape
    s2 = s2 if s2 is not None else torch.empty(k, dtype=torch.float32, device=C.device)
    _req(s2, torch.float32, (k,), "s2")
    _same_device(C, s2=s2)
    c = _ctx(ctx, C)
    c.check(load().kmeans_center_separation(c.handle, _ptr(C), k, d, _ptr(s2)))
    return s2


def kmeans_learned_assign(net, X, Xh, C, s2, topm=32, labels=None, n_fallback=None, cand_out=None, ctx=None):
    _req(X, torch.float32, name="X")
    n, d = X.shape
    if d != net.d_in:
        raise ValueError(f"X must be n x {net.d_in} (the network's input width)")
    _req(Xh, torch.bfloat16, (n, d), "Xh")
    _req(C, torch.float32, (net.k, d), "C")
    k = C.shape[0]
    _req(s2, torch.float32, (k,), "s2")
    labels = labels if labels is not None else torch.empty(n, dtype=torch.int32, device=X.device)
    n_fallback = n_fallback if n_fallback is not None else torch.zeros(1, dtype=torch.int64, device=X.device)
    _req(labels, torch.int32, (n,), "labels")
    _req(n_fallback, torch.int64, (1,), "n_fallback")
    if cand_out is not None:
        _req(cand_out, torch.int32, (n, topm), "cand_out")
    _same_device(X, params=net.params, Xh=Xh, C=C, s2=s2, labels=labels, n_fallback=n_fallback,
                 cand_out=cand_out)
    m = _mlp_struct(net)
    c = _ctx(ctx, X)
    c.check(load().kmeans_learned_assign(c.handle, ct.byref(m), _ptr(X), _ptr(Xh), n, d, _ptr(C), k, _ptr(s2), topm,
                                         _ptr(labels), _ptr(n_fallback), _ptr(cand_out)))
    return labels, n_fallback


# ------------------------------------------------------------------ BICO-style query
def kmeans_bico_query(X, R, N, S, Q, T, w=None, Xop=None, Xop_scales=None, xnorm=None, compute="f32",
                      engine="auto", ref_out=None, d2_out=None, take_out=None, ctx=None):
    """Nearest reference of every point (R: m x d) and the copies w' its feature takes under the
    threshold T, against the snapshot N (m), S (m x d), Q (m) in FP64.  Returns (ref, d2, take)."""
    _req(X, torch.float32, name="X")
    n, d = X.shape
    _req(R, torch.float32, name="R")
    if R.dim() != 2 or R.shape[1] != d:
        raise ValueError(f"R must be m x {d}")
    m = R.shape[0]
    _req(N, torch.float64, (m,), "N")
    _req(S, torch.float64, (m, d), "S")
    _req(Q, torch.float64, (m,), "Q")
    if w is not None:
        _req(w, torch.float32, (n,), "w")
    if compute == "bf16":
        _req(Xop, torch.bfloat16, (n, d), "Xop")
    if xnorm is not None:
        _req(xnorm, torch.float32, (n,), "xnorm")
    dev = X.device
    ref_out = ref_out if ref_out is not None else torch.empty(n, dtype=torch.int32, device=dev)
    d2_out = d2_out if d2_out is not None else torch.empty(n, dtype=torch.float64, device=dev)
    take_out = take_out if take_out is not None else torch.empty(n, dtype=torch.float64, device=dev)
    _req(ref_out, torch.int32, (n,), "ref_out")
    _req(d2_out, torch.float64, (n,), "d2_out")
    _req(take_out, torch.float64, (n,), "take_out")
    _same_device(X, R=R, N=N, S=S, Q=Q, w=w, Xop=Xop, Xop_scales=Xop_scales, xnorm=xnorm, ref_out=ref_out,
                 d2_out=d2_out, take_out=take_out)
    opts = AssignOpts(DTYPES[compute], ENGINES[engine], 1, 1)
    c = _ctx(ctx, X)
    c.check(load().kmeans_bico_query(c.handle, _ptr(Xop), _ptr(Xop_scales), _ptr(X), _ptr(xnorm), n, d, _ptr(w),
                                     _ptr(R), m, _ptr(N), _ptr(S), _ptr(Q), float(T), ct.byref(opts),
                                     _ptr(ref_out), _ptr(d2_out), _ptr(take_out)))
    return ref_out, d2_out, take_out
