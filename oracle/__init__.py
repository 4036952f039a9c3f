"""FP64 CPU oracle for the k-means hot path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline and
reference arms may import this package.  The product path (the CUDA library
and its binding) never imports it, and it imports nothing from the product.

The arithmetic lives in plain C (``kmeans_oracle.c``, FP64 loops, optional
OpenMP over points); this module only marshals numpy arrays.  The brute-force
optimum for tiny inputs is in ``oracle.bruteforce``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kmeans_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

ORC_OK = 0
ORC_EINVAL = -1
ORC_EDEGENERATE = -6


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP) into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u16p = np.ctypeslib.ndpointer(dtype=np.uint16, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")
_vp = ct.c_void_p
_i64 = ct.c_int64


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ct.CDLL(path)
        sigs = {
            "orc_set_threads": (ct.c_int, [ct.c_int]),
            "orc_has_openmp": (ct.c_int, []),
            "orc_row_norms": (ct.c_int, [_f32p, _i64, _i64, _f64p]),
            "orc_assign": (ct.c_int, [_f32p, _i64, _i64, _f64p, _i64, _i32p, _vp, _vp]),
            "orc_update": (ct.c_int, [_f32p, _i64, _i64, _vp, _i32p, _i64, _f64p, _f64p, _f64p,
                                      _f64p, _f64p, _vp, _vp, _vp]),
            "orc_cost": (ct.c_int, [_f32p, _i64, _i64, _vp, _f64p, _i64, _vp]),
            "orc_cost_cf": (ct.c_int, [_f64p, _f64p, _f64p, _f64p, _i64, _i64, _vp]),
            "orc_pp_pick": (ct.c_int, [_f64p, _vp, _i64, ct.c_double, _vp]),
            "orc_seed_pp": (ct.c_int, [_f32p, _i64, _i64, _vp, _i64, _f64p, _i64p, _vp, _vp]),
            "orc_lloyd": (ct.c_int, [_f32p, _i64, _i64, _vp, _f64p, _i64, _i64, _f64p, _i32p,
                                     _vp, _vp]),
            "orc_project": (ct.c_int, [_f32p, _i64, _i64, _f64p, _i64, _f64p, _vp]),
            "orc_quant_bf16": (ct.c_int, [_f32p, _i64, _u16p]),
            "orc_quant_e4m3": (ct.c_int, [_f32p, _i64, _i64, _i64, _u8p, _f32p]),
            "orc_e4m3_decode": (ct.c_double, [ct.c_uint8]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _x(X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    assert X.ndim == 2
    return X


def _w(w, n):
    if w is None:
        return None
    w = np.ascontiguousarray(w, dtype=np.float64)
    assert w.shape == (n,)
    return w


def _check(rc, what):
    if rc != ORC_OK:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def set_threads(t: int) -> int:
    """Set the OpenMP thread count the oracle uses; returns the count in effect."""
    return lib().orc_set_threads(int(t))


def row_norms(X):
    X = _x(X)
    out = np.empty(X.shape[0], np.float64)
    _check(lib().orc_row_norms(X, X.shape[0], X.shape[1], out), "row_norms")
    return out


def assign(X, C):
    """Nearest center by full scan: (labels int32, d1, d2) with d1/d2 the best/second FP64 distances."""
    X = _x(X)
    C = np.ascontiguousarray(C, dtype=np.float64)
    n, d = X.shape
    k = C.shape[0]
    assert C.shape[1] == d
    labels = np.empty(n, np.int32)
    d1 = np.empty(n, np.float64)
    d2 = np.empty(n, np.float64)
    _check(lib().orc_assign(X, n, d, C, k, labels, _ptr(d1), _ptr(d2)), "assign")
    return labels, d1, d2


def near_tie_gap(X, d1, d2):
    """Relative top-2 gap (d2 - d1) / max(d1, 1e-30 (||x||^2 + 1)) of every point."""
    xn = row_norms(X)
    den = np.maximum(d1, 1e-30 * (xn + 1.0))
    with np.errstate(invalid="ignore", divide="ignore"):
        g = (d2 - d1) / den
    g[np.isnan(g)] = 0.0
    return g


def update(X, labels, C_old, w=None):
    """Centroid update through clustering features.

    Returns a dict with C_new (k x d FP64), N (k), S (k x d), Q (k),
    cost_old = cost(C_old, labels), cost_new = cost(C_new, labels), n_empty.
    """
    X = _x(X)
    n, d = X.shape
    C_old = np.ascontiguousarray(C_old, dtype=np.float64)
    k = C_old.shape[0]
    labels = np.ascontiguousarray(labels, dtype=np.int32)
    w = _w(w, n)
    C_new = np.empty((k, d), np.float64)
    N = np.empty(k, np.float64)
    S = np.empty((k, d), np.float64)
    Q = np.empty(k, np.float64)
    co = ct.c_double()
    cn = ct.c_double()
    ne = ct.c_int64()
    _check(lib().orc_update(X, n, d, _ptr(w), labels, k, C_old, C_new, N, S, Q,
                            ct.byref(co), ct.byref(cn), ct.byref(ne)), "update")
    return {"C_new": C_new, "N": N, "S": S, "Q": Q, "cost_old": co.value,
            "cost_new": cn.value, "n_empty": ne.value}


def cost(X, C, w=None):
    X = _x(X)
    n, d = X.shape
    C = np.ascontiguousarray(C, dtype=np.float64)
    w = _w(w, n)
    out = ct.c_double()
    _check(lib().orc_cost(X, n, d, _ptr(w), C, C.shape[0], ct.byref(out)), "cost")
    return out.value


def cost_cf(N, S, Q, C):
    N = np.ascontiguousarray(N, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    Q = np.ascontiguousarray(Q, np.float64)
    C = np.ascontiguousarray(C, np.float64)
    k, d = C.shape
    out = ct.c_double()
    _check(lib().orc_cost_cf(N, S, Q, C, k, d, ct.byref(out)), "cost_cf")
    return out.value


def pp_pick(D2, u, w=None):
    D2 = np.ascontiguousarray(D2, np.float64)
    n = D2.shape[0]
    w = _w(w, n)
    idx = ct.c_int64()
    rc = lib().orc_pp_pick(D2, _ptr(w), n, float(u), ct.byref(idx))
    if rc == ORC_EDEGENERATE:
        return None
    _check(rc, "pp_pick")
    return idx.value


def seed_pp(X, k, u, w=None):
    """k-means++ seeding; returns (idx int64[k], C FP64 k x d, final D2, status)."""
    X = _x(X)
    n, d = X.shape
    u = np.ascontiguousarray(u, np.float64)
    assert u.shape[0] >= k
    w = _w(w, n)
    idx = np.full(k, -1, np.int64)
    C = np.zeros((k, d), np.float64)
    D2 = np.empty(n, np.float64)
    rc = lib().orc_seed_pp(X, n, d, _ptr(w), k, u, idx, _ptr(C), _ptr(D2))
    if rc not in (ORC_OK, ORC_EDEGENERATE):
        _check(rc, "seed_pp")
    return idx, C, D2, rc


def lloyd(X, C0, iters, w=None):
    """Lloyd iterations from C0: (C, labels, cost_trace[2*iters], conv_iter)."""
    X = _x(X)
    n, d = X.shape
    C0 = np.ascontiguousarray(C0, np.float64)
    k = C0.shape[0]
    w = _w(w, n)
    C = np.empty((k, d), np.float64)
    labels = np.empty(n, np.int32)
    trace = np.empty(2 * max(iters, 1), np.float64)
    conv = ct.c_int64()
    _check(lib().orc_lloyd(X, n, d, _ptr(w), C0, k, iters, C, labels, _ptr(trace),
                           ct.byref(conv)), "lloyd")
    return C, labels, trace[: 2 * iters], conv.value


def project(X, V, lift=False):
    """Y = X V (n x r, FP64) and optionally the lift Y V^T (n x d)."""
    X = _x(X)
    n, d = X.shape
    V = np.ascontiguousarray(V, np.float64)
    r = V.shape[1]
    assert V.shape[0] == d
    Y = np.empty((n, r), np.float64)
    L = np.empty((n, d), np.float64) if lift else None
    _check(lib().orc_project(X, n, d, V, r, Y, _ptr(L)), "project")
    return (Y, L) if lift else Y


def quant_bf16(x):
    """bfloat16 bit patterns (uint16) of an FP32 array, round to nearest even."""
    x = np.ascontiguousarray(x, np.float32)
    out = np.empty(x.shape, np.uint16)
    _check(lib().orc_quant_bf16(x.reshape(-1), x.size, out.reshape(-1)), "quant_bf16")
    return out


def bf16_to_f32(bits):
    return (np.asarray(bits, np.uint32) << 16).view(np.float32)


def quant_e4m3(X, block=128):
    """E4M3 codes (uint8, n x d) and power-of-two scales (n x ceil(d/block))."""
    X = _x(X)
    n, d = X.shape
    nb = (d + block - 1) // block
    q = np.empty((n, d), np.uint8)
    s = np.empty((n, nb), np.float32)
    _check(lib().orc_quant_e4m3(X, n, d, block, q, s), "quant_e4m3")
    return q, s


def e4m3_decode(codes):
    table = np.array([lib().orc_e4m3_decode(c) for c in range(256)], np.float64)
    return table[np.asarray(codes, np.uint8)]
