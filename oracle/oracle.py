"""ctypes wrapper around the C oracle (kg_oracle.c).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg load this module; the product path never does.  It shares no
code with the CUDA path.  The *_omp functions (kg_oracle_omp.c) are the timed
CPU baseline on all host cores; parity is checked against the serial ones.

All functions take and return float64 numpy arrays.  FP32 workloads are
checked by calling these on the FP32-rounded inputs (the oracle itself always
computes in double precision).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kg_oracle.c")
_LIB = os.path.join(_HERE, "libkg_oracle.so")
_lock = threading.Lock()
_lib = None

# -ffp-contract=off keeps a*b+c unfused on every host (Arm contracts by default),
# so the oracle rounds the same way on x86 and aarch64.
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile kg_oracle.c into libkg_oracle.so next to it (gcc, no intrinsics)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


_SRC_OMP = os.path.join(_HERE, "kg_oracle_omp.c")
_LIB_OMP = os.path.join(_HERE, "libkg_oracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """Compile kg_oracle_omp.c (the OpenMP CPU baseline) into libkg_oracle_omp.so."""
    if (not force and os.path.exists(_LIB_OMP)
            and os.path.getmtime(_LIB_OMP) >= os.path.getmtime(_SRC_OMP)):
        return _LIB_OMP
    tmp = _LIB_OMP + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, "-fopenmp", "-o", tmp, _SRC_OMP, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def _load_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = ctypes.CDLL(build_omp())
            i64, dp, d = ctypes.c_int64, ctypes.c_void_p, ctypes.c_double
            lib.kgo_omp_threads.argtypes = []
            lib.kgo_omp_threads.restype = ctypes.c_int
            lib.kgo_quadform_grad_omp.argtypes = [i64, i64, dp, dp, d, dp, dp, dp]
            lib.kgo_quadform_grad_omp.restype = ctypes.c_int
            lib.kgo_tet_grad_omp.argtypes = [i64, i64, dp, dp, dp, d, dp, dp, dp]
            lib.kgo_tet_grad_omp.restype = ctypes.c_int
            _lib_omp = lib
    return _lib_omp


def omp_threads() -> int:
    """Threads the OpenMP CPU baseline uses (OMP_NUM_THREADS, else all cores)."""
    return int(_load_omp().kgo_omp_threads())


def quadform_grad_omp(A, x, fbar=1.0):
    """CPU baseline on all cores: (f, gx, threads used).  Not a parity reference."""
    A, x = _f64(A), _f64(x)
    m, n = A.shape
    f = np.zeros(1)
    gx = np.empty(n)
    t = ctypes.c_int(0)
    _check(_load_omp().kgo_quadform_grad_omp(m, n, _p(A), _p(x), float(fbar), _p(f), _p(gx),
                                             ctypes.addressof(t)), "quadform_grad_omp")
    return float(f[0]), gx, t.value


def tet_grad_omp(conn, G, u, fbar=1.0):
    """CPU baseline on all cores: (f, gu, threads used).  Not a parity reference."""
    conn, G, u = _i32(conn), _f64(G), _f64(u)
    f = np.zeros(1)
    gu = np.empty(u.shape[0])
    t = ctypes.c_int(0)
    _check(_load_omp().kgo_tet_grad_omp(conn.shape[0], u.shape[0], _p(conn), _p(G), _p(u),
                                        float(fbar), _p(f), _p(gu), ctypes.addressof(t)),
           "tet_grad_omp")
    return float(f[0]), gu, t.value


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, dp, ip = ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
            d = ctypes.c_double
            sig = {
                "kgo_quadform_value": [i64, i64, dp, dp, dp, dp],
                "kgo_quadform_grad": [i64, i64, dp, dp, d, dp, dp, dp],
                "kgo_tet_value": [i64, i64, ip, dp, dp, dp],
                "kgo_tet_adjoint_local": [i64, i64, ip, dp, dp, d, dp],
                "kgo_tet_grad": [i64, i64, ip, dp, dp, d, dp, dp],
                "kgo_tet_descent": [i64, i64, ip, dp, dp, d, ctypes.c_int, dp],
                "kgo_spquadform_value": [i64, i64, i64, ip, ip, dp, dp, dp, dp],
                "kgo_spquadform_grad": [i64, i64, i64, ip, ip, dp, dp, d, dp, dp, dp],
                "kgo_tet_hvp": [i64, i64, ip, dp, dp, dp, d, dp],
                "kgo_laplace1d_hvp": [i64, dp, d, dp],
                "kgo_laplace1d_value": [i64, dp, dp, dp],
                "kgo_laplace1d_grad": [i64, dp, dp, d, dp, dp, dp],
            }
            for name, args in sig.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, name):
    if rc != 0:
        raise ValueError(f"{name} failed with status {rc}")


# ------------------------------------------------------------ ||A x||^2
def quadform_value(A, x, return_y=False):
    A, x = _f64(A), _f64(x)
    m, n = A.shape
    y = np.empty(m)
    f = np.zeros(1)
    _check(_load().kgo_quadform_value(m, n, _p(A), _p(x), _p(y), _p(f)), "quadform_value")
    return (float(f[0]), y) if return_y else float(f[0])


def quadform_grad(A, x, fbar=1.0, want_gA=False):
    """Returns (f, gx) or (f, gx, gA)."""
    A, x = _f64(A), _f64(x)
    m, n = A.shape
    f = np.zeros(1)
    gx = np.empty(n)
    gA = np.empty((m, n)) if want_gA else None
    _check(_load().kgo_quadform_grad(m, n, _p(A), _p(x), float(fbar), _p(f), _p(gx), _p(gA)),
           "quadform_grad")
    return (float(f[0]), gx, gA) if want_gA else (float(f[0]), gx)


# ------------------------------------------------------------ sparse ||A x||^2
def spquadform_value(rowptr, col, val, x, n=None, return_y=False):
    rowptr, col, val, x = _i32(rowptr), _i32(col), _f64(val), _f64(x)
    m = rowptr.shape[0] - 1
    n = x.shape[0] if n is None else n
    y = np.empty(max(m, 1))
    f = np.zeros(1)
    _check(_load().kgo_spquadform_value(m, n, col.shape[0], _p(rowptr), _p(col), _p(val), _p(x),
                                        _p(y), _p(f)), "spquadform_value")
    return (float(f[0]), y[:m]) if return_y else float(f[0])


def spquadform_grad(rowptr, col, val, x, fbar=1.0, want_gval=False):
    """Returns (f, gx) or (f, gx, gval) for A in CSR form (rowptr, col, val), A m x len(x)."""
    rowptr, col, val, x = _i32(rowptr), _i32(col), _f64(val), _f64(x)
    m, n = rowptr.shape[0] - 1, x.shape[0]
    f = np.zeros(1)
    gx = np.empty(max(n, 1))
    gval = np.empty(max(col.shape[0], 1)) if want_gval else None
    _check(_load().kgo_spquadform_grad(m, n, col.shape[0], _p(rowptr), _p(col), _p(val), _p(x),
                                       float(fbar), _p(f), _p(gx), _p(gval)), "spquadform_grad")
    if want_gval:
        return float(f[0]), gx[:n], gval[:col.shape[0]]
    return float(f[0]), gx[:n]


# ------------------------------------------------------------ tet energy
def tet_value(conn, G, u):
    conn, G, u = _i32(conn), _f64(G), _f64(u)
    f = np.zeros(1)
    _check(_load().kgo_tet_value(conn.shape[0], u.shape[0], _p(conn), _p(G), _p(u), _p(f)),
           "tet_value")
    return float(f[0])


def tet_adjoint_local(conn, G, u, fbar=1.0):
    conn, G, u = _i32(conn), _f64(G), _f64(u)
    c = np.empty((conn.shape[0], 4))
    _check(_load().kgo_tet_adjoint_local(conn.shape[0], u.shape[0], _p(conn), _p(G), _p(u),
                                         float(fbar), _p(c)), "tet_adjoint_local")
    return c


def tet_grad(conn, G, u, fbar=1.0):
    conn, G, u = _i32(conn), _f64(G), _f64(u)
    f = np.zeros(1)
    gu = np.empty(u.shape[0])
    _check(_load().kgo_tet_grad(conn.shape[0], u.shape[0], _p(conn), _p(G), _p(u), float(fbar),
                                _p(f), _p(gu)), "tet_grad")
    return float(f[0]), gu


def tet_hvp(conn, G, u, v, fbar=1.0):
    """fbar * Hessian(u) @ v of the tet energy (forward over reverse)."""
    conn, G, u, v = _i32(conn), _f64(G), _f64(u), _f64(v)
    hv = np.empty(u.shape[0])
    _check(_load().kgo_tet_hvp(conn.shape[0], u.shape[0], _p(conn), _p(G), _p(u), _p(v), float(fbar),
                               _p(hv)), "tet_hvp")
    return hv


def tet_descent(conn, G, u0, eta, steps):
    """Returns (u after `steps` steps, f history of length steps + 1)."""
    conn, G = _i32(conn), _f64(G)
    u = _f64(u0).copy()
    hist = np.empty(steps + 1)
    _check(_load().kgo_tet_descent(conn.shape[0], u.shape[0], _p(conn), _p(G), _p(u),
                                   float(eta), int(steps), _p(hist)), "tet_descent")
    return u, hist


# ------------------------------------------------------------ 1-D Laplacian
def laplace1d_value(x, b):
    x, b = _f64(x), _f64(b)
    f = np.zeros(1)
    _check(_load().kgo_laplace1d_value(x.shape[0], _p(x), _p(b), _p(f)), "laplace1d_value")
    return float(f[0])


def laplace1d_grad(x, b, fbar=1.0):
    x, b = _f64(x), _f64(b)
    n = x.shape[0]
    f = np.zeros(1)
    gx = np.empty(n)
    gb = np.empty(n)
    _check(_load().kgo_laplace1d_grad(n, _p(x), _p(b), float(fbar), _p(f), _p(gx), _p(gb)),
           "laplace1d_grad")
    return float(f[0]), gx, gb


def laplace1d_hvp(v, fbar=1.0):
    """fbar * Hessian @ v of the 1-D example (independent of x and b)."""
    v = _f64(v)
    hv = np.empty(v.shape[0])
    _check(_load().kgo_laplace1d_hvp(v.shape[0], _p(v), float(fbar), _p(hv)), "laplace1d_hvp")
    return hv
