"""ctypes binding of the CPU FP64 oracle -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package.  The library under
``paper_1811_01277_gb300`` never imports it and shares no code with it.

All matrices are column-major (Fortran order) float64 / complex128 numpy
arrays.  The reflector storage layout is described in ``oracle.h``.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i, ll, p = ctypes.c_int, ctypes.c_longlong, ctypes.c_void_p
        L.or_hh_count.argtypes = [i, i]; L.or_hh_count.restype = ll
        L.or_hh_index.argtypes = [i, i, i, i]; L.or_hh_index.restype = ll
        L.or_larfg_d.argtypes = [i, p, p, p]; L.or_larfg_d.restype = i
        L.or_larfg_z.argtypes = [i, p, p, p]; L.or_larfg_z.restype = i
        for nm in ("or_bulge_chase_d", "or_bulge_chase_z"):
            getattr(L, nm).argtypes = [i, i, p, i, p, p, p, p]
            getattr(L, nm).restype = i
        for nm in ("or_trans_ev_d", "or_trans_ev_z"):
            getattr(L, nm).argtypes = [i, i, i, p, p, p, i]
            getattr(L, nm).restype = i
        L.or_tridiag_ql.argtypes = [i, p, p, p, i]; L.or_tridiag_ql.restype = i
        L.or_jacobi_d.argtypes = [i, p, i, p, p, i]; L.or_jacobi_d.restype = i
        L.or_sytrd_d.argtypes = [i, p, i, p, p, p, i, p]; L.or_sytrd_d.restype = i
        L.or_sytrd_apply_d.argtypes = [i, i, p, i, p, p, i]; L.or_sytrd_apply_d.restype = i
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} returned {rc}")


def hh_count(n, b):
    return int(lib().or_hh_count(n, b))


def hh_index(n, b, s, k):
    return int(lib().or_hh_index(n, b, s, k))


def larfg(alpha, x):
    """Return (beta, v, tau) with v = [1, v_1..v_m]; real or complex by dtype."""
    x = np.array(x, copy=True)
    cplx = np.iscomplexobj(x) or np.iscomplexobj(alpha)
    dt = np.complex128 if cplx else np.float64
    x = np.ascontiguousarray(x, dtype=dt)
    a = np.array([alpha], dtype=dt)
    t = np.zeros(1, dtype=dt)
    f = lib().or_larfg_z if cplx else lib().or_larfg_d
    _check(f(x.size, _ptr(a), _ptr(x), _ptr(t)), "larfg")
    return a[0], np.concatenate([np.ones(1, dt), x]), t[0]


def bulge_chase(B, b):
    """Band -> tridiagonal.  Returns (d, e, hh_v, hh_tau, T_dense)."""
    cplx = np.iscomplexobj(B)
    dt = np.complex128 if cplx else np.float64
    A = np.array(B, dtype=dt, order="F", copy=True)
    n = A.shape[0]
    cnt = hh_count(n, b)
    hv = np.zeros(cnt * b, dtype=dt)
    ht = np.zeros(max(cnt, 1), dtype=dt)
    d = np.zeros(n)
    e = np.zeros(max(n - 1, 1))
    f = lib().or_bulge_chase_z if cplx else lib().or_bulge_chase_d
    _check(f(n, b, _ptr(A), n, _ptr(d), _ptr(e), _ptr(hv), _ptr(ht)), "bulge_chase")
    return d, e[:n - 1], hv, ht[:cnt], A


def trans_ev(n, b, hh_v, hh_tau, Z):
    """Return Q2 @ Z (a new array); Z is n x nev, real or complex."""
    cplx = np.iscomplexobj(Z) or np.iscomplexobj(hh_v)
    dt = np.complex128 if cplx else np.float64
    Zo = np.array(Z, dtype=dt, order="F", copy=True)
    if Zo.ndim == 1:
        Zo = Zo.reshape(n, 1, order="F")
    hv = np.ascontiguousarray(hh_v, dtype=dt)
    ht = np.ascontiguousarray(hh_tau, dtype=dt)
    if ht.size == 0:
        ht = np.zeros(1, dtype=dt)
    if hv.size == 0:
        hv = np.zeros(1, dtype=dt)
    f = lib().or_trans_ev_z if cplx else lib().or_trans_ev_d
    _check(f(n, b, Zo.shape[1], _ptr(hv), _ptr(ht), _ptr(Zo), max(Zo.strides[1] // Zo.itemsize, n)),
           "trans_ev")
    return Zo


def tridiag_ql(d, e, Z=None):
    """Eigen-decomposition of the symmetric tridiagonal (d, e): (w, V)."""
    n = len(d)
    dd = np.array(d, dtype=np.float64, copy=True)
    ee = np.zeros(max(n, 1))
    ee[:n - 1] = e
    V = np.eye(n, order="F") if Z is None else np.array(Z, dtype=np.float64, order="F", copy=True)
    _check(lib().or_tridiag_ql(n, _ptr(dd), _ptr(ee), _ptr(V), n), "tridiag_ql")
    return dd, V


def jacobi(A):
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    w = np.zeros(n)
    V = np.zeros((n, n), order="F")
    _check(lib().or_jacobi_d(n, _ptr(A), n, _ptr(w), _ptr(V), n), "jacobi")
    return w, V


def sytrd(A):
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    n = A.shape[0]
    d = np.zeros(n)
    e = np.zeros(max(n, 1))
    v = np.zeros((n, max(n - 1, 1)), order="F")
    tau = np.zeros(max(n - 1, 1))
    _check(lib().or_sytrd_d(n, _ptr(A), n, _ptr(d), _ptr(e), _ptr(v), n, _ptr(tau)), "sytrd")
    return d, e[:n - 1], v, tau


def sytrd_apply(v, tau, Z):
    Zo = np.array(Z, dtype=np.float64, order="F", copy=True)
    n = Zo.shape[0]
    _check(lib().or_sytrd_apply_d(n, Zo.shape[1], _ptr(np.asfortranarray(v)), n,
                                  _ptr(np.ascontiguousarray(tau)), _ptr(Zo), n), "sytrd_apply")
    return Zo
