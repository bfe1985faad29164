"""Python access to the 2D FP64 CPU oracle with quadratic (TSC) shapes
(relsim_oracle_q.c).

TEST INFRASTRUCTURE: only ``tests/`` and the benchmark's CPU-baseline leg
may import it. The 2D scheme with the linear shape replaced by the quadratic
B-spline (3 x 3 nodes per particle, 25 neighbour offsets in the mass
matrix), base scheme only. Configs and particles are the 2D oracle's; the
mass matrix is (nn, 25, 3, 3) with offset o = (dj+2)*5 + (di+2).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Ledger, OracleConfig, Particles, load as _load2

__all__ = ["node_weightsq", "gather_Eq", "gather_Bq", "depositq", "apply_Mq", "apply_Aq", "gmresq", "pushq",
           "stepq", "offsetq"]

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_C = ctypes.POINTER(OracleConfig)
_dbl = ctypes.c_double
_done = False


def load():
    global _done
    lib = _load2()
    if not _done:
        sig = {
            "orcq_node_weights": (None, [_C, _dbl, _dbl, _I64, _D]),
            "orcq_gather_E": (None, [_C, _D, _dbl, _dbl, _D]),
            "orcq_gather_B": (None, [_C, _D, _dbl, _dbl, _D]),
            "orcq_deposit": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
            "orcq_apply_M": (None, [_C, _D, _D, _D]),
            "orcq_apply_A": (None, [_C, _D, _D, _D]),
            "orcq_gmres": (ctypes.c_int, [_C, _D, _D, _D, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double)]),
            "orcq_push": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
            "orcq_step": (ctypes.c_int, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.POINTER(Ledger),
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _done = True
    return lib


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def offsetq(di, dj):
    return (dj + 2) * 5 + (di + 2)


def node_weightsq(c, x, y):
    g = np.zeros(9, dtype=np.int64)
    W = np.zeros(9)
    load().orcq_node_weights(ctypes.byref(c), x, y, g, W)
    return g, W


def gather_Eq(c, E, x, y):
    out = np.zeros(3)
    load().orcq_gather_E(ctypes.byref(c), _f(E).ravel(), x, y, out)
    return out


def gather_Bq(c, B, x, y):
    out = np.zeros(3)
    load().orcq_gather_B(ctypes.byref(c), _f(B).ravel(), x, y, out)
    return out


def depositq(c, P: Particles, B):
    nn = c.nx * c.ny
    J = np.zeros(3 * nn)
    M = np.zeros(225 * nn)
    load().orcq_deposit(ctypes.byref(c), P.off, P.x, P.y, P.ux, P.uy, P.uz, P.w, _f(B).ravel(), J, M)
    return J.reshape(3, nn), M.reshape(nn, 25, 3, 3)


def apply_Mq(c, M, v):
    out = np.zeros(3 * c.nx * c.ny)
    load().orcq_apply_M(ctypes.byref(c), _f(M).ravel(), _f(v).ravel(), out)
    return out.reshape(3, -1)


def apply_Aq(c, M, v):
    out = np.zeros(3 * c.nx * c.ny)
    load().orcq_apply_A(ctypes.byref(c), _f(M).ravel(), _f(v).ravel(), out)
    return out.reshape(3, -1)


def gmresq(c, M, b, x0=None):
    x = np.zeros(3 * c.nx * c.ny) if x0 is None else _f(x0).ravel().copy()
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = load().orcq_gmres(ctypes.byref(c), _f(M).ravel(), _f(b).ravel(), x, ctypes.byref(it), ctypes.byref(rr))
    return x.reshape(3, -1), it.value, rr.value, st


def pushq(c, P: Particles, Et, B):
    sums = np.zeros(4)
    load().orcq_push(ctypes.byref(c), P.off, P.x, P.y, P.ux, P.uy, P.uz, P.w, _f(Et).ravel(), _f(B).ravel(), sums)
    return sums


def stepq(c, P: Particles, E, B, want_matrices=False):
    """One full step in place on P; returns (E, B, ledger dict, extras)."""
    nn = c.nx * c.ny
    E = _f(E).ravel().copy()
    B = _f(B).ravel().copy()
    led = Ledger()
    extras = {}
    if want_matrices:
        J = np.zeros(3 * nn)
        M = np.zeros(225 * nn)
        Et = np.zeros(3 * nn)
        ptrs = [J.ctypes.data, M.ctypes.data, Et.ctypes.data]
    else:
        ptrs = [None, None, None]
    st = load().orcq_step(ctypes.byref(c), P.off, P.x, P.y, P.ux, P.uy, P.uz, P.w, E, B, ctypes.byref(led), *ptrs)
    if want_matrices:
        extras = {"J": J.reshape(3, nn), "M": M.reshape(nn, 25, 3, 3), "Etheta": Et.reshape(3, nn)}
    d = led.asdict()
    d["status"] = st
    return E.reshape(3, nn), B.reshape(3, nn), d, extras
