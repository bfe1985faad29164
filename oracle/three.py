"""Python access to the 3D FP64 CPU oracle (relsim_oracle3.c).

TEST INFRASTRUCTURE: only ``tests/`` and the benchmark's CPU-baseline leg
may import it. The same scheme as the 2D oracle (Sec. 2: explicit pusher,
implicit field solve through the mass matrices) on a periodic
nx x ny x nz grid with trilinear shape functions (the 27-node stencil),
base scheme only. Node and cell (i, j, k) have linear index
(k*ny + j)*nx + i; fields are (3, nn); the mass matrix is (nn, 27, 3, 3)
with offset o = (dk+1)*9 + (dj+1)*3 + (di+1).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import Ledger, load as _load2

__all__ = ["OracleConfig3", "make_config3", "Particles3", "deposit3", "curl_c3", "curl_n3", "apply_M3",
           "apply_A3", "rhs3", "gmres3", "field_update3", "push3", "energies3", "cell_keys3", "step3",
           "gather_E3", "gather_B3", "node_weights3", "offset3"]


class OracleConfig3(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("theta", ctypes.c_double),
                ("nspecies", ctypes.c_int),
                ("q", ctypes.c_double * 4), ("m", ctypes.c_double * 4),
                ("gmres_tol", ctypes.c_double),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int)]


_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_C = ctypes.POINTER(OracleConfig3)
_dbl = ctypes.c_double
_sigs_done = False


def load():
    global _sigs_done
    lib = _load2()
    if not _sigs_done:
        sig = {
            "orc3_node_weights": (None, [_C, _dbl, _dbl, _dbl, _I64, _D]),
            "orc3_gather_E": (None, [_C, _D, _dbl, _dbl, _dbl, _D]),
            "orc3_gather_B": (None, [_C, _D, _dbl, _dbl, _dbl, _D]),
            "orc3_deposit": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
            "orc3_curl_c": (None, [_C, _D, _D]),
            "orc3_curl_n": (None, [_C, _D, _D]),
            "orc3_apply_M": (None, [_C, _D, _D, _D]),
            "orc3_apply_A": (None, [_C, _D, _D, _D]),
            "orc3_rhs": (None, [_C, _D, _D, _D, _D]),
            "orc3_gmres": (ctypes.c_int, [_C, _D, _D, _D, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_double)]),
            "orc3_field_update": (None, [_C, _D, _D, _D]),
            "orc3_push": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
            "orc3_energies": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D]),
            "orc3_cell_keys": (None, [_C, ctypes.c_int64, _D, _D, _D, _I32]),
            "orc3_step": (ctypes.c_int, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D,
                                         ctypes.POINTER(Ledger), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _sigs_done = True
    return lib


def make_config3(nx, ny, nz, dx=1.0, dy=1.0, dz=1.0, dt=0.5, theta=0.5, q=(1.0, -1.0), m=(1.0, 1.0),
                 gmres_tol=1e-12, gmres_restart=50, gmres_maxit=2000) -> OracleConfig3:
    c = OracleConfig3()
    c.nx, c.ny, c.nz = nx, ny, nz
    c.dx, c.dy, c.dz, c.dt, c.theta = dx, dy, dz, dt, theta
    c.nspecies = len(q)
    for s in range(len(q)):
        c.q[s] = q[s]
        c.m[s] = m[s]
    c.gmres_tol, c.gmres_restart, c.gmres_maxit = gmres_tol, gmres_restart, gmres_maxit
    return c


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _nn(c):
    return c.nx * c.ny * c.nz


def offset3(di, dj, dk):
    return (dk + 1) * 9 + (dj + 1) * 3 + (di + 1)


class Particles3:
    """Concatenated FP64 particle arrays of all species (x, y, z, ux, uy, uz, w)."""

    KEYS = ("x", "y", "z", "ux", "uy", "uz", "w")

    def __init__(self, species):
        self.off = np.zeros(len(species) + 1, dtype=np.int64)
        for s, sp in enumerate(species):
            self.off[s + 1] = self.off[s] + len(sp["x"])
        for k in self.KEYS:
            setattr(self, k, _f(np.concatenate([np.asarray(sp[k], dtype=np.float64) for sp in species])))

    def species(self, s):
        a, b = self.off[s], self.off[s + 1]
        return {k: getattr(self, k)[a:b].copy() for k in self.KEYS}

    def copy(self):
        p = Particles3.__new__(Particles3)
        p.off = self.off.copy()
        for k in self.KEYS:
            setattr(p, k, getattr(self, k).copy())
        return p


def node_weights3(c, x, y, z):
    g = np.zeros(8, dtype=np.int64)
    W = np.zeros(8)
    load().orc3_node_weights(ctypes.byref(c), x, y, z, g, W)
    return g, W


def gather_E3(c, E, x, y, z):
    out = np.zeros(3)
    load().orc3_gather_E(ctypes.byref(c), _f(E).ravel(), x, y, z, out)
    return out


def gather_B3(c, B, x, y, z):
    out = np.zeros(3)
    load().orc3_gather_B(ctypes.byref(c), _f(B).ravel(), x, y, z, out)
    return out


def deposit3(c, P: Particles3, B):
    nn = _nn(c)
    J = np.zeros(3 * nn)
    M = np.zeros(243 * nn)
    load().orc3_deposit(ctypes.byref(c), P.off, P.x, P.y, P.z, P.ux, P.uy, P.uz, P.w, _f(B).ravel(), J, M)
    return J.reshape(3, nn), M.reshape(nn, 27, 3, 3)


def _unary(name, c, v):
    out = np.zeros(3 * _nn(c))
    getattr(load(), name)(ctypes.byref(c), _f(v).ravel(), out)
    return out.reshape(3, -1)


def curl_c3(c, E):
    return _unary("orc3_curl_c", c, E)


def curl_n3(c, B):
    return _unary("orc3_curl_n", c, B)


def apply_M3(c, M, v):
    out = np.zeros(3 * _nn(c))
    load().orc3_apply_M(ctypes.byref(c), _f(M).ravel(), _f(v).ravel(), out)
    return out.reshape(3, -1)


def apply_A3(c, M, v):
    out = np.zeros(3 * _nn(c))
    load().orc3_apply_A(ctypes.byref(c), _f(M).ravel(), _f(v).ravel(), out)
    return out.reshape(3, -1)


def rhs3(c, E, B, J):
    out = np.zeros(3 * _nn(c))
    load().orc3_rhs(ctypes.byref(c), _f(E).ravel(), _f(B).ravel(), _f(J).ravel(), out)
    return out.reshape(3, -1)


def gmres3(c, M, b, x0=None):
    x = np.zeros(3 * _nn(c)) if x0 is None else _f(x0).ravel().copy()
    it = ctypes.c_int()
    rr = ctypes.c_double()
    st = load().orc3_gmres(ctypes.byref(c), _f(M).ravel(), _f(b).ravel(), x, ctypes.byref(it), ctypes.byref(rr))
    return x.reshape(3, -1), it.value, rr.value, st


def field_update3(c, Et, E, B):
    E = _f(E).ravel().copy()
    B = _f(B).ravel().copy()
    load().orc3_field_update(ctypes.byref(c), _f(Et).ravel(), E, B)
    return E.reshape(3, -1), B.reshape(3, -1)


def push3(c, P: Particles3, Et, B):
    """Push in place; returns the sums (K0, K1, work, mismatch)."""
    sums = np.zeros(4)
    load().orc3_push(ctypes.byref(c), P.off, P.x, P.y, P.z, P.ux, P.uy, P.uz, P.w, _f(Et).ravel(),
                     _f(B).ravel(), sums)
    return sums


def energies3(c, P: Particles3, E, B):
    out = np.zeros(3)
    load().orc3_energies(ctypes.byref(c), P.off, P.ux, P.uy, P.uz, P.w, _f(E).ravel(), _f(B).ravel(), out)
    return out


def cell_keys3(c, x, y, z):
    x = _f(x)
    keys = np.zeros(len(x), dtype=np.int32)
    load().orc3_cell_keys(ctypes.byref(c), len(x), x, _f(y), _f(z), keys)
    return keys


def step3(c, P: Particles3, E, B, want_matrices=False):
    """One full step in place on P; returns (E, B, ledger dict, extras)."""
    nn = _nn(c)
    E = _f(E).ravel().copy()
    B = _f(B).ravel().copy()
    led = Ledger()
    extras = {}
    if want_matrices:
        J = np.zeros(3 * nn)
        M = np.zeros(243 * nn)
        Et = np.zeros(3 * nn)
        ptrs = [J.ctypes.data, M.ctypes.data, Et.ctypes.data]
    else:
        ptrs = [None, None, None]
    st = load().orc3_step(ctypes.byref(c), P.off, P.x, P.y, P.z, P.ux, P.uy, P.uz, P.w, E, B,
                          ctypes.byref(led), *ptrs)
    if want_matrices:
        extras = {"J": J.reshape(3, nn), "M": M.reshape(nn, 27, 3, 3), "Etheta": Et.reshape(3, nn)}
    d = led.asdict()
    d["status"] = st
    return E.reshape(3, nn), B.reshape(3, nn), d, extras
