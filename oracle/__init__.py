"""Python access to the plain FP64 CPU oracle (relsim_oracle.c).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. The CUDA library and its
binding never do. The oracle is compiled from C with gcc on first use (or by
``oracle.build.build()``), with no fast-math and no FMA contraction.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build, lib_path

__all__ = ["OracleConfig", "Ledger", "load", "deposit", "apply_A", "apply_M", "curl_c",
           "curl_n", "rhs", "gmres", "field_update", "push", "energies", "cell_keys",
           "stable_sort", "step", "gather_E", "gather_B", "alpha", "node_weights",
           "to_full_offsets", "make_config", "spectrum", "field_modes", "growth_fit", "field_adjoint",
           "push_adjoint", "deposit_adjoint", "step_adjoint",
           "mode_energy", "window_gradient", "mode_growth_rates", "dispersion_fit",
           "tearing_dispersion"]


class OracleConfig(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("dt", ctypes.c_double), ("theta", ctypes.c_double),
                ("nspecies", ctypes.c_int),
                ("q", ctypes.c_double * 4), ("m", ctypes.c_double * 4),
                ("gmres_tol", ctypes.c_double),
                ("gmres_restart", ctypes.c_int), ("gmres_maxit", ctypes.c_int),
                ("gamma_pred", ctypes.c_int)]


class Ledger(ctypes.Structure):
    _fields_ = [("W_E0", ctypes.c_double), ("W_B0", ctypes.c_double), ("K0", ctypes.c_double),
                ("W_E1", ctypes.c_double), ("W_B1", ctypes.c_double), ("K1", ctypes.c_double),
                ("work_grid", ctypes.c_double), ("work_particles", ctypes.c_double),
                ("mismatch", ctypes.c_double), ("dissipation", ctypes.c_double),
                ("residual", ctypes.c_double), ("gmres_iters", ctypes.c_int),
                ("gmres_relres", ctypes.c_double)]

    def asdict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_C = ctypes.POINTER(OracleConfig)


def load():
    """Load (building if needed) the oracle shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        build()
    lib = ctypes.CDLL(path)
    sig = {
        "orc_version": (ctypes.c_int, []),
        "orc_node_weights": (None, [_C, ctypes.c_double, ctypes.c_double, _I64, _D]),
        "orc_gather_E": (None, [_C, _D, ctypes.c_double, ctypes.c_double, _D]),
        "orc_gather_B": (None, [_C, _D, ctypes.c_double, ctypes.c_double, _D]),
        "orc_alpha": (None, [ctypes.c_double, ctypes.c_double, _D, _D]),
        "orc_deposit": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
        "orc_curl_c": (None, [_C, _D, _D]),
        "orc_curl_n": (None, [_C, _D, _D]),
        "orc_apply_M": (None, [_C, _D, _D, _D]),
        "orc_apply_A": (None, [_C, _D, _D, _D]),
        "orc_rhs": (None, [_C, _D, _D, _D, _D]),
        "orc_gmres": (ctypes.c_int, [_C, _D, _D, _D, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_double)]),
        "orc_field_update": (None, [_C, _D, _D, _D]),
        "orc_push": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]),
        "orc_energies": (None, [_C, _I64, _D, _D, _D, _D, _D, _D, _D]),
        "orc_cell_keys": (None, [_C, ctypes.c_int64, _D, _D, _I32]),
        "orc_stable_sort": (None, [ctypes.c_int64, _I32, ctypes.c_int32, _I64, _I64]),
        "orc_step": (ctypes.c_int, [_C, _I64, _D, _D, _D, _D, _D, _D, _D, _D,
                                    ctypes.POINTER(Ledger), ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def make_config(nx, ny, dx=1.0, dy=1.0, dt=0.5, theta=0.5, q=(1.0, -1.0), m=(1.0, 1.0),
                gmres_tol=1e-12, gmres_restart=50, gmres_maxit=2000, gamma_pred=0) -> OracleConfig:
    """gamma_pred = 1: the Lorentz factor in alpha and M is that of the
    predicted half-step momentum u^n + beta E^n(x) instead of u^n."""
    c = OracleConfig()
    c.gamma_pred = int(gamma_pred)
    c.nx, c.ny, c.dx, c.dy, c.dt, c.theta = nx, ny, dx, dy, dt, theta
    c.nspecies = len(q)
    for s in range(len(q)):
        c.q[s] = q[s]
        c.m[s] = m[s]
    c.gmres_tol, c.gmres_restart, c.gmres_maxit = gmres_tol, gmres_restart, gmres_maxit
    return c


def _f(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Particles:
    """Concatenated FP64 particle arrays of all species (oracle layout)."""

    def __init__(self, species):
        self.off = np.zeros(len(species) + 1, dtype=np.int64)
        for s, sp in enumerate(species):
            self.off[s + 1] = self.off[s] + len(sp["x"])
        cat = lambda k: _f(np.concatenate([np.asarray(sp[k], dtype=np.float64) for sp in species]))
        self.x, self.y = cat("x"), cat("y")
        self.ux, self.uy, self.uz = cat("ux"), cat("uy"), cat("uz")
        self.w = cat("w")

    def species(self, s):
        a, b = self.off[s], self.off[s + 1]
        return {k: getattr(self, k)[a:b].copy() for k in ("x", "y", "ux", "uy", "uz", "w")}

    def copy(self):
        p = Particles.__new__(Particles)
        p.off = self.off.copy()
        for k in ("x", "y", "ux", "uy", "uz", "w"):
            setattr(p, k, getattr(self, k).copy())
        return p


def node_weights(c, x, y):
    g = np.zeros(4, dtype=np.int64)
    W = np.zeros(4)
    load().orc_node_weights(ctypes.byref(c), x, y, g, W)
    return g, W


def gather_E(c, E, x, y):
    out = np.zeros(3)
    load().orc_gather_E(ctypes.byref(c), _f(E).ravel(), x, y, out)
    return out


def gather_B(c, B, x, y):
    out = np.zeros(3)
    load().orc_gather_B(ctypes.byref(c), _f(B).ravel(), x, y, out)
    return out


def alpha(beta, gbar, Bp):
    out = np.zeros(9)
    load().orc_alpha(beta, gbar, _f(Bp), out)
    return out.reshape(3, 3)


def deposit(c, P: Particles, B, E=None):
    """Jhat and M; E (E^n) is used by the predicted-gamma variant only."""
    nn = c.nx * c.ny
    J = np.zeros(3 * nn)
    M = np.zeros(81 * nn)
    E = np.zeros(3 * nn) if E is None else _f(E).ravel()
    load().orc_deposit(ctypes.byref(c), P.off, P.x, P.y, P.ux, P.uy, P.uz, P.w,
                       _f(B).ravel(), E, J, M)
    return J.reshape(3, nn), M.reshape(nn, 9, 3, 3)


def curl_c(c, E):
    out = np.zeros(3 * c.nx * c.ny)
    load().orc_curl_c(ctypes.byref(c), _f(E).ravel(), out)
    return out.reshape(3, -1)


def curl_n(c, B):
    out = np.zeros(3 * c.nx * c.ny)
    load().orc_curl_n(ctypes.byref(c), _f(B).ravel(), out)
    return out.reshape(3, -1)


def apply_M(c, M, v):
    out = np.zeros(3 * c.nx * c.ny)
    load().orc_apply_M(ctypes.byref(c), _f(M).ravel(), _f(v).ravel(), out)
    return out.reshape(3, -1)


def apply_A(c, M, v):
    out = np.zeros(3 * c.nx * c.ny)
    load().orc_apply_A(ctypes.byref(c), _f(M).ravel(), _f(v).ravel(), out)
    return out.reshape(3, -1)


def rhs(c, E, B, J):
    out = np.zeros(3 * c.nx * c.ny)
    load().orc_rhs(ctypes.byref(c), _f(E).ravel(), _f(B).ravel(), _f(J).ravel(), out)
    return out.reshape(3, -1)


def gmres(c, M, b, x0):
    x = _f(x0).ravel().copy()
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load().orc_gmres(ctypes.byref(c), _f(M).ravel(), _f(b).ravel(), x,
                          ctypes.byref(it), ctypes.byref(rr))
    return x.reshape(3, -1), st, it.value, rr.value


def field_update(c, Etheta, E, B):
    E = _f(E).ravel().copy()
    B = _f(B).ravel().copy()
    load().orc_field_update(ctypes.byref(c), _f(Etheta).ravel(), E, B)
    return E.reshape(3, -1), B.reshape(3, -1)


def push(c, P: Particles, Etheta, B, E=None):
    """Push in place; returns sums (K0, K1, work_particles, mismatch). E
    (E^n) is used by the predicted-gamma variant only."""
    sums = np.zeros(4)
    E = np.zeros(3 * c.nx * c.ny) if E is None else _f(E).ravel()
    load().orc_push(ctypes.byref(c), P.off, P.x, P.y, P.ux, P.uy, P.uz, P.w,
                    _f(Etheta).ravel(), _f(B).ravel(), E, sums)
    return sums


def energies(c, P: Particles, E, B):
    out = np.zeros(3)
    load().orc_energies(ctypes.byref(c), P.off, P.ux, P.uy, P.uz, P.w, _f(E).ravel(),
                        _f(B).ravel(), out)
    return out


def cell_keys(c, x, y):
    x, y = _f(x), _f(y)
    keys = np.zeros(x.size, dtype=np.int32)
    load().orc_cell_keys(ctypes.byref(c), x.size, x, y, keys)
    return keys


def stable_sort(keys, nkeys):
    keys = np.ascontiguousarray(keys, dtype=np.int32)
    perm = np.zeros(keys.size, dtype=np.int64)
    start = np.zeros(nkeys + 1, dtype=np.int64)
    load().orc_stable_sort(keys.size, keys, nkeys, perm, start)
    return perm, start


def step(c, P: Particles, E, B, want_matrices=False):
    """One full step in place on P; returns (E, B, ledger dict, extras)."""
    nn = c.nx * c.ny
    E = _f(E).ravel().copy()
    B = _f(B).ravel().copy()
    led = Ledger()
    extras = {}
    if want_matrices:
        J = np.zeros(3 * nn)
        M = np.zeros(81 * nn)
        Et = np.zeros(3 * nn)
        ptrs = [J.ctypes.data, M.ctypes.data, Et.ctypes.data]
    else:
        ptrs = [None, None, None]
    st = load().orc_step(ctypes.byref(c), P.off, P.x, P.y, P.ux, P.uy, P.uz, P.w, E, B,
                         ctypes.byref(led), *ptrs)
    if want_matrices:
        extras = {"J": J.reshape(3, nn), "M": M.reshape(nn, 9, 3, 3),
                  "Etheta": Et.reshape(3, nn)}
    d = led.asdict()
    d["status"] = st
    return E.reshape(3, nn), B.reshape(3, nn), d, extras


# the five neighbour offsets (di, dj) a half-stored mass matrix keeps: the
# other four follow from M_{g,g+o} = M_{g+o,g}
HALF_OFFSETS = ((0, 0), (1, 0), (-1, 1), (0, 1), (1, 1))


def to_full_offsets(o):
    di, dj = o
    return (dj + 1) * 3 + (di + 1)


def spectrum(ux, uy, uz, w, edges, variable=0, precision=64):
    """Weighted and counted particle spectrum: the paper's spectra (Sec. 3.2,
    "Nonlinear reconnection and spectra") are weighted particle distributions
    over the Lorentz factor or the proper speed u/c.

    x = gamma - 1 = |u|^2/(gamma + 1) (variable 0) or x = |u| (variable 1),
    formed in the given precision (32 or 64: the bin is an integer decided in
    floating point, so it is decided in the precision of the form being
    compared), with |u|^2 summed x, y, z in that order. Bins: [0] below
    edges[0], [b] for edges[b-1] <= x < edges[b], [nbins+1] at or above
    edges[nbins]. Returns (weights, counts), each of length nbins + 2.
    """
    t = np.float32 if precision == 32 else np.float64
    ux, uy, uz = (np.asarray(a, dtype=np.float64).astype(t) for a in (ux, uy, uz))
    u2 = ux * ux + uy * uy + uz * uz
    one = t(1)
    x = u2 / (np.sqrt(one + u2) + one) if variable == 0 else np.sqrt(u2)
    e = np.asarray(edges, dtype=np.float64)
    idx = np.searchsorted(e, x.astype(np.float64), side="right")
    nb = e.size + 1
    return (np.bincount(idx, weights=np.asarray(w, dtype=np.float64), minlength=nb),
            np.bincount(idx, minlength=nb).astype(np.int64))


def field_modes(c, B, component=1, nmodes=8):
    """Energy in the Fourier modes along x of one B component, the
    linear-tearing diagnostic of Sec. 3.1 (Fig. 1: the B_y energy, its
    low-pass part and single modes, whose growth gives the tearing rate).

    B is the (3, ny*nx) cell-centre field. With F_{m,j} the DFT along x of
    row j (numpy's FFT, FP64), the energy of mode m = 0 .. nmodes-1 is
    (1/2) dV (c_m / nx) sum_j |F_{m,j}|^2, c_m = 1 for m = 0 and m = nx/2,
    else 2 (mode m and its mirror nx - m), so that modes 0 .. nx/2 add up to
    (1/2) sum B_c^2 dV by Parseval. Mode m has k = 2 pi m / L_x.
    """
    nx, ny = c.nx, c.ny
    Bc = np.asarray(B, dtype=np.float64).reshape(3, ny, nx)[component]
    F = np.fft.rfft(Bc, axis=1)
    e = (np.abs(F) ** 2).sum(axis=0)
    cm = np.full(e.size, 2.0)
    cm[0] = 1.0
    if nx % 2 == 0:
        cm[-1] = 1.0
    dV = c.dx * c.dy
    return (0.5 * dV * cm * e / nx)[:nmodes]


def growth_fit(s, dt, window):
    """Exponential growth rate of a positive series (Sec. 3.1 measures the
    tearing rate as a best fit over the linear phase): for every run of
    `window` consecutive samples spaced dt, the least-squares slope of log s
    against time (numpy's polyfit, degree 1); returns the largest slope and
    the index of its run's first sample. Runs with a non-positive sample are
    skipped."""
    s = np.asarray(s, dtype=np.float64)
    t = np.arange(window) * dt
    best = None
    for a in range(s.size - window + 1):
        seg = s[a:a + window]
        if np.any(~(seg > 0)) or not np.all(np.isfinite(seg)):
            continue
        slope = np.polyfit(t, np.log(seg), 1)[0]
        if best is None or slope > best[0]:
            best = (slope, a)
    if best is None:
        raise ValueError("no admissible window")
    return best


def mode_growth_rates(modes, dt, first, window):
    """Amplitude growth rate of every Fourier mode over one fixed window
    (Sec. 3.1: each mode's growth is a best fit over the linear phase).

    modes is (nsamples, nmodes) mode energies sampled every dt; for mode m
    the rate is half the least-squares slope (numpy polyfit) of log energy
    against time over samples first .. first+window-1 (the amplitude grows
    at half the energy's rate); NaN for mode 0 and for modes with a
    non-positive or non-finite sample in the window."""
    e = np.asarray(modes, dtype=np.float64)
    t = np.arange(window) * dt
    out = np.full(e.shape[1], np.nan)
    for m in range(1, e.shape[1]):
        seg = e[first:first + window, m]
        if seg.size == window and np.all(np.isfinite(seg)) and np.all(seg > 0):
            out[m] = 0.5 * np.polyfit(t, np.log(seg), 1)[0]
    return out


def dispersion_fit(x, rates):
    """Least-squares fit of the tearing dispersion of Sec. 2, f(k) = ka
    (1 - k^2 a^2), with a free scale and a free width: rate = A x b (1 -
    x^2 b^2) in x = ka. For each b, A is the closed-form linear least
    squares; b is the minimiser of the residual over a dense grid on
    [0.2, 4] (step 1e-5). Non-finite rates are left out. Returns (A, b):
    the fitted curve peaks at x = 1/(sqrt(3) b) and vanishes at x = 1/b."""
    x = np.asarray(x, dtype=np.float64)
    r = np.asarray(rates, dtype=np.float64)
    keep = np.isfinite(r)
    x, r = x[keep], r[keep]
    if x.size < 2:
        raise ValueError("fewer than two finite rates")
    b = np.linspace(0.2, 4.0, 380001)
    xb = np.outer(b, x)
    g = xb * (1.0 - xb * xb)
    A = (g @ r) / np.einsum("ij,ij->i", g, g)
    res = ((A[:, None] * g - r[None, :]) ** 2).sum(axis=1)
    i = int(np.argmin(res))
    return float(A[i]), float(b[i])


def tearing_dispersion(modes, dt, first, window, Lx, a):
    """Per-mode rates over the window and their dispersion fit, with mode m
    at x = 2 pi m a / Lx: returns (rates, A, b)."""
    rates = mode_growth_rates(modes, dt, first, window)
    x = 2.0 * np.pi * np.arange(rates.size) * a / Lx
    A, b = dispersion_fit(x[1:], rates[1:])
    return rates, A, b


def field_adjoint(c, M, Etheta, gE1, gB1, gEt=None):
    """Adjoint of the field part of one step with the particles (hence M and
    Jhat) held fixed. The forward map (Sec. 2: the implicit field solve) is
      b = E0 + theta dt curl_n B0 - theta dt J,   A Et = b,
      E1 = (Et - (1 - theta) E0)/theta,           B1 = B0 - dt curl_c Et,
    with A = I + (theta dt)^2 curl_n curl_c + theta dt M (M in the oracle's
    full layout, (nn, 9, 3, 3)). For L with dL/dE1 = gE1, dL/dB1 = gB1 this
    returns dL/dE0, dL/dB0, dL/dJ and dL/dM (full layout) (gEt, if given, is
    a further dL/dEt, e.g. from the push), by the chain rule
    written out with dense matrices: A, curl_c and curl_n are assembled
    column by column from the oracle's own operators and transposed with
    numpy, and A^T lambda = dL/dEt is solved densely. For small grids only.
    """
    nn = c.nx * c.ny
    N = 3 * nn
    M = np.asarray(M, dtype=np.float64)

    def dense(f):
        out = np.empty((N, N))
        e = np.zeros(N)
        for k in range(N):
            e[k] = 1.0
            out[:, k] = np.asarray(f(e)).ravel()
            e[k] = 0.0
        return out

    A = dense(lambda v: apply_A(c, M, v))
    Cc = dense(lambda v: curl_c(c, v))
    Cn = dense(lambda v: curl_n(c, v))
    th, dt = c.theta, c.dt
    gE1 = np.asarray(gE1, dtype=np.float64).ravel()
    gB1 = np.asarray(gB1, dtype=np.float64).ravel()
    gEt = gE1 / th - dt * (Cc.T @ gB1) + (0.0 if gEt is None else np.asarray(gEt, dtype=np.float64).ravel())
    lam = np.linalg.solve(A.T, gEt)
    gE0 = lam - (1.0 - th) / th * gE1
    gB0 = gB1 + th * dt * (Cn.T @ lam)
    gJ = -th * dt * lam
    # dL/dA = -lambda Et^T; A holds theta dt M_{g g'} in the 3x3 block of
    # rows g, columns g'
    Et = np.asarray(Etheta, dtype=np.float64).reshape(3, nn)
    L3 = lam.reshape(3, nn)
    gM = np.zeros((nn, 9, 3, 3))
    for g in range(nn):
        i, j = g % c.nx, g // c.nx
        for slot in range(9):
            di, dj = slot % 3 - 1, slot // 3 - 1
            h = ((j + dj) % c.ny) * c.nx + (i + di) % c.nx
            gM[g, slot] = -th * dt * np.outer(L3[:, g], Et[:, h])
    return {"E0": gE0.reshape(3, nn), "B0": gB0.reshape(3, nn), "J": gJ.reshape(3, nn), "M": gM,
            "lambda": lam.reshape(3, nn)}


def _cic(c, x, y, shift):
    """Linear weights of the 4 lattice points around (x, y) on a lattice
    shifted by `shift` cells (0: nodes, 0.5: cell centres), with their x and
    y derivatives: indices (4, n), W, dW/dx, dW/dy (4, n)."""
    tx, ty = x / c.dx - shift, y / c.dy - shift
    fi, fj = np.floor(tx), np.floor(ty)
    fx, fy = tx - fi, ty - fj
    i, j = fi.astype(np.int64) % c.nx, fj.astype(np.int64) % c.ny
    i1, j1 = (i + 1) % c.nx, (j + 1) % c.ny
    g = np.stack([j * c.nx + i, j * c.nx + i1, j1 * c.nx + i, j1 * c.nx + i1])
    W = np.stack([(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy])
    Wx = np.stack([-(1 - fy), 1 - fy, -fy, fy]) / c.dx
    Wy = np.stack([-(1 - fx), -fx, 1 - fx, fx]) / c.dy
    return g, W, Wx, Wy


def _gbar_back(c, ggb, u, s, gb, beta, gN, WN, WNx, WNy, En, gEn, gx0, gy0, a0, a1):
    """dL/dgbar carried back through gbar: to u (base scheme, gbar =
    gamma(u)), or, with the predicted gbar = gamma(s), s = u + beta E^n(x), to
    u, to E^n on the nodes (the gather's transpose) and to x through the
    gather's weights. Returns dL/du's share."""
    gs = ggb * s / gb
    if not c.gamma_pred:
        return gs
    gEp = beta * gs
    for k in range(4):
        for comp in range(3):
            np.add.at(gEn[comp], gN[k], WN[k] * gEp[comp])
        eg = (En[:, gN[k]] * gEp).sum(axis=0)
        gx0[a0:a1] += WNx[k] * eg
        gy0[a0:a1] += WNy[k] * eg
    return gs


def push_adjoint(c, P: Particles, Etheta, B, gu1, gx1, gy1, En=None):
    """Adjoint of the push (Sec. 2: the pusher is explicit) with the fields
    held fixed. Forward, per particle:
      Ep = sum_g W_g(x) E_g (nodes),  Bp = sum_c W_c(x) B_c (centres),
      gbar = sqrt(1 + |s|^2) with s = u (base scheme) or, with gamma_pred,
      s = u + beta E^n(x) (E^n = En on the nodes),
      a = beta Bp/gbar,  alpha = (I + [a]x)^{-1},
      ubar = alpha (u + beta Ep),  u1 = 2 ubar - u,  x1 = x + dt u1/gamma(u1).
    Given dL/du1 (gu1, (3, N)) and dL/dx1, dL/dy1 (N each), returns dL/du,
    dL/dx, dL/dy per particle and dL/dE (nodes), dL/dB (centres), (3, nn),
    and with gamma_pred dL/dEn (nodes), by the chain rule in reverse: the
    transposes of the gathers are the scatters with the same weights,
    alpha's transpose is applied to the gradient of ubar, and d alpha =
    -alpha d[a]x alpha.
    """
    nn = c.nx * c.ny
    E = np.asarray(Etheta, dtype=np.float64).reshape(3, nn)
    if c.gamma_pred and En is None:
        raise ValueError("the predicted-gamma push adjoint needs E^n")
    En = np.zeros((3, nn)) if En is None else np.asarray(En, dtype=np.float64).reshape(3, nn)
    gEn = np.zeros((3, nn))
    Bf = np.asarray(B, dtype=np.float64).reshape(3, nn)
    gu1 = np.asarray(gu1, dtype=np.float64).reshape(3, -1)
    gx1 = np.asarray(gx1, dtype=np.float64).ravel()
    gy1 = np.asarray(gy1, dtype=np.float64).ravel()
    N = P.x.size
    gu0 = np.zeros((3, N))
    gx0 = gx1.copy()
    gy0 = gy1.copy()
    gE = np.zeros((3, nn))
    gB = np.zeros((3, nn))
    for s in range(int(c.nspecies)):
        a0, a1 = int(P.off[s]), int(P.off[s + 1])
        if a1 == a0:
            continue
        beta = c.q[s] * c.dt / (2.0 * c.m[s])
        x, y = P.x[a0:a1], P.y[a0:a1]
        u = np.stack([P.ux[a0:a1], P.uy[a0:a1], P.uz[a0:a1]])
        gN, WN, WNx, WNy = _cic(c, x, y, 0.0)
        gC, WC, WCx, WCy = _cic(c, x, y, 0.5)
        Ep = sum(WN[k] * E[:, gN[k]] for k in range(4))
        Bp = sum(WC[k] * Bf[:, gC[k]] for k in range(4))
        sv = u + beta * sum(WN[k] * En[:, gN[k]] for k in range(4)) if c.gamma_pred else u
        gb = np.sqrt(1.0 + (sv * sv).sum(axis=0))
        a = beta * Bp / gb
        n = a1 - a0
        ax = np.zeros((n, 3, 3))   # [a]x v = a x v
        ax[:, 0, 1], ax[:, 0, 2] = -a[2], a[1]
        ax[:, 1, 0], ax[:, 1, 2] = a[2], -a[0]
        ax[:, 2, 0], ax[:, 2, 1] = -a[1], a[0]
        alpha = np.linalg.inv(np.eye(3)[None] + ax)
        w = u + beta * Ep
        ub = np.einsum("nij,jn->in", alpha, w)
        u1 = 2.0 * ub - u
        g1 = np.sqrt(1.0 + (u1 * u1).sum(axis=0))
        # x1 = x + dt u1/g1 (x and y components)
        gpos = np.stack([gx1[a0:a1], gy1[a0:a1], np.zeros(n)])
        gu1t = gu1[:, a0:a1] + c.dt * (gpos / g1 - u1 * (u1 * gpos).sum(axis=0) / g1 ** 3)
        gub = 2.0 * gu1t
        gu = -gu1t
        gw = np.einsum("nji,jn->in", alpha, gub)          # alpha^T gubar
        galpha = np.einsum("in,jn->nij", gub, w)           # gubar w^T
        gu += gw
        gEp = beta * gw
        G = -np.einsum("nji,njk,nlk->nil", alpha, galpha, alpha)   # -alpha^T galpha alpha^T
        ga = np.stack([G[:, 2, 1] - G[:, 1, 2], G[:, 0, 2] - G[:, 2, 0], G[:, 1, 0] - G[:, 0, 1]])
        gBp = beta * ga / gb
        ggb = -beta * (ga * Bp).sum(axis=0) / gb ** 2
        gu += _gbar_back(c, ggb, u, sv, gb, beta, gN, WN, WNx, WNy, En, gEn, gx0, gy0, a0, a1)
        for k in range(4):
            for comp in range(3):
                np.add.at(gE[comp], gN[k], WN[k] * gEp[comp])
                np.add.at(gB[comp], gC[k], WC[k] * gBp[comp])
            eg = (E[:, gN[k]] * gEp).sum(axis=0)
            bg = (Bf[:, gC[k]] * gBp).sum(axis=0)
            gx0[a0:a1] += WNx[k] * eg + WCx[k] * bg
            gy0[a0:a1] += WNy[k] * eg + WCy[k] * bg
        gu0[:, a0:a1] = gu
    out = {"u": gu0, "x": gx0, "y": gy0, "E": gE, "B": gB}
    if c.gamma_pred:
        out["En"] = gEn
    return out


def deposit_adjoint(c, P: Particles, B, gJ, gM, En=None):
    """Adjoint of the deposit. Forward, per particle: Bp = sum_c W_c(x) B_c,
    gbar = gamma(u^n) (base scheme) or, with gamma_pred, gamma(u^n + beta
    E^n(x)) (E^n = En on the nodes), a = beta Bp/gbar, alpha = (I + [a]x)^-1,
      Jhat_g += (w q/dV) W_g(x) alpha u/gbar,
      M_{g g'} += (w q beta/dV) W_g(x) W_g'(x) alpha/gbar  (ordered pairs, full layout).
    Given dL/dJhat (gJ, (3, nn)) and dL/dM (gM, (nn, 9, 3, 3) full layout),
    returns dL/du (3, N), dL/dx, dL/dy (N), dL/dw (N) and dL/dB (3, nn): the
    gradient of alpha collects the current and every node pair's block
    gradient, then flows through a (d alpha = -alpha d[a]x alpha) to Bp and
    gbar (and, with gamma_pred, through gbar to E^n: dL/dEn in the result);
    J and M are linear in w, so dL/dw is the particle's contribution to
    <gJ, Jhat> + <gM, M> per unit weight."""
    nn = c.nx * c.ny
    dV = c.dx * c.dy
    Bf = np.asarray(B, dtype=np.float64).reshape(3, nn)
    if c.gamma_pred and En is None:
        raise ValueError("the predicted-gamma deposit adjoint needs E^n")
    En = np.zeros((3, nn)) if En is None else np.asarray(En, dtype=np.float64).reshape(3, nn)
    gEn = np.zeros((3, nn))
    gJ = np.asarray(gJ, dtype=np.float64).reshape(3, nn)
    gM = np.asarray(gM, dtype=np.float64).reshape(nn, 9, 3, 3)
    N = P.x.size
    gu0 = np.zeros((3, N))
    gx0 = np.zeros(N)
    gy0 = np.zeros(N)
    gw0 = np.zeros(N)
    gB = np.zeros((3, nn))
    for s in range(int(c.nspecies)):
        a0, a1 = int(P.off[s]), int(P.off[s + 1])
        if a1 == a0:
            continue
        q, m = c.q[s], c.m[s]
        beta = q * c.dt / (2.0 * m)
        x, y = P.x[a0:a1], P.y[a0:a1]
        u = np.stack([P.ux[a0:a1], P.uy[a0:a1], P.uz[a0:a1]])
        w = P.w[a0:a1]
        n = a1 - a0
        gN, WN, WNx, WNy = _cic(c, x, y, 0.0)
        gC, WC, WCx, WCy = _cic(c, x, y, 0.5)
        Bp = sum(WC[k] * Bf[:, gC[k]] for k in range(4))
        sv = u + beta * sum(WN[k] * En[:, gN[k]] for k in range(4)) if c.gamma_pred else u
        gb = np.sqrt(1.0 + (sv * sv).sum(axis=0))
        a = beta * Bp / gb
        ax = np.zeros((n, 3, 3))
        ax[:, 0, 1], ax[:, 0, 2] = -a[2], a[1]
        ax[:, 1, 0], ax[:, 1, 2] = a[2], -a[0]
        ax[:, 2, 0], ax[:, 2, 1] = -a[1], a[0]
        alpha = np.linalg.inv(np.eye(3)[None] + ax)
        cJ = w * q / dV
        cM = w * q * beta / dV
        au = np.einsum("nij,jn->in", alpha, u)
        galpha = np.zeros((n, 3, 3))
        gWn = np.zeros((4, n))
        ggb = np.zeros(n)
        gu = np.zeros((3, n))
        for k in range(4):
            gj = gJ[:, gN[k]]                                   # (3, n)
            # Jhat: cJ W alpha u / gbar
            galpha += (cJ * WN[k] / gb)[:, None, None] * np.einsum("in,jn->nij", gj, u)
            gu += cJ * WN[k] / gb * np.einsum("nji,jn->in", alpha, gj)
            sJ = (gj * au).sum(axis=0)
            gWn[k] += cJ * sJ / gb
            ggb -= cJ * WN[k] * sJ / gb ** 2
            gw0[a0:a1] += (q / dV) * WN[k] * sJ / gb
            # M: every ordered node pair (k, l) of the cell
            for l in range(4):
                # the slot of node l seen from node k (offsets of the cell's nodes)
                dk = (k % 2, k // 2)
                dl = (l % 2, l // 2)
                slot = (dl[1] - dk[1] + 1) * 3 + (dl[0] - dk[0] + 1)
                G = gM[gN[k], slot]                              # (n, 3, 3)
                s2 = np.einsum("nij,nij->n", G, alpha)
                coef = cM * WN[k] * WN[l] / gb
                galpha += coef[:, None, None] * G
                gWn[k] += cM * WN[l] * s2 / gb
                gWn[l] += cM * WN[k] * s2 / gb
                ggb -= cM * WN[k] * WN[l] * s2 / gb ** 2
                gw0[a0:a1] += (q * beta / dV) * WN[k] * WN[l] * s2 / gb
        Gm = -np.einsum("nji,njk,nlk->nil", alpha, galpha, alpha)   # -alpha^T galpha alpha^T
        ga = np.stack([Gm[:, 2, 1] - Gm[:, 1, 2], Gm[:, 0, 2] - Gm[:, 2, 0], Gm[:, 1, 0] - Gm[:, 0, 1]])
        gBp = beta * ga / gb
        ggb -= beta * (ga * Bp).sum(axis=0) / gb ** 2
        gu += _gbar_back(c, ggb, u, sv, gb, beta, gN, WN, WNx, WNy, En, gEn, gx0, gy0, a0, a1)
        for k in range(4):
            for comp in range(3):
                np.add.at(gB[comp], gC[k], WC[k] * gBp[comp])
            bg = (Bf[:, gC[k]] * gBp).sum(axis=0)
            gx0[a0:a1] += WNx[k] * gWn[k] + WCx[k] * bg
            gy0[a0:a1] += WNy[k] * gWn[k] + WCy[k] * bg
        gu0[:, a0:a1] = gu
    out = {"u": gu0, "x": gx0, "y": gy0, "w": gw0, "B": gB}
    if c.gamma_pred:
        out["En"] = gEn
    return out


def step_adjoint(c, P: Particles, E, B, gu1, gx1, gy1, gE1, gB1):
    """Gradient of a loss of one full step's outputs (u^{n+1}, x^{n+3/2},
    E^{n+1}, B^{n+1}) with respect to its inputs (u^n, x^{n+1/2}, E^n, B^n):
    the push's adjoint (fields fixed) gives dL/dEt and part of dL/dB^n; the
    field adjoint with that dL/dEt gives dL/dE^n, dL/dJhat, dL/dM and the
    field part of dL/dB^n; the deposit's adjoint carries dL/dJhat and dL/dM
    back to the particles and B^n. P is the state before the step."""
    nn = c.nx * c.ny
    En = E if c.gamma_pred else None
    J, M = deposit(c, P, B, En)
    b = rhs(c, E, B, J)
    Et, _, _, _ = gmres(c, M, b, np.zeros_like(b))
    gp = push_adjoint(c, P, Et, B, gu1, gx1, gy1, En)
    gf = field_adjoint(c, M, Et, gE1, gB1, gEt=gp["E"])
    gd = deposit_adjoint(c, P, B, gf["J"], gf["M"], En)
    gE0 = gf["E0"] + (gp["En"] + gd["En"] if c.gamma_pred else 0.0)
    return {"u": gp["u"] + gd["u"], "x": gp["x"] + gd["x"], "y": gp["y"] + gd["y"], "w": gd["w"],
            "E": gE0, "B": gf["B0"] + gp["B"] + gd["B"], "push": gp, "field": gf, "deposit": gd}


def mode_energy(c, B, mode=1, component=1):
    """Energy of Fourier mode m along x of one B component, and its gradient
    with respect to B (3, nn): with F_j the DFT of row j (numpy's FFT), the
    energy (1/2) dV (2/nx) sum_j |F_j|^2 has derivative
    (2 dV/nx) Re(conj(F_j) exp(-2 pi sqrt(-1) m i/nx)) at cell (i, j)."""
    nx, ny = c.nx, c.ny
    dV = c.dx * c.dy
    Bc = np.asarray(B, dtype=np.float64).reshape(3, ny, nx)[component]
    F = np.fft.fft(Bc, axis=1)[:, mode]
    W = 0.5 * dV * (2.0 / nx) * float(np.sum(np.abs(F) ** 2))
    ph = np.exp(-2j * np.pi * mode * np.arange(nx) / nx)
    g = np.zeros((3, ny, nx))
    g[component] = (2.0 * dV / nx) * np.real(np.conj(F)[:, None] * ph[None, :])
    return W, g.reshape(3, nx * ny)


def window_gradient(c, species, E, B, nsteps, mode=1):
    """Loss = mode_energy of B_y after nsteps oracle steps from the given
    state, and its gradient with respect to the initial E, B and particles
    (the oracle keeps the particles' order): the step adjoints chained
    backwards over the stored start states."""
    P = Particles(species)
    E = np.asarray(E, dtype=np.float64).reshape(3, -1).copy()
    B = np.asarray(B, dtype=np.float64).reshape(3, -1).copy()
    pres = []
    for n in range(nsteps):
        pres.append((P.copy(), E.copy(), B.copy()))
        E, B, _, _ = step(c, P, E, B)
    W, gB = mode_energy(c, B, mode)
    gE = np.zeros_like(E)
    N = P.x.size
    gu, gx, gy, gw = np.zeros((3, N)), np.zeros(N), np.zeros(N), np.zeros(N)
    for n in range(nsteps - 1, -1, -1):
        Pn, En, Bn = pres[n]
        g = step_adjoint(c, Pn, En, Bn, gu, gx, gy, gE, gB)
        gu, gx, gy, gE, gB = g["u"], g["x"], g["y"], g["E"], g["B"]
        gw = gw + g["w"]   # the weights are the same at every step
    return W, {"E": gE, "B": gB, "u": gu, "x": gx, "y": gy, "w": gw}
