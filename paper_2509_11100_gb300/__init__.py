"""Python binding of the GB300 RelSIM hot-path library (librelsim.so).

Argument marshalling only: every step of the method runs in the CUDA
kernels behind the C ABI declared in include/relsim.h. The functions keep the
C names (relsim_init, relsim_load_particles, relsim_build_mass_matrix,
relsim_field_solve, relsim_push, relsim_energy_ledger, ...). Arrays may be
numpy arrays (host memory) or CUDA torch tensors (device memory); torch
supplies device memory and the CUDA stream, nothing else.

If the shared library has not been built, importing works but the first call
raises RelsimUnavailable: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

__all__ = [
    "RelsimError", "RelsimUnavailable", "relsim_config", "relsim_energy", "lib", "lib_path",
    "make_config", "relsim_init", "relsim_destroy", "relsim_last_error", "relsim_load_particles",
    "relsim_set_fields", "relsim_get_fields", "relsim_num_particles", "relsim_get_particles",
    "relsim_get_cell_start", "relsim_build_mass_matrix", "relsim_get_mass_matrix",
    "relsim_set_mass_matrix", "relsim_field_solve", "relsim_get_E_theta", "relsim_apply_operator",
    "relsim_push", "relsim_energy_ledger", "relsim_step", "relsim_version", "Simulation",
    "relsim_profile_enable", "relsim_profile_read", "relsim_kernel_launches", "PROFILE_SLOTS",
    "relsim_kinetic_energy_noalloc", "relsim_energy_spectrum", "RELSIM_ERR_TOO_LARGE", "RELSIM_NOALLOC_MAX_PARTICLES",
    "RELSIM_HOST", "RELSIM_DEVICE", "RELSIM_OK", "RELSIM_ERR_NOT_CONVERGED",
    "relsim_field_modes", "relsim_field_mode_gradient", "relsim_growth_fit", "relsim_dispersion_fit", "relsim_batch_create", "relsim_batch_run",
    "relsim_batch_set_shared", "relsim_batch_last_path", "relsim_batch_destroy", "Batch", "relsim_graph_info", "relsim_field_adjoint", "relsim_autotune",
    "relsim_tuning", "relsim_push_adjoint", "relsim_deposit_adjoint", "relsim_step_adjoint",
    "relsim_relabel_particles", "relsim_set_launch_shapes", "relsim_get_particles_native",
    "relsim_load_particles_native",
]

HERE = os.path.dirname(os.path.abspath(__file__))

RELSIM_OK = 0
RELSIM_ERR_INVALID_ARG = -1
RELSIM_ERR_BAD_STATE = -2
RELSIM_ERR_CUDA = -3
RELSIM_ERR_OOM = -4
RELSIM_ERR_NOT_CONVERGED = -5
RELSIM_ERR_NONFINITE = -6
RELSIM_ERR_TIMEOUT = -7
RELSIM_ERR_INTERNAL = -8
RELSIM_ERR_TOO_LARGE = -9
RELSIM_NOALLOC_MAX_PARTICLES = 33554432
RELSIM_HOST = 0
RELSIM_DEVICE = 1

_ERRNAMES = {-1: "INVALID_ARG", -2: "BAD_STATE", -3: "CUDA", -4: "OOM", -5: "NOT_CONVERGED",
             -6: "NONFINITE", -7: "TIMEOUT", -8: "INTERNAL",
             -9: "TOO_LARGE"}


class RelsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"relsim error {code} ({_ERRNAMES.get(code, '?')}): {msg}")
        self.code = code


class RelsimUnavailable(RuntimeError):
    pass


class relsim_config(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("dt", ctypes.c_double), ("theta_implicit", ctypes.c_double),
                ("precision", ctypes.c_int), ("nspecies", ctypes.c_int),
                ("q", ctypes.c_double * 4), ("m", ctypes.c_double * 4),
                ("gmres_tol", ctypes.c_double), ("gmres_restart", ctypes.c_int),
                ("gmres_maxit", ctypes.c_int), ("track_ids", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("gamma_pred", ctypes.c_int), ("shape", ctypes.c_int),
                ("gmres_fp64", ctypes.c_int)]


class relsim_energy(ctypes.Structure):
    _fields_ = [("W_E", ctypes.c_double), ("W_B", ctypes.c_double), ("K", ctypes.c_double),
                ("total", ctypes.c_double), ("K_species", ctypes.c_double * 4),
                ("W_E0", ctypes.c_double), ("W_B0", ctypes.c_double), ("K0", ctypes.c_double),
                ("dW_E", ctypes.c_double), ("dW_B", ctypes.c_double), ("dK", ctypes.c_double),
                ("work_grid", ctypes.c_double), ("work_particles", ctypes.c_double),
                ("mismatch", ctypes.c_double), ("dissipation", ctypes.c_double),
                ("residual", ctypes.c_double), ("gmres_iters", ctypes.c_int),
                ("gmres_restarts", ctypes.c_int), ("gmres_relres", ctypes.c_double),
                ("step", ctypes.c_int64), ("n_particles", ctypes.c_int64)]

    def asdict(self) -> dict:
        d = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            d[k] = list(v) if k == "K_species" else v
        return d


_P = ctypes.c_void_p
_CTX = ctypes.c_void_p
_SIGS = {
    "relsim_version": (ctypes.c_int, []),
    "relsim_init": (ctypes.c_int, [ctypes.POINTER(relsim_config), _P, ctypes.POINTER(_CTX)]),
    "relsim_destroy": (None, [_CTX]),
    "relsim_last_error": (ctypes.c_char_p, [_CTX]),
    "relsim_load_particles": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int64, _P, _P, _P, ctypes.c_int]),
    "relsim_set_fields": (ctypes.c_int, [_CTX, _P, _P, ctypes.c_int]),
    "relsim_get_fields": (ctypes.c_int, [_CTX, _P, _P, ctypes.c_int]),
    "relsim_num_particles": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)]),
    "relsim_get_particles": (ctypes.c_int, [_CTX, ctypes.c_int, _P, _P, _P, _P, ctypes.c_int]),
    "relsim_get_cell_start": (ctypes.c_int, [_CTX, ctypes.c_int, _P, ctypes.c_int]),
    "relsim_build_mass_matrix": (ctypes.c_int, [_CTX]),
    "relsim_get_mass_matrix": (ctypes.c_int, [_CTX, _P, _P, ctypes.c_int]),
    "relsim_set_mass_matrix": (ctypes.c_int, [_CTX, _P, _P, ctypes.c_int]),
    "relsim_field_solve": (ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "relsim_get_E_theta": (ctypes.c_int, [_CTX, _P, ctypes.c_int]),
    "relsim_apply_operator": (ctypes.c_int, [_CTX, _P, _P, ctypes.c_int]),
    "relsim_push": (ctypes.c_int, [_CTX]),
    "relsim_energy_ledger": (ctypes.c_int, [_CTX, ctypes.POINTER(relsim_energy)]),
    "relsim_step": (ctypes.c_int, [_CTX, ctypes.POINTER(relsim_energy)]),
    "relsim_profile_enable": (ctypes.c_int, [_CTX, ctypes.c_int]),
    "relsim_profile_read": (ctypes.c_int, [_CTX, ctypes.c_void_p, ctypes.c_int]),
    "relsim_kernel_launches": (ctypes.c_int64, []),
    "relsim_kinetic_energy_noalloc": (ctypes.c_int, [_P, _P, ctypes.c_int64, ctypes.c_double, _P, _P]),
    "relsim_energy_spectrum": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P,
                                              ctypes.c_int]),
    "relsim_field_modes": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int]),
    "relsim_field_mode_gradient": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _P, _P, ctypes.c_int]),
    "relsim_growth_fit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_int, _P, _P]),
    "relsim_dispersion_fit": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, ctypes.c_double, _P, _P, _P]),
    "relsim_batch_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P]),
    "relsim_batch_run": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "relsim_batch_set_shared": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "relsim_batch_last_path": (ctypes.c_int, [_P]),
    "relsim_batch_destroy": (None, [_P]),
    "relsim_graph_info": (ctypes.c_int, [_CTX, _P, _P, _P]),
    "relsim_field_adjoint": (ctypes.c_int, [_CTX, _P, _P, _P, _P, _P, _P, _P, _P, _P, ctypes.c_int]),
    "relsim_deposit_adjoint": (ctypes.c_int, [_CTX, ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_int]),
    "relsim_autotune": (ctypes.c_int, [_CTX, _P]),
    "relsim_push_adjoint": (ctypes.c_int, [_CTX, ctypes.c_int, _P, _P, _P, _P, _P, _P, ctypes.c_int]),
    "relsim_set_launch_shapes": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "relsim_step_adjoint": (ctypes.c_int, [_CTX, _P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double)]),
    "relsim_relabel_particles": (ctypes.c_int, [_CTX, ctypes.c_int, _P, ctypes.c_int]),
    "relsim_get_particles_native": (ctypes.c_int, [_CTX, ctypes.c_int, _P, _P, _P, _P, _P, ctypes.c_int]),
    "relsim_load_particles_native": (ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int64, _P, _P, _P, _P, _P,
                                                    ctypes.c_int]),
}

PROFILE_SLOTS = ("deposit", "push", "sort_tables", "permute", "gmres_apply",
                 "gmres_ortho", "field_update", "rhs", "load", "general_sort")


class relsim_tuning(ctypes.Structure):
    _fields_ = [("ncand", ctypes.c_int), ("deposit_blocks", ctypes.c_int * 8),
                ("deposit_ms", ctypes.c_float * 8), ("push_blocks", ctypes.c_int * 8),
                ("push_ms", ctypes.c_float * 8), ("deposit_choice", ctypes.c_int),
                ("push_choice", ctypes.c_int), ("op_nrows", ctypes.c_int), ("op_rows", ctypes.c_int * 4),
                ("op_ms", ctypes.c_float * 4), ("op_choice", ctypes.c_int)]

    def asdict(self) -> dict:
        n = self.ncand
        return {"deposit": [(self.deposit_blocks[k], self.deposit_ms[k]) for k in range(n)],
                "push": [(self.push_blocks[k], self.push_ms[k]) for k in range(n)],
                "deposit_blocks": self.deposit_blocks[self.deposit_choice],
                "push_blocks": self.push_blocks[self.push_choice],
                "op_tile_rows": [(self.op_rows[k], self.op_ms[k]) for k in range(self.op_nrows)],
                "op_rows": self.op_rows[self.op_choice]}


class relsim_profile(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 16), ("groups", ctypes.c_int64 * 16),
                ("kernels", ctypes.c_int64 * 16)]

_lib = None


def lib_path() -> str:
    return os.path.join(HERE, "librelsim.so")


def lib():
    """The loaded librelsim.so; raises RelsimUnavailable if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RelsimUnavailable(
            f"{path} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
            "(the RelSIM path has no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


# ---------------------------------------------------------------------------
# marshalling helpers

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, dtype=np.float64, writable=False):
    """(pointer, where, keepalive) of a numpy array or torch tensor."""
    if a is None:
        return None, RELSIM_HOST, None
    if _is_torch(a):
        import torch
        want = {np.float64: torch.float64, np.float32: torch.float32, np.int64: torch.int64,
                np.int32: torch.int32}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"tensor must be contiguous {want}")
        return a.data_ptr(), (RELSIM_DEVICE if a.is_cuda else RELSIM_HOST), a
    arr = np.asarray(a)
    if arr.dtype != dtype or not arr.flags["C_CONTIGUOUS"] or (writable and not arr.flags["WRITEABLE"]):
        if writable:
            raise TypeError(f"output array must be a writable C-contiguous {np.dtype(dtype)} array")
        arr = np.ascontiguousarray(arr, dtype=dtype)
    return arr.ctypes.data, RELSIM_HOST, arr


def _where(*items):
    ws = {w for (p, w, k) in items if p is not None}
    if len(ws) > 1:
        raise ValueError("mix of host and device arrays in one call")
    return ws.pop() if ws else RELSIM_HOST


def _check(ctx, code, allow=()):
    if code != RELSIM_OK and code not in allow:
        msg = lib().relsim_last_error(ctx)
        raise RelsimError(code, msg.decode() if msg else "")
    return code


def _stream(stream=None) -> int:
    if stream is not None:
        return int(stream)
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


# ---------------------------------------------------------------------------
# the C entry points, one Python function each

def make_config(nx, ny, dx=1.0, dy=1.0, dt=0.5, theta_implicit=0.5, precision=32,
                q=(1.0, -1.0), m=(1.0, 1.0), gmres_tol=0.0, gmres_restart=0, gmres_maxit=0,
                track_ids=False, gamma_pred=False, nz=None, dz=1.0, shape=1, gmres_fp64=False) -> relsim_config:
    """gamma_pred: the Lorentz factor in alpha and M is that of the
    predicted half-step momentum u^n + beta E^n(x) instead of u^n. nz: the
    3D form on an nx x ny x nz grid (cell size dz along z). gmres_fp64: FP64
    GMRES vectors in the FP32 form too (default: double-float pairs in the
    2D FP32 form with linear shapes)."""
    c = relsim_config()
    c.dim, c.nx, c.ny, c.nz = (2, nx, ny, 1) if nz is None else (3, nx, ny, nz)
    c.dx, c.dy, c.dz, c.dt, c.theta_implicit = dx, dy, (1.0 if nz is None else dz), dt, theta_implicit
    c.precision, c.nspecies = precision, len(q)
    for s in range(len(q)):
        c.q[s] = q[s]
        c.m[s] = m[s]
    c.gmres_tol, c.gmres_restart, c.gmres_maxit = gmres_tol, gmres_restart, gmres_maxit
    c.track_ids = 1 if track_ids else 0
    c.gamma_pred = 1 if gamma_pred else 0
    c.shape = int(shape)
    c.gmres_fp64 = 1 if gmres_fp64 else 0
    return c


def relsim_version() -> int:
    return lib().relsim_version()


def relsim_init(cfg: relsim_config, stream=None):
    ctx = _CTX()
    code = lib().relsim_init(ctypes.byref(cfg), _P(_stream(stream)), ctypes.byref(ctx))
    if code != RELSIM_OK:
        raise RelsimError(code, "relsim_init failed (check the config)")
    return ctx


def relsim_destroy(ctx):
    if ctx:
        lib().relsim_destroy(ctx)


def relsim_last_error(ctx) -> str:
    m = lib().relsim_last_error(ctx)
    return m.decode() if m else ""


def relsim_load_particles(ctx, species, x, u, w):
    n = int(len(w))
    px, pu, pw = _ptr(x), _ptr(u), _ptr(w)
    return _check(ctx, lib().relsim_load_particles(ctx, species, n, px[0], pu[0], pw[0],
                                                   _where(px, pu, pw)))


def relsim_set_fields(ctx, E=None, B=None):
    pE, pB = _ptr(E), _ptr(B)
    return _check(ctx, lib().relsim_set_fields(ctx, pE[0], pB[0], _where(pE, pB)))


def _out(shape, dtype, device):
    if device:
        import torch
        td = {np.float64: torch.float64, np.float32: torch.float32, np.int64: torch.int64,
              np.int32: torch.int32}[dtype]
        return torch.empty(shape, dtype=td, device="cuda")
    return np.empty(shape, dtype=dtype)


def _ncell(ctx_cfg):
    return ctx_cfg.nx * ctx_cfg.ny


def relsim_get_fields(ctx, ncell, device=False):
    E, B = _out((3, ncell), np.float64, device), _out((3, ncell), np.float64, device)
    pE, pB = _ptr(E, writable=True), _ptr(B, writable=True)
    _check(ctx, lib().relsim_get_fields(ctx, pE[0], pB[0], _where(pE, pB)))
    return E, B


def relsim_num_particles(ctx, species) -> int:
    n = ctypes.c_int64(0)
    _check(ctx, lib().relsim_num_particles(ctx, species, ctypes.byref(n)))
    return n.value


def relsim_get_particles(ctx, species, ids=False, device=False, dim=2):
    n = relsim_num_particles(ctx, species)
    x = _out((n, dim), np.float64, device)
    u = _out((n, 3), np.float64, device)
    w = _out((n,), np.float64, device)
    i = _out((n,), np.int32, device) if ids else None
    px, pu, pw = _ptr(x, writable=True), _ptr(u, writable=True), _ptr(w, writable=True)
    pi = _ptr(i, np.int32, writable=True) if ids else (None, RELSIM_HOST, None)
    _check(ctx, lib().relsim_get_particles(ctx, species, px[0], pu[0], pw[0], pi[0], _where(px, pu, pw)))
    return (x, u, w, i) if ids else (x, u, w)


def relsim_get_particles_native(ctx, species, ncell, precision=32, ids=False, device=False, dim=2):
    """The species in the library's own form: (start[ncell + 1] int32,
    off (dim, n), u (3, n), w (n,), [id (n,) int32]), the floating arrays in
    the context's precision (float32 or float64)."""
    n = relsim_num_particles(ctx, species)
    ft = np.float32 if precision == 32 else np.float64
    st = _out((ncell + 1,), np.int32, device)
    off, u, w = _out((dim, n), ft, device), _out((3, n), ft, device), _out((n,), ft, device)
    i = _out((n,), np.int32, device) if ids else None
    ps = _ptr(st, np.int32, writable=True)
    po, pu, pw = (_ptr(a, ft, writable=True) for a in (off, u, w))
    pi = _ptr(i, np.int32, writable=True) if ids else (None, RELSIM_HOST, None)
    _check(ctx, lib().relsim_get_particles_native(ctx, species, ps[0], po[0], pu[0], pw[0], pi[0],
                                                  _where(ps, po, pu, pw)))
    return (st, off, u, w, i) if ids else (st, off, u, w)


def relsim_load_particles_native(ctx, species, start, off, u, w, ids=None, precision=32):
    """Replace a species by particles in the library's own form (see
    relsim_get_particles_native); no conversion and no sort."""
    ft = np.float32 if precision == 32 else np.float64
    n = int(w.shape[0])
    ps = _ptr(start, np.int32)
    po, pu, pw = _ptr(off, ft), _ptr(u, ft), _ptr(w, ft)
    pi = _ptr(ids, np.int32) if ids is not None else (None, RELSIM_HOST, None)
    return _check(ctx, lib().relsim_load_particles_native(ctx, species, n, ps[0], po[0], pu[0], pw[0], pi[0],
                                                          _where(ps, po, pu, pw, pi)))


def relsim_get_cell_start(ctx, species, ncell, device=False):
    s = _out((ncell + 1,), np.int64, device)
    ps = _ptr(s, np.int64, writable=True)
    _check(ctx, lib().relsim_get_cell_start(ctx, species, ps[0], ps[1]))
    return s


def relsim_build_mass_matrix(ctx):
    return _check(ctx, lib().relsim_build_mass_matrix(ctx))


def relsim_get_mass_matrix(ctx, ncell, device=False, nhalf=5):
    """The stored blocks (ncell, nhalf, 3, 3): 5 offsets in 2D, 14 in 3D."""
    M = _out((ncell, nhalf, 3, 3), np.float64, device)
    J = _out((3, ncell), np.float64, device)
    pM, pJ = _ptr(M, writable=True), _ptr(J, writable=True)
    _check(ctx, lib().relsim_get_mass_matrix(ctx, pM[0], pJ[0], _where(pM, pJ)))
    return M, J


def relsim_set_mass_matrix(ctx, M, J):
    pM, pJ = _ptr(M), _ptr(J)
    return _check(ctx, lib().relsim_set_mass_matrix(ctx, pM[0], pJ[0], _where(pM, pJ)))


def relsim_field_solve(ctx):
    """Returns (iters, rel_residual, status); status may be NOT_CONVERGED."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    code = _check(ctx, lib().relsim_field_solve(ctx, ctypes.byref(it), ctypes.byref(rr)),
                  allow=(RELSIM_ERR_NOT_CONVERGED,))
    return it.value, rr.value, code


def relsim_get_E_theta(ctx, ncell, device=False):
    E = _out((3, ncell), np.float64, device)
    pE = _ptr(E, writable=True)
    _check(ctx, lib().relsim_get_E_theta(ctx, pE[0], pE[1]))
    return E


def relsim_apply_operator(ctx, v, device=False):
    pv = _ptr(v)
    out = _out(tuple(np.shape(v)) if not _is_torch(v) else tuple(v.shape), np.float64,
               pv[1] == RELSIM_DEVICE)
    po = _ptr(out, writable=True)
    _check(ctx, lib().relsim_apply_operator(ctx, pv[0], po[0], _where(pv, po)))
    return out


def relsim_energy_spectrum(ctx, species, edges, variable=0, device=False):
    """Weighted and counted histogram of gamma - 1 (variable 0) or |u|
    (variable 1) over the bins between the FP64 edges (host array), plus the
    bins below and above them. Returns (weight[nbins + 2], count[nbins + 2])."""
    e = np.ascontiguousarray(edges, dtype=np.float64)
    nb = e.size - 1
    wgt = _out((nb + 2,), np.float64, device)
    cnt = _out((nb + 2,), np.int64, device)
    pw, pc = _ptr(wgt, writable=True), _ptr(cnt, np.int64, writable=True)
    _check(ctx, lib().relsim_energy_spectrum(ctx, species, variable, nb, e.ctypes.data, pw[0], pc[0],
                                             _where(pw, pc)))
    return wgt, cnt


def relsim_field_modes(ctx, component, nmodes, device=False):
    """Energy in the Fourier modes m = 0 .. nmodes-1 (along x) of one
    component of B: (1/2) dV (c_m / nx) sum_j |DFT_x(B_c)(m, j)|^2."""
    out = _out((nmodes,), np.float64, device)
    po = _ptr(out, writable=True)
    _check(ctx, lib().relsim_field_modes(ctx, component, nmodes, po[0], po[1]))
    return out


def relsim_field_mode_gradient(ctx, component, mode, ncell, device=False):
    """(energy (1,), gB (3, ncell)): the energy of mode m of a B component
    and its gradient in B, computed on the device."""
    e = _out((1,), np.float64, device)
    g = _out((3, ncell), np.float64, device)
    pe, pg = _ptr(e, writable=True), _ptr(g, writable=True)
    _check(ctx, lib().relsim_field_mode_gradient(ctx, component, mode, pe[0], pg[0], pe[1]))
    return e, g


def relsim_dispersion_fit(modes, dt, first, window, Lx, a):
    """(rates, A, b): per-mode amplitude growth rates of an (nsamples, nmodes)
    array of mode energies over samples first .. first+window-1 (rates[0] and
    modes without a positive window are NaN), and the fit of
    A x b (1 - x^2 b^2), x = 2 pi m a / Lx, to them."""
    e = np.ascontiguousarray(modes, dtype=np.float64)
    if e.ndim != 2:
        raise ValueError("modes must be (nsamples, nmodes)")
    rates = np.empty(e.shape[1])
    A = ctypes.c_double()
    b = ctypes.c_double()
    code = lib().relsim_dispersion_fit(e.ctypes.data, e.shape[0], e.shape[1], float(dt), int(first), int(window),
                                       float(Lx), float(a), rates.ctypes.data, ctypes.byref(A), ctypes.byref(b))
    if code != RELSIM_OK:
        raise RelsimError(code, "dispersion fit: bad arguments or fewer than two growing modes")
    return rates, A.value, b.value


def relsim_growth_fit(s, dt, window):
    """(rate, first): the largest least-squares slope of log s over runs of
    `window` consecutive samples spaced dt, and the run's first index."""
    a = np.ascontiguousarray(s, dtype=np.float64)
    rate = ctypes.c_double()
    first = ctypes.c_int()
    code = lib().relsim_growth_fit(a.ctypes.data, a.size, float(dt), int(window), ctypes.byref(rate),
                                   ctypes.byref(first))
    if code != RELSIM_OK:
        raise RelsimError(code, "growth fit: bad arguments or no admissible window")
    return rate.value, first.value


def relsim_field_adjoint(ctx, ncell, gE1, gB1, mass=True, device=False, gEt=None):
    """Adjoint of the solved step's field part (particles fixed): returns
    {"E0", "B0", "J": (3, ncell), "M": (ncell, 5, 3, 3) or None, "iters",
    "relres", "status"} for upstream gradients gE1, gB1 of E^{n+1}, B^{n+1}
    and an optional further gradient gEt of E^{n+theta}."""
    p1, p2, p3 = _ptr(gE1), _ptr(gB1), _ptr(gEt)
    dev = _where(p1, p2, p3) == RELSIM_DEVICE
    outs = {k: _out((3, ncell), np.float64, dev) for k in ("E0", "B0", "J")}
    outs["M"] = _out((ncell, 5, 3, 3), np.float64, dev) if mass else None
    ptrs = {k: _ptr(v, writable=True) for k, v in outs.items() if v is not None}
    it = ctypes.c_int()
    rr = ctypes.c_double()
    code = _check(ctx, lib().relsim_field_adjoint(
        ctx, p1[0], p2[0], p3[0], ptrs["E0"][0], ptrs["B0"][0], ptrs["J"][0], ptrs["M"][0] if mass else None,
        ctypes.byref(it), ctypes.byref(rr), RELSIM_DEVICE if dev else RELSIM_HOST),
        allow=(RELSIM_ERR_NOT_CONVERGED,))
    outs.update(iters=it.value, relres=rr.value, status=code)
    return outs


def relsim_deposit_adjoint(ctx, species, ncell, gJ, gM):
    """Adjoint of one species' deposit: from dL/dJhat (3, ncell) and dL/dM
    (ncell, 5, 3, 3), returns {"u": (n, 3), "x": (n, 2), "w": (n,),
    "B": (3, ncell)}."""
    p1, p2 = _ptr(gJ), _ptr(gM)
    dev = _where(p1, p2) == RELSIM_DEVICE
    n = relsim_num_particles(ctx, species)
    outs = {"u": _out((n, 3), np.float64, dev), "x": _out((n, 2), np.float64, dev),
            "w": _out((n,), np.float64, dev), "B": _out((3, ncell), np.float64, dev)}
    pp = {k: _ptr(v, writable=True) for k, v in outs.items()}
    _check(ctx, lib().relsim_deposit_adjoint(ctx, species, p1[0], p2[0], pp["u"][0], pp["x"][0], pp["B"][0],
                                             pp["w"][0], RELSIM_DEVICE if dev else RELSIM_HOST))
    return outs


def relsim_push_adjoint(ctx, species, ncell, gu1, gx1, device=False):
    """Adjoint of one species' push with the fields fixed: from dL/du^{n+1}
    (n, 3) and dL/dx^{n+3/2} (n, 2) in the particles' current order, returns
    {"u": (n, 3), "x": (n, 2), "E": (3, ncell), "B": (3, ncell)}."""
    p1, p2 = _ptr(gu1), _ptr(gx1)
    dev = _where(p1, p2) == RELSIM_DEVICE
    n = relsim_num_particles(ctx, species)
    outs = {"u": _out((n, 3), np.float64, dev), "x": _out((n, 2), np.float64, dev),
            "E": _out((3, ncell), np.float64, dev), "B": _out((3, ncell), np.float64, dev)}
    pp = {k: _ptr(v, writable=True) for k, v in outs.items()}
    _check(ctx, lib().relsim_push_adjoint(ctx, species, p1[0], p2[0], pp["u"][0], pp["x"][0], pp["E"][0],
                                          pp["B"][0], RELSIM_DEVICE if dev else RELSIM_HOST))
    return outs


def relsim_step_adjoint(ctx, gE, gB, gu, gx, gw=None):
    """One whole step's adjoint in place on CUDA float64 tensors: gE, gB
    (3, ncell) and per species gu[s] (n_s, 3), gx[s] (n_s, 2) indexed by
    particle id; dL/d(state after the step) in, dL/d(state before) out.
    gw (optional, per species (n_s,) by id): the step's dL/dw is added.
    Returns (adjoint iters, relative residual, status)."""
    items = [_ptr(gE, writable=True), _ptr(gB, writable=True)]
    pu = [_ptr(a, writable=True) for a in gu]
    px = [_ptr(a, writable=True) for a in gx]
    pw = [_ptr(a, writable=True) for a in gw] if gw is not None else []
    if _where(*(items + pu + px + pw)) != RELSIM_DEVICE:
        raise ValueError("relsim_step_adjoint takes device arrays only")
    au = (ctypes.c_void_p * len(pu))(*[p[0] for p in pu])
    ax = (ctypes.c_void_p * len(px))(*[p[0] for p in px])
    aw = (ctypes.c_void_p * len(pw))(*[p[0] for p in pw]) if pw else None
    it = ctypes.c_int()
    rr = ctypes.c_double()
    code = _check(ctx, lib().relsim_step_adjoint(ctx, items[0][0], items[1][0], au, ax, aw, ctypes.byref(it),
                                                 ctypes.byref(rr)), allow=(RELSIM_ERR_NOT_CONVERGED,))
    return it.value, rr.value, code


def relsim_relabel_particles(ctx, species, ids):
    """Each particle of the species carrying id j gets ids[j] (int32, host
    array or CUDA tensor)."""
    p = _ptr(ids, np.int32)
    return _check(ctx, lib().relsim_relabel_particles(ctx, species, p[0], p[1]))


def relsim_set_launch_shapes(ctx, deposit_blocks=0, push_blocks=0, op_rows=0):
    """Apply launch shapes (as relsim_autotune chooses them): deposit blocks,
    push grid cap (0: defaults) and the 2D operator's tile rows."""
    return _check(ctx, lib().relsim_set_launch_shapes(ctx, int(deposit_blocks), int(push_blocks), int(op_rows)))


def relsim_autotune(ctx) -> dict:
    """Time candidate launch shapes of the deposit and the push on the loaded
    state and keep the fastest; returns the candidates and the choice."""
    t = relsim_tuning()
    _check(ctx, lib().relsim_autotune(ctx, ctypes.byref(t)))
    return t.asdict()


def relsim_graph_info(ctx) -> dict:
    """{"graph_steps": steps run as a CUDA graph, "disabled": capture failed,
    "why": the failure}."""
    n = ctypes.c_int64()
    d = ctypes.c_int()
    why = ctypes.c_char_p()
    _check(ctx, lib().relsim_graph_info(ctx, ctypes.byref(n), ctypes.byref(d), ctypes.byref(why)))
    return {"graph_steps": n.value, "disabled": bool(d.value), "why": (why.value or b"").decode()}


def relsim_batch_create(ctxs, nworkers):
    arr = (_CTX * len(ctxs))(*ctxs)
    b = _P()
    code = lib().relsim_batch_create(arr, len(ctxs), int(nworkers), ctypes.byref(b))
    if code != RELSIM_OK:
        raise RelsimError(code, "batch create: bad arguments")
    return b


def relsim_batch_run(b, count, nsteps, component=1, nmodes=0):
    """Advance every instance nsteps steps. Returns (modes[count, nsteps,
    nmodes] or None, status[count], iters[count, nsteps], code)."""
    modes = np.zeros((count, nsteps, nmodes)) if nmodes > 0 else None
    status = np.zeros(count, dtype=np.int32)
    iters = np.zeros((count, nsteps), dtype=np.int32)
    code = lib().relsim_batch_run(b, int(nsteps), int(component), int(nmodes),
                                  modes.ctypes.data if modes is not None else None, status.ctypes.data,
                                  iters.ctypes.data)
    return modes, status, iters, code


def relsim_batch_set_shared(b, on=True, groups=1, deposit_blocks=0, push_blocks=0):
    """Shared launches over the batch's instances (per group of instances,
    one deposit, push and re-sort launch per species) on or off."""
    code = lib().relsim_batch_set_shared(b, 1 if on else 0, int(groups), int(deposit_blocks), int(push_blocks))
    if code != RELSIM_OK:
        raise RelsimError(code, "batch set_shared: bad arguments")


def relsim_batch_last_path(b):
    """0 host-driven, 1 per-instance step graphs, 2 shared launches, -1 no run yet."""
    return int(lib().relsim_batch_last_path(b))


def relsim_batch_destroy(b):
    lib().relsim_batch_destroy(b)


def relsim_push(ctx):
    return _check(ctx, lib().relsim_push(ctx))


def relsim_energy_ledger(ctx) -> dict:
    e = relsim_energy()
    _check(ctx, lib().relsim_energy_ledger(ctx, ctypes.byref(e)))
    return e.asdict()


def relsim_step(ctx, ledger=True):
    """One full step; returns (ledger dict or None, status)."""
    e = relsim_energy()
    code = _check(ctx, lib().relsim_step(ctx, ctypes.byref(e) if ledger else None),
                  allow=(RELSIM_ERR_NOT_CONVERGED,))
    return (e.asdict() if ledger else None), code


def relsim_profile_enable(ctx, on=True):
    return _check(ctx, lib().relsim_profile_enable(ctx, 1 if on else 0))


def relsim_profile_read(ctx, reset=True) -> dict:
    """{slot name: (ms, timed groups, kernel launches)} since the last reset."""
    p = relsim_profile()
    _check(ctx, lib().relsim_profile_read(ctx, ctypes.byref(p), 1 if reset else 0))
    return {name: (p.ms[k], p.groups[k], p.kernels[k]) for k, name in enumerate(PROFILE_SLOTS)}


def relsim_kernel_launches() -> int:
    return int(lib().relsim_kernel_launches())


def relsim_kinetic_energy_noalloc(u, w, m, out, stream=None) -> int:
    """Allocation-free kinetic energy sum w m (gamma - 1) of device arrays
    u (n, 3) and w (n,) (CUDA float64 tensors) into out (a one-element CUDA
    float64 tensor). Returns the C status code unchanged (0 on success) so a
    caller can see TOO_LARGE; asynchronous on the stream."""
    pu, pw, po = _ptr(u), _ptr(w), _ptr(out, writable=True)
    if _where(pu, pw, po) != RELSIM_DEVICE:
        raise ValueError("relsim_kinetic_energy_noalloc takes device arrays only")
    n = int(w.shape[0]) if _is_torch(w) else int(np.shape(w)[0])
    return lib().relsim_kinetic_energy_noalloc(pu[0], pw[0], n, float(m), po[0], _P(_stream(stream)))


class Simulation:
    """Owns one relsim context; methods forward to the C entry points."""

    def __init__(self, cfg: relsim_config, stream=None):
        self.cfg = cfg
        self.ncell = cfg.nx * cfg.ny * (cfg.nz if cfg.dim == 3 else 1)
        self.ctx = relsim_init(cfg, stream)

    def close(self):
        if getattr(self, "ctx", None):
            relsim_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_species(self, s, x, u, w):
        return relsim_load_particles(self.ctx, s, x, u, w)

    def load_state(self, state: dict):
        """Load a state dict as produced by relsim_inputs (species + E + B);
        3D states carry z as well."""
        keys = ("x", "y", "z") if self.cfg.dim == 3 else ("x", "y")
        for s, sp in enumerate(state["species"]):
            x = np.stack([np.asarray(sp[k], np.float64) for k in keys], axis=1)
            u = np.stack([np.asarray(sp[k], np.float64) for k in ("ux", "uy", "uz")], axis=1)
            self.load_species(s, x, u, np.asarray(sp["w"], np.float64))
        relsim_set_fields(self.ctx, np.asarray(state["E"], np.float64), np.asarray(state["B"], np.float64))

    def set_fields(self, E=None, B=None):
        return relsim_set_fields(self.ctx, E, B)

    def fields(self, device=False):
        return relsim_get_fields(self.ctx, self.ncell, device)

    def particles(self, s, ids=False, device=False):
        return relsim_get_particles(self.ctx, s, ids, device, self.cfg.dim)

    def cell_start(self, s, device=False):
        return relsim_get_cell_start(self.ctx, s, self.ncell, device)

    def particles_native(self, s, ids=False, device=False):
        """(start, off, u, w[, id]) in the library's own form."""
        return relsim_get_particles_native(self.ctx, s, self.ncell, self.cfg.precision, ids, device,
                                           self.cfg.dim)

    def load_species_native(self, s, start, off, u, w, ids=None):
        return relsim_load_particles_native(self.ctx, s, start, off, u, w, ids, self.cfg.precision)

    def build(self):
        return relsim_build_mass_matrix(self.ctx)

    def mass_matrix(self, device=False):
        nhalf = 14 if self.cfg.dim == 3 else (13 if self.cfg.shape == 2 else 5)
        return relsim_get_mass_matrix(self.ctx, self.ncell, device, nhalf)

    def set_mass_matrix(self, M, J):
        return relsim_set_mass_matrix(self.ctx, M, J)

    def solve(self):
        return relsim_field_solve(self.ctx)

    def E_theta(self, device=False):
        return relsim_get_E_theta(self.ctx, self.ncell, device)

    def apply_operator(self, v):
        return relsim_apply_operator(self.ctx, v)

    def spectrum(self, s, edges, variable=0, device=False):
        return relsim_energy_spectrum(self.ctx, s, edges, variable, device)

    def push(self):
        return relsim_push(self.ctx)

    def ledger(self):
        return relsim_energy_ledger(self.ctx)

    def step(self, ledger=True):
        return relsim_step(self.ctx, ledger)

    def profile(self, on=True):
        return relsim_profile_enable(self.ctx, on)

    def profile_read(self, reset=True):
        return relsim_profile_read(self.ctx, reset)

    def graph_info(self):
        return relsim_graph_info(self.ctx)

    def autotune(self):
        return relsim_autotune(self.ctx)

    def set_launch_shapes(self, deposit_blocks=0, push_blocks=0, op_rows=0):
        return relsim_set_launch_shapes(self.ctx, deposit_blocks, push_blocks, op_rows)

    def push_adjoint(self, s, gu1, gx1, device=False):
        return relsim_push_adjoint(self.ctx, s, self.ncell, gu1, gx1, device)

    def field_adjoint(self, gE1, gB1, mass=True, device=False, gEt=None):
        return relsim_field_adjoint(self.ctx, self.ncell, gE1, gB1, mass, device, gEt)

    def step_adjoint(self, gE, gB, gu, gx, gw=None):
        return relsim_step_adjoint(self.ctx, gE, gB, gu, gx, gw)

    def relabel(self, s, ids):
        return relsim_relabel_particles(self.ctx, s, ids)

    def deposit_adjoint(self, s, gJ, gM):
        return relsim_deposit_adjoint(self.ctx, s, self.ncell, gJ, gM)

    def field_modes(self, component=1, nmodes=8, device=False):
        return relsim_field_modes(self.ctx, component, nmodes, device)

    def field_mode_gradient(self, component=1, mode=1, device=False):
        return relsim_field_mode_gradient(self.ctx, component, mode, self.ncell, device)


class Batch:
    """Independent Simulations advanced concurrently by `nworkers` host
    threads (each Simulation should have a CUDA stream of its own). The
    batch does not own the simulations."""

    def __init__(self, sims, nworkers=8, shared=False, groups=1, deposit_blocks=0, push_blocks=0):
        self.sims = list(sims)
        self.b = relsim_batch_create([s.ctx for s in self.sims], nworkers)
        if shared:
            relsim_batch_set_shared(self.b, True, groups, deposit_blocks, push_blocks)

    def set_shared(self, on=True, groups=1, deposit_blocks=0, push_blocks=0):
        relsim_batch_set_shared(self.b, on, groups, deposit_blocks, push_blocks)

    @property
    def last_path(self):
        """How the last run stepped: "host", "graphs", "shared" or None."""
        return {0: "host", 1: "graphs", 2: "shared"}.get(relsim_batch_last_path(self.b))

    def run(self, nsteps, component=1, nmodes=0):
        """Returns (modes[count, nsteps, nmodes] or None, status[count],
        iters[count, nsteps]); raises if an instance failed with anything
        but NOT_CONVERGED."""
        modes, status, iters, code = relsim_batch_run(self.b, len(self.sims), nsteps, component, nmodes)
        bad = [i for i, s in enumerate(status) if s not in (RELSIM_OK, RELSIM_ERR_NOT_CONVERGED)]
        if bad:
            i = bad[0]
            raise RelsimError(int(status[i]), f"instance {i}: " + relsim_last_error(self.sims[i].ctx))
        if code not in (RELSIM_OK, RELSIM_ERR_NOT_CONVERGED):
            raise RelsimError(code, "batch run failed")
        return modes, status, iters

    def close(self):
        if getattr(self, "b", None):
            relsim_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
