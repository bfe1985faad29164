"""Seeded synthetic inputs in 3D: the relativistic double Harris sheet of
Sec. 2 extended uniformly along z, and a generic random state for tests.

Like harris.py this only builds initial states; none of the method's
arithmetic lives here. The sheet is the 2D one (profile in y, B_x reversing
through both sheets, drifting Maxwell-Juettner members carrying J_z) made
uniform in z. Readings where the paper is silent (listed in the design
notes): the perturbation is a sum of B_y modes
  dB_y = pert B0 sum_{mx, mz = 1..4} a_{mx,mz} cos(2 pi (mx x/L_x + mz z/L_z) + phi_{mx,mz})
with seeded random amplitudes a (summing to 1) and phases phi, uniform in y,
so divergence free; cells hold exactly ppc particles per species at uniform
random positions, weight n(y) dx dy dz / ppc.
"""
from __future__ import annotations

import math
from dataclasses import asdict, dataclass

import numpy as np

from .harris import _rng, boost_flip, harris_derived, sample_maxwell_juettner, HarrisConfig

__all__ = ["HarrisConfig3", "make_harris3", "random_state3"]


@dataclass
class HarrisConfig3:
    """A 3D relativistic double Harris sheet in a periodic box."""

    nx: int = 32
    ny: int = 16
    nz: int = 16
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    ppc: int = 16
    theta_T: float = 0.3
    delta: float = 1.0
    sigma: float = 10.0
    pert: float = 0.01
    modes: int = 4           # x and z mode numbers 1..modes
    dt: float = 0.5
    theta: float = 0.5
    seed: int = 0
    q: tuple = (1.0, -1.0)
    m: tuple = (1.0, 1.0)

    def asdict(self) -> dict:
        return asdict(self)


def make_harris3(cfg: HarrisConfig3) -> dict:
    """species: list of dicts with x, y, z, ux, uy, uz, w (cell by cell, x
    fastest, then y, then z); E: (3, nn) zero; B: (3, nn) on cell centres."""
    d = harris_derived(HarrisConfig(nx=cfg.nx, ny=cfg.ny, dx=cfg.dx, dy=cfg.dy, theta_T=cfg.theta_T,
                                    delta=cfg.delta, sigma=cfg.sigma))
    nx, ny, nz, ppc = cfg.nx, cfg.ny, cfg.nz, cfg.ppc
    Lx, Ly, Lz = nx * cfg.dx, ny * cfg.dy, nz * cfg.dz
    a = cfg.delta
    nn = nx * ny * nz
    n = nn * ppc
    rpos = _rng(cfg.seed, 0xFF, 11)
    cell = np.repeat(np.arange(nn, dtype=np.int64), ppc)
    ci = cell % nx
    cj = (cell // nx) % ny
    ck = cell // (nx * ny)
    x = (ci + rpos.random(n)) * cfg.dx
    y = (cj + rpos.random(n)) * cfg.dy
    z = (ck + rpos.random(n)) * cfg.dz
    x = np.minimum(x, np.nextafter((ci + 1) * cfg.dx, -np.inf))
    y = np.minimum(y, np.nextafter((cj + 1) * cfg.dy, -np.inf))
    z = np.minimum(z, np.nextafter((ck + 1) * cfg.dz, -np.inf))
    n1 = (1.0 / np.cosh((y - 0.25 * Ly) / a)) ** 2
    n2 = (1.0 / np.cosh((y - 0.75 * Ly) / a)) ** 2
    ntot = n1 + n2 + d["n_b"]
    w = ntot * cfg.dx * cfg.dy * cfg.dz / ppc
    rmem = _rng(cfg.seed, 0xFF, 12).random(n)
    sheet = np.where(rmem < n1 / ntot, 1, np.where(rmem < (n1 + n2) / ntot, 2, 0))
    species = []
    for s, (q, m) in enumerate(zip(cfg.q, cfg.m)):
        r = _rng(cfg.seed, s, 13)
        u = sample_maxwell_juettner(r, cfg.theta_T, n)
        sgn_q = 1.0 if q > 0 else -1.0
        beta = np.where(sheet == 1, -sgn_q * d["beta_d"], np.where(sheet == 2, sgn_q * d["beta_d"], 0.0))
        u = boost_flip(r, u, beta)
        species.append({"x": x, "y": y, "z": z, "ux": u[0], "uy": u[1], "uz": u[2], "w": w,
                        "q": float(q), "m": float(m)})
    xc = (np.arange(nx) + 0.5) * cfg.dx
    yc = (np.arange(ny) + 0.5) * cfg.dy
    zc = (np.arange(nz) + 0.5) * cfg.dz
    Bx = d["B0"] * (np.tanh((yc - 0.25 * Ly) / a) - np.tanh((yc - 0.75 * Ly) / a) - 1.0)
    rp = _rng(cfg.seed, 0xFF, 14)
    amp = rp.random((cfg.modes, cfg.modes))
    amp /= amp.sum()
    phase = 2.0 * math.pi * rp.random((cfg.modes, cfg.modes))
    By = np.zeros((nz, nx))
    for mx in range(1, cfg.modes + 1):
        for mz in range(1, cfg.modes + 1):
            By += amp[mx - 1, mz - 1] * np.cos(2.0 * math.pi * (mx * xc[None, :] / Lx + mz * zc[:, None] / Lz)
                                               + phase[mx - 1, mz - 1])
    B = np.zeros((3, nz, ny, nx))
    B[0] = Bx[None, :, None]
    B[1] = cfg.pert * d["B0"] * By[:, None, :]
    return {"species": species, "E": np.zeros((3, nn)), "B": B.reshape(3, nn), "derived": d,
            "sheet": sheet, "config": cfg.asdict()}


def random_state3(nx: int, ny: int, nz: int, n_per_species, seed: int = 0, dx: float = 1.0, dy: float = 1.0,
                  dz: float = 1.0, u_scale: float = 1.0, field_scale: float = 0.5, q=(1.0, -1.0),
                  m=(1.0, 1.0)) -> dict:
    """Uniform positions, normal momenta, weights in [0.5, 1.5), random E on
    nodes and B on cell centres."""
    if np.isscalar(n_per_species):
        n_per_species = [int(n_per_species)] * len(q)
    L = (nx * dx, ny * dy, nz * dz)
    species = []
    for s, nps in enumerate(n_per_species):
        r = _rng(seed, s, 17)
        pos = [r.random(nps) * Lk for Lk in L]
        pos = [np.where(p >= Lk, 0.0, p) for p, Lk in zip(pos, L)]
        u = r.normal(0.0, u_scale, (3, nps))
        w = 0.5 + r.random(nps)
        species.append({"x": pos[0], "y": pos[1], "z": pos[2], "ux": u[0], "uy": u[1], "uz": u[2], "w": w,
                        "q": float(q[s]), "m": float(m[s])})
    rf = _rng(seed, 0xFE, 19)
    nn = nx * ny * nz
    return {"species": species, "E": field_scale * rf.normal(size=(3, nn)),
            "B": field_scale * rf.normal(size=(3, nn))}
