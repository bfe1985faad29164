"""Seeded synthetic inputs: the relativistic double Harris sheet of Sec. 2.

This module only *builds* initial states (particle positions, momenta, weights
and the initial E/B fields). It contains none of the semi-implicit method's
arithmetic (no shape-function deposit, no rotation matrix, no field solve, no
push), so both the CPU oracle and the CUDA library can be fed from it.

Units are rationalised (Heaviside-Lorentz) with c = 1, m_e = 1, |q| = 1, the
sheet-centre density n0 = 1 and omega_pe0 = 1, so the n0-based skin depth
d_0e = 1. In these units the Gaussian formulas of Sec. 2 become:

* density profile, Eq. 3:  n(y) = n0 sech^2((y - y_s)/a) + n_b   (per species)
* force balance, Eq. 5:    B0^2 = 2 (2 n0) T / Gamma_d = 4 theta_T / Gamma_d
* Ampere, Eq. 6:           a = B0 / (2 n0 e v_d)

Combining Eqs. 5 and 6 for a given half-thickness a fixes the drift:
Gamma_d beta_d^2 = theta_T / a^2.

Readings taken where the paper is silent or garbled (they are listed in the
design notes of this repository):

* B_x on the periodic domain [0, L_y) with sheets at L_y/4 and 3L_y/4 is
  B_x = B0 [tanh((y - L_y/4)/a) - tanh((y - 3L_y/4)/a) - 1]  (Eq. 4 as printed
  has a sign garble that would give 3 B0 between the sheets).
* sigma is measured against the background density: n_b = B0^2 / (sigma m).
* "ppc per species": every cell gets exactly ppc particles per species at
  uniform random positions; each particle is a sheet member with probability
  n_sheet(y)/n(y) and carries the weight w = n(y) dx dy / ppc. Electrons and
  positrons are co-located (zero initial charge density).
* Sheet members are drifting Maxwell-Juettner: the rest-frame speed is drawn
  by exact rejection (an energy-space Gamma-mixture envelope when cold,
  Sobol's method when hot) and the boost uses Zenitani's flipping method
  (Zenitani 2015, "Loading relativistic Maxwell distributions in particle
  simulations"), all written here from the mathematics.
* The initial perturbation is dB_y = pert * B0 * cos(2 pi m x / L_x) at cell
  centres (divergence free, uniform in y), m = pert_mode (1 by default).
* loader = "weighted" is a second loading of the same equilibrium whose
  particles are smooth functions of the parameters for fixed random numbers
  (for gradients in delta, theta_T, ... by central differences): each cell's
  ppc particles take fixed roles by their index in the cell (k mod 3:
  background, sheet 1, sheet 2), a role's weight is its density n_role(y) dx
  dy over the role's count in the cell, and the drifting members are boosted
  without the flip, their weight multiplied by 1 + beta v'_z instead (the
  rest-frame draw has density f'(u'); the drifting Maxwell-Juettner law is
  (gamma/gamma') f'(u') = Gamma (1 + beta v'_z) f'(u'), and the mean of
  1 + beta v'_z over the isotropic rest frame is 1, so the lab density stays
  n_role). No discrete choice depends on a parameter.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

__all__ = [
    "HarrisConfig",
    "harris_derived",
    "make_harris",
    "random_state",
    "sample_maxwell_juettner",
    "boost_flip",
    "boost_weighted",
]


@dataclass
class HarrisConfig:
    """A 2D relativistic double Harris sheet in a periodic box (Sec. 2)."""

    nx: int = 64
    ny: int = 32
    dx: float = 1.0
    dy: float = 1.0
    ppc: int = 16            # particles per cell per species
    theta_T: float = 0.3     # temperature kT/(m c^2), both species
    delta: float = 1.0       # sheet half-thickness a, in d_0e
    sigma: float = 10.0      # B0^2 / (n_b m c^2): background magnetization
    pert: float = 0.01       # dB_y / B0, single cosine mode in x
    pert_mode: int = 1       # its mode number m: k_x = 2 pi m / L_x
    loader: str = "sampled"  # "sampled" (sheet membership drawn, flip boost) or "weighted"
    dt: float = 0.5          # time step, in 1/omega_pe0
    theta: float = 0.5       # implicitness parameter of the field solve
    seed: int = 0
    q: tuple = (1.0, -1.0)   # positrons, electrons
    m: tuple = (1.0, 1.0)

    def asdict(self) -> dict:
        return asdict(self)


def harris_derived(cfg: HarrisConfig) -> dict:
    """Drift, field amplitude and background density fixed by Eqs. 5 and 6."""
    s = cfg.theta_T / cfg.delta ** 2          # Gamma_d beta_d^2 = s
    beta2 = 0.5 * (-s * s + math.sqrt(s ** 4 + 4.0 * s * s))
    beta_d = math.sqrt(beta2)
    gamma_d = 1.0 / math.sqrt(1.0 - beta2)
    u_d = gamma_d * beta_d
    B0 = math.sqrt(4.0 * cfg.theta_T / gamma_d)
    n_b = B0 * B0 / cfg.sigma
    return {
        "beta_d": beta_d,
        "Gamma_d": gamma_d,
        "u_d": u_d,
        "B0": B0,
        "n_b": n_b,
        "sigma_n0": B0 * B0,
        "Lx": cfg.nx * cfg.dx,
        "Ly": cfg.ny * cfg.dy,
    }


def _rng(seed: int, species: int, purpose: int) -> np.random.Generator:
    # Philox counter-based generator keyed by (seed, species, purpose).
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, (species << 32) | purpose], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def _mj_speed_sobol(rng, theta_T, n):
    # Sobol's rejection method: u ~ Gamma(3, theta) (sum of three
    # exponentials), eta = u + Exp(theta), accept when eta^2 - u^2 > 1; the
    # accepted density is u^2 exp(-sqrt(1+u^2)/theta). Efficient when hot.
    out = np.empty(n)
    filled = 0
    while filled < n:
        want = n - filled
        m = max(int(want * 5.0) + 64, 1024)
        X = 1.0 - rng.random((4, m))          # uniform on (0, 1]
        l3 = np.log(X[0] * X[1] * X[2])
        u = -theta_T * l3
        eta = -theta_T * (l3 + np.log(X[3]))
        acc = u[eta * eta - u * u > 1.0]
        take = min(acc.size, want)
        out[filled:filled + take] = acc[:take]
        filled += take
    return out


def _mj_speed_energy_mixture(rng, theta_T, n):
    # Rejection in the kinetic energy e = gamma - 1, whose density is
    # sqrt(e (e+2)) (1+e) exp(-e/theta). Since sqrt(e+2) <= sqrt(2) (1+e)^(1/2)
    # <= sqrt(2) (1+e), the envelope sqrt(2) e^(1/2) (1 + 2e + e^2) exp(-e/theta)
    # is a mixture of Gamma(3/2), Gamma(5/2), Gamma(7/2) (scale theta) with
    # weights proportional to Gamma(k) theta^k * (1, 2, 1); a draw is accepted
    # with probability sqrt((e+2)/2)/(1+e). Efficient when cold.
    from math import gamma as G
    shapes = np.array([1.5, 2.5, 3.5])
    wts = np.array([G(1.5) * theta_T ** 1.5, 2 * G(2.5) * theta_T ** 2.5,
                    G(3.5) * theta_T ** 3.5])
    wts = wts / wts.sum()
    out = np.empty(n)
    filled = 0
    while filled < n:
        want = n - filled
        m = max(int(want * 1.6) + 64, 1024)
        comp = rng.choice(3, size=m, p=wts)
        e = rng.gamma(shapes[comp], theta_T)
        acc = rng.random(m) < np.sqrt(0.5 * (e + 2.0)) / (1.0 + e)
        e = e[acc]
        take = min(e.size, want)
        out[filled:filled + take] = np.sqrt(e[:take] * (e[:take] + 2.0))
        filled += take
    return out


def sample_maxwell_juettner(rng: np.random.Generator, theta_T: float, n: int) -> np.ndarray:
    """Isotropic Maxwell-Juettner momenta u = gamma v, shape (3, n).

    The speed follows f(u) ~ u^2 exp(-sqrt(1+u^2)/theta_T), drawn exactly by
    one of two rejection samplers (cold: an energy-space Gamma-mixture
    envelope; hot, theta_T > 1: Sobol's method). Direction: uniform on the
    sphere.
    """
    if theta_T > 1.0:
        out = _mj_speed_sobol(rng, theta_T, n)
    else:
        out = _mj_speed_energy_mixture(rng, theta_T, n)
    mu = 2.0 * rng.random(n) - 1.0            # cos(polar angle)
    phi = 2.0 * math.pi * rng.random(n)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return np.stack([out * st * np.cos(phi), out * st * np.sin(phi), out * mu])


def boost_flip(rng: np.random.Generator, u: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Boost rest-frame momenta along z by a per-particle signed speed beta.

    Zenitani's flipping method: u_z is mirrored with probability
    max(0, -beta v_z), which turns the rest-frame distribution into one
    weighted by (1 + beta v_z), then u_z' = Gamma (u_z + beta gamma).
    Particles with beta = 0 are returned unchanged.
    """
    u = u.copy()
    g = np.sqrt(1.0 + (u * u).sum(axis=0))
    vz = u[2] / g
    flip = (-beta * vz) > rng.random(u.shape[1])
    u[2] = np.where(flip, -u[2], u[2])
    G = 1.0 / np.sqrt(1.0 - beta * beta)
    u[2] = G * (u[2] + beta * g)
    return u


def boost_weighted(u: np.ndarray, beta: np.ndarray, w: np.ndarray):
    """Boost rest-frame momenta along z by beta without flipping: u_z' =
    Gamma (u_z + beta gamma), the weight multiplied by 1 + beta v_z (the
    factor the flip method realises by mirroring). Returns (u', w')."""
    u = u.copy()
    g = np.sqrt(1.0 + (u * u).sum(axis=0))
    vz = u[2] / g
    G = 1.0 / np.sqrt(1.0 - beta * beta)
    u[2] = G * (u[2] + beta * g)
    return u, w * (1.0 + beta * vz)


def make_harris(cfg: HarrisConfig, dtype=np.float64) -> dict:
    """Build the seeded initial state of the double Harris sheet.

    Returns a dict with
      ``species``: list of dicts (one per species) with x, y (absolute
      positions in [0, L)), ux, uy, uz, w (all float64 arrays, particles
      ordered cell by cell, x fastest), q and m;
      ``E``: (3, ny*nx) node field, zero;
      ``B``: (3, ny*nx) cell-centre field (equilibrium + perturbation);
      ``derived``: the values fixed by Eqs. 5-6 and the readings above.
    """
    d = harris_derived(cfg)
    nx, ny, ppc = cfg.nx, cfg.ny, cfg.ppc
    Lx, Ly = d["Lx"], d["Ly"]
    a = cfg.delta
    ncell = nx * ny
    n = ncell * ppc

    # positions: ppc uniform random points per cell, shared by both species
    rpos = _rng(cfg.seed, 0xFF, 1)
    cell = np.repeat(np.arange(ncell, dtype=np.int64), ppc)
    ci = cell % nx
    cj = cell // nx
    x = (ci + rpos.random(n)) * cfg.dx
    y = (cj + rpos.random(n)) * cfg.dy
    # guard the half-open interval against rounding up to the upper cell edge
    x = np.minimum(x, np.nextafter((ci + 1) * cfg.dx, -np.inf))
    y = np.minimum(y, np.nextafter((cj + 1) * cfg.dy, -np.inf))

    n1 = (1.0 / np.cosh((y - 0.25 * Ly) / a)) ** 2   # sech^2, no overflow far out
    n2 = (1.0 / np.cosh((y - 0.75 * Ly) / a)) ** 2
    ntot = n1 + n2 + d["n_b"]
    if cfg.loader == "sampled":
        w = ntot * cfg.dx * cfg.dy / ppc
        rmem = _rng(cfg.seed, 0xFF, 2).random(n)
        sheet = np.where(rmem < n1 / ntot, 1, np.where(rmem < (n1 + n2) / ntot, 2, 0))
    elif cfg.loader == "weighted":
        if ppc < 3:
            raise ValueError("the weighted loader needs ppc >= 3 (one particle per role)")
        sheet = np.tile(np.arange(ppc) % 3, ncell)
        count = np.array([(np.arange(ppc) % 3 == r).sum() for r in range(3)])
        dens = np.where(sheet == 1, n1, np.where(sheet == 2, n2, d["n_b"]))
        w = dens * cfg.dx * cfg.dy / count[sheet]
    else:
        raise ValueError(f"unknown loader {cfg.loader!r}")

    species = []
    for s, (q, m) in enumerate(zip(cfg.q, cfg.m)):
        r = _rng(cfg.seed, s, 3)
        u = sample_maxwell_juettner(r, cfg.theta_T, n)
        # sheet 1 carries J_z < 0, sheet 2 J_z > 0 (B_x reverses through both)
        sgn_q = 1.0 if q > 0 else -1.0
        beta = np.where(sheet == 1, -sgn_q * d["beta_d"],
                        np.where(sheet == 2, sgn_q * d["beta_d"], 0.0))
        if cfg.loader == "sampled":
            u = boost_flip(r, u, beta)
            ws = w
        else:
            u, ws = boost_weighted(u, beta, w)
        species.append({
            "x": x.astype(dtype), "y": y.astype(dtype),
            "ux": u[0].astype(dtype), "uy": u[1].astype(dtype), "uz": u[2].astype(dtype),
            "w": ws.astype(dtype), "q": float(q), "m": float(m),
        })

    # fields: E = 0 on nodes; B on cell centres
    xc = (np.arange(nx) + 0.5) * cfg.dx
    yc = (np.arange(ny) + 0.5) * cfg.dy
    Bx = d["B0"] * (np.tanh((yc - 0.25 * Ly) / a) - np.tanh((yc - 0.75 * Ly) / a) - 1.0)
    By = cfg.pert * d["B0"] * np.cos(2.0 * math.pi * cfg.pert_mode * xc / Lx)
    B = np.zeros((3, ny, nx))
    B[0] = Bx[:, None]
    B[1] = By[None, :]
    E = np.zeros((3, ncell))
    return {
        "species": species,
        "E": E.astype(dtype),
        "B": B.reshape(3, ncell).astype(dtype),
        "derived": d,
        "sheet": sheet,
        "config": cfg.asdict(),
    }


def random_state(nx: int, ny: int, n_per_species, seed: int = 0, dx: float = 1.0,
                 dy: float = 1.0, u_scale: float = 1.0, field_scale: float = 0.5,
                 q=(1.0, -1.0), m=(1.0, 1.0)) -> dict:
    """Generic seeded state for unit tests: uniform positions, normal momenta,
    weights in [0.5, 1.5), random E on nodes and B on cell centres."""
    if np.isscalar(n_per_species):
        n_per_species = [int(n_per_species)] * len(q)
    Lx, Ly = nx * dx, ny * dy
    species = []
    for s, nps in enumerate(n_per_species):
        r = _rng(seed, s, 7)
        x = r.random(nps) * Lx
        y = r.random(nps) * Ly
        x = np.where(x >= Lx, 0.0, x)
        y = np.where(y >= Ly, 0.0, y)
        u = r.normal(0.0, u_scale, (3, nps))
        w = 0.5 + r.random(nps)
        species.append({"x": x, "y": y, "ux": u[0], "uy": u[1], "uz": u[2], "w": w,
                        "q": float(q[s]), "m": float(m[s])})
    rf = _rng(seed, 0xFE, 9)
    E = field_scale * rf.normal(size=(3, nx * ny))
    B = field_scale * rf.normal(size=(3, nx * ny))
    return {"species": species, "E": E, "B": B}
