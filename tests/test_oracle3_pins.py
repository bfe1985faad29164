"""Pins of the 3D FP64 oracle (relsim_oracle3.c) against what the scheme and
the mathematics fix, independently of the oracle's own code:

* nz = 1 reduces the 3D scheme to the 2D one (the z derivatives vanish and
  the z weights add to one): one 3D step equals one step of the separately
  pinned 2D oracle, fields, particles and every ledger term;
* a cyclic permutation of the axes (x, y, z) -> (z, x, y) is a proper
  rotation, under which the scheme is equivariant: rotating the input state
  rotates the step's output (on a grid with three different sizes, so a
  mixed-up stride or cell size shows);
* the mass matrix and the predicted current on a 3x3x3 grid against a brute
  force double sum over all node pairs, with trilinear weights from
  periodic distances and alpha = (I + [a]x)^{-1} by a dense inverse;
* curl_n is the transpose of curl_c (discrete integration by parts, what
  makes the field energy balance close);
* the discrete energy identity closes to the solve tolerance at theta = 0.5
  and 0.7;
* a single particle in a uniform B (any direction) keeps |u| to rounding
  and turns by 2 atan(|a|) per step, |a| = beta |B| / gamma.
"""
import numpy as np
import pytest

import oracle
from oracle.three import (Particles3, apply_A3, curl_c3, curl_n3, deposit3, make_config3, offset3, step3)
from relsim_inputs import random_state3

pytestmark = pytest.mark.filterwarnings("ignore")


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def test_nz1_reduces_to_the_2d_scheme():
    nx, ny = 7, 5
    st = random_state3(nx, ny, 1, [180, 150], seed=3, u_scale=0.8, field_scale=0.4)
    c3 = make_config3(nx, ny, 1, dt=0.6, theta=0.6, gmres_tol=1e-14, gmres_restart=200)
    c2 = oracle.make_config(nx, ny, dt=0.6, theta=0.6, gmres_tol=1e-14, gmres_restart=200)
    P3 = Particles3(st["species"])
    P2 = oracle.Particles([{k: sp[k] for k in ("x", "y", "ux", "uy", "uz", "w")} for sp in st["species"]])
    E3, B3, L3, _ = step3(c3, P3, st["E"], st["B"])
    E2, B2, L2, _ = oracle.step(c2, P2, st["E"], st["B"])
    assert rel(E3, E2) < 1e-11 and rel(B3, B2) < 1e-11
    for k2, k3 in (("x", "x"), ("y", "y"), ("ux", "ux"), ("uy", "uy"), ("uz", "uz")):
        assert rel(getattr(P3, k3), getattr(P2, k2)) < 1e-11
    for k in ("W_E1", "W_B1", "K1", "work_grid", "work_particles", "mismatch", "dissipation"):
        assert abs(L3[k] - L2[k]) <= 1e-10 * max(abs(L2[k]), L2["K1"] * 1e-6)


def _rotate_field(F, nx, ny, nz):
    """(x, y, z) -> (z, x, y): node (i, j, k) goes to (k, i, j) on the grid
    (nz, nx, ny), vector components (Fx, Fy, Fz) -> (Fz, Fx, Fy)."""
    F = np.asarray(F).reshape(3, nz, ny, nx)   # [comp][k][j][i]
    # new array indexed [comp'][k'=j][j'=i][i'=k]
    G = np.transpose(F, (0, 2, 3, 1))           # [comp][j][i][k]
    return G[[2, 0, 1]].reshape(3, -1)


def test_step_is_equivariant_under_a_cyclic_axis_permutation():
    nx, ny, nz = 5, 4, 3
    dx, dy, dz = 1.0, 0.8, 1.3
    st = random_state3(nx, ny, nz, [250, 200], seed=5, dx=dx, dy=dy, dz=dz, u_scale=0.9, field_scale=0.4)
    c = make_config3(nx, ny, nz, dx=dx, dy=dy, dz=dz, dt=0.5, theta=0.5, gmres_tol=1e-14, gmres_restart=300)
    cr = make_config3(nz, nx, ny, dx=dz, dy=dx, dz=dy, dt=0.5, theta=0.5, gmres_tol=1e-14, gmres_restart=300)
    P = Particles3(st["species"])
    rot_species = [{"x": sp["z"], "y": sp["x"], "z": sp["y"], "ux": sp["uz"], "uy": sp["ux"], "uz": sp["uy"],
                    "w": sp["w"]} for sp in st["species"]]
    Pr = Particles3(rot_species)
    E, B, L, _ = step3(c, P, st["E"], st["B"])
    Er, Br, Lr, _ = step3(cr, Pr, _rotate_field(st["E"], nx, ny, nz), _rotate_field(st["B"], nx, ny, nz))
    assert rel(Er, _rotate_field(E, nx, ny, nz)) < 1e-11
    assert rel(Br, _rotate_field(B, nx, ny, nz)) < 1e-11
    assert rel(Pr.x, P.z) < 1e-12 and rel(Pr.y, P.x) < 1e-12 and rel(Pr.z, P.y) < 1e-12
    assert rel(Pr.ux, P.uz) < 1e-11 and rel(Pr.uy, P.ux) < 1e-11 and rel(Pr.uz, P.uy) < 1e-11
    for k in ("W_E1", "W_B1", "K1", "mismatch"):
        assert abs(Lr[k] - L[k]) <= 1e-10 * abs(L[k]) + 1e-15


def _tri(s, L, n, d):
    """Trilinear node weights along one axis by periodic distance."""
    g = np.arange(n) * d
    dist = np.abs(((s - g) + 0.5 * L) % L - 0.5 * L)
    return np.maximum(0.0, 1.0 - dist / d)


def test_mass_matrix_against_a_brute_force_pair_sum():
    n = 3
    dx, dy, dz = 1.0, 0.9, 1.1
    st = random_state3(n, n, n, [40, 30], seed=8, dx=dx, dy=dy, dz=dz, u_scale=1.0, field_scale=0.6,
                       q=(1.0, -2.0), m=(1.0, 3.0))
    dt = 0.7
    c = make_config3(n, n, n, dx=dx, dy=dy, dz=dz, dt=dt, q=(1.0, -2.0), m=(1.0, 3.0))
    P = Particles3(st["species"])
    J, M = deposit3(c, P, st["B"])
    nn = n ** 3
    dV = dx * dy * dz
    Mfull = np.zeros((nn, nn, 3, 3))
    Jb = np.zeros((3, nn))
    Bf = st["B"].reshape(3, n, n, n)   # [comp][k][j][i]
    for s, sp in enumerate(st["species"]):
        q, m = (1.0, -2.0)[s], (1.0, 3.0)[s]
        beta = q * dt / (2 * m)
        for p in range(len(sp["w"])):
            wx = _tri(sp["x"][p], n * dx, n, dx)
            wy = _tri(sp["y"][p], n * dy, n, dy)
            wz = _tri(sp["z"][p], n * dz, n, dz)
            W = (wz[:, None, None] * wy[None, :, None] * wx[None, None, :]).ravel()
            # B at the particle: trilinear on the centre lattice (shifted by half a cell)
            cx = _tri(sp["x"][p] - 0.5 * dx, n * dx, n, dx)
            cy = _tri(sp["y"][p] - 0.5 * dy, n * dy, n, dy)
            cz = _tri(sp["z"][p] - 0.5 * dz, n * dz, n, dz)
            Bp = np.einsum("ckji,k,j,i->c", Bf, cz, cy, cx)
            u = np.array([sp["ux"][p], sp["uy"][p], sp["uz"][p]])
            g = np.sqrt(1 + u @ u)
            a = beta * Bp / g
            ax = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
            al = np.linalg.inv(np.eye(3) + ax)
            Mfull += sp["w"][p] * q * beta / (g * dV) * W[:, None, None, None] * W[None, :, None, None] * al
            Jb += sp["w"][p] * q / dV * (al @ u / g)[:, None] * W[None, :]
    assert rel(J, Jb) < 1e-13
    Mo = np.zeros((nn, nn, 3, 3))
    for g in range(nn):
        i, j, k = g % n, (g // n) % n, g // (n * n)
        for dk in (-1, 0, 1):
            for dj in (-1, 0, 1):
                for di in (-1, 0, 1):
                    h = ((k + dk) % n * n + (j + dj) % n) * n + (i + di) % n
                    Mo[g, h] += M[g, offset3(di, dj, dk)]
    assert rel(Mo, Mfull) < 1e-13


def test_curl_n_is_the_transpose_of_curl_c():
    nx, ny, nz = 4, 5, 3
    c = make_config3(nx, ny, nz, dx=1.2, dy=0.7, dz=0.9)
    rng = np.random.default_rng(4)
    E = rng.normal(size=(3, nx * ny * nz))
    B = rng.normal(size=(3, nx * ny * nz))
    assert abs(np.sum(curl_c3(c, E) * B) - np.sum(E * curl_n3(c, B))) < 1e-12 * np.abs(E).sum()
    # and curl_c of a gradient-free uniform field vanishes
    assert np.abs(curl_c3(c, np.ones((3, nx * ny * nz)))).max() < 1e-14


@pytest.mark.parametrize("theta", [0.5, 0.7])
def test_energy_identity_closes(theta):
    nx, ny, nz = 4, 3, 3
    st = random_state3(nx, ny, nz, [150, 120], seed=9, u_scale=1.2, field_scale=0.5)
    c = make_config3(nx, ny, nz, dt=0.8, theta=theta, gmres_tol=1e-13, gmres_restart=300)
    P = Particles3(st["species"])
    E, B, L, _ = step3(c, P, st["E"], st["B"])
    total = L["W_E1"] + L["W_B1"] + L["K1"]
    assert abs(L["residual"]) < 1e-10 * total
    # the field-side and particle-side work agree (the mass matrix is exact)
    assert abs(L["work_grid"] - L["work_particles"]) < 1e-10 * abs(L["work_grid"])
    if theta > 0.5:
        assert L["dissipation"] > 0


@pytest.mark.parametrize("bdir", [(0.0, 0.0, 1.0), (1.0, 0.0, 0.0), (0.3, -0.5, 0.8)])
def test_single_particle_gyration(bdir):
    n = 4
    b = np.array(bdir) / np.linalg.norm(bdir)
    B0 = 0.7
    c = make_config3(n, n, n, dt=0.3, q=(1.0,), m=(1.0,), gmres_tol=1e-14)
    u0 = np.cross(b, [0.2, 0.9, -0.4])
    u0 = 1.5 * u0 / np.linalg.norm(u0)           # perpendicular to B
    sp = {"x": np.array([1.3]), "y": np.array([2.2]), "z": np.array([0.7]),
          "ux": np.array([u0[0]]), "uy": np.array([u0[1]]), "uz": np.array([u0[2]]), "w": np.array([1e-12])}
    P = Particles3([sp])
    nn = n ** 3
    E = np.zeros((3, nn))
    B = np.tile((B0 * b)[:, None], (1, nn))
    g = np.sqrt(1 + u0 @ u0)
    a = 0.5 * c.dt * B0 / g
    phi = 2 * np.arctan(a)
    u_prev = u0.copy()
    for _ in range(5):
        E, B, L, _ = step3(c, P, E, B)
        u = np.array([P.ux[0], P.uy[0], P.uz[0]])
        assert abs(np.linalg.norm(u) - 1.5) < 1e-9
        # the turn angle about -b (a positive charge gyrates clockwise about B)
        cosang = u_prev @ u / (np.linalg.norm(u_prev) * np.linalg.norm(u))
        assert abs(np.arccos(np.clip(cosang, -1, 1)) - phi) < 1e-8
        assert np.cross(u_prev, u) @ b < 0
        u_prev = u
