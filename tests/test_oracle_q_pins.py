"""Pins of the 2D FP64 oracle with quadratic (TSC) shapes (relsim_oracle_q.c)
against what the quadratic B-spline and the scheme fix, independently of
the oracle's code:

* the weights form a partition of unity and reproduce linear functions
  exactly (first moment), with the B-spline's second moment 1/4 cell^2, on
  the node and on the centre lattice;
* gathering a field that is linear in x and y (on nodes, and on centres)
  returns its value at the particle;
* the mass matrix and the predicted current on a 5x5 grid against a brute
  force double sum over all node pairs, with weights from the closed form of
  the quadratic B-spline of the periodic distance and alpha by a dense
  inverse; each block equals its mirror, M_{g,g+o} = M_{g+o,g};
* the discrete energy identity closes to the solve tolerance at theta = 0.5
  and 0.7 (the mass matrix is consistent with the push);
* a particle in a uniform B keeps |u| and turns by 2 atan(|a|) per step.
"""
import numpy as np
import pytest

import oracle
from oracle.quad import depositq, gather_Bq, gather_Eq, node_weightsq, offsetq, stepq
from relsim_inputs import random_state


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def test_weights_partition_and_moments():
    nx, ny = 9, 7
    c = oracle.make_config(nx, ny, dx=1.3, dy=0.7)
    rng = np.random.default_rng(1)
    for _ in range(200):
        x, y = rng.random() * nx * 1.3, rng.random() * ny * 0.7
        g, W = node_weightsq(c, x, y)
        assert abs(W.sum() - 1) < 1e-14
        gi, gj = g % nx, g // nx
        # unwrap node coordinates around the particle
        X = (gi * 1.3 - x + 0.5 * nx * 1.3) % (nx * 1.3) - 0.5 * nx * 1.3
        Y = (gj * 0.7 - y + 0.5 * ny * 0.7) % (ny * 0.7) - 0.5 * ny * 0.7
        assert abs(W @ X) < 1e-12 and abs(W @ Y) < 1e-12
        # second moment of the quadratic B-spline: 1/4 cell^2 per axis
        assert abs(W @ (X / 1.3) ** 2 - 0.25) < 1e-12
        assert abs(W @ (Y / 0.7) ** 2 - 0.25) < 1e-12


def test_gathers_reproduce_linear_fields():
    nx, ny = 12, 10
    c = oracle.make_config(nx, ny)
    # a field linear in x and y away from the periodic seam: test particles
    # in the interior, where the 3x3 support does not wrap
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    E = np.stack([0.3 + 0.2 * i + 0.1 * j, -0.5 * i + 0.4 * j, 1.0 + 0.0 * i]).reshape(3, -1).astype(float)
    B = np.stack([0.3 + 0.2 * (i + 0.5) + 0.1 * (j + 0.5), -0.5 * (i + 0.5) + 0.4 * (j + 0.5),
                  1.0 + 0.0 * i]).reshape(3, -1).astype(float)
    rng = np.random.default_rng(2)
    for _ in range(100):
        x, y = 2.5 + rng.random() * (nx - 5), 2.5 + rng.random() * (ny - 5)
        want = np.array([0.3 + 0.2 * x + 0.1 * y, -0.5 * x + 0.4 * y, 1.0])
        assert np.abs(gather_Eq(c, E, x, y) - want).max() < 1e-12
        assert np.abs(gather_Bq(c, B, x, y) - want).max() < 1e-12


def _b2(t):
    t = np.abs(t)
    return np.where(t <= 0.5, 0.75 - t * t, np.where(t <= 1.5, 0.5 * (1.5 - t) ** 2, 0.0))


def test_mass_matrix_against_a_brute_force_pair_sum():
    n = 5
    dx, dy, dt = 1.0, 0.8, 0.6
    q, m = (1.0, -2.0), (1.0, 3.0)
    st = random_state(n, n, [30, 25], seed=12, dx=dx, dy=dy, u_scale=1.0, field_scale=0.6, q=q, m=m)
    c = oracle.make_config(n, n, dx=dx, dy=dy, dt=dt, q=q, m=m)
    P = oracle.Particles(st["species"])
    J, M = depositq(c, P, st["B"])
    nn = n * n
    dV = dx * dy
    Mf = np.zeros((nn, nn, 3, 3))
    Jb = np.zeros((3, nn))
    Bf = st["B"].reshape(3, n, n)
    L = (n * dx, n * dy)
    for s, sp in enumerate(st["species"]):
        beta = q[s] * dt / (2 * m[s])
        for p in range(len(sp["w"])):
            px, py = sp["x"][p], sp["y"][p]
            dxn = ((np.arange(n) * dx - px) + 0.5 * L[0]) % L[0] - 0.5 * L[0]
            dyn = ((np.arange(n) * dy - py) + 0.5 * L[1]) % L[1] - 0.5 * L[1]
            W = (_b2(dyn / dy)[:, None] * _b2(dxn / dx)[None, :]).ravel()
            dxc = (((np.arange(n) + 0.5) * dx - px) + 0.5 * L[0]) % L[0] - 0.5 * L[0]
            dyc = (((np.arange(n) + 0.5) * dy - py) + 0.5 * L[1]) % L[1] - 0.5 * L[1]
            Bp = np.einsum("cji,j,i->c", Bf, _b2(dyc / dy), _b2(dxc / dx))
            u = np.array([sp["ux"][p], sp["uy"][p], sp["uz"][p]])
            g = np.sqrt(1 + u @ u)
            a = beta * Bp / g
            ax = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
            al = np.linalg.inv(np.eye(3) + ax)
            Mf += sp["w"][p] * q[s] * beta / (g * dV) * W[:, None, None, None] * W[None, :, None, None] * al
            Jb += sp["w"][p] * q[s] / dV * (al @ u / g)[:, None] * W[None, :]
    assert rel(J, Jb) < 1e-13
    Mo = np.zeros((nn, nn, 3, 3))
    for gg in range(nn):
        i, j = gg % n, gg // n
        for dj in range(-2, 3):
            for di in range(-2, 3):
                h = ((j + dj) % n) * n + (i + di) % n
                Mo[gg, h] += M[gg, offsetq(di, dj)]
                # the mirror block is the same block (to the rounding of the
                # product order of the two weights)
                hi, hj = (i + di) % n, (j + dj) % n
                mb = M[hj * n + hi, offsetq(-di, -dj)]
                assert np.abs(M[gg, offsetq(di, dj)] - mb).max() <= 1e-15 * max(np.abs(mb).max(), 1e-300)
    assert rel(Mo, Mf) < 1e-13


@pytest.mark.parametrize("theta", [0.5, 0.7])
def test_energy_identity_closes(theta):
    st = random_state(7, 6, [180, 150], seed=13, u_scale=1.2, field_scale=0.5)
    c = oracle.make_config(7, 6, dt=0.8, theta=theta, gmres_tol=1e-13, gmres_restart=200)
    P = oracle.Particles(st["species"])
    E, B, L, _ = stepq(c, P, st["E"], st["B"])
    total = L["W_E1"] + L["W_B1"] + L["K1"]
    assert abs(L["residual"]) < 1e-10 * total
    assert abs(L["work_grid"] - L["work_particles"]) < 1e-10 * abs(L["work_grid"])


def test_single_particle_gyration():
    n = 6
    B0 = 0.7
    c = oracle.make_config(n, n, dt=0.3, q=(1.0,), m=(1.0,), gmres_tol=1e-14)
    u0 = np.array([1.2, -0.4, 0.0])
    sp = {"x": np.array([2.3]), "y": np.array([3.1]), "ux": u0[:1], "uy": u0[1:2], "uz": u0[2:],
          "w": np.array([1e-12])}
    P = oracle.Particles([sp])
    E = np.zeros((3, n * n))
    B = np.zeros((3, n * n))
    B[2] = B0
    g = np.sqrt(1 + u0 @ u0)
    phi = 2 * np.arctan(0.5 * c.dt * B0 / g)
    up = u0.copy()
    for _ in range(5):
        E, B, L, _ = stepq(c, P, E, B)
        u = np.array([P.ux[0], P.uy[0], P.uz[0]])
        assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-9
        ang = np.arccos(np.clip(up @ u / (np.linalg.norm(up) * np.linalg.norm(u)), -1, 1))
        assert abs(ang - phi) < 1e-8
        up = u
