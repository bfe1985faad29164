"""The 2D step with quadratic (TSC) shapes on the GPU against the FP64
oracle with the same shapes (relsim_oracle_q.c): deposit (Jhat and the 13
stored mass-matrix offsets against the oracle's 25), the operator with the
GPU's own mass matrix, one full step (fields, particles matched by id,
ledger terms), three FP64 steps with the energy identity, and the calls that
cover only the linear shape.

Tolerances relative to the largest entry: FP64 form 1e-11 (deposit,
operator), 1e-9 after a step; FP32 form 2e-6 (deposit), 1e-5 (operator),
2e-5 (fields and momenta after a step).
"""
import numpy as np
import pytest

from relsim_inputs import HarrisConfig, make_harris, random_state

pytestmark = pytest.mark.gpu

HALFQ = [(0, 0), (1, 0), (2, 0)] + [(di, 1) for di in range(-2, 3)] + [(di, 2) for di in range(-2, 3)]


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    return rs


@pytest.fixture(scope="module")
def oq():
    from oracle import quad
    quad.load()
    return quad


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def f32(st):
    for sp in st["species"]:
        for k in ("x", "y", "ux", "uy", "uz", "w"):
            sp[k] = np.asarray(sp[k]).astype(np.float32).astype(np.float64)
    st["E"] = st["E"].astype(np.float32).astype(np.float64)
    st["B"] = st["B"].astype(np.float32).astype(np.float64)
    return st


def full_from_half_q(Mh, nx, ny):
    nn = nx * ny
    M = np.zeros((nn, 25, 3, 3))
    for g in range(nn):
        i, j = g % nx, g // nx
        for h, (di, dj) in enumerate(HALFQ):
            M[g, (dj + 2) * 5 + di + 2] = Mh[g, h]
            gn = ((j + dj) % ny) * nx + (i + di) % nx
            M[gn, (-dj + 2) * 5 + (-di) + 2] = Mh[g, h]
    return M


def simq(rs, prec, st, nx, ny, dt=0.5, q=(1.0, -1.0), m=(1.0, 1.0)):
    cfg = rs.make_config(nx, ny, dt=dt, precision=prec, q=q, m=m, track_ids=True, shape=2,
                         gmres_tol=1e-13 if prec == 64 else 1e-7, gmres_restart=100)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    return sim


@pytest.mark.parametrize("prec", [64, 32])
def test_deposit_q_matches_oracle(rs, oq, prec):
    import oracle
    nx, ny = 11, 7
    q, m = (1.0, -2.0), (1.0, 3.0)
    st = f32(random_state(nx, ny, [30 * nx * ny, 20 * nx * ny], seed=51, u_scale=1.0, field_scale=0.6, q=q, m=m))
    sim = simq(rs, prec, st, nx, ny, dt=0.7, q=q, m=m)
    sim.build()
    Mh, J = sim.mass_matrix()
    c = oracle.make_config(nx, ny, dt=0.7, q=q, m=m)
    Jo, Mo = oq.depositq(c, oracle.Particles(st["species"]), st["B"])
    t = 1e-11 if prec == 64 else 2e-6
    assert rel(J, Jo) < t
    assert rel(full_from_half_q(Mh, nx, ny), Mo) < t
    sim.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_operator_q_matches_oracle(rs, oq, prec):
    import oracle
    nx, ny = 37, 11   # more than one tile along x and y, ragged tails
    st = f32(random_state(nx, ny, [6 * nx * ny, 6 * nx * ny], seed=52))
    sim = simq(rs, prec, st, nx, ny)
    sim.build()
    Mh, J = sim.mass_matrix()
    v = np.random.default_rng(3).normal(size=(3, nx * ny))
    Av = sim.apply_operator(v)
    c = oracle.make_config(nx, ny, dt=0.5)
    Ao = oq.apply_Aq(c, full_from_half_q(Mh, nx, ny), v)
    assert rel(Av, Ao) < (1e-11 if prec == 64 else 1e-5)
    sim.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_step_q_matches_oracle(rs, oq, prec):
    import oracle
    hc = HarrisConfig(nx=32, ny=16, ppc=8, pert=0.05, dt=0.5)
    st = f32(make_harris(hc))
    st["E"] = (0.02 * np.random.default_rng(5).normal(size=st["E"].shape)).astype(np.float32).astype(np.float64)
    sim = simq(rs, prec, st, hc.nx, hc.ny)
    led, code = sim.step()
    assert code == 0
    E, B = sim.fields()
    c = oracle.make_config(hc.nx, hc.ny, dt=0.5, gmres_tol=1e-14, gmres_restart=200)
    P = oracle.Particles(st["species"])
    Eo, Bo, Lo, _ = oq.stepq(c, P, st["E"], st["B"])
    tf = 1e-9 if prec == 64 else 2e-5
    assert rel(E, Eo) < tf and rel(B, Bo) < tf
    n0 = P.off[1]
    for s, sl in enumerate((slice(0, n0), slice(n0, None))):
        x, u, w, ids = sim.particles(s, ids=True)
        o = np.argsort(ids)
        uo = np.stack([P.ux[sl], P.uy[sl], P.uz[sl]], axis=1)
        xo = np.stack([P.x[sl], P.y[sl]], axis=1)
        assert rel(u[o], uo) < tf
        L = np.array([hc.nx, hc.ny], dtype=float)
        d = (x[o] - xo + 0.5 * L) % L - 0.5 * L
        assert np.abs(d).max() < (1e-10 if prec == 64 else 2e-5)
    total = Lo["W_E1"] + Lo["W_B1"] + Lo["K1"]
    tl = 1e-9 if prec == 64 else 1e-5
    for kg, ko in (("K", "K1"), ("W_E", "W_E1"), ("W_B", "W_B1"), ("work_grid", "work_grid"),
                   ("work_particles", "work_particles"), ("dissipation", "dissipation")):
        assert abs(led[kg] - Lo[ko]) < tl * total, kg
    assert abs(led["residual"]) < (1e-10 if prec == 64 else 1e-6) * total
    sim.close()


def test_three_fp64_steps_and_energy_identity(rs, oq):
    import oracle
    nx, ny = 9, 8
    st = random_state(nx, ny, [200, 150], seed=53, u_scale=0.8, field_scale=0.4)
    sim = simq(rs, 64, st, nx, ny, dt=0.6)
    c = oracle.make_config(nx, ny, dt=0.6, gmres_tol=1e-14, gmres_restart=200)
    P = oracle.Particles(st["species"])
    E, B = st["E"], st["B"]
    for _ in range(3):
        led, code = sim.step()
        assert code == 0
        E, B, Lo, _ = oq.stepq(c, P, E, B)
        total = Lo["W_E1"] + Lo["W_B1"] + Lo["K1"]
        assert abs(led["residual"]) < 1e-10 * total
    Eg, Bg = sim.fields()
    assert rel(Eg, E) < 1e-9 and rel(Bg, B) < 1e-9
    # the second and third steps ran as CUDA graphs
    gi = sim.graph_info()
    assert gi["graph_steps"] == 2 and not gi["disabled"], gi
    sim.close()


def test_quadratic_config_checks(rs):
    with pytest.raises(rs.RelsimError):
        rs.Simulation(rs.make_config(8, 8, nz=4, shape=2))
    with pytest.raises(rs.RelsimError):
        rs.Simulation(rs.make_config(8, 8, shape=2, gamma_pred=True))
    st = random_state(8, 8, [100, 100], seed=54)
    sim = simq(rs, 32, st, 8, 8)
    sim.build()
    sim.solve()
    with pytest.raises(rs.RelsimError):
        sim.push_adjoint(0, np.zeros((100, 3)), np.zeros((100, 2)))
    sim.push()
    sim.close()
