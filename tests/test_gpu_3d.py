"""The 3D form on the GPU against the 3D FP64 oracle (relsim_oracle3.c).

Deposit (Jhat and the 14 stored mass-matrix offsets against the oracle's 27),
the operator with the GPU's own mass matrix, one full step (fields,
particles matched by id, every ledger term) and three FP64 steps, the
energy identity of the GPU's ledger, the field-mode diagnostic over the
ny*nz rows, and the entry points that cover only the 2D form.

Tolerances relative to the largest entry: FP64 form 1e-11 for the deposit
and the operator (summation order), 1e-9 after a step (GMRES at 1e-13);
FP32 form 2e-6 for the deposit (FP32 accumulation over a cell's particles
and the 8 cells around a node), 1e-5 for the operator, 2e-5 for fields and
momenta after a step (GMRES at 1e-7 with an FP32 operator).
"""
import numpy as np
import pytest

from relsim_inputs import HarrisConfig3, make_harris3, random_state3

pytestmark = pytest.mark.gpu

NX, NY, NZ = 6, 5, 4
HALF3 = [(0, 0, 0), (1, 0, 0), (-1, 1, 0), (0, 1, 0), (1, 1, 0)] + \
        [(di, dj, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]


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
def o3():
    from oracle import three
    three.load()
    return three


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def f32(st):
    for sp in st["species"]:
        for k in ("x", "y", "z", "ux", "uy", "uz", "w"):
            sp[k] = np.asarray(sp[k]).astype(np.float32).astype(np.float64)
    st["E"] = st["E"].astype(np.float32).astype(np.float64)
    st["B"] = st["B"].astype(np.float32).astype(np.float64)
    return st


def full_from_half3(Mh, nx, ny, nz):
    """(nn, 14, 3, 3) stored blocks -> the oracle's (nn, 27, 3, 3)."""
    nn = nx * ny * nz
    M = np.zeros((nn, 27, 3, 3))
    for g in range(nn):
        i, j, k = g % nx, (g // nx) % ny, g // (nx * ny)
        for h, (di, dj, dk) in enumerate(HALF3):
            M[g, (dk + 1) * 9 + (dj + 1) * 3 + di + 1] = Mh[g, h]
            gn = (((k + dk) % nz) * ny + (j + dj) % ny) * nx + (i + di) % nx
            M[gn, (-dk + 1) * 9 + (-dj + 1) * 3 + (-di) + 1] = Mh[g, h]
    return M


def sim3(rs, prec, st, dt=0.5, tol=None, q=(1.0, -1.0), m=(1.0, 1.0), nx=NX, ny=NY, nz=NZ):
    cfg = rs.make_config(nx, ny, nz=nz, dt=dt, precision=prec, q=q, m=m, track_ids=True,
                         gmres_tol=tol or (1e-13 if prec == 64 else 1e-7), gmres_restart=100)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    return sim


@pytest.mark.parametrize("prec", [64, 32])
def test_deposit3_matches_oracle(rs, o3, prec):
    q, m = (1.0, -2.0), (1.0, 3.0)
    st = f32(random_state3(NX, NY, NZ, [20 * NX * NY * NZ, 15 * NX * NY * NZ], seed=31, u_scale=1.0,
                           field_scale=0.6, q=q, m=m))
    sim = sim3(rs, prec, st, dt=0.7, q=q, m=m)
    sim.build()
    Mh, J = sim.mass_matrix()
    c = o3.make_config3(NX, NY, NZ, dt=0.7, q=q, m=m)
    Jo, Mo = o3.deposit3(c, o3.Particles3(st["species"]), st["B"])
    t = 1e-11 if prec == 64 else 2e-6
    assert rel(J, Jo) < t
    assert rel(full_from_half3(Mh, NX, NY, NZ), Mo) < t
    sim.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_operator3_matches_oracle(rs, o3, prec):
    st = f32(random_state3(NX, NY, NZ, [10 * NX * NY * NZ, 10 * NX * NY * NZ], seed=32))
    sim = sim3(rs, prec, st)
    sim.build()
    Mh, J = sim.mass_matrix()
    v = np.random.default_rng(3).normal(size=(3, NX * NY * NZ))
    Av = sim.apply_operator(v)
    c = o3.make_config3(NX, NY, NZ, dt=0.5)
    Ao = o3.apply_A3(c, full_from_half3(Mh, NX, NY, NZ), v)
    assert rel(Av, Ao) < (1e-11 if prec == 64 else 1e-5)
    sim.close()


def _by_id(sim, s, ids_total_offset):
    x, u, w, ids = sim.particles(s, ids=True)
    order = np.argsort(ids)
    return x[order], u[order], w[order]


@pytest.mark.parametrize("prec", [64, 32])
def test_step3_matches_oracle(rs, o3, prec):
    st = f32(make_harris3(HarrisConfig3(nx=8, ny=8, nz=4, ppc=8, pert=0.05, dt=0.5)))
    st["E"] = (0.02 * np.random.default_rng(5).normal(size=st["E"].shape)).astype(np.float32).astype(np.float64)
    sim = sim3(rs, prec, st, dt=0.5, nx=8, ny=8, nz=4)
    led, code = sim.step()
    assert code == 0
    E, B = sim.fields()
    c = o3.make_config3(8, 8, 4, dt=0.5, gmres_tol=1e-14, gmres_restart=200)
    P = o3.Particles3(st["species"])
    Eo, Bo, Lo, _ = o3.step3(c, P, st["E"], st["B"])
    tf = 1e-9 if prec == 64 else 2e-5
    assert rel(E, Eo) < tf and rel(B, Bo) < tf
    n0 = P.off[1]
    for s, sl in enumerate((slice(0, n0), slice(n0, None))):
        x, u, w = _by_id(sim, s, 0)
        uo = np.stack([P.ux[sl], P.uy[sl], P.uz[sl]], axis=1)
        xo = np.stack([P.x[sl], P.y[sl], P.z[sl]], axis=1)
        assert rel(u, uo) < tf
        # positions: periodic difference
        L = np.array([8.0, 8.0, 4.0])
        d = (x - xo + 0.5 * L) % L - 0.5 * L
        assert np.abs(d).max() < (1e-10 if prec == 64 else 2e-5)
    tl = 1e-9 if prec == 64 else 1e-5
    total = Lo["W_E1"] + Lo["W_B1"] + Lo["K1"]
    assert abs(led["K"] - Lo["K1"]) < tl * total
    assert abs(led["W_E"] - Lo["W_E1"]) < tl * total
    assert abs(led["W_B"] - Lo["W_B1"]) < tl * total
    assert abs(led["work_grid"] - Lo["work_grid"]) < tl * total
    assert abs(led["work_particles"] - Lo["work_particles"]) < tl * total
    assert abs(led["dissipation"] - Lo["dissipation"]) < tl * total
    assert abs(led["mismatch"] - Lo["mismatch"]) < 1e-3 * abs(Lo["mismatch"]) + tl * total * 1e-2
    assert abs(led["residual"]) < (1e-10 if prec == 64 else 1e-6) * total
    sim.close()


def test_three_fp64_steps_and_energy_identity(rs, o3):
    st = random_state3(5, 4, 3, [150, 120], seed=33, u_scale=0.8, field_scale=0.4)
    sim = sim3(rs, 64, st, dt=0.6, nx=5, ny=4, nz=3)
    c = o3.make_config3(5, 4, 3, dt=0.6, gmres_tol=1e-14, gmres_restart=200)
    P = o3.Particles3(st["species"])
    E, B = st["E"], st["B"]
    for _ in range(3):
        led, code = sim.step()
        assert code == 0
        E, B, Lo, _ = o3.step3(c, P, E, B)
        total = Lo["W_E1"] + Lo["W_B1"] + Lo["K1"]
        assert abs(led["residual"]) < 1e-10 * total
    Eg, Bg = sim.fields()
    assert rel(Eg, E) < 1e-9 and rel(Bg, B) < 1e-9
    # the second and third steps ran as CUDA graphs
    gi = sim.graph_info()
    assert gi["graph_steps"] == 2 and not gi["disabled"], gi
    sim.close()


def test_field_modes_3d_over_all_rows(rs):
    st = f32(make_harris3(HarrisConfig3(nx=16, ny=6, nz=4, ppc=2)))
    sim = sim3(rs, 64, st, nx=16, ny=6, nz=4)
    W = sim.field_modes(component=1, nmodes=5)
    By = st["B"][1].reshape(4 * 6, 16)
    F = np.fft.rfft(By, axis=1)
    cm = np.full(9, 2.0)
    cm[0] = 1.0
    cm[-1] = 1.0
    want = (0.5 * cm * (np.abs(F) ** 2).sum(axis=0) / 16)[:5]
    assert rel(W, want) < 1e-12
    sim.close()


def test_3d_config_checks_and_2d_only_calls(rs):
    with pytest.raises(rs.RelsimError):
        rs.Simulation(rs.make_config(8, 8, nz=2))
    with pytest.raises(rs.RelsimError):
        rs.Simulation(rs.make_config(8, 8, nz=4, gamma_pred=True))
    st = random_state3(5, 4, 3, [60, 60], seed=34)
    sim = sim3(rs, 32, st, nx=5, ny=4, nz=3)
    sim.build()
    sim.solve()
    with pytest.raises(rs.RelsimError):
        sim.field_adjoint(np.zeros((3, 60)), np.zeros((3, 60)))
    sim.push()
    x, u, w = sim.particles(0)
    assert x.shape == (60, 3) and np.all(x >= 0) and np.all(x[:, 2] < 3.0)
    sim.close()
