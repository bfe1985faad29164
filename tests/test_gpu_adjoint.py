"""The adjoint of the field part of a step on the GPU against the oracle's.

Both sides use the GPU's mass matrix and E^{n+theta} (read back after the
forward solve), so they differ only in the adjoint solve: the GPU's
transposed operator applied in the form's precision with GMRES to the
context's tolerance, the oracle's dense solve in FP64. Tolerances relative
to the largest entry: FP64 form 1e-9 (GMRES tolerance 1e-12), FP32 form 2e-5
(an FP32 operator application carries ~1e-7 relative error, GMRES stops at
1e-7).
"""
import numpy as np
import pytest

from relsim_inputs import random_state

pytestmark = pytest.mark.gpu

HALF = ((0, 0), (1, 0), (-1, 1), (0, 1), (1, 1))


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
def orc():
    import oracle
    oracle.load()
    return oracle


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def full_from_half(Mh, nx, ny):
    nn = nx * ny
    full = np.zeros((nn, 9, 3, 3))
    idx = np.arange(nn)
    i, j = idx % nx, idx // nx
    for k, (di, dj) in enumerate(HALF):
        full[:, (dj + 1) * 3 + di + 1] = Mh[:, k]
        if k:
            nb = ((j + dj) % ny) * nx + (i + di) % nx
            full[nb, (-dj + 1) * 3 - di + 1] = Mh[:, k]
    return full


def half_grad_from_full(G, nx, ny):
    # a stored block serves the pairs (g, g+o) and (g+o, g)
    nn = nx * ny
    out = np.zeros((nn, 5, 3, 3))
    idx = np.arange(nn)
    i, j = idx % nx, idx // nx
    for k, (di, dj) in enumerate(HALF):
        out[:, k] = G[:, (dj + 1) * 3 + di + 1]
        if k:
            nb = ((j + dj) % ny) * nx + (i + di) % nx
            out[:, k] += G[nb, (-dj + 1) * 3 - di + 1]
    return out


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("nx,ny,theta", [(13, 7, 0.5), (24, 16, 0.6)])
def test_field_adjoint_matches_oracle(rs, orc, prec, nx, ny, theta):
    dt = 0.7
    st = random_state(nx, ny, [20 * nx * ny, 20 * nx * ny], seed=41, u_scale=1.0, field_scale=0.6)
    cfg = rs.make_config(nx, ny, dt=dt, theta_implicit=theta, precision=prec,
                         gmres_tol=1e-12 if prec == 64 else 1e-7, gmres_restart=60)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    sim.build()
    Mh, _ = sim.mass_matrix()
    sim.solve()
    Et = sim.E_theta()
    rng = np.random.default_rng(5)
    gE1, gB1 = rng.normal(size=(3, nx * ny)), rng.normal(size=(3, nx * ny))
    g = sim.field_adjoint(gE1, gB1)
    assert g["status"] == 0 and g["iters"] > 0
    c = orc.make_config(nx, ny, dt=dt, theta=theta)
    o = orc.field_adjoint(c, full_from_half(np.asarray(Mh).reshape(nx * ny, 5, 3, 3), nx, ny), Et, gE1, gB1)
    t = 1e-9 if prec == 64 else 2e-5
    for k in ("E0", "B0", "J"):
        assert rel(g[k], o[k]) < t, (k, rel(g[k], o[k]))
    assert rel(g["M"], half_grad_from_full(o["M"], nx, ny)) < t
    # the adjoint leaves the forward step intact: the push still runs
    sim.push()
    sim.close()


def test_field_adjoint_device_arrays_and_call_order(rs):
    import torch
    nx, ny = 16, 8
    st = random_state(nx, ny, [500, 500], seed=42)
    sim = rs.Simulation(rs.make_config(nx, ny, precision=64, gmres_tol=1e-12))
    sim.load_state(st)
    g1 = torch.randn(3, nx * ny, dtype=torch.float64, device="cuda")
    g2 = torch.randn(3, nx * ny, dtype=torch.float64, device="cuda")
    with pytest.raises(rs.RelsimError) as e:
        sim.field_adjoint(g1, g2)   # no solved step yet
    assert e.value.code == rs.RELSIM_ERR_BAD_STATE
    sim.build()
    sim.solve()
    gd = sim.field_adjoint(g1, g2, mass=False)
    gh = sim.field_adjoint(g1.cpu().numpy(), g2.cpu().numpy(), mass=False)
    assert gd["E0"].is_cuda and gd["M"] is None
    for k in ("E0", "B0", "J"):
        assert rel(gd[k].cpu().numpy(), gh[k]) < 1e-13
    sim.push()
    with pytest.raises(rs.RelsimError):
        sim.field_adjoint(g1, g2)   # after the push
    sim.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_push_adjoint_matches_oracle(rs, orc, prec):
    """Both sides replay the push in FP64 from the same stored values (the
    GPU's offsets, momenta and fields, read back), so they agree to
    summation order: 1e-10 of the largest entry in either form."""
    nx, ny, dt = 19, 11, 0.7
    q, m = (1.0, -1.0), (1.0, 2.0)
    st = random_state(nx, ny, [3000, 2500], seed=61, u_scale=1.2, field_scale=0.7, q=q, m=m)
    cfg = rs.make_config(nx, ny, dt=dt, precision=prec, q=q, m=m, track_ids=True,
                         gmres_tol=1e-12 if prec == 64 else 1e-7)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    sim.build()
    Bn = sim.fields()[1]
    parts = [sim.particles(s, ids=True) for s in range(2)]
    sim.solve()
    Et = sim.E_theta()
    rng = np.random.default_rng(17)
    gE_tot = np.zeros((3, nx * ny))
    for s in range(2):
        x, u, w, ids = parts[s]
        n = len(w)
        gu1, gx1 = rng.normal(size=(n, 3)), rng.normal(size=(n, 2))
        g = sim.push_adjoint(s, gu1, gx1)
        c = orc.make_config(nx, ny, dt=dt, q=(q[s],), m=(m[s],))
        P = orc.Particles([{"x": x[:, 0], "y": x[:, 1], "ux": u[:, 0], "uy": u[:, 1], "uz": u[:, 2], "w": w}])
        o = orc.push_adjoint(c, P, Et, Bn, gu1.T, gx1[:, 0], gx1[:, 1])
        assert rel(g["u"], o["u"].T) < 1e-10
        assert rel(g["x"], np.stack([o["x"], o["y"]], axis=1)) < 1e-10
        assert rel(g["E"], o["E"]) < 1e-10
        assert rel(g["B"], o["B"]) < 1e-10
        gE_tot += g["E"]
    assert np.abs(gE_tot).max() > 0
    sim.push()   # the forward step is intact
    sim.close()


def test_push_adjoint_device_arrays(rs):
    import torch
    nx, ny = 16, 8
    st = random_state(nx, ny, [700, 0], seed=62)
    sim = rs.Simulation(rs.make_config(nx, ny, precision=32))
    sim.load_state(st)
    sim.build()
    sim.solve()
    n = rs.relsim_num_particles(sim.ctx, 0)
    gu1 = torch.randn(n, 3, dtype=torch.float64, device="cuda")
    gx1 = torch.randn(n, 2, dtype=torch.float64, device="cuda")
    gd = sim.push_adjoint(0, gu1, gx1)
    gh = sim.push_adjoint(0, gu1.cpu().numpy(), gx1.cpu().numpy())
    assert gd["u"].is_cuda
    # the field gradients come from float atomics in either order: rounding only
    assert rel(gd["u"].cpu().numpy(), gh["u"]) < 1e-13
    assert rel(gd["E"].cpu().numpy(), gh["E"]) < 1e-12
    # an empty species gives zero field gradients
    ge = sim.push_adjoint(1, np.zeros((0, 3)), np.zeros((0, 2)))
    assert not np.any(ge["E"]) and not np.any(ge["B"])
    sim.close()


def _gpu_state(rs, nx, ny, prec, dt, q, m, seed, tol=None):
    st = random_state(nx, ny, [8 * nx * ny, 6 * nx * ny], seed=seed, u_scale=1.0, field_scale=0.5, q=q, m=m)
    cfg = rs.make_config(nx, ny, dt=dt, precision=prec, q=q, m=m, track_ids=True,
                         gmres_tol=tol or (1e-13 if prec == 64 else 1e-7), gmres_restart=100)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    sim.build()
    E0, B0 = sim.fields()
    parts = [sim.particles(s, ids=True) for s in range(2)]
    return sim, E0, B0, parts


@pytest.mark.parametrize("prec", [64, 32])
def test_deposit_adjoint_matches_oracle(rs, orc, prec):
    nx, ny, dt = 17, 9, 0.6
    q, m = (1.0, -2.0), (1.0, 3.0)
    sim, E0, B0, parts = _gpu_state(rs, nx, ny, prec, dt, q, m, seed=63)
    rng = np.random.default_rng(19)
    gJ = rng.normal(size=(3, nx * ny))
    gMh = rng.normal(size=(nx * ny, 5, 3, 3))
    # the oracle's full layout: each stored block's gradient on its (g, g+o) slot
    gMf = np.zeros((nx * ny, 9, 3, 3))
    for k, (di, dj) in enumerate(HALF):
        gMf[:, (dj + 1) * 3 + di + 1] = gMh[:, k]
    for s in range(2):
        x, u, w, ids = parts[s]
        g = sim.deposit_adjoint(s, gJ, gMh)
        c = orc.make_config(nx, ny, dt=dt, q=(q[s],), m=(m[s],))
        P = orc.Particles([{"x": x[:, 0], "y": x[:, 1], "ux": u[:, 0], "uy": u[:, 1], "uz": u[:, 2], "w": w}])
        o = orc.deposit_adjoint(c, P, B0, gJ, gMf)
        assert rel(g["u"], o["u"].T) < 1e-10
        assert rel(g["x"], np.stack([o["x"], o["y"]], axis=1)) < 1e-10
        assert rel(g["B"], o["B"]) < 1e-10
    sim.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_one_step_adjoint_chain_matches_oracle(rs, orc, prec):
    """One full step's gradient on the GPU, chained as the header describes
    (push adjoints, field adjoint with their dL/dE^{n+theta}, deposit
    adjoints), against the oracle's step adjoint on the GPU's own state and
    fields (the oracle's chain is pinned by central differences of its full
    step). The GPU solves with its FP64 or FP32 operator: FP64 1e-8, FP32
    2e-4 of the largest entry (the FP32 form's adjoint solve)."""
    nx, ny, dt = 12, 8, 0.6
    q, m = (1.0, -1.0), (1.0, 1.0)
    sim, E0, B0, parts = _gpu_state(rs, nx, ny, prec, dt, q, m, seed=64)
    Mh, Jh = sim.mass_matrix()
    sim.solve()
    rng = np.random.default_rng(21)
    nn = nx * ny
    gE1, gB1 = rng.normal(size=(3, nn)), rng.normal(size=(3, nn))
    gu1 = [rng.normal(size=(len(p[2]), 3)) for p in parts]
    gx1 = [rng.normal(size=(len(p[2]), 2)) for p in parts]
    gp = [sim.push_adjoint(s, gu1[s], gx1[s]) for s in range(2)]
    gEt = gp[0]["E"] + gp[1]["E"]
    gf = sim.field_adjoint(gE1, gB1, gEt=gEt)
    gd = [sim.deposit_adjoint(s, gf["J"], gf["M"]) for s in range(2)]
    gB = gf["B0"] + sum(g["B"] for g in gp) + sum(g["B"] for g in gd)
    # the oracle on the same particles (both species, GPU order) and fields
    allp = [{"x": p[0][:, 0], "y": p[0][:, 1], "ux": p[1][:, 0], "uy": p[1][:, 1], "uz": p[1][:, 2], "w": p[2]}
            for p in parts]
    c = orc.make_config(nx, ny, dt=dt, q=q, m=m, gmres_tol=1e-14, gmres_restart=200)
    P = orc.Particles(allp)
    o = orc.step_adjoint(c, P, E0, B0, np.concatenate(gu1).T, np.concatenate(gx1)[:, 0],
                         np.concatenate(gx1)[:, 1], gE1, gB1)
    t = 1e-8 if prec == 64 else 2e-4
    gu = np.concatenate([gp[s]["u"] + gd[s]["u"] for s in range(2)])
    gx = np.concatenate([gp[s]["x"] + gd[s]["x"] for s in range(2)])
    assert rel(gu, o["u"].T) < t
    assert rel(gx, np.stack([o["x"], o["y"]], axis=1)) < t
    assert rel(gf["E0"], o["E"]) < t
    assert rel(gB, o["B"]) < t
    sim.push()
    sim.close()
