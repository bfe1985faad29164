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
    """Both sides replay the push from the same stored values (the GPU's
    offsets, momenta and fields, read back). The FP64 form replays in FP64
    and agrees to summation order, 1e-10 of the largest entry; the FP32 form
    replays in FP32 (a few hundred operations per particle at 6e-8 each as
    a linear bound, the per-cell warp sums of at most 32 terms on top):
    2e-5."""
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
        t = 1e-10 if prec == 64 else 2e-5
        assert rel(g["u"], o["u"].T) < t
        assert rel(g["x"], np.stack([o["x"], o["y"]], axis=1)) < t
        assert rel(g["E"], o["E"]) < t
        assert rel(g["B"], o["B"]) < t
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
        t = 1e-10 if prec == 64 else 2e-5   # FP32 form: FP32 replay, as for the push
        assert rel(g["u"], o["u"].T) < t
        assert rel(g["x"], np.stack([o["x"], o["y"]], axis=1)) < t
        assert rel(g["w"], o["w"]) < t
        assert rel(g["B"], o["B"]) < t
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


@pytest.mark.parametrize("prec,pred", [(64, 0), (32, 0), (64, 1), (32, 1)])
def test_step_adjoint_in_place_by_id_matches_oracle(rs, orc, prec, pred):
    """relsim_step_adjoint (build, solve and the three adjoints in one call,
    gradients in place and indexed by particle id) on particles relabelled by
    a random permutation, against the oracle's step adjoint on the same
    state: the label-indexed gradients map to the GPU order through the ids
    read back. Both readings of gbar (pred: gamma(u^n + beta E^n(x)), whose
    chain also reaches E^n and u^n through gbar). FP64 1e-8, FP32 2e-4 of
    the largest entry."""
    import torch
    nx, ny, dt = 12, 8, 0.6
    q, m = (1.0, -1.0), (1.0, 1.0)
    st = random_state(nx, ny, [8 * nx * ny, 6 * nx * ny], seed=71, u_scale=1.0, field_scale=0.5, q=q, m=m)
    cfg = rs.make_config(nx, ny, dt=dt, precision=prec, q=q, m=m, track_ids=True, gamma_pred=pred,
                         gmres_tol=1e-13 if prec == 64 else 1e-7, gmres_restart=100)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    rng = np.random.default_rng(5)
    for s in range(2):
        sim.relabel(s, rng.permutation(len(st["species"][s]["w"])).astype(np.int32))
    E0, B0 = sim.fields()
    parts = [sim.particles(s, ids=True) for s in range(2)]
    nn = nx * ny
    gE1, gB1 = rng.normal(size=(3, nn)), rng.normal(size=(3, nn))
    gu_lab = [rng.normal(size=(len(p[2]), 3)) for p in parts]
    gx_lab = [rng.normal(size=(len(p[2]), 2)) for p in parts]
    dev = lambda a: torch.tensor(a, dtype=torch.float64, device="cuda")
    gE, gB = dev(gE1), dev(gB1)
    gu, gx = [dev(a) for a in gu_lab], [dev(a) for a in gx_lab]
    gw = [torch.zeros(len(p[2]), dtype=torch.float64, device="cuda") for p in parts]
    it, rr, code = sim.step_adjoint(gE, gB, gu, gx, gw)
    assert code == 0 and it > 0
    # the oracle in the GPU's order: particle k carries label ids[k]
    allp = [{"x": p[0][:, 0], "y": p[0][:, 1], "ux": p[1][:, 0], "uy": p[1][:, 1], "uz": p[1][:, 2], "w": p[2]}
            for p in parts]
    c = orc.make_config(nx, ny, dt=dt, q=q, m=m, gmres_tol=1e-14, gmres_restart=200, gamma_pred=pred)
    gu1 = np.concatenate([gu_lab[s][parts[s][3]] for s in range(2)])
    gx1 = np.concatenate([gx_lab[s][parts[s][3]] for s in range(2)])
    o = orc.step_adjoint(c, orc.Particles(allp), E0, B0, gu1.T, gx1[:, 0], gx1[:, 1], gE1, gB1)
    t = 1e-8 if prec == 64 else 2e-4
    n0 = len(parts[0][2])
    ou, ox = o["u"].T, np.stack([o["x"], o["y"]], axis=1)
    for s, sl in enumerate((slice(0, n0), slice(n0, None))):
        ids = parts[s][3]
        want_u = np.empty_like(gu_lab[s])
        want_x = np.empty_like(gx_lab[s])
        want_w = np.empty(len(ids))
        want_u[ids] = ou[sl]
        want_x[ids] = ox[sl]
        want_w[ids] = o["w"][sl]
        assert rel(gu[s].cpu().numpy(), want_u) < t
        assert rel(gx[s].cpu().numpy(), want_x) < t
        assert rel(gw[s].cpu().numpy(), want_w) < t
    assert rel(gE.cpu().numpy(), o["E"]) < t
    assert rel(gB.cpu().numpy(), o["B"]) < t
    sim.push()   # the context is left solved
    sim.close()


def test_relabel_particles(rs):
    """Relabelling composes (id j -> ids[j]), is range-checked before it
    changes anything, and follows the particles through a step."""
    import torch
    nx, ny = 8, 8
    st = random_state(nx, ny, [300, 200], seed=9)
    cfg = rs.make_config(nx, ny, dt=0.5, precision=32, track_ids=True)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    ids0 = sim.particles(0, ids=True)[3]
    rng = np.random.default_rng(2)
    p1 = rng.permutation(300).astype(np.int32)
    p2 = torch.tensor(rng.permutation(300), dtype=torch.int32, device="cuda")
    sim.relabel(0, p1)
    assert np.array_equal(sim.particles(0, ids=True)[3], p1[ids0])
    sim.relabel(0, p2)
    assert np.array_equal(sim.particles(0, ids=True)[3], p2.cpu().numpy()[p1[ids0]])
    bad = p1.copy()
    bad[17] = 300
    before = sim.particles(0, ids=True)[3]
    with pytest.raises(rs.RelsimError) as e:
        sim.relabel(0, bad)
    assert e.value.code == rs.RELSIM_ERR_INVALID_ARG
    assert np.array_equal(sim.particles(0, ids=True)[3], before)
    # a step carries the labels with the particles: each label keeps its
    # particle's weight through the push and the re-sort
    x0, u0, w0, l0 = sim.particles(1, ids=True)
    sim.step()
    x1, u1, w1, l1 = sim.particles(1, ids=True)
    assert sorted(l1) == list(range(200))
    o0, o1 = np.argsort(l0), np.argsort(l1)
    assert np.array_equal(w0[o0], w1[o1])
    sim.close()
    cfg2 = rs.make_config(nx, ny, dt=0.5, precision=32)
    sim2 = rs.Simulation(cfg2)
    sim2.load_state(st)
    with pytest.raises(rs.RelsimError):
        sim2.relabel(0, p1)
    sim2.close()


@pytest.mark.parametrize("prec", [64, 32])
def test_adjoint_scatters_on_clustered_particles(rs, orc, prec):
    """The per-cell warp sums of the push and deposit adjoints' scatters on
    a clustered layout: 300 particles in one cell (runs that fill whole
    warps), 40 in its neighbour, one each in a few cells and most cells
    empty, against the oracle (tolerances as for the uniform layouts)."""
    nx, ny, dt = 16, 8, 0.6
    q, m = (1.0, -1.0), (1.0, 1.0)
    st = random_state(nx, ny, [360, 8], seed=77, u_scale=1.0, field_scale=0.5, q=q, m=m)
    rng = np.random.default_rng(78)
    sp0 = st["species"][0]
    cx = np.concatenate([np.full(300, 5), np.full(40, 6), rng.integers(0, nx, 20)])
    cy = np.concatenate([np.full(300, 3), np.full(40, 3), rng.integers(0, ny, 20)])
    sp0["x"] = cx + rng.random(360)
    sp0["y"] = cy + rng.random(360)
    cfg = rs.make_config(nx, ny, dt=dt, precision=prec, q=q, m=m, track_ids=True,
                         gmres_tol=1e-13 if prec == 64 else 1e-7, gmres_restart=100)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    sim.build()
    E0, B0 = sim.fields()
    parts = [sim.particles(s, ids=True) for s in range(2)]
    sim.solve()
    Et = sim.E_theta()
    t = 1e-10 if prec == 64 else 2e-5
    gJ = rng.normal(size=(3, nx * ny))
    gMh = rng.normal(size=(nx * ny, 5, 3, 3))
    gMf = np.zeros((nx * ny, 9, 3, 3))
    for k, (di, dj) in enumerate(HALF):
        gMf[:, (dj + 1) * 3 + di + 1] = gMh[:, k]
    for s in range(2):
        x, u, w, ids = parts[s]
        n = len(w)
        c = orc.make_config(nx, ny, dt=dt, q=(q[s],), m=(m[s],))
        P = orc.Particles([{"x": x[:, 0], "y": x[:, 1], "ux": u[:, 0], "uy": u[:, 1], "uz": u[:, 2], "w": w}])
        gu1, gx1 = rng.normal(size=(n, 3)), rng.normal(size=(n, 2))
        g = sim.push_adjoint(s, gu1, gx1)
        o = orc.push_adjoint(c, P, Et, B0, gu1.T, gx1[:, 0], gx1[:, 1])
        assert rel(g["u"], o["u"].T) < t
        assert rel(g["x"], np.stack([o["x"], o["y"]], axis=1)) < t
        assert rel(g["E"], o["E"]) < t
        assert rel(g["B"], o["B"]) < t
        gd = sim.deposit_adjoint(s, gJ, gMh)
        od = orc.deposit_adjoint(c, P, B0, gJ, gMf)
        assert rel(gd["u"], od["u"].T) < t
        assert rel(gd["x"], np.stack([od["x"], od["y"]], axis=1)) < t
        assert rel(gd["B"], od["B"]) < t
    sim.close()
