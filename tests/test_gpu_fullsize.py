"""Parity at the benchmark's full size and launch configuration: the 1024x512
double Harris sheet with 64 particles per cell per species (67.1M
particles), FP32 form, GMRES tol 1e-6, restart 30, ids not tracked.

* mass matrix and predicted current on sampled nodes: each sampled node's
  blocks depend only on the particles of its four cells, so the oracle
  deposits those particles on a small local grid carrying the same B and
  gives the exact value (FP64) at that node;
* one full step against one full oracle step (FP64, tol 1e-12): fields and
  per-species moments, within the FP32 tolerance;
* the cell sort: cell starts are monotone and conserve every particle;
* the energy identity of the step holds to the FP32 floor.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NX, NY, PPC = 1024, 512, 64
HALF = ((0, 0), (1, 0), (-1, 1), (0, 1), (1, 1))


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    import oracle
    from relsim_inputs import HarrisConfig, make_harris
    hc = HarrisConfig(nx=NX, ny=NY, ppc=PPC, dt=1.0, theta=0.5, seed=0)
    st = make_harris(hc)
    cfg = rs.make_config(NX, NY, dt=1.0, theta_implicit=0.5, precision=32, gmres_tol=1e-6,
                         gmres_restart=30)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    yield rs, oracle, hc, st, sim
    sim.close()


def local_oracle_node(oracle, st, hc, gi, gj):
    """Exact (FP64) M blocks and Jhat at node (gi, gj) from the particles of
    its four cells, deposited on a 6x6 local periodic grid around it."""
    i0, j0 = gi - 3, gj - 3
    sp_local = []
    for sp in st["species"]:
        idx = []
        for dj in (-1, 0):
            for di in (-1, 0):
                c = ((gj + dj) % NY) * NX + (gi + di) % NX
                idx.append(np.arange(c * PPC, (c + 1) * PPC))
        idx = np.concatenate(idx)
        x = (sp["x"][idx] - i0 * hc.dx) % (NX * hc.dx)
        y = (sp["y"][idx] - j0 * hc.dy) % (NY * hc.dy)
        d = {k: sp[k][idx] for k in ("ux", "uy", "uz", "w")}
        d["x"], d["y"] = x, y
        sp_local.append(d)
    B = st["B"].reshape(3, NY, NX)
    jj = (np.arange(j0, j0 + 6)) % NY
    ii = (np.arange(i0, i0 + 6)) % NX
    Bl = B[:, jj][:, :, ii].reshape(3, 36)
    c = oracle.make_config(6, 6, dt=hc.dt, theta=hc.theta)
    J, M = oracle.deposit(c, oracle.Particles(sp_local), Bl)
    g = 3 * 6 + 3
    Mh = np.stack([M[g, (dj + 1) * 3 + di + 1] for di, dj in HALF])
    return Mh, J[:, g]


def test_fullsize_sampled_mass_matrix(setup):
    rs, oracle, hc, st, sim = setup
    sim.build()
    M, J = sim.mass_matrix()
    rng = np.random.default_rng(0)
    nodes = [(int(rng.integers(NX)), int(rng.integers(NY))) for _ in range(12)]
    nodes += [(0, 0), (NX - 1, NY - 1), (5, NY // 4), (700, 3 * NY // 4)]   # wrap and sheets
    for gi, gj in nodes:
        Mo, Jo = local_oracle_node(oracle, st, hc, gi, gj)
        g = gj * NX + gi
        assert np.abs(M[g] - Mo).max() <= 2e-5 * np.abs(Mo).max(), (gi, gj)
        assert np.abs(J[:, g] - Jo).max() <= 2e-5 * max(np.abs(Jo).max(), 1e-30) + 1e-7, (gi, gj)


def test_fullsize_step_against_oracle(setup):
    rs, oracle, hc, st, sim = setup
    # the test above built the mass matrix; finish this step
    it, relres, status = sim.solve()
    assert status == 0 and relres <= 1e-6
    sim.push()
    led = sim.ledger()
    E, B = sim.fields()
    start0 = sim.cell_start(0)
    assert np.all(np.diff(start0) >= 0) and start0[-1] == NX * NY * PPC
    assert abs(led["residual"]) < 2e-5 * led["total"]
    assert abs(led["work_grid"] - led["work_particles"]) < 1e-5 * led["total"]
    c = oracle.make_config(NX, NY, dt=hc.dt, theta=hc.theta, gmres_tol=1e-12, gmres_restart=50)
    P = oracle.Particles(st["species"])
    Eo, Bo, lo, _ = oracle.step(c, P, st["E"], st["B"])
    assert np.linalg.norm(E - Eo) <= 1e-5 * np.linalg.norm(Eo)
    assert np.linalg.norm(B - Bo) <= 1e-6 * np.linalg.norm(Bo)
    assert abs(led["K"] - lo["K1"]) <= 1e-6 * lo["K1"]
    assert abs(led["W_E"] - lo["W_E1"]) <= 1e-5 * lo["W_E1"]
    for s in range(2):
        x, u, w = sim.particles(s)
        o = P.species(s)
        mom = (w[:, None] * u).sum(axis=0)
        mom_o = np.array([(o["w"] * o[k]).sum() for k in ("ux", "uy", "uz")])
        scale = (o["w"] * np.sqrt(o["ux"] ** 2 + o["uy"] ** 2 + o["uz"] ** 2)).sum()
        assert np.abs(mom - mom_o).max() <= 1e-6 * scale
        # cell populations agree except where FP32 and FP64 put a particle on
        # different sides of a cell edge
        keys = np.floor(x[:, 1]).astype(np.int64) * NX + np.floor(x[:, 0]).astype(np.int64)
        ko = np.floor(o["y"]).astype(np.int64) % NY * NX + np.floor(o["x"]).astype(np.int64) % NX
        cnt = np.bincount(keys, minlength=NX * NY)
        cnt_o = np.bincount(ko, minlength=NX * NY)
        assert np.abs(cnt - cnt_o).sum() <= 200
