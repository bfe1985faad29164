"""Parity of the 3D form at the full 3D benchmark size and launch
configuration: the 256x128x128 double Harris sheet with 16 particles per
cell per species (134,217,728 particles), FP32 form, GMRES tol 1e-6,
restart 30 (ids tracked, to follow sampled particles).

A full 3D oracle step at this size takes the single-core oracle many
minutes, so the step is checked on sampled outputs the oracle computes one
by one, and by properties that hold at any size:

* mass-matrix blocks of all 27 offsets and the current at sampled nodes:
  they depend only on the particles of the 8 cells around the node, which
  the oracle deposits on a small local periodic grid carrying the same B;
* the push of sampled particles (matched by id) against the oracle's push of
  the same particles in the GPU's own E^{n+theta} and B^n (FP64);
* the re-sort keeps every particle and puts each in the cell of its new
  position; the energy identity of the step holds to the FP32 floor.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NX, NY, NZ, PPC = 256, 128, 128, 16
HALF3 = [(0, 0, 0), (1, 0, 0), (-1, 1, 0), (0, 1, 0), (1, 1, 0)] + \
        [(di, dj, 1) for dj in (-1, 0, 1) for di in (-1, 0, 1)]


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    from oracle import three
    from relsim_inputs import HarrisConfig3, make_harris3
    hc = HarrisConfig3(nx=NX, ny=NY, nz=NZ, ppc=PPC, dt=0.5, seed=0)
    st = make_harris3(hc)
    cfg = rs.make_config(NX, NY, nz=NZ, dt=0.5, theta_implicit=0.5, precision=32, gmres_tol=1e-6,
                         gmres_restart=30, track_ids=True)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    yield rs, three, hc, st, sim
    sim.close()


def node_index(i, j, k):
    return ((k % NZ) * NY + (j % NY)) * NX + (i % NX)


def local_oracle_node(three, st, hc, gi, gj, gk):
    """Exact (FP64) blocks M[g][o] for all 27 offsets and Jhat at node g from
    the particles of its 8 cells, on a 6x6x6 local periodic grid around it."""
    i0, j0, k0 = gi - 3, gj - 3, gk - 3
    sp_local = []
    for sp in st["species"]:
        idx = []
        for dk in (-1, 0):
            for dj in (-1, 0):
                for di in (-1, 0):
                    c = node_index(gi + di, gj + dj, gk + dk)
                    idx.append(np.arange(c * PPC, (c + 1) * PPC))   # loader order: cell by cell
        idx = np.concatenate(idx)
        d = {k: sp[k][idx] for k in ("ux", "uy", "uz", "w")}
        d["x"] = (sp["x"][idx] - i0 * hc.dx) % (NX * hc.dx)
        d["y"] = (sp["y"][idx] - j0 * hc.dy) % (NY * hc.dy)
        d["z"] = (sp["z"][idx] - k0 * hc.dz) % (NZ * hc.dz)
        sp_local.append(d)
    B = st["B"].reshape(3, NZ, NY, NX)
    kk, jj, ii = (np.arange(k0, k0 + 6) % NZ), (np.arange(j0, j0 + 6) % NY), (np.arange(i0, i0 + 6) % NX)
    Bl = B[:, kk][:, :, jj][:, :, :, ii].reshape(3, 216)
    c = three.make_config3(6, 6, 6, dt=hc.dt, theta=hc.theta)
    J, M = three.deposit3(c, three.Particles3(sp_local), Bl)
    g = (3 * 6 + 3) * 6 + 3
    return M[g], J[:, g]


def test_fullsize3d_sampled_mass_matrix(setup):
    import torch
    rs, three, hc, st, sim = setup
    sim.build()
    M, J = sim.mass_matrix(device=True)   # (nn, 14, 3, 3), (3, nn) on the device
    rng = np.random.default_rng(0)
    nodes = [(int(rng.integers(NX)), int(rng.integers(NY)), int(rng.integers(NZ))) for _ in range(8)]
    nodes += [(0, 0, 0), (NX - 1, NY - 1, NZ - 1), (7, NY // 4, 5), (200, 3 * NY // 4, NZ - 1)]
    for gi, gj, gk in nodes:
        Mo, Jo = local_oracle_node(three, st, hc, gi, gj, gk)
        g = node_index(gi, gj, gk)
        # the GPU's 27 blocks of node g: own stored offsets, the rest from
        # the neighbour that stores the pair
        full = np.zeros((27, 3, 3))
        for h, (di, dj, dk) in enumerate(HALF3):
            full[(dk + 1) * 9 + (dj + 1) * 3 + di + 1] = M[g, h].double().cpu().numpy()
            gn = node_index(gi - di, gj - dj, gk - dk)
            full[(-dk + 1) * 9 + (-dj + 1) * 3 + (-di) + 1] = M[gn, h].double().cpu().numpy()
        assert np.abs(full - Mo).max() <= 2e-5 * np.abs(Mo).max(), (gi, gj, gk)
        Jg = J[:, g].double().cpu().numpy()
        assert np.abs(Jg - Jo).max() <= 2e-5 * max(np.abs(Jo).max(), 1e-30) + 1e-7, (gi, gj, gk)
    del M, J
    torch.cuda.empty_cache()


def test_fullsize3d_step_sampled_push_and_properties(setup):
    import torch
    rs, three, hc, st, sim = setup
    # the test above built the mass matrix; B^n is current until the solve
    Bn = sim.fields()[1]
    it, relres, status = sim.solve()
    assert status == 0 and relres <= 1e-6
    Et = sim.E_theta()
    rng = np.random.default_rng(1)
    samples = []
    for s in range(2):
        n = len(st["species"][s]["w"])
        ids = np.sort(rng.choice(n, 400, replace=False))
        samples.append(ids)
    sim.push()
    led = sim.ledger()
    assert abs(led["residual"]) < 2e-5 * led["total"]
    assert abs(led["work_grid"] - led["work_particles"]) < 1e-5 * led["total"]
    for s in range(2):
        sp = st["species"][s]
        x, u, w, ids = sim.particles(s, ids=True, device=True)
        n = len(sp["w"])
        assert ids.shape[0] == n
        # every particle once, in the cell of its new position
        assert torch.equal(torch.sort(ids.long())[0], torch.arange(n, device=ids.device))
        start = sim.cell_start(s, device=True)
        cnt = (start[1:] - start[:-1]).long()
        cell = (torch.floor(x[:, 2]).long() * NY + torch.floor(x[:, 1]).long()) * NX + torch.floor(x[:, 0]).long()
        assert torch.equal(torch.repeat_interleave(torch.arange(NX * NY * NZ, device=x.device), cnt), cell)
        # sampled particles against the oracle's push in the GPU's fields
        inv = torch.empty_like(ids)
        inv[ids.long()] = torch.arange(n, device=ids.device, dtype=ids.dtype)
        pos = inv[torch.as_tensor(samples[s], device=ids.device)].long()
        xs, us = x[pos].cpu().numpy(), u[pos].cpu().numpy()
        sel = {k: np.asarray(sp[k])[samples[s]].astype(np.float32).astype(np.float64)
               for k in ("x", "y", "z", "ux", "uy", "uz", "w")}
        c = three.make_config3(NX, NY, NZ, dt=hc.dt, theta=hc.theta, q=(sp["q"],), m=(sp["m"],))
        P = three.Particles3([sel])
        three.push3(c, P, Et, Bn)
        uo = np.stack([P.ux, P.uy, P.uz], axis=1)
        xo = np.stack([P.x, P.y, P.z], axis=1)
        assert np.abs(us - uo).max() <= 2e-5 * max(np.abs(uo).max(), 1.0)
        L = np.array([NX, NY, NZ], dtype=float)
        d = (xs - xo + 0.5 * L) % L - 0.5 * L
        assert np.abs(d).max() <= 1e-4
