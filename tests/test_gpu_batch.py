"""Field-mode diagnostic and batched instances on the GPU, through the C ABI.

* relsim_field_modes against the oracle's FFT mode energies on the same
  fields (FP64 form: 1e-11 of the component's field energy; FP32 form: the
  DFT along x runs in FP32 over <= nx terms per row from FP32 twiddles, so
  5e-6 of the component's energy), and bit-identical on repeated calls.
* relsim_batch_run: instances of uneven sizes advanced concurrently equal
  the same instances stepped one by one (the deposit's float atomics make
  both runs differ in the last bits, so 1e-4 of the mode energies after a
  few steps), and the batched run's tearing growth rates match the oracle's.
* shared launches over the instances (relsim_batch_set_shared) equal the
  per-instance step graphs on the same instances.
"""
import numpy as np
import pytest

from relsim_inputs import HarrisConfig, make_harris, random_state

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("nx,ny", [(64, 32), (37, 11), (130, 9)])
def test_field_modes_match_oracle(rs, orc, precision, nx, ny):
    st = random_state(nx, ny, [0, 0], seed=3, dx=0.8, dy=1.1, field_scale=0.7)
    B = st["B"].copy()
    # a few strong modes on top of the noise, as on a tearing sheet
    xc = (np.arange(nx) + 0.5)
    B.reshape(3, ny, nx)[1] += 0.3 * np.cos(2 * np.pi * xc / nx)[None, :] + 0.1 * np.sin(6 * np.pi * xc / nx)
    if precision == 32:
        B = B.astype(np.float32).astype(np.float64)
    sim = rs.Simulation(rs.make_config(nx, ny, dx=0.8, dy=1.1, precision=precision))
    sim.set_fields(np.zeros_like(B), B)
    c = orc.make_config(nx, ny, dx=0.8, dy=1.1)
    for comp in range(3):
        for nm in (1, 5, nx // 2 + 1):
            g = sim.field_modes(comp, nm)
            o = orc.field_modes(c, B, comp, nm)
            tot = 0.5 * c.dx * c.dy * np.sum(B[comp] ** 2)
            tol = (5e-6 if precision == 32 else 1e-11) * tot
            assert np.max(np.abs(g - o)) <= tol, (comp, nm, np.max(np.abs(g - o)) / tot)
            assert np.array_equal(g, sim.field_modes(comp, nm))
    sim.close()


def test_field_modes_device_output_and_arguments(rs):
    import torch
    nx, ny = 48, 16
    st = random_state(nx, ny, [0, 0], seed=4)
    sim = rs.Simulation(rs.make_config(nx, ny))
    sim.set_fields(st["E"], st["B"])
    d = sim.field_modes(1, 7, device=True)
    assert d.is_cuda
    torch.cuda.synchronize()
    assert np.array_equal(d.cpu().numpy(), sim.field_modes(1, 7))
    for comp, nm in [(3, 1), (-1, 1), (1, 0), (1, nx // 2 + 2)]:
        with pytest.raises(rs.RelsimError):
            rs.relsim_field_modes(sim.ctx, comp, nm)
    sim.close()


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("nx,ny", [(64, 32), (37, 11)])
def test_field_mode_gradient_matches_oracle(rs, orc, precision, nx, ny):
    """The window's loss (one mode's B_y energy) and its gradient in B,
    computed on the device, against the oracle's (numpy FFT); host and
    device outputs agree bit for bit."""
    st = random_state(nx, ny, [0, 0], seed=5, dx=0.8, dy=1.1, field_scale=0.7)
    B = st["B"].copy()
    xc = (np.arange(nx) + 0.5)
    B.reshape(3, ny, nx)[1] += 0.3 * np.cos(2 * np.pi * xc / nx)[None, :]
    if precision == 32:
        B = B.astype(np.float32).astype(np.float64)
    sim = rs.Simulation(rs.make_config(nx, ny, dx=0.8, dy=1.1, precision=precision))
    sim.set_fields(np.zeros_like(B), B)
    c = orc.make_config(nx, ny, dx=0.8, dy=1.1)
    for comp in (1, 2):
        for m in (1, 3, (nx - 1) // 2):
            e, g = sim.field_mode_gradient(comp, m)
            W, gW = orc.mode_energy(c, B, m, comp)
            tot = 0.5 * c.dx * c.dy * np.sum(B[comp] ** 2)
            tol = 5e-6 if precision == 32 else 1e-11
            assert abs(e[0] - W) <= tol * tot, (comp, m, e[0], W)
            assert np.max(np.abs(g - gW)) <= tol * np.max(np.abs(gW)) + 1e-15, (comp, m)
            ed, gd = sim.field_mode_gradient(comp, m, device=True)
            assert ed.is_cuda and gd.is_cuda
            assert np.array_equal(ed.cpu().numpy(), e) and np.array_equal(gd.cpu().numpy(), g)
            # the energy equals relsim_field_modes' value of that mode
            fm = sim.field_modes(comp, m + 1)[m]
            assert abs(e[0] - fm) <= 1e-13 * abs(fm), (e[0], fm)
    for comp, m in [(3, 1), (-1, 1), (1, -1), (1, nx // 2 + 1)]:
        with pytest.raises(rs.RelsimError):
            rs.relsim_field_mode_gradient(sim.ctx, comp, m, sim.ncell)
    sim.close()


def _instance(rs, hc, stream, precision=32):
    sim = rs.Simulation(rs.make_config(hc.nx, hc.ny, dt=hc.dt, precision=precision, gmres_tol=1e-6),
                        stream=stream.cuda_stream)
    sim.load_state(make_harris(hc))
    return sim


SIZES = [HarrisConfig(nx=48, ny=24, ppc=8, dt=0.5, delta=1.0, sigma=10.0, seed=1),
         HarrisConfig(nx=96, ny=48, ppc=8, dt=0.5, delta=0.5, sigma=40.0, seed=2),
         HarrisConfig(nx=64, ny=32, ppc=4, dt=0.5, delta=2.0, sigma=1.0, seed=3)]


def test_batch_equals_instances_stepped_one_by_one(rs):
    import torch
    steps, nm = 4, 6
    streams = [torch.cuda.Stream() for _ in SIZES]
    sims = [_instance(rs, hc, s) for hc, s in zip(SIZES, streams)]
    batch = rs.Batch(sims, nworkers=3)
    modes, status, iters = batch.run(steps, component=1, nmodes=nm)
    assert modes.shape == (len(SIZES), steps, nm)
    assert list(status) == [0] * len(SIZES)
    assert np.all(iters > 0)
    after = [s.fields()[1] for s in sims]
    # after one host-driven step each instance stepped as enqueued graphs
    assert all(s.graph_info()["graph_steps"] == steps - 1 for s in sims)
    batch.close()
    # the batch's last mode energies are those of the final fields
    for k, s in enumerate(sims):
        assert np.array_equal(modes[k, -1], s.field_modes(1, nm))
        s.close()
    # the same instances, one at a time on the default stream
    for k, hc in enumerate(SIZES):
        sim = _instance(rs, hc, torch.cuda.current_stream())
        ref = []
        for _ in range(steps):
            _, code = sim.step(ledger=False)
            assert code == 0
            ref.append(sim.field_modes(1, nm))
        ref = np.array(ref)
        scale = np.abs(ref).max()
        assert np.max(np.abs(modes[k] - ref)) <= 1e-4 * scale, k
        B1 = sim.fields()[1]
        assert np.max(np.abs(after[k] - B1)) <= 1e-4 * np.abs(B1).max(), k
        sim.close()


@pytest.mark.parametrize("precision,pred,groups", [(32, 0, 1), (32, 1, 2), (64, 0, 3)])
def test_shared_launches_equal_per_instance_graphs(rs, precision, pred, groups):
    """Shared launches (per group of instances one deposit, push and re-sort
    launch per species; each instance's solve a branch of the group's graph;
    1, 2 or 3 groups on streams of their own) give
    the per-instance graphs' results on the same uneven instances: fields,
    mode energies, every particle by id, the energy ledger and the GMRES
    iteration counts, up to the order of the deposit's and the ledger's
    floating-point atomics (FP32: 1e-4 of each quantity's scale after 6
    steps; FP64: 1e-9)."""
    import torch
    steps, nm = 6, 6
    tol = 1e-4 if precision == 32 else 1e-9
    out = {}
    for shared in (True, False):
        streams = [torch.cuda.Stream() for _ in SIZES]
        sims = []
        for hc, stream in zip(SIZES, streams):
            sim = rs.Simulation(rs.make_config(hc.nx, hc.ny, dt=hc.dt, precision=precision, gmres_tol=1e-6,
                                               gamma_pred=pred, track_ids=True), stream=stream.cuda_stream)
            sim.load_state(make_harris(hc))
            sims.append(sim)
        batch = rs.Batch(sims, nworkers=3, shared=shared, groups=groups)
        assert batch.last_path is None
        for bad in (dict(groups=5000), dict(deposit_blocks=1 << 21)):
            with pytest.raises(rs.RelsimError):
                rs.relsim_batch_set_shared(batch.b, True, **bad)
        batch.set_shared(shared, groups=groups)
        modes, status, iters = batch.run(steps, component=1, nmodes=nm)
        assert list(status) == [0] * len(SIZES)
        assert batch.last_path == ("shared" if shared else "graphs")
        res = []
        for sim in sims:
            E, B = sim.fields()
            parts = []
            for s in range(2):
                x, u, w, ids = sim.particles(s, ids=True)
                o = np.argsort(ids)
                parts.append((x[o], u[o], w[o]))
            res.append((E, B, parts, sim.ledger()))
        out[shared] = (modes, iters, res)
        # a second run continues from where the first stopped
        modes2, status2, _ = batch.run(2, component=1, nmodes=nm)
        assert list(status2) == [0] * len(SIZES)
        out[shared] += (modes2,)
        batch.close()
        for sim in sims:
            sim.close()
    (mA, iA, rA, m2A), (mB, iB, rB, m2B) = out[True], out[False]
    assert np.max(np.abs(mA - mB)) <= tol * np.abs(mB).max()
    assert np.max(np.abs(m2A - m2B)) <= tol * np.abs(m2B).max()
    assert np.max(np.abs(iA - iB)) <= 1
    for k in range(len(SIZES)):
        EA, BA, pA, lA = rA[k]
        EB, BB, pB, lB = rB[k]
        assert np.max(np.abs(EA - EB)) <= tol * np.abs(EB).max(), k
        assert np.max(np.abs(BA - BB)) <= tol * np.abs(BB).max(), k
        for (xa, ua, wa), (xb, ub, wb) in zip(pA, pB):
            assert np.array_equal(wa, wb)
            assert np.max(np.abs(ua - ub)) <= tol * max(1.0, np.abs(ub).max()), k
            assert np.max(np.abs(xa - xb)) <= tol, k
        for key in ("W_E", "W_B", "K", "work_particles", "mismatch", "total"):
            assert abs(lA[key] - lB[key]) <= tol * abs(lB["total"]), (k, key, lA[key], lB[key])


def test_batch_more_workers_than_instances_and_zero_steps(rs):
    import torch
    hc = SIZES[0]
    stream = torch.cuda.Stream()
    sims = [_instance(rs, hc, stream)]
    batch = rs.Batch(sims, nworkers=8)
    modes, status, iters = batch.run(0, nmodes=3)
    assert modes.shape == (1, 0, 3) and status[0] == 0
    modes, status, iters = batch.run(2, nmodes=0)
    assert modes is None and status[0] == 0 and np.all(iters > 0)
    batch.close()
    sims[0].close()


TEARING = [HarrisConfig(nx=64, ny=32, ppc=16, dt=0.5, delta=0.5, sigma=10.0),
           HarrisConfig(nx=80, ny=40, ppc=16, dt=0.5, delta=0.5, sigma=40.0),
           HarrisConfig(nx=96, ny=48, ppc=16, dt=0.5, delta=1.0, sigma=10.0)]
STEPS, WINDOW = 160, 40


def test_batched_tearing_growth_rates_match_oracle(rs, orc):
    """Three uneven tearing instances (1% B_y perturbation at k_x = 2 pi/L_x,
    16 ppc per species) advanced by the batch runner: the growth rate of the
    m = 1 B_y mode energy, fitted over the best 40-step window, agrees with
    the FP64 oracle's on the same initial state within 5%, and the mode
    energy itself within 1e-3 over the first 80 steps (measured on GB300:
    1e-8 after one step, 1e-5 after 80, below 1e-3 after 160; the particle
    orbits diverge slowly and the collective mode follows them late)."""
    import torch
    states = []
    for hc in TEARING:
        st = make_harris(hc)
        for sp in st["species"]:   # FP32-representable: both sides start from the same state
            for k in ("x", "y", "ux", "uy", "uz", "w"):
                sp[k] = sp[k].astype(np.float32).astype(np.float64)
        st["B"] = st["B"].astype(np.float32).astype(np.float64)
        states.append(st)
    sims = []
    streams = [torch.cuda.Stream() for _ in TEARING]
    for hc, st, stream in zip(TEARING, states, streams):
        sim = rs.Simulation(rs.make_config(hc.nx, hc.ny, dt=hc.dt, precision=32, gmres_tol=1e-6),
                            stream=stream.cuda_stream)
        sim.load_state(st)
        sims.append(sim)
    batch = rs.Batch(sims, nworkers=3)
    modes, status, _ = batch.run(STEPS, component=1, nmodes=6)
    batch.close()
    for s in sims:
        s.close()
    assert list(status) == [0] * len(TEARING)
    for k, (hc, st) in enumerate(zip(TEARING, states)):
        c = orc.make_config(hc.nx, hc.ny, dt=hc.dt, gmres_tol=1e-10)
        P = orc.Particles(st["species"])
        E, B = st["E"], st["B"]
        Wall = []
        for _ in range(STEPS):
            E, B, _, _ = orc.step(c, P, E, B)
            Wall.append(orc.field_modes(c, B, 1, 6))
        Wall = np.array(Wall)
        W = Wall[:, 1]
        g_orc, _ = orc.growth_fit(W, hc.dt, WINDOW)
        g_gpu, _ = rs.relsim_growth_fit(modes[k, :, 1], hc.dt, WINDOW)
        dev = np.abs(modes[k, :, 1] / W - 1.0)
        print(f"instance {k} ({hc.nx}x{hc.ny}, delta {hc.delta}, sigma {hc.sigma}): "
              f"m=1 energy growth rate GPU {g_gpu:.6f}, oracle {g_orc:.6f} / omega_pe; "
              f"|W_gpu/W_oracle - 1| at steps 1, 40, 80, 160: {dev[0]:.2e} {dev[39]:.2e} {dev[79]:.2e} {dev[-1]:.2e}")
        assert g_orc > 0.05 and g_gpu > 0.05, (k, g_gpu, g_orc)
        assert abs(g_gpu - g_orc) < 0.05 * g_orc, (k, g_gpu, g_orc)
        # the mode energy is a grid-collective quantity: the FP32 run tracks
        # the FP64 one closely until the orbits' divergence reaches it
        assert np.all(dev[:80] < 1e-3), (k, dev[:80].max())
        # the per-mode fit (modes 1 .. 5, steps 10 .. 80) and its dispersion
        # fit (Sec. 3.1, Fig. 1 b, d) on the GPU's mode energies against the
        # oracle's fit of the oracle's energies
        Lx = hc.nx * hc.dx
        rates, A, b = rs.relsim_dispersion_fit(modes[k], hc.dt, 9, 71, Lx, hc.delta)
        orates, oA, ob = orc.tearing_dispersion(Wall, hc.dt, 9, 71, Lx, hc.delta)
        print(f"   per-mode rates GPU {np.round(rates[1:], 4)}, oracle {np.round(orates[1:], 4)}; "
              f"fit peak ka GPU {1 / (np.sqrt(3) * b):.3f}, oracle {1 / (np.sqrt(3) * ob):.3f}")
        assert np.all(np.abs(rates[1:] - orates[1:]) < 2e-3 + 0.02 * np.abs(orates[1:])), (k, rates, orates)
