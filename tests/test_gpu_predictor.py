"""The predicted-gamma variant on the GPU against the oracle's.

With gamma_pred the Lorentz factor in alpha and M is that of the predicted
half-step momentum u^n + beta E^n(x). Tolerances as for the base scheme: FP64
form 1e-11 of the largest entry (summation order only), FP32 form 2e-5 (sums
of O(100) FP32 products); ledger terms as in the base one-step test.
"""
import numpy as np
import pytest

from relsim_inputs import HarrisConfig, make_harris, random_state

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


def fp32_state(st):
    # offsets, momenta, weights and fields exactly representable in FP32
    for sp in st["species"]:
        for k in ("x", "y"):
            s = np.asarray(sp[k])
            fl = np.floor(s)
            f = np.minimum((s - fl).astype(np.float32).astype(np.float64),
                           np.float64(np.nextafter(np.float32(1.0), np.float32(0.0))))
            sp[k] = fl + f
        for k in ("ux", "uy", "uz", "w"):
            sp[k] = np.asarray(sp[k]).astype(np.float32).astype(np.float64)
    st["E"] = np.asarray(st["E"]).astype(np.float32).astype(np.float64)
    st["B"] = np.asarray(st["B"]).astype(np.float32).astype(np.float64)
    return st


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def sim_for(rs, nx, ny, prec, dt, pred=True, tol=None):
    tol = tol if tol is not None else (1e-12 if prec == 64 else 1e-7)
    cfg = rs.make_config(nx, ny, dt=dt, precision=prec, gmres_tol=tol, track_ids=True, gamma_pred=pred)
    return rs.Simulation(cfg)


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("case", ["tiny", "ragged"])
def test_predicted_deposit_matches_oracle(rs, orc, prec, case):
    if case == "tiny":
        nx, ny, dt = 3, 3, 0.7
        st = random_state(nx, ny, [40, 25], seed=5, u_scale=2.0, field_scale=1.5)
    else:
        nx, ny, dt = 37, 11, 0.9
        st = random_state(nx, ny, [5000, 4000], seed=6, u_scale=1.0, field_scale=1.0)
    st = fp32_state(st)
    sim = sim_for(rs, nx, ny, prec, dt)
    sim.load_state(st)
    sim.build()
    M, J = sim.mass_matrix()
    c = orc.make_config(nx, ny, dt=dt, gamma_pred=1)
    Jo, Mo = orc.deposit(c, orc.Particles(st["species"]), st["B"], st["E"])
    Mh = np.stack([Mo[:, (dj + 1) * 3 + di + 1] for di, dj in HALF], axis=1)
    t = 1e-11 if prec == 64 else 2e-5
    assert rel(M, Mh) < t
    assert rel(J, Jo) < t
    # and it differs from the base scheme's deposit (E^n is not zero here)
    Jb, Mb = orc.deposit(orc.make_config(nx, ny, dt=dt), orc.Particles(st["species"]), st["B"])
    assert rel(Jb, Jo) > 1e-4
    sim.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_predicted_one_step_matches_oracle(rs, orc, prec):
    nx, ny, dt = 24, 16, 0.5
    st = fp32_state(random_state(nx, ny, [3000, 3000], seed=21, u_scale=1.5, field_scale=0.4))
    sim = sim_for(rs, nx, ny, prec, dt)
    sim.load_state(st)
    led, status = sim.step()
    assert status == 0
    c = orc.make_config(nx, ny, dt=dt, gmres_tol=1e-12, gmres_restart=50, gamma_pred=1)
    P = orc.Particles(st["species"])
    Eo, Bo, lo, _ = orc.step(c, P, st["E"], st["B"])
    t = 1e-11 if prec == 64 else 2e-5
    for s in range(2):
        x, u, w, ids = sim.particles(s, ids=True)
        o = P.species(s)
        assert rel(u, np.stack([o["ux"], o["uy"], o["uz"]], axis=1)[ids]) < t
    Eg, Bg = sim.fields()
    assert rel(Eg, Eo) < (1e-10 if prec == 64 else 2e-5)
    assert rel(Bg, Bo) < (1e-10 if prec == 64 else 2e-5)
    tt = 1e-9 if prec == 64 else 1e-5
    assert abs(led["K"] - lo["K1"]) < tt * lo["K1"]
    assert abs(led["work_particles"] - lo["work_particles"]) < (1e-9 if prec == 64 else 1e-3) * abs(
        lo["work_particles"])
    assert abs(led["mismatch"] - lo["mismatch"]) < (1e-8 if prec == 64 else 1e-2) * abs(lo["mismatch"])
    sim.close()


def test_predicted_fp64_steps_match_oracle_and_close_the_ledger(rs, orc):
    # a hot sheet after the first step (E^n no longer zero), through the
    # graph-captured steps: fields against the oracle, and the ledger
    # residual at round-off
    nx, ny, dt = 32, 16, 0.5
    st = make_harris(HarrisConfig(nx=nx, ny=ny, ppc=8, theta_T=1.0, dt=dt, sigma=10.0))
    sim = sim_for(rs, nx, ny, 64, dt)
    sim.load_state(st)
    c = orc.make_config(nx, ny, dt=dt, gmres_tol=1e-12, gmres_restart=50, gamma_pred=1)
    P = orc.Particles(st["species"])
    E, B = st["E"], st["B"]
    for n in range(6):
        led, status = sim.step()
        E, B, lo, _ = orc.step(c, P, E, B)
        assert status == 0
        assert abs(led["residual"]) < 1e-9 * led["total"]
        assert abs(led["mismatch"] - lo["mismatch"]) < 1e-6 * abs(lo["mismatch"]) + 1e-14 * led["total"]
    assert sim.graph_info()["graph_steps"] == 5
    Eg, Bg = sim.fields()
    assert rel(Eg, E) < 1e-8
    assert rel(Bg, B) < 1e-9
    sim.close()


def test_predicted_gamma_shrinks_the_gpu_energy_error(rs):
    # the same hot sheet, FP64 form, 20 steps: the per-step mismatch (the
    # relativistic energy error) falls by more than tenfold with the
    # predicted gamma, as in the oracle
    nx, ny, dt = 32, 16, 0.5
    st = make_harris(HarrisConfig(nx=nx, ny=ny, ppc=8, theta_T=1.0, dt=dt, sigma=10.0))
    mean = []
    for pred in (False, True):
        sim = sim_for(rs, nx, ny, 64, dt, pred=pred)
        sim.load_state(st)
        mis = []
        for n in range(20):
            led, status = sim.step()
            assert status == 0
            mis.append(abs(led["mismatch"]) / led["total"])
        mean.append(np.mean(mis[5:]))
        sim.close()
    print(f"mean per-step |mismatch| / total: gamma(u^n) {mean[0]:.3e}, predicted {mean[1]:.3e}")
    assert mean[1] < mean[0] / 10, mean
