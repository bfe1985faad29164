"""Energy over a run on the GPU against the oracle (Sec. 2: RelSIM keeps the
total energy accurately; the scheme's only energy error at theta = 1/2 is
the relativistic mismatch term).

A 64x32 double Harris sheet in the workload's regime (theta_T = 0.3,
sigma = 10, dt = 1, 16 particles per cell and species) runs 200 steps in
the FP32 form with each reading of the Lorentz factor in alpha, Jhat, M and
the push, and 200 steps in the FP64 oracle with the same reading. The
trajectories separate (FP32 against FP64, particle noise), but the total
energy's drift is a systematic effect of the reading: the GPU's drift is
within a factor 1.5 of the oracle's for both readings, the predicted
gamma keeps it below 1e-3, and gamma(u^n) loses at least 20 times more.
The ledger's mismatch term, which carries that loss, is also compared
directly: summed over the first 10 steps (while the FP32 and FP64 orbits
still agree closely) it equals the oracle's within 1e-2 for both readings.
"""
import numpy as np
import pytest

from relsim_inputs import HarrisConfig, make_harris

pytestmark = pytest.mark.gpu

NX, NY, PPC, DT, NSTEPS = 64, 32, 16, 1.0, 200


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    return rs


def gpu_drift(rs, st, pred):
    cfg = rs.make_config(NX, NY, dt=DT, theta_implicit=0.5, precision=32, gmres_tol=1e-6, gamma_pred=pred)
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    tot0 = None
    mis10 = 0.0
    for n in range(NSTEPS):
        led, code = sim.step(ledger=True)
        assert code == 0
        if tot0 is None:
            tot0 = led["W_E0"] + led["W_B0"] + led["K0"]
        assert abs(led["residual"]) < 2e-5 * tot0
        if n < 10:
            mis10 += led["mismatch"]
    sim.close()
    return (led["total"] - tot0) / tot0, mis10


def oracle_drift(st, pred):
    import oracle as orc
    sp = st["species"]
    c = orc.make_config(NX, NY, dt=DT, theta=0.5, q=(sp[0]["q"], sp[1]["q"]), m=(sp[0]["m"], sp[1]["m"]),
                        gmres_tol=1e-12, gamma_pred=pred)
    P = orc.Particles(sp)
    E, B = st["E"], st["B"]
    tot0 = None
    mis10 = 0.0
    for n in range(NSTEPS):
        E, B, led, _ = orc.step(c, P, E, B)
        if tot0 is None:
            tot0 = led["W_E0"] + led["W_B0"] + led["K0"]
        if n < 10:
            mis10 += led["mismatch"]
    return (led["W_E1"] + led["W_B1"] + led["K1"] - tot0) / tot0, mis10


def test_energy_over_200_steps_both_readings(rs):
    st = make_harris(HarrisConfig(nx=NX, ny=NY, ppc=PPC, dt=DT))
    gm = {pred: gpu_drift(rs, st, pred) for pred in (False, True)}
    om = {pred: oracle_drift(st, int(pred)) for pred in (False, True)}
    g = {k: v[0] for k, v in gm.items()}
    o = {k: v[0] for k, v in om.items()}
    for pred in (False, True):
        mg, mo = gm[pred][1], om[pred][1]
        assert abs(mg - mo) < 1e-2 * abs(mo), (pred, mg, mo)
    assert abs(g[True]) < 1e-3 and abs(o[True]) < 1e-3, (g, o)
    assert abs(g[False]) > 20 * abs(g[True]), g
    for pred in (False, True):
        if pred:
            # both tiny: the FP32 ledger's own floor (GMRES at 1e-6) sets the scale
            assert abs(g[pred] - o[pred]) < 5e-4, (g, o)
        else:
            assert o[pred] < 0 and g[pred] < 0, (g, o)
            assert 1 / 1.5 < g[pred] / o[pred] < 1.5, (g, o)
