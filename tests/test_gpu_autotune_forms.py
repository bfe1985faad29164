"""The launch-shape autotuner on the 3D form and on the quadratic shapes.

It times the deposit's block count (2, 4, 8, 16 blocks per SM) and the
push's grid cap (4, 8, 16, 32 per SM) on the loaded state; the operator has
one tile shape in these forms, so no operator shape is tried. The choice
only changes launch shapes: after it, steps agree with an untuned context's
to rounding (the deposit's float atomics, and the counting sort's order
within a cell, so particles are compared by id), and the GMRES iteration
counts agree within one. A choice applied to another context by
relsim_set_launch_shapes gives the same agreement.
"""
import numpy as np
import pytest

from relsim_inputs import HarrisConfig, HarrisConfig3, make_harris, make_harris3

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


def setup(rs, form):
    if form == "3d":
        st = make_harris3(HarrisConfig3(nx=16, ny=12, nz=8, ppc=6, dt=0.5))
        cfg = rs.make_config(16, 12, nz=8, dt=0.5, precision=32, gmres_tol=1e-7, track_ids=True)
        return st, cfg, np.array([16.0, 12.0, 8.0])
    st = make_harris(HarrisConfig(nx=40, ny=20, ppc=12, dt=0.5, pert=0.05))
    cfg = rs.make_config(40, 20, dt=0.5, precision=32, gmres_tol=1e-7, track_ids=True, shape=2)
    return st, cfg, np.array([40.0, 20.0])


def by_id(sim, s):
    x, u, w, i = sim.particles(s, ids=True)
    o = np.argsort(i)
    return x[o], u[o], w[o]


@pytest.mark.parametrize("form", ["3d", "quadratic"])
def test_autotune_3d_and_quadratic(rs, form):
    st, cfg, L = setup(rs, form)
    sims = [rs.Simulation(cfg) for _ in range(3)]
    for s in sims:
        s.load_state(st)
    t = sims[0].autotune()
    assert len(t["deposit"]) == 4 and all(ms > 0 for _, ms in t["deposit"] + t["push"])
    assert t["deposit_blocks"] in [b for b, _ in t["deposit"]]
    assert t["push_blocks"] in [b for b, _ in t["push"]]
    assert t["op_tile_rows"] == []
    # the tuned shapes applied to the third context (the push's block count
    # as its cap gives the same grid); the second stays untuned
    sims[2].set_launch_shapes(t["deposit_blocks"], t["push_blocks"], 0)
    its = [[], [], []]
    for _ in range(3):
        for k, s in enumerate(sims):
            led, code = s.step()
            assert code == 0
            its[k].append(led["gmres_iters"])
    assert all(abs(a - b) <= 1 for a, b in zip(its[0], its[1]))
    for k in (0, 2):
        for a, b in zip(sims[k].fields(), sims[1].fields()):
            assert np.max(np.abs(a - b)) <= 2e-5 * np.abs(b).max()
        for s in range(2):
            xa, ua, wa = by_id(sims[k], s)
            xb, ub, wb = by_id(sims[1], s)
            assert np.max(np.abs(ua - ub)) <= 2e-5 * np.abs(ub).max()
            d = np.abs(xa - xb)   # periodic: a particle may sit across the box edge
            assert np.max(np.minimum(d, L - d)) <= 1e-4
            assert np.array_equal(wa, wb)
    assert sims[0].graph_info()["graph_steps"] == 2
    for s in sims:
        s.close()
