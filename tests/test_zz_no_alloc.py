"""The allocation-free kinetic energy entry point agrees with the energy ledger.

relsim_kinetic_energy_noalloc is for callers that cannot allocate device
memory where they need the kinetic energy: a diagnostics hook inside a time
loop whose device memory is all reserved up front by its own pool, or code
where a cudaMalloc would synchronise the device or is not allowed. It keeps
its partial sums in a fixed array inside the library. Here it must return,
on two calls in a row, the per-species kinetic energy that relsim_energy_ledger
reports for a context holding the same particles and an independent numpy
FP64 sum of w m |u|^2/(gamma + 1) on the host (FP64 tolerance 1e-11
relative), and it must refuse more particles than its fixed array can take. This file is collected last so that a failure here comes after every
other test has run.
"""
import ctypes
import math

import numpy as np
import pytest

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


def states():
    from relsim_inputs import HarrisConfig, make_harris, random_state
    yield "harris", 64, 32, make_harris(HarrisConfig(nx=64, ny=32, ppc=16)), (1.0, -1.0), (1.0, 1.0)
    # one species spanning many blocks and a partial last block
    yield ("random", 40, 30, random_state(40, 30, [1_500_001, 777], seed=12, u_scale=2.0),
           (1.0, -1.0), (1.0, 3.0))


def test_noalloc_matches_ledger_two_calls(rs):
    import torch
    for name, nx, ny, st, q, m in states():
        cfg = rs.make_config(nx, ny, dt=0.5, precision=64, q=q, m=m)
        sim = rs.Simulation(cfg)
        sim.load_state(st)
        led = sim.ledger()
        for s, sp in enumerate(st["species"]):
            u = torch.tensor(np.stack([sp["ux"], sp["uy"], sp["uz"]], axis=1), device="cuda")
            w = torch.tensor(np.asarray(sp["w"]), device="cuda")
            out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            vals = []
            for call in range(2):
                out.fill_(float("nan"))
                code = rs.relsim_kinetic_energy_noalloc(u, w, m[s], out)
                torch.cuda.synchronize()
                assert code == rs.RELSIM_OK, (name, s, code)
                vals.append(out.item())
            K = led["K_species"][s]
            assert abs(vals[0] - K) <= 1e-11 * abs(K), (name, s, vals[0], K)
            # an independent host sum, compensated (math.fsum)
            uu = np.stack([sp["ux"], sp["uy"], sp["uz"]], axis=1).astype(np.float64)
            u2 = (uu * uu).sum(axis=1)
            K_np = math.fsum(np.asarray(sp["w"], np.float64) * m[s] * (u2 / (np.sqrt(1.0 + u2) + 1.0)))
            assert abs(vals[0] - K_np) <= 1e-11 * abs(K_np), (name, s, vals[0], K_np)
            assert vals[1] == vals[0], (name, s, vals)
        sim.close()


def test_noalloc_refuses_too_many_particles_and_handles_empty(rs):
    import torch
    u = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    w = torch.zeros(4, dtype=torch.float64, device="cuda")
    out = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
    L = rs.lib()
    # the size check happens on the host before anything touches the arrays
    code = L.relsim_kinetic_energy_noalloc(ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(w.data_ptr()),
                                           rs.RELSIM_NOALLOC_MAX_PARTICLES + 1, 1.0,
                                           ctypes.c_void_p(out.data_ptr()), None)
    assert code == rs.RELSIM_ERR_TOO_LARGE
    assert L.relsim_kinetic_energy_noalloc(None, None, -1, 1.0, ctypes.c_void_p(out.data_ptr()), None) \
        == rs.RELSIM_ERR_INVALID_ARG
    code = L.relsim_kinetic_energy_noalloc(None, None, 0, 1.0, ctypes.c_void_p(out.data_ptr()), None)
    torch.cuda.synchronize()
    assert code == rs.RELSIM_OK and out.item() == 0.0
