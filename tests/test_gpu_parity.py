"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Both sides get the same seeded inputs from relsim_inputs; nothing the CUDA
path computes is fed to the oracle. Tolerances:
* integer work (cell sort, cell starts): bit-exact;
* FP64 form: 1e-11 relative to the largest entry (the two sides differ only
  in summation order and in the GMRES iterate, both solved to 1e-12);
* FP32 form: inputs are FP32-representable; per-entry sums of O(100)
  products carry ~1e-7 relative rounding each, so 2e-5 of the largest entry
  (deposit, operator, one-step fields and momenta) is the bound used.
"""
import math

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


def fp32_state(st, nx, ny, dx=1.0, dy=1.0):
    """Round a state so that cell offsets, momenta, weights and fields are
    exactly representable in FP32 (both sides then start identical)."""
    for sp in st["species"]:
        for k, d in (("x", dx), ("y", dy)):
            s = np.asarray(sp[k]) / d
            fl = np.floor(s)
            f = (s - fl).astype(np.float32).astype(np.float64)
            f = np.minimum(f, np.float64(np.nextafter(np.float32(1.0), np.float32(0.0))))
            sp[k] = (fl + f) * d
        for k in ("ux", "uy", "uz", "w"):
            sp[k] = np.asarray(sp[k]).astype(np.float32).astype(np.float64)
    st["E"] = np.asarray(st["E"]).astype(np.float32).astype(np.float64)
    st["B"] = np.asarray(st["B"]).astype(np.float32).astype(np.float64)
    return st


def make_sim(rs, nx, ny, prec, dt=0.5, dx=1.0, dy=1.0, theta=0.5, q=(1.0, -1.0), m=(1.0, 1.0),
             tol=None, restart=0, ids=True):
    if tol is None:
        tol = 1e-12 if prec == 64 else 1e-7
    cfg = rs.make_config(nx, ny, dx=dx, dy=dy, dt=dt, theta_implicit=theta, precision=prec, q=q, m=m,
                         gmres_tol=tol, gmres_restart=restart, track_ids=ids)
    return rs.Simulation(cfg)


def ocfg(orc, nx, ny, dt=0.5, dx=1.0, dy=1.0, theta=0.5, q=(1.0, -1.0), m=(1.0, 1.0), tol=1e-12):
    return orc.make_config(nx, ny, dx=dx, dy=dy, dt=dt, theta=theta, q=q, m=m, gmres_tol=tol,
                           gmres_restart=50)


def rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def tol_for(prec):
    return 1e-11 if prec == 64 else 2e-5


def half_from_full(Mfull, nx, ny):
    nn = nx * ny
    out = np.zeros((nn, 5, 3, 3))
    for k, (di, dj) in enumerate(HALF):
        out[:, k] = Mfull[:, (dj + 1) * 3 + (di + 1)]
    return out


# ---------------------------------------------------------------------------
# cell sort (integer, bit-exact)

@pytest.mark.parametrize("prec", [32, 64])
def test_load_sort_is_oracle_stable_sort(rs, orc, prec):
    nx, ny = 13, 7   # ragged: not a multiple of any tile
    st = random_state(nx, ny, [3001, 1], seed=11)
    # many particles share cells: duplicates of a few positions
    sp = st["species"][0]
    sp["x"][::7] = sp["x"][3]
    sp["y"][::7] = sp["y"][3]
    sim = make_sim(rs, nx, ny, prec)
    sim.load_state(st)
    c = ocfg(orc, nx, ny)
    for s, n in ((0, 3001), (1, 1)):
        keys = orc.cell_keys(c, st["species"][s]["x"], st["species"][s]["y"])
        perm, start = orc.stable_sort(keys, nx * ny)
        x, u, w, ids = sim.particles(s, ids=True)
        np.testing.assert_array_equal(ids, perm)
        np.testing.assert_array_equal(sim.cell_start(s), start)
        np.testing.assert_array_equal(w, np.asarray(st["species"][s]["w"])[perm]
                                      .astype(np.float32 if prec == 32 else np.float64))
    sim.close()


def test_empty_species_and_single_cell(rs, orc):
    nx, ny = 5, 4
    sim = make_sim(rs, nx, ny, 32)
    n = 257
    x = np.stack([np.full(n, 2.25), np.full(n, 1.5)], axis=1)
    u = np.zeros((n, 3))
    w = np.ones(n)
    sim.load_species(0, x, u, w)
    sim.load_species(1, np.zeros((0, 2)), np.zeros((0, 3)), np.zeros(0))
    rs.relsim_set_fields(sim.ctx, np.zeros((3, 20)), np.zeros((3, 20)))
    start = sim.cell_start(0)
    assert start[1 * nx + 2] == 0 and start[1 * nx + 3] == n and start[-1] == n
    assert sim.cell_start(1)[-1] == 0
    led, status = sim.step()
    assert status == 0 and led["n_particles"] == n
    # a cold, field-free plasma stays put
    x1, u1, w1, ids = sim.particles(0, ids=True)
    np.testing.assert_array_equal(u1, 0.0)
    np.testing.assert_allclose(x1, x, atol=1e-6)
    sim.close()


# ---------------------------------------------------------------------------
# deposit

def harris_small(nx=64, ny=32, ppc=4, seed=0):
    return make_harris(HarrisConfig(nx=nx, ny=ny, ppc=ppc, seed=seed))


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("case", ["tiny", "ragged", "harris"])
def test_deposit_matches_oracle(rs, orc, prec, case):
    if case == "tiny":
        nx, ny, dt = 3, 3, 0.7
        st = random_state(nx, ny, [40, 25], seed=5, u_scale=2.0, field_scale=1.5)
    elif case == "ragged":
        nx, ny, dt = 37, 11, 0.9
        st = random_state(nx, ny, [5000, 4000], seed=6, u_scale=1.0)
    else:
        nx, ny, dt = 64, 32, 0.5
        st = harris_small(nx, ny, 16)
    st = fp32_state(st, nx, ny)
    q, m = (1.0, -1.0), (1.0, 1.0)
    sim = make_sim(rs, nx, ny, prec, dt=dt, q=q, m=m)
    sim.load_state(st)
    sim.build()
    M, J = sim.mass_matrix()
    c = ocfg(orc, nx, ny, dt=dt, q=q, m=m)
    Jo, Mo = orc.deposit(c, orc.Particles(st["species"]), st["B"])
    Mh = half_from_full(Mo, nx, ny)
    assert rel(M, Mh) < tol_for(prec)
    assert rel(J, Jo) < tol_for(prec)
    sim.close()


# ---------------------------------------------------------------------------
# implicit operator, field solve

@pytest.mark.parametrize("prec", [32, 64])
def test_operator_matches_oracle(rs, orc, prec):
    nx, ny, dt = 19, 9, 0.8
    st = fp32_state(random_state(nx, ny, [800, 800], seed=7, u_scale=1.0, field_scale=1.0), nx, ny)
    c = ocfg(orc, nx, ny, dt=dt)
    Jo, Mo = orc.deposit(c, orc.Particles(st["species"]), st["B"])
    Mh = half_from_full(Mo, nx, ny).astype(np.float32).astype(np.float64)
    Jo = Jo.astype(np.float32).astype(np.float64)
    # rebuild the full-offset matrix from the rounded halves for the oracle
    Mfull = np.zeros_like(Mo)
    for k, (di, dj) in enumerate(HALF):
        Mfull[:, (dj + 1) * 3 + di + 1] = Mh[:, k]
        if k:
            idx = np.arange(nx * ny)
            i, j = idx % nx, idx // nx
            nb = ((j + dj) % ny) * nx + (i + di) % nx
            Mfull[nb, (-dj + 1) * 3 - di + 1] = Mh[:, k]
    sim = make_sim(rs, nx, ny, prec, dt=dt)
    sim.load_state(st)
    sim.set_mass_matrix(Mh, Jo)
    v = np.random.default_rng(3).normal(size=(3, nx * ny)).astype(np.float32).astype(np.float64)
    Av = sim.apply_operator(v)
    Avo = orc.apply_A(c, Mfull, v)
    assert rel(Av, Avo) < (1e-13 if prec == 64 else 2e-6)
    sim.close()


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("theta", [0.5, 0.7])
def test_field_solve_matches_oracle(rs, orc, prec, theta):
    nx, ny, dt = 64, 32, 0.5
    st = fp32_state(harris_small(nx, ny, 8), nx, ny)
    sim = make_sim(rs, nx, ny, prec, dt=dt, theta=theta, restart=7 if prec == 64 else 0)
    sim.load_state(st)
    sim.build()
    it, relres, status = sim.solve()
    assert status == 0
    Eth = sim.E_theta()
    E1, B1 = sim.fields()
    c = ocfg(orc, nx, ny, dt=dt, theta=theta)
    P = orc.Particles(st["species"])
    Eo, Bo, lo, ex = orc.step(c, P, st["E"], st["B"], want_matrices=True)
    t = 1e-9 if prec == 64 else 2e-5
    assert rel(Eth, ex["Etheta"]) < t
    assert rel(E1, Eo) < t * (1 / theta)
    assert rel(B1, Bo) < t
    if prec == 64:
        assert relres < 1e-12 and it >= 7   # restarts were exercised
    sim.close()


# ---------------------------------------------------------------------------
# push and full steps

@pytest.mark.parametrize("prec", [32, 64])
def test_one_step_particles_match_oracle(rs, orc, prec):
    nx, ny, dt = 64, 32, 0.5
    st = fp32_state(harris_small(nx, ny, 8), nx, ny)
    sim = make_sim(rs, nx, ny, prec, dt=dt)
    sim.load_state(st)
    led, status = sim.step()
    assert status == 0
    c = ocfg(orc, nx, ny, dt=dt)
    P = orc.Particles(st["species"])
    Eo, Bo, lo, _ = orc.step(c, P, st["E"], st["B"])
    t = 1e-11 if prec == 64 else 2e-5
    Lx, Ly = nx * 1.0, ny * 1.0
    for s in range(2):
        x, u, w, ids = sim.particles(s, ids=True)
        o = P.species(s)
        uo = np.stack([o["ux"], o["uy"], o["uz"]], axis=1)[ids]
        xo = np.stack([o["x"], o["y"]], axis=1)[ids]
        assert rel(u, uo) < t
        d = x - xo
        d[:, 0] = (d[:, 0] + Lx / 2) % Lx - Lx / 2
        d[:, 1] = (d[:, 1] + Ly / 2) % Ly - Ly / 2
        assert np.abs(d).max() < (1e-11 if prec == 64 else 2e-5)
        # the sort after the push is the stable sort of the new cells
        keys = (np.floor(x[:, 1]).astype(np.int64) * nx + np.floor(x[:, 0]).astype(np.int64))
        assert np.all(np.diff(keys) >= 0)
    # ledger terms
    tt = 1e-9 if prec == 64 else 1e-5
    assert abs(led["K"] - lo["K1"]) < tt * lo["K1"]
    assert abs(led["W_B"] - lo["W_B1"]) < tt * lo["W_B1"]
    assert abs(led["work_grid"] - lo["work_grid"]) < (1e-9 if prec == 64 else 1e-3) * abs(lo["work_grid"])
    assert abs(led["mismatch"] - lo["mismatch"]) < (1e-8 if prec == 64 else 1e-2) * abs(lo["mismatch"])
    sim.close()


def test_fp64_ten_steps_match_oracle(rs, orc):
    nx, ny, dt = 64, 32, 0.5
    st = harris_small(nx, ny, 16)
    sim = make_sim(rs, nx, ny, 64, dt=dt)
    sim.load_state(st)
    c = ocfg(orc, nx, ny, dt=dt)
    P = orc.Particles(st["species"])
    E, B = st["E"], st["B"]
    for n in range(10):
        led, status = sim.step()
        E, B, lo, _ = orc.step(c, P, E, B)
        assert status == 0
        assert abs(led["residual"] - lo["residual"]) < 1e-9 * lo["W_B1"]
    Eg, Bg = sim.fields()
    assert rel(Eg, E) < 1e-8
    assert rel(Bg, B) < 1e-9
    x, u, w, ids = sim.particles(0, ids=True)
    o = P.species(0)
    assert rel(u, np.stack([o["ux"], o["uy"], o["uz"]], axis=1)[ids]) < 1e-8
    sim.close()


def test_fp32_error_curve_config0(rs, orc):
    """FP32 form vs FP64 oracle on the 64x32 Harris sheet, 16 ppc per species,
    100 steps. Orbits in the sheet are chaotic, so any round-off grows
    exponentially (about e-fold per 12 steps here). Checked: (a) the 1e-5
    relative field error holds over the steps where the divergence has not
    yet grown (B through step 50, E through step 30); (b) at every step the
    FP32 error is within 10x of the error between the oracle and the oracle
    started from momenta perturbed at the FP32 rounding level (6e-8), i.e.
    the FP32 path adds nothing beyond the conditioning of the dynamics."""
    nx, ny, dt = 64, 32, 0.5
    st = fp32_state(harris_small(nx, ny, 16), nx, ny)
    sim = make_sim(rs, nx, ny, 32, dt=dt, tol=1e-7)
    sim.load_state(st)
    c = ocfg(orc, nx, ny, dt=dt)
    P = orc.Particles(st["species"])
    Pp = P.copy()
    rng = np.random.default_rng(1)
    for k in ("ux", "uy", "uz"):
        a_ = getattr(Pp, k)
        a_ *= 1.0 + 6e-8 * rng.choice([-1.0, 1.0], size=a_.size)
    E, B = st["E"], st["B"]
    Ep, Bp = st["E"], st["B"]
    errs = []
    for n in range(100):
        led, status = sim.step(ledger=False)
        E, B, lo, _ = orc.step(c, P, E, B)
        Ep, Bp, _, _ = orc.step(c, Pp, Ep, Bp)
        Eg, Bg = sim.fields()
        nE, nB = np.linalg.norm(E), np.linalg.norm(B)
        errs.append((n + 1, np.linalg.norm(Eg - E) / nE, np.linalg.norm(Bg - B) / nB,
                     np.linalg.norm(Ep - E) / nE, np.linalg.norm(Bp - B) / nB))
    msg = " ".join(f"{n}:{eE:.1e}/{eB:.1e}(pert {pE:.1e}/{pB:.1e})"
                   for n, eE, eB, pE, pB in errs[::10])
    assert all(eB < 1e-5 for n, _, eB, _, _ in errs if n <= 50), msg
    assert all(eE < 1e-5 for n, eE, _, _, _ in errs if n <= 30), msg
    for n, eE, eB, pE, pB in errs:
        assert eE <= 10 * max(pE, 1e-7) and eB <= 10 * max(pB, 1e-8), msg
    sim.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_long_move_general_sort_path(rs, orc, prec):
    # c dt > dx: particles may cross more than one cell per step
    nx, ny, dt, dx = 16, 12, 1.6, 0.5
    st = fp32_state(random_state(nx, ny, [2000, 2000], seed=8, dx=dx, dy=dx, u_scale=3.0,
                                 field_scale=0.3), nx, ny, dx, dx)
    sim = make_sim(rs, nx, ny, prec, dt=dt, dx=dx, dy=dx)
    sim.load_state(st)
    c = ocfg(orc, nx, ny, dt=dt, dx=dx, dy=dx)
    P = orc.Particles(st["species"])
    E, B = st["E"], st["B"]
    for n in range(2):
        led, status = sim.step()
        E, B, lo, _ = orc.step(c, P, E, B)
    x, u, w, ids = sim.particles(1, ids=True)
    o = P.species(1)
    assert rel(u, np.stack([o["ux"], o["uy"], o["uz"]], axis=1)[ids]) < (1e-10 if prec == 64 else 1e-4)
    keys = np.floor(x[:, 1] / dx).astype(np.int64) * nx + np.floor(x[:, 0] / dx).astype(np.int64)
    assert np.all(np.diff(keys) >= 0)
    sim.close()


def test_per_step_sort_is_stable(rs, orc):
    nx, ny = 32, 16
    st = fp32_state(harris_small(nx, ny, 8), nx, ny)
    sim = make_sim(rs, nx, ny, 32, dt=0.9)
    sim.load_state(st)
    for n in range(3):
        _, _, _, ids0 = sim.particles(0, ids=True)
        sim.step(ledger=False)
        x1, _, _, ids1 = sim.particles(0, ids=True)
        # new keys listed in the previous order, then stably sorted by the oracle
        keys_new = (np.floor(x1[:, 1]).astype(np.int64) * nx + np.floor(x1[:, 0]).astype(np.int64))
        pos_of = np.empty(len(ids1), dtype=np.int64)
        pos_of[ids1] = np.arange(len(ids1))
        keys_in_prev_order = keys_new[pos_of[ids0]].astype(np.int32)
        perm, start = orc.stable_sort(keys_in_prev_order, nx * ny)
        np.testing.assert_array_equal(ids0[perm], ids1)
        np.testing.assert_array_equal(sim.cell_start(0), start)
    sim.close()


@pytest.mark.parametrize("case", ["cell", "row"])
def test_crowded_cell_sort_is_stable(rs, orc, case):
    # "cell": one cell holds far more particles than a warp stages at once
    # (the two-pass big-cell path of the push); "row": one row of cells holds
    # more particles than the deposit's staging buffer (the permutation goes
    # through global memory). Particles leave in every direction; a second
    # step runs the deposit that completes the first step's sort.
    nx, ny, dt = 8, 8, 0.9
    rng = np.random.default_rng(11)
    nbig, nrest = (400, 300) if case == "cell" else (4000, 300)
    lo, span = ((3.0, 3.0), (1.0, 1.0)) if case == "cell" else ((0.0, 3.0), (nx, 1.0))
    x = np.concatenate([np.array(lo) + rng.random((nbig, 2)) * span, rng.random((nrest, 2)) * [nx, ny]])
    u = rng.normal(scale=1.5, size=(nbig + nrest, 3))
    w = rng.random(nbig + nrest) + 0.5
    st = {"species": [dict(x=x[:, 0], y=x[:, 1], ux=u[:, 0], uy=u[:, 1], uz=u[:, 2], w=w)] * 2,
          "E": rng.normal(scale=0.1, size=(3, nx * ny)), "B": rng.normal(scale=0.5, size=(3, nx * ny))}
    st = fp32_state(st, nx, ny)
    sim = make_sim(rs, nx, ny, 32, dt=dt)
    sim.load_state(st)
    counts = np.diff(sim.cell_start(0))
    assert (counts.max() if case == "cell" else counts.reshape(ny, nx).sum(axis=1).max()) >= nbig
    _, _, _, ids0 = sim.particles(0, ids=True)
    led, status = sim.step()
    assert status == 0
    # the next deposit completes this step's sort (fused) before anything reads
    # the particles
    sim.build()
    M, J = sim.mass_matrix()
    x1, u1, _, ids1 = sim.particles(0, ids=True)
    keys_new = (np.floor(x1[:, 1]).astype(np.int64) * nx + np.floor(x1[:, 0]).astype(np.int64))
    pos_of = np.empty(len(ids1), dtype=np.int64)
    pos_of[ids1] = np.arange(len(ids1))
    perm, start = orc.stable_sort(keys_new[pos_of[ids0]].astype(np.int32), nx * ny)
    np.testing.assert_array_equal(ids0[perm], ids1)
    np.testing.assert_array_equal(sim.cell_start(0), start)
    # the pushed momenta and the next deposit are the oracle's
    c = ocfg(orc, nx, ny, dt=dt)
    P = orc.Particles(st["species"])
    E1o, B1o, _, _ = orc.step(c, P, st["E"], st["B"])
    o = P.species(0)
    assert rel(u1, np.stack([o["ux"], o["uy"], o["uz"]], axis=1)[ids1]) < 2e-5
    Jo, Mo = orc.deposit(c, P, B1o)
    assert rel(M, half_from_full(Mo, nx, ny)) < 1e-4
    assert rel(J, Jo) < 1e-4
    sim.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_spectrum_matches_oracle(rs, orc, prec):
    nx, ny, dt = 64, 32, 0.5
    st = harris_small(nx, ny, 16)
    sim = make_sim(rs, nx, ny, prec, dt=dt)
    sim.load_state(st)
    for _ in range(2):
        sim.step(ledger=False)
    edges0 = np.geomspace(1e-2, 1e4, 257)    # 256 log bins of gamma - 1
    edges1 = np.geomspace(1e-3, 1e3, 97)     # 96 log bins of |u|
    for s in range(2):
        x, u, w, ids = sim.particles(s, ids=True)
        for var, edges in ((0, edges0), (1, edges1)):
            wt, ct = sim.spectrum(s, edges, var)
            wo, co = orc.spectrum(u[:, 0], u[:, 1], u[:, 2], w, edges, var, prec)
            # the bin of every particle is decided exactly as the oracle does
            np.testing.assert_array_equal(ct, co)
            np.testing.assert_allclose(wt, wo, rtol=1e-12, atol=1e-12 * w.sum())
            assert ct.sum() == len(w)
    wd, cd = sim.spectrum(0, edges0, 0, device=True)
    np.testing.assert_array_equal(cd.cpu().numpy(), sim.spectrum(0, edges0, 0)[1])
    for bad in (np.array([1.0]), np.array([1.0, 1.0]), np.array([2.0, 1.0]), np.array([1.0, np.nan])):
        with pytest.raises(rs.RelsimError):
            sim.spectrum(0, bad, 0)
    with pytest.raises(rs.RelsimError):
        sim.spectrum(0, edges0, 2)
    sim.close()


def test_ledger_identity_on_gpu(rs):
    nx, ny = 64, 32
    st = harris_small(nx, ny, 16)
    for prec, bound in ((64, 1e-10), (32, 2e-5)):
        sim = make_sim(rs, nx, ny, prec, dt=0.5, tol=1e-12 if prec == 64 else 1e-7)
        sim.load_state(st)
        for n in range(5):
            led, status = sim.step()
            assert abs(led["residual"]) < bound * led["total"], (prec, led)
            assert abs(led["work_grid"] - led["work_particles"]) < bound * led["total"]
        sim.close()


def test_call_order_is_enforced(rs):
    sim = make_sim(rs, 8, 8, 32)
    sim.load_state(random_state(8, 8, 10, seed=1))
    with pytest.raises(rs.RelsimError) as e:
        sim.push()
    assert e.value.code == rs.RELSIM_ERR_BAD_STATE
    with pytest.raises(rs.RelsimError):
        sim.solve()
    sim.build()
    with pytest.raises(rs.RelsimError):
        sim.build()
    sim.solve()
    sim.push()
    sim.close()


def test_nonfinite_input_is_rejected(rs):
    sim = make_sim(rs, 8, 8, 32)
    x = np.array([[1.0, 1.0], [np.nan, 2.0]])
    with pytest.raises(rs.RelsimError) as e:
        sim.load_species(0, x, np.zeros((2, 3)), np.ones(2))
    assert e.value.code == rs.RELSIM_ERR_NONFINITE
    sim.close()


def test_not_converged_is_reported(rs):
    sim = make_sim(rs, 16, 8, 64, tol=1e-14)
    cfg = sim.cfg
    sim.close()
    cfg.gmres_maxit = 1
    sim = rs.Simulation(cfg)
    sim.load_state(harris_small(16, 8, 4))
    sim.build()
    it, relres, status = sim.solve()
    assert status == rs.RELSIM_ERR_NOT_CONVERGED and it == 1
    sim.push()   # the state still advances
    sim.close()


def test_device_pointers_roundtrip(rs):
    import torch
    nx, ny = 16, 8
    st = harris_small(nx, ny, 4)
    sim = make_sim(rs, nx, ny, 32)
    sp = st["species"][0]
    x = torch.tensor(np.stack([sp["x"], sp["y"]], axis=1), device="cuda")
    u = torch.tensor(np.stack([sp["ux"], sp["uy"], sp["uz"]], axis=1), device="cuda")
    w = torch.tensor(sp["w"], device="cuda")
    sim.load_species(0, x, u, w)
    xd, ud, wd = sim.particles(0, device=True)
    xh, uh, wh = sim.particles(0)
    np.testing.assert_array_equal(xd.cpu().numpy(), xh)
    np.testing.assert_array_equal(ud.cpu().numpy(), uh)
    sim.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_graph_steps_match_host_driven_steps(rs, precision):
    """After the first step, relsim_step runs each step as one CUDA graph
    (the solve's loops as conditional while nodes). With event profiling on,
    the same steps are driven from the host. Both routes run the same
    kernels; the deposit's float atomics make their sums differ in the last
    bits, so the fields agree to rounding (FP64 1e-11, FP32 2e-5 of the
    largest entry after 3 steps) and the GMRES iteration counts match."""
    nx, ny = 24, 16
    st = harris_small(nx, ny, 4)
    sims = [make_sim(rs, nx, ny, precision) for _ in range(2)]
    for s in sims:
        s.load_state(st)
    sims[1].profile(True)   # host-driven route
    its = [[], []]
    for _ in range(4):
        for k, s in enumerate(sims):
            led, code = s.step(ledger=True)
            assert code == 0
            its[k].append(led["gmres_iters"])
    info = sims[0].graph_info()
    assert not info["disabled"], info["why"]
    assert info["graph_steps"] == 3
    assert sims[1].graph_info()["graph_steps"] == 0
    # FP32: a residual estimate within rounding of the tolerance may stop
    # one iteration apart
    assert all(abs(a - b) <= (0 if precision == 64 else 1) for a, b in zip(*its)), its
    tol = 1e-11 if precision == 64 else 2e-5
    for a, b in zip(sims[0].fields(), sims[1].fields()):
        assert np.max(np.abs(a - b)) <= tol * np.abs(b).max()
    for s in range(2):
        xa, ua, wa = sims[0].particles(s)
        xb, ub, wb = sims[1].particles(s)
        assert np.max(np.abs(ua - ub)) <= tol * np.abs(ub).max()
    for s in sims:
        s.close()


def test_graph_step_after_reload_and_not_converged(rs):
    """A reload invalidates the captured graphs (new buffers and layout);
    NOT_CONVERGED is reported from a graph step as from a host-driven one."""
    nx, ny = 16, 8
    sim = make_sim(rs, nx, ny, 32)
    st = harris_small(nx, ny, 4)
    sim.load_state(st)
    for _ in range(3):
        _, code = sim.step()
        assert code == 0
    assert sim.graph_info()["graph_steps"] == 2
    sim.load_state(st)
    for _ in range(3):
        _, code = sim.step()
        assert code == 0
    assert sim.graph_info()["graph_steps"] == 4
    sim.close()
    cfg = rs.make_config(nx, ny, precision=32, gmres_tol=1e-14)
    cfg.gmres_maxit = 1
    sim = rs.Simulation(cfg)
    sim.load_state(st)
    for _ in range(3):
        led, code = sim.step()
        assert code == rs.RELSIM_ERR_NOT_CONVERGED and led["gmres_iters"] == 1
    assert sim.graph_info()["graph_steps"] == 2
    sim.close()


def test_autotuned_launch_shapes_give_the_same_steps(rs):
    """The autotuner only changes launch shapes: after it, steps agree with
    an untuned context's to rounding (the deposit's float atomics), with the
    same GMRES iteration counts, and the choice is one of the candidates."""
    nx, ny = 48, 24
    st = harris_small(nx, ny, 8)
    sims = [make_sim(rs, nx, ny, 32) for _ in range(2)]
    for s in sims:
        s.load_state(st)
    t = sims[0].autotune()
    assert t["deposit_blocks"] in [b for b, _ in t["deposit"]]
    assert t["push_blocks"] in [b for b, _ in t["push"]]
    assert all(ms > 0 for _, ms in t["deposit"] + t["push"])
    its = [[], []]
    for _ in range(4):
        for k, s in enumerate(sims):
            led, code = s.step()
            assert code == 0
            its[k].append(led["gmres_iters"])
    assert all(abs(a - b) <= 1 for a, b in zip(*its))
    for a, b in zip(sims[0].fields(), sims[1].fields()):
        assert np.max(np.abs(a - b)) <= 2e-5 * np.abs(b).max()
    x0, u0, w0 = sims[0].particles(0)[:3]
    x1, u1, w1 = sims[1].particles(0)[:3]
    assert np.max(np.abs(u0 - u1)) <= 2e-5 * np.abs(u1).max()
    built = make_sim(rs, nx, ny, 32)
    built.load_state(st)
    built.build()
    with pytest.raises(rs.RelsimError) as e:
        built.autotune()
    assert e.value.code == rs.RELSIM_ERR_BAD_STATE
    for s in sims + [built]:
        s.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_operator_tile_heights_agree(rs, prec):
    """The operator's two compiled tile heights (8 and 4 rows in FP32, 4 and
    2 in FP64) give the same A v on a grid with ragged tiles in both
    directions (41 x 19), bit for bit (each node's arithmetic is the same;
    only the tiling differs), and GMRES solves agree to rounding."""
    nx, ny = 41, 19
    st = harris_small(nx, ny, 8)
    sims = [make_sim(rs, nx, ny, prec) for _ in range(2)]
    alt = 4 if prec == 32 else 2
    v = np.random.default_rng(9).normal(size=(3, nx * ny))
    # one context, one deposited M, both tilings
    sims[0].load_state(st)
    sims[0].build()
    a0 = sims[0].apply_operator(v)
    sims[0].set_launch_shapes(0, 0, alt)
    a1 = sims[0].apply_operator(v)
    sims[0].set_launch_shapes(0, 0, 0)
    assert np.array_equal(a0, a1)
    # solves on two contexts (each with its own deposit) agree to rounding
    sims[1].set_launch_shapes(0, 0, alt)
    sims[1].load_state(st)
    sims[1].build()
    its = [s.solve()[0] for s in sims]
    assert abs(its[0] - its[1]) <= 1
    E0, E1 = sims[0].E_theta(), sims[1].E_theta()
    assert np.max(np.abs(E0 - E1)) <= (1e-6 if prec == 32 else 1e-12) * np.abs(E0).max()
    with pytest.raises(rs.RelsimError):
        sims[0].set_launch_shapes(0, 0, 3)
    for s in sims:
        s.close()


@pytest.mark.parametrize("case", ["harris", "ragged"])
def test_double_float_krylov_matches_fp64_krylov(rs, orc, case):
    """The FP32 form keeps its GMRES vectors as double-float pairs (FP32
    arithmetic, ~48-bit values) unless gmres_fp64 is set. Over ten steps the
    two agree: the same iteration counts (within one), E within the solve
    tolerance's reach (1e-5) and B within 5e-6, ledger residuals at the FP32
    floor, and both match the oracle's first solve (E^{n+theta}) to the FP32
    bound. The FP32 form's deposit adds the cells' mass-matrix and current
    sums into the nodes with atomics in no fixed order, so two runs of the
    same configuration differ too: over these ten steps by up to 9.4e-7 in B
    and 1.7e-6 in E on the ragged case (four runs each, both Krylov forms),
    as much as the two Krylov forms differ from each other; the B bound
    stands about five times above that spread."""
    if case == "harris":
        nx, ny, dt = 64, 32, 0.5
        st = fp32_state(harris_small(nx, ny, 16), nx, ny)
    else:
        nx, ny, dt = 37, 11, 0.7
        st = fp32_state(random_state(nx, ny, [900, 700], seed=21, u_scale=0.5, field_scale=0.3), nx, ny)
    res = {}
    for fp64 in (False, True):
        sim = rs.Simulation(rs.make_config(nx, ny, dt=dt, precision=32, gmres_tol=1e-7, gmres_fp64=fp64))
        sim.load_state(st)
        sim.build()
        it0, rr0, status = sim.solve()
        assert status == 0 and rr0 <= 1e-7
        Et0 = sim.E_theta()
        sim.push()
        iters, resid = [it0], []
        for _ in range(9):
            led, status = sim.step()
            assert status == 0
            iters.append(led["gmres_iters"])
            resid.append(abs(led["residual"]) / led["total"])
        E, B = sim.fields()
        res[fp64] = (np.array(iters), Et0, E, B, max(resid))
        sim.close()
    (itd, Etd, Ed, Bd, rd), (itf, Etf, Ef, Bf, rf) = res[False], res[True]
    print(f"{case}: GMRES iterations double-float {itd.tolist()}, FP64 {itf.tolist()}; "
          f"max ledger residual {rd:.1e} / {rf:.1e}")
    assert np.all(np.abs(itd - itf) <= 1), (itd, itf)
    assert rel(Ed, Ef) <= 1e-5 and rel(Bd, Bf) <= 5e-6
    assert rd < 1e-6 and rf < 1e-6
    c = ocfg(orc, nx, ny, dt=dt)
    P = orc.Particles(st["species"])
    _, _, _, ex = orc.step(c, P, st["E"], st["B"], want_matrices=True)
    for Et in (Etd, Etf):
        assert rel(Et, ex["Etheta"]) <= 2e-5
