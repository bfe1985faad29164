"""The particles in the library's own form (relsim_get_particles_native /
relsim_load_particles_native) on the GPU.

* A state read out in this form and loaded into a fresh context is the
  same state bit for bit (both records, the start table, ids), in the FP32
  and FP64 forms, 2D and 3D, from host and from device arrays; it then
  steps as the original to the form's tolerance (the deposit's atomic
  additions land in a different order in another context, so the two runs
  are not bitwise equal after a step: FP32 2e-5, FP64 1e-10 relative to the
  largest entry).
* The form agrees with the FP64 record: absolute position = (cell index +
  offset) x cell size, exactly, for every particle; momenta and weights
  equal; the start table equals relsim_get_cell_start.
* Ids: carried through a native load, or 0..n-1 when none are given.
* The device check: a start table that does not end at n or decreases, an
  offset of 1.0 or below 0, a NaN momentum, an id out of range each fail
  with the documented code and leave the species empty.
"""
import numpy as np
import pytest

from relsim_inputs import HarrisConfig, HarrisConfig3, make_harris, make_harris3

pytestmark = pytest.mark.gpu

NX, NY = 24, 12


@pytest.fixture(scope="module")
def rs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_11100_gb300 as rs
    return rs


def sim2(rs, prec, ids=True):
    cfg = rs.make_config(NX, NY, dt=0.5, theta_implicit=0.5, precision=prec,
                         gmres_tol=1e-6 if prec == 32 else 1e-12, track_ids=ids)
    return rs.Simulation(cfg)


def harris2():
    return make_harris(HarrisConfig(nx=NX, ny=NY, ppc=8, dt=0.5, pert=0.05))


def snapshot(sim, nsp, by_id=False):
    """Fields and both records; by_id: particles in id order (two runs that
    differ by rounding may sort a particle at a cell line differently)."""
    E, B = sim.fields()
    parts = []
    for s in range(nsp):
        x, u, w, i = sim.particles(s, ids=True)
        if by_id:
            o = np.argsort(i, kind="stable")
            x, u, w, i = x[o], u[o], w[o], i[o]
        parts.append((x, u, w, i))
    return E, B, parts


def same(a, b, tol=0.0):
    assert len(a) == len(b)
    for x, y in zip(a, b):
        if isinstance(x, (list, tuple)):
            same(x, y, tol)
        elif tol == 0.0 or np.asarray(x).dtype.kind in "iu":
            assert np.array_equal(np.asarray(x), np.asarray(y))
        else:
            x, y = np.asarray(x, np.float64), np.asarray(y, np.float64)
            assert np.abs(x - y).max() <= tol * max(np.abs(y).max(), 1e-300)


def native_same(a, b, nsp):
    for s in range(nsp):
        same(a.particles_native(s, ids=True), b.particles_native(s, ids=True))


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("device", [False, True])
def test_native_round_trip(rs, prec, device):
    st = harris2()
    a = sim2(rs, prec)
    a.load_state(st)
    a.step()
    b = sim2(rs, prec)
    b.set_fields(*a.fields())
    for s in range(2):
        b.load_species_native(s, *a.particles_native(s, ids=True, device=device))
    same(snapshot(a, 2), snapshot(b, 2))
    native_same(a, b, 2)
    for _ in range(3):
        a.step()
        b.step()
    tol = 2e-5 if prec == 32 else 1e-10
    same(snapshot(a, 2, True), snapshot(b, 2, True), tol)
    la, lb = a.ledger(), b.ledger()
    for k in ("W_E", "W_B", "K", "total", "work_grid", "work_particles"):
        assert abs(la[k] - lb[k]) <= tol * abs(la["total"]), k
    a.close()
    b.close()


@pytest.mark.parametrize("prec", [32, 64])
def test_native_form_equals_fp64_record(rs, prec):
    st = harris2()
    a = sim2(rs, prec)
    a.load_state(st)
    a.step()
    for s in range(2):
        start, off, u, w, ids = a.particles_native(s, ids=True)
        x, u64, w64, ids64 = a.particles(s, ids=True)
        n = w.shape[0]
        assert start.dtype == np.int32 and start.shape == (NX * NY + 1,)
        assert off.dtype == (np.float32 if prec == 32 else np.float64) and off.shape == (2, n)
        assert start[0] == 0 and start[-1] == n and np.all(np.diff(start) >= 0)
        assert np.array_equal(start.astype(np.int64), a.cell_start(s))
        cell = np.repeat(np.arange(NX * NY), np.diff(start))
        i, j = cell % NX, cell // NX
        assert np.all((off >= 0) & (off < 1))
        # absolute positions (cell size 1 here): FP64 sums of an integer and an offset
        assert np.array_equal(x[:, 0], i + off[0].astype(np.float64))
        assert np.array_equal(x[:, 1], j + off[1].astype(np.float64))
        assert np.array_equal(u64, u.T.astype(np.float64))
        assert np.array_equal(w64, w.astype(np.float64))
        assert np.array_equal(ids64, ids)
    a.close()


def test_native_ids_carried_or_counted(rs):
    st = harris2()
    a = sim2(rs, 32)
    a.load_state(st)
    a.step()   # the re-sort moves particles, so the ids are no longer 0..n-1
    start, off, u, w, ids = a.particles_native(0, ids=True)
    assert not np.array_equal(ids, np.arange(len(ids)))
    b = sim2(rs, 32)
    b.load_species_native(0, start, off, u, w, ids)
    assert np.array_equal(b.particles_native(0, ids=True)[4], ids)
    b.load_species_native(0, start, off, u, w)
    assert np.array_equal(b.particles_native(0, ids=True)[4], np.arange(len(ids), dtype=np.int32))
    a.close()
    b.close()


def test_native_check_rejects_bad_state(rs):
    st = harris2()
    a = sim2(rs, 32)
    a.load_state(st)
    start, off, u, w, ids = a.particles_native(0, ids=True)
    n = w.shape[0]
    b = sim2(rs, 32)

    def expect(code, **kw):
        args = dict(start=start, off=off, u=u, w=w, ids=ids)
        args.update(kw)
        with pytest.raises(rs.RelsimError) as e:
            b.load_species_native(0, args["start"], args["off"], args["u"], args["w"], args["ids"])
        assert e.value.code == code
        assert rs.relsim_num_particles(b.ctx, 0) == 0
        assert np.all(b.cell_start(0) == 0)
        # a good load still works after a rejected one
        b.load_species_native(0, start, off, u, w, ids)
        assert rs.relsim_num_particles(b.ctx, 0) == n

    bad = start.copy()
    bad[-1] = n - 1
    expect(-1, start=bad)
    bad = start.copy()
    k = int(np.argmax(np.diff(start) > 0))   # a cell with particles
    bad[k + 1] = bad[k + 2] + 1
    expect(-1, start=bad)
    for val in (1.0, -1e-7, np.nan):
        o = off.copy()
        o[1, n // 2] = val
        expect(-1, off=o)
    uu = u.copy()
    uu[2, 7] = np.nan
    expect(-6, u=uu)
    ww = w.copy()
    ww[-1] = np.inf
    expect(-6, w=ww)
    ii = ids.copy()
    ii[3] = n
    expect(-1, ids=ii)
    a.close()
    b.close()


def test_native_round_trip_3d(rs):
    hc = HarrisConfig3(nx=12, ny=8, nz=6, ppc=4, dt=0.5)
    st = make_harris3(hc)
    cfg = rs.make_config(12, 8, nz=6, dt=0.5, theta_implicit=0.5, precision=32, gmres_tol=1e-6, track_ids=True)
    a = rs.Simulation(cfg)
    a.load_state(st)
    a.step()
    b = rs.Simulation(cfg)
    b.set_fields(*a.fields())
    for s in range(2):
        start, off, u, w, ids = a.particles_native(s, ids=True)
        assert off.shape[0] == 3
        b.load_species_native(s, start, off, u, w, ids)
    same(snapshot(a, 2), snapshot(b, 2))
    native_same(a, b, 2)
    for _ in range(2):
        a.step()
        b.step()
    same(snapshot(a, 2, True), snapshot(b, 2, True), 2e-5)
    a.close()
    b.close()
