"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares. No compute call is made (no GPU needed)."""
import ctypes
import glob
import os
import re
import shutil

import numpy as np

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(relsim_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def librelsim():
    import paper_2509_11100_gb300 as rs
    if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
        from paper_2509_11100_gb300 import build
        build.build()
    if not os.path.exists(rs.lib_path()):
        pytest.skip("librelsim.so not built and no nvcc available")
    return rs


def test_header_declares_the_step_api():
    names = declared_symbols()
    for must in ("relsim_init", "relsim_load_particles", "relsim_build_mass_matrix",
                 "relsim_field_solve", "relsim_push", "relsim_energy_ledger", "relsim_destroy",
                 "relsim_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(librelsim):
    L = ctypes.CDLL(librelsim.lib_path())
    missing = [n for n in declared_symbols() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_symbol(librelsim):
    for n in declared_symbols():
        assert hasattr(librelsim, n), n


def test_version_and_config_validation_without_gpu(librelsim):
    rs = librelsim
    assert rs.relsim_version() >= 100
    bad = [
        dict(nx=2, ny=8),                 # grid too small
        dict(nx=8, ny=8, precision=16),   # unsupported precision
        dict(nx=8, ny=8, dt=-1.0),
        dict(nx=8, ny=8, theta_implicit=0.0),
        dict(nx=8, ny=8, gmres_restart=101),
    ]
    for kw in bad:
        cfg = rs.make_config(**kw)
        ctx = ctypes.c_void_p()
        code = rs.lib().relsim_init(ctypes.byref(cfg), None, ctypes.byref(ctx))
        assert code == rs.RELSIM_ERR_INVALID_ARG and not ctx.value, kw
    cfg = rs.make_config(8, 8, m=(1.0, 0.0))
    ctx = ctypes.c_void_p()
    assert rs.lib().relsim_init(ctypes.byref(cfg), None, ctypes.byref(ctx)) == rs.RELSIM_ERR_INVALID_ARG
    cfg = rs.make_config(8, 8)
    cfg.dim = 3
    assert rs.lib().relsim_init(ctypes.byref(cfg), None, ctypes.byref(ctx)) == rs.RELSIM_ERR_INVALID_ARG


def test_null_arguments_are_rejected(librelsim):
    L = librelsim.lib()
    assert L.relsim_build_mass_matrix(None) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_push(None) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_energy_ledger(None, None) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_init(None, None, None) == librelsim.RELSIM_ERR_INVALID_ARG
    L.relsim_destroy(None)
    assert L.relsim_last_error(None) == b"null context"


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2509_11100_gb300 as rs
    monkeypatch.setattr(rs, "_lib", None)
    monkeypatch.setattr(rs, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(rs.RelsimUnavailable):
        rs.lib()


def test_dispersion_fit_host_code_matches_oracle(librelsim):
    # relsim_dispersion_fit is host code: it runs without a GPU. Noisy mode
    # energies of a tearing-like dispersion and one mode without a positive
    # window, against the oracle's per-mode fit and its dense-grid fit of b
    import oracle
    rng = np.random.default_rng(11)
    dt, n, nm, Lx, a = 0.5, 90, 9, 32.0, 1.0
    t = np.arange(n) * dt
    x = 2 * np.pi * np.arange(nm) * a / Lx
    g = 0.16 * x * 0.93 * (1 - (x * 0.93) ** 2)
    e = np.exp(2.0 * g[None, :] * t[:, None] + 0.05 * rng.normal(size=(n, nm))) * 1e-3
    e[30, 5] = -1.0
    for first, window in ((20, 60), (0, 90), (10, 2)):
        rates, A, b = librelsim.relsim_dispersion_fit(e, dt, first, window, Lx, a)
        orates, oA, ob = oracle.tearing_dispersion(e, dt, first, window, Lx, a)
        assert np.array_equal(np.isnan(rates), np.isnan(orates))
        ok = ~np.isnan(orates)
        assert np.allclose(rates[ok], orates[ok], rtol=1e-10, atol=1e-13)
        assert abs(b - ob) < 2e-5 * ob and abs(A - oA) < 1e-4 * abs(oA), (A, b, oA, ob)
    L = librelsim.lib()
    r = np.zeros(nm)
    A, b = ctypes.c_double(), ctypes.c_double()
    D = e.ctypes.data
    for args in [(None, n, nm, dt, 0, 10, Lx, a), (D, 1, nm, dt, 0, 10, Lx, a), (D, n, 2, dt, 0, 10, Lx, a),
                 (D, n, nm, 0.0, 0, 10, Lx, a), (D, n, nm, dt, -1, 10, Lx, a), (D, n, nm, dt, 85, 10, Lx, a),
                 (D, n, nm, dt, 0, 1, Lx, a), (D, n, nm, dt, 0, 10, 0.0, a), (D, n, nm, dt, 0, 10, Lx, float("nan"))]:
        assert L.relsim_dispersion_fit(*args, r.ctypes.data, ctypes.byref(A), ctypes.byref(b)) == \
            librelsim.RELSIM_ERR_INVALID_ARG, args
    # fewer than two modes with a positive window
    neg = -np.ones((n, nm))
    neg[:, 1] = 1.0
    assert L.relsim_dispersion_fit(neg.ctypes.data, n, nm, dt, 0, 10, Lx, a, r.ctypes.data, ctypes.byref(A),
                                   ctypes.byref(b)) == librelsim.RELSIM_ERR_INVALID_ARG


def test_growth_fit_host_code_matches_oracle(librelsim):
    # relsim_growth_fit is host code: it runs without a GPU
    import oracle
    rng = np.random.default_rng(5)
    for n, window, dt in [(40, 8, 0.5), (200, 50, 0.25), (7, 7, 1.0), (12, 2, 2.0)]:
        t = np.arange(n) * dt
        s = np.exp(0.3 * t - 0.002 * t * t + 0.05 * rng.normal(size=n))
        rate, first = librelsim.relsim_growth_fit(s, dt, window)
        orate, ofirst = oracle.growth_fit(s, dt, window)
        assert first == ofirst
        assert abs(rate - orate) < 1e-10 * max(1.0, abs(orate))
    s = np.exp(np.arange(10.0))
    s[4] = -1.0
    rate, first = librelsim.relsim_growth_fit(s, 1.0, 3)
    assert not (first <= 4 < first + 3) and abs(rate - 1.0) < 1e-12
    L = librelsim.lib()
    r, f = ctypes.c_double(), ctypes.c_int()
    for args in [(None, 5, 1.0, 2), (s.ctypes.data, 1, 1.0, 2), (s.ctypes.data, 10, 1.0, 11),
                 (s.ctypes.data, 10, 0.0, 3), (s.ctypes.data, 10, 1.0, 1)]:
        assert L.relsim_growth_fit(*args, ctypes.byref(r), ctypes.byref(f)) == librelsim.RELSIM_ERR_INVALID_ARG
    neg = -np.ones(6)
    assert L.relsim_growth_fit(neg.ctypes.data, 6, 1.0, 3, ctypes.byref(r), None) == librelsim.RELSIM_ERR_INVALID_ARG


def test_batch_rejects_bad_arguments(librelsim):
    L = librelsim.lib()
    out = ctypes.c_void_p()
    assert L.relsim_batch_create(None, 1, 1, ctypes.byref(out)) == librelsim.RELSIM_ERR_INVALID_ARG
    arr = (ctypes.c_void_p * 2)(None, None)
    assert L.relsim_batch_create(arr, 2, 1, ctypes.byref(out)) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_batch_create(arr, 0, 1, ctypes.byref(out)) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_batch_create(arr, 2, 1, None) == librelsim.RELSIM_ERR_INVALID_ARG
    assert not out.value
    st = np.zeros(1, dtype=np.int32)
    assert L.relsim_batch_run(None, 1, 1, 0, None, st.ctypes.data, None) == librelsim.RELSIM_ERR_INVALID_ARG
    L.relsim_batch_destroy(None)
    assert L.relsim_field_modes(None, 1, 1, None, 0) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_autotune(None, None) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_field_adjoint(None, None, None, None, None, None, None, None, None, None, 0) == \
        librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_step_adjoint(None, None, None, None, None, None, None, None) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_relabel_particles(None, 0, None, 0) == librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_get_particles_native(None, 0, None, None, None, None, None, 0) == \
        librelsim.RELSIM_ERR_INVALID_ARG
    assert L.relsim_load_particles_native(None, 0, 0, None, None, None, None, None, 0) == \
        librelsim.RELSIM_ERR_INVALID_ARG
