"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/*.h declares. No compute call is made (no GPU needed)."""
import ctypes
import glob
import os
import re
import shutil

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
