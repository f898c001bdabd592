"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, exports every
symbol ``include/rs.h`` declares, and its pure-host entry points behave."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_09218_gb300 import _lib, build
    build.build()
    return _lib.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "rs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    from paper_1606_09218_gb300 import _lib
    names = declared_functions()
    assert set(names) == set(_lib.EXPORTED)
    for nm in names:
        assert hasattr(lib, nm), nm


def test_version_and_workspace(lib):
    from paper_1606_09218_gb300 import config_from_workload
    from workloads import load_config
    assert b"sm_103a" in lib.rs_version()
    c1 = config_from_workload(load_config("c1_box64_n129"))
    c2 = config_from_workload(load_config("c2_protein1000_n513"))
    w1 = lib.rs_workspace_bytes(C.byref(c1))
    w2 = lib.rs_workspace_bytes(C.byref(c2))
    assert 0 < w1 < w2
    # T2 (rank bound x n x n, FP32) dominates at n = 513
    assert w2 > 4 * load_config("c2_protein1000_n513")["max_rank"] * 513 * 513


def test_invalid_config_is_rejected_on_host(lib):
    from paper_1606_09218_gb300 import _lib, config_from_workload
    from workloads import load_config
    for bad in (dict(n=128), dict(R_s=20), dict(eps=0.0), dict(b=-1.0), dict(snap=False)):
        cfg = dict(load_config("c1_box64_n129"))
        cfg.update(bad)
        c = config_from_workload(cfg)
        assert lib.rs_workspace_bytes(C.byref(c)) == 0
        h = C.c_void_p()
        assert lib.rs_create(C.byref(c), None, C.byref(h)) == _lib.RS_ERR_INVALID_ARG
        assert h.value is None
        assert lib.rs_last_error(None)


def test_als_entry_rejects_a_null_context(lib):
    """rs_tucker_als checks its context before any device work."""
    from paper_1606_09218_gb300 import _lib
    assert lib.rs_tucker_als(None, 1, 0, None) == _lib.RS_ERR_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library the binding raises; there is no CPU fallback."""
    from paper_1606_09218_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(_lib.RSError) as e:
        _lib.load(str(tmp_path / "librs_gb300.so"))
    assert "missing" in str(e.value)
