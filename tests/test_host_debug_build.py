"""The bounds-checked debug build (-DQSA_DEBUG_BOUNDS, libqsa_debug.so) builds
beside the release library, exports the same ABI plus the bounds-status calls,
and says which build it is.  No GPU: only entry points that touch no device."""
import ctypes
import os

import pytest


@pytest.fixture(scope="module")
def libs():
    import __graft_entry__
    mod = __graft_entry__._build_module()
    release = mod.build()
    debug = mod.build(debug_bounds=True)
    return ctypes.CDLL(release), ctypes.CDLL(debug)


def test_debug_build_reports_itself(libs):
    rel, dbg = libs
    rel.qsa_debug_bounds_enabled.restype = ctypes.c_int
    dbg.qsa_debug_bounds_enabled.restype = ctypes.c_int
    assert rel.qsa_debug_bounds_enabled() == 0
    assert dbg.qsa_debug_bounds_enabled() == 1


def test_release_status_needs_no_device(libs):
    rel, _ = libs
    rel.qsa_debug_bounds_status.restype = ctypes.c_uint64
    assert rel.qsa_debug_bounds_status() == 0


def test_debug_build_exports_the_abi(libs):
    rel, dbg = libs
    from test_host_abi import _declared
    missing = [n for n in sorted(_declared()) if not hasattr(dbg, n)]
    assert not missing, missing


def test_binding_selects_the_variant():
    import subprocess
    import sys
    code = ("import paper_2608_16940_gb300 as q, os; "
            "print(os.path.basename(q.LIB_PATH), q.qsa_debug_bounds_enabled())")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, QSA_LIB_VARIANT="debug")
    out = subprocess.run([sys.executable, "-c", code], cwd=root, env=env, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    assert out.stdout.split() == ["libqsa_debug.so", "True"]
