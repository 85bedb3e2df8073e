"""The C-ABI library builds for sm_103a, loads without a GPU and exports every symbol include/mfs.h declares."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mfs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mfs_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2409_04215_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["mfs_setup", "mfs_matvec", "mfs_precond_apply", "mfs_solve_elastance", "mfs_solve_mobility",
              "mfs_mobility_vjp", "mfs_update_centers", "mfs_pair_sum", "mfs_destroy", "mfs_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mfs_\w+)", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_reports(lib_path):
    from paper_2409_04215_gb300.api import EXPORTED, Options, load_library

    lib = load_library(lib_path)
    assert lib.mfs_abi_version() == 1
    o = Options()
    lib.mfs_default_options(o)
    assert o.mu == 1.0 and o.gmres_tol == 1e-7 and o.max_rhs == 4 and o.precision == 0
    assert set(EXPORTED) == set(_declared())


def test_setup_rejects_bad_input_without_gpu(lib_path):
    """Argument checks run before any device work, so they answer on a machine without a GPU too."""
    import ctypes

    from paper_2409_04215_gb300.api import load_library

    lib = load_library(lib_path)
    out = ctypes.c_void_p()
    rc = lib.mfs_setup(ctypes.byref(out), 1, None, 1, None, None, None, None)
    assert rc == 1  # MFS_ERR_INVALID_ARG
    assert b"invalid" in lib.mfs_setup_error()
