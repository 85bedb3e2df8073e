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

    from paper_2409_04215_gb300.api import ABI_VERSION

    lib = load_library(lib_path)
    assert lib.mfs_abi_version() == ABI_VERSION
    o = Options()
    lib.mfs_default_options(o)
    assert o.mu == 1.0 and o.gmres_tol == 1e-7 and o.max_rhs == 4 and o.precision == 0
    assert o.tensor_cores == 1 and o.autotune == 1 and o.profile == 0 and o.pair_variant == -1
    assert set(EXPORTED) == set(_declared())


def test_setup_rejects_bad_input_without_gpu(lib_path):
    """Argument checks run before any device work, so they answer on a machine without a GPU too."""
    import ctypes

    from paper_2409_04215_gb300.api import load_library

    lib = load_library(lib_path)
    assert lib.mfs_pair_variant(None, 1) == b""
    out = ctypes.c_void_p()
    rc = lib.mfs_setup(ctypes.byref(out), 1, None, 1, None, None, None, None)
    assert rc == 1  # MFS_ERR_INVALID_ARG
    assert b"invalid" in lib.mfs_setup_error()
    val = ctypes.c_double(-1.0)
    assert lib.mfs_fp32_fma_rate(5, ctypes.byref(val), None) == 1  # mode must be 0..4
    assert lib.mfs_fp32_fma_rate(-1, ctypes.byref(val), None) == 1
    assert lib.mfs_fp32_fma_rate(1, None, None) == 1
    assert lib.mfs_selftest_bounded_wait(2, 10, None) == 1  # arrive must be 0 or 1
    assert lib.mfs_selftest_bounded_wait(0, 0, None) == 1  # at least one poll


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors have the header's field offsets and sizes (a C probe compiled with gcc)."""
    import ctypes

    from paper_2409_04215_gb300.api import Options, _Bodies, _Info, _PointSet

    mirrors = {"mfs_options": Options, "mfs_solve_info": _Info, "mfs_bodies": _Bodies, "mfs_pointset": _PointSet}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mfs.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, val = line.split()
        got[(cname, field)] = int(val)
    for cname, py in mirrors.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_pair_variant_table(lib_path):
    from paper_2409_04215_gb300.api import pair_variants

    table = pair_variants()
    names = [t[1] for t in table]
    assert len(names) == len(set(names))
    for d in (1, 3):  # every (d, nrhs) has at least one forward pair-sum variant
        for r in (1, 2, 3, 4):
            assert any(t[2] == d and t[3] == r and not t[4] for t in table), (d, r)
    assert any(n.startswith("PackedLaplaceReg") for n in names) and any(n.startswith("GradStokes") for n in names)
