"""The C-ABI library builds, loads and exports every entry point include/amg.h declares.

CPU-only: nothing here launches GPU work (host-only entry points are called).
"""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2102_07417_gb300 import amg, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "amg.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(amg_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return amg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("amg_setup", "amg_pcg_solve", "amg_free", "amg_hierarchy_info", "amg_hierarchy_export",
                 "amg_vcycle_apply", "amg_spmv", "amg_solve", "amg_params_default", "amg_status_string"):
        assert must in names
    assert sorted(amg.EXPORTS) == names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", build.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (amg_[a-z_0-9]+)$", out, flags=re.M))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)


def test_host_only_entry_points(lib):
    p = amg.default_params()
    assert p.theta == 0.25 and p.max_coarse == 64 and p.nu1 == 1 and p.nu2 == 1
    assert abs(p.omega - 2.0 / 3.0) < 1e-16 and p.precision == amg.PREC_FP64
    assert lib.amg_params_default(None) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_status_string(amg.AMG_ERR_NOT_SPD).decode().startswith("matrix is not")
    assert lib.amg_status_string(12345) == b"unknown status"
    # argument checks happen before any device work
    h = C.c_void_p()
    assert lib.amg_setup(None, None, None, None, C.byref(h)) == amg.AMG_ERR_INVALID_ARG
    csr = amg.Csr(0, 0, None, None, None, 0)
    assert lib.amg_setup(C.byref(csr), None, None, None, C.byref(h)) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_pcg_solve(None, None, None, 1e-8, 10, None, None, None, 0) == amg.AMG_ERR_INVALID_ARG
    assert lib.amg_hierarchy_bytes(None) == 0
    lib.amg_free(None)


def test_bad_params_rejected_without_gpu(lib):
    import numpy as np

    rp = np.array([0, 1], np.int32)
    ci = np.array([0], np.int32)
    v = np.array([1.0])
    csr = amg.Csr(1, 1, rp.ctypes.data, ci.ctypes.data, v.ctypes.data, 0)
    h = C.c_void_p()
    for kw, code in (({"theta": 0.0}, amg.AMG_ERR_INVALID_ARG), ({"max_levels": 0}, amg.AMG_ERR_INVALID_ARG),
                     ({"omega": 2.5}, amg.AMG_ERR_INVALID_ARG), ({"nu1": -1}, amg.AMG_ERR_INVALID_ARG),
                     ({"precision": 7}, amg.AMG_ERR_INVALID_ARG), ({"block_size": 0}, amg.AMG_ERR_INVALID_ARG),
                     ({"block_size": 9}, amg.AMG_ERR_INVALID_ARG), ({"smoother": 5}, amg.AMG_ERR_INVALID_ARG),
                     ({"interp": 7}, amg.AMG_ERR_INVALID_ARG),
                     ({"block_size": 3}, amg.AMG_ERR_INVALID_ARG)):  # n = 1 is not a multiple of 3
        p = amg.default_params(**kw)
        assert lib.amg_setup(C.byref(csr), C.byref(p), None, None, C.byref(h)) == code
        assert h.value is None


def test_noalloc_arguments_refused_without_gpu(lib):
    """amg_spmv_dot_noalloc checks its arguments before any CUDA call (the pointers below are
    never dereferenced): NULL pointers and n < 1 are invalid, n above its scratch's 16,777,216 rows
    unsupported.  The Python wrapper refuses host tensors before reaching the library."""
    torch = pytest.importorskip("torch")
    f = lib.amg_spmv_dot_noalloc
    assert len(f.argtypes) == 9
    fake = 256  # a non-NULL address that the refused calls never touch
    assert f(4, 4, None, fake, fake, fake, fake, fake, None) == amg.AMG_ERR_INVALID_ARG
    assert f(4, 4, fake, None, fake, fake, fake, fake, None) == amg.AMG_ERR_INVALID_ARG
    assert f(4, 4, fake, fake, fake, fake, fake, None, None) == amg.AMG_ERR_INVALID_ARG
    assert f(0, 0, fake, None, None, fake, fake, fake, None) == amg.AMG_ERR_INVALID_ARG
    assert f(4, -1, fake, fake, fake, fake, fake, fake, None) == amg.AMG_ERR_INVALID_ARG
    assert f(16_777_217, 0, fake, None, None, fake, fake, fake, None) == amg.AMG_ERR_UNSUPPORTED
    assert b"exceeds the limit" in lib.amg_last_error()
    rp = torch.tensor([0, 1], dtype=torch.int32)
    ci = torch.tensor([0], dtype=torch.int32)
    v = torch.ones(1, dtype=torch.float64)
    x = torch.ones(1, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA tensor"):
        amg.spmv_dot_noalloc(rp, ci, v, x, x.clone(), x.clone())
