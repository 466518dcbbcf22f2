"""Host-side checks of the C ABI that need no GPU: the library builds, loads,
exports every symbol that include/psatd.h declares, and rejects bad arguments
before touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2010_00409_gb300.build import build_library
    from paper_2010_00409_gb300 import psatd
    build_library()
    return psatd


def declared_functions():
    src = open(os.path.join(ROOT, "include", "psatd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(psatd_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree(L):
    assert declared_functions() == sorted(L.EXPORTS)


def test_library_exports_every_declared_symbol(L):
    lib = L.load_library()
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_nm_shows_exports(L):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(r"\bT %s\b" % name, out), name


def grid(Nx=8, Ny=8, Nz=8, d=1.0):
    from paper_2010_00409_gb300.psatd import PsatdGrid
    return PsatdGrid(Nx, Ny, Nz, d, d, d, 0.0, 0.0, 0.0, 1.0)


@pytest.mark.parametrize("dims", [(7, 8, 8), (8, 14, 8), (8, 8, 0), (4096, 8, 8), (8, 8, 22)])
def test_bad_sizes_rejected_without_device(L, dims):
    lib = L.load_library()
    out = C.c_void_p()
    st = lib.psatd_init_grid(C.byref(grid(*dims)), None, 0.1, 64, None, 0, C.byref(out))
    assert st == L.ERR_SIZE
    assert out.value is None
    assert b"prime factors" in lib.psatd_last_error(None)


def test_bad_arguments_rejected_without_device(L):
    lib = L.load_library()
    out = C.c_void_p()
    assert lib.psatd_init_grid(C.byref(grid()), None, 0.1, 16, None, 0, C.byref(out)) == L.ERR_ARG
    assert lib.psatd_init_grid(C.byref(grid(d=-1.0)), None, 0.1, 64, None, 0, C.byref(out)) == L.ERR_ARG
    assert lib.psatd_init_grid(C.byref(grid()), None, float("nan"), 64, None, 0, C.byref(out)) == L.ERR_ARG
    assert lib.psatd_init_grid(None, None, 0.1, 64, None, 0, C.byref(out)) == L.ERR_ARG
    assert lib.psatd_advance(None, 1) == L.ERR_ARG
    assert lib.psatd_time(None) == 0.0
    assert lib.psatd_status_string(L.ERR_SIZE) == b"PSATD_ERR_SIZE"
    buf = C.c_void_p(8)   # never dereferenced: every call below fails its argument check first
    assert lib.psatd_fp64_fma_probe(None, 1, 32, 1, None) == L.ERR_ARG
    assert lib.psatd_fp64_fma_probe(buf, 0, 32, 1, None) == L.ERR_ARG
    assert lib.psatd_fp64_fma_probe(buf, 1, 48, 1, None) == L.ERR_ARG
    assert lib.psatd_fp64_fma_probe(buf, 1, 2048, 1, None) == L.ERR_ARG
    assert lib.psatd_fp64_fma_probe(buf, 1, 32, 0, None) == L.ERR_ARG
    ctxs = (C.c_void_p * 2)(None, None)
    ms = C.c_double()
    steps = (C.c_int * 2)(1, 1)
    assert lib.psatd_multi_advance(None, 0, steps) == L.ERR_ARG
    assert lib.psatd_multi_advance(ctxs, 2, steps) == L.ERR_ARG
    assert lib.psatd_multi_autotune(ctxs, 0, 1, C.byref(ms)) == L.ERR_ARG
    assert lib.psatd_selftest_grid_barrier_timeout(None) == L.ERR_ARG


def test_d_min_host_helper_matches_oracle(L):
    from oracle import psatd_oracle as O
    for th in (0.3, 0.8, 1.0, 1.2):
        assert abs(L.d_min(16.0, 2.0, th) - O.d_min(16.0, 2.0, th)) < 1e-12


def test_build_flags_target_sm103a():
    from paper_2010_00409_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH
