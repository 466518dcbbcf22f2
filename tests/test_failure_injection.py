"""Host-side failure injection: out-of-memory from a capped allocator and CUDA
errors returned in place of a call, each reported as its status with the
context usable afterwards.  Nothing here faults the GPU: the failures are made
on the host."""
import ctypes as C

import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

CUDA_ERROR_INVALID_VALUE = 1
CUDA_ERROR_MEMORY_ALLOCATION = 2


@pytest.fixture
def hooks():
    from paper_2010_00409_gb300 import psatd
    L = psatd.lib()
    yield L
    L.psatd_debug_set_alloc_limit(-1)
    L.psatd_debug_inject_cuda_error(0, 0)


def ogrid(g):
    return O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def test_hooks_need_no_device(hooks):
    hooks.psatd_debug_set_alloc_limit(0)
    assert hooks.psatd_debug_alloc_live() >= 0
    hooks.psatd_debug_inject_cuda_error(3, CUDA_ERROR_INVALID_VALUE)
    hooks.psatd_debug_inject_cuda_error(0, 0)


@pytest.mark.gpu
def test_capped_allocator_reports_oom_and_releases(lib, hooks):
    g = W.GridSpec(24, 20, 16, 0.5, 0.6, 0.7, 0.0, 0.0, 0.0, 1.0)
    live0 = hooks.psatd_debug_alloc_live()
    hooks.psatd_debug_set_alloc_limit(live0)             # nothing more may be allocated
    out = C.c_void_p()
    st = hooks.psatd_init_grid(C.byref(lib.make_grid(g)), None, 0.1, 64, None, 0, C.byref(out))
    assert st == lib.ERR_OOM and out.value is None
    assert hooks.psatd_debug_alloc_live() == live0     # the partial context gave everything back
    hooks.psatd_debug_set_alloc_limit(-1)
    f = W.random_complex_field((6, g.Nz, g.Ny, g.Nx), seed=5)
    with lib.Context(g, None, 0.1, 64) as ctx:
        ctx.set_fields(f)
        hooks.psatd_debug_set_alloc_limit(hooks.psatd_debug_alloc_live())
        with pytest.raises(lib.PsatdError) as e:
            ctx.diagnostics()                            # its scratch is allocated on first use
        assert e.value.status == lib.ERR_OOM
        hooks.psatd_debug_set_alloc_limit(-1)
        d = ctx.diagnostics()                            # usable once memory is there
        ref = O.diagnostics(f, ogrid(g))
        assert abs(d["energy"] - ref["energy"]) <= 1e-12 * ref["energy"]
    assert hooks.psatd_debug_alloc_live() == live0


@pytest.mark.gpu
def test_injected_cuda_errors_are_reported_and_the_context_survives(lib, hooks):
    g = W.GridSpec(24, 20, 16, 0.5, 0.6, 0.7, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, g.Nz, g.Ny, g.Nx), seed=6)
    dt = 0.3
    with lib.Context(g, None, dt, 64) as ctx:
        ctx.set_fields(f)
        hooks.psatd_debug_inject_cuda_error(1, CUDA_ERROR_INVALID_VALUE)
        with pytest.raises(lib.PsatdError) as e:
            ctx.get_field(-1)                            # its copy is the checked call
        assert e.value.status == lib.ERR_CUDA
        assert np.array_equal(ctx.get_field(-1), f)      # nothing was lost
        hooks.psatd_debug_inject_cuda_error(1, CUDA_ERROR_INVALID_VALUE)
        with pytest.raises(lib.PsatdError) as e:
            ctx.advance(2)                               # the first step's launch
        assert e.value.status == lib.ERR_CUDA
        assert ctx.time == 0.0
        hooks.psatd_debug_inject_cuda_error(1, CUDA_ERROR_MEMORY_ALLOCATION)
        with pytest.raises(lib.PsatdError) as e:
            ctx.advance(1)
        assert e.value.status == lib.ERR_OOM
        ctx.advance(2)                                   # the field was not touched by the failed calls
        got = ctx.get_field(-1)
    ref = O.advance(f, ogrid(g), dt, 2)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-12
