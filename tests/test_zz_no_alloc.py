"""The allocation-free energy entry point (psatd_energy_noalloc) against the
energy that psatd_diagnostics computes with its own scratch buffers.

This file is named so that pytest collects it last: if it fails, a run that
stops at the first failure has already run every other test.  It must also
pass on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-12   # float64 accumulation on both sides; only the summation order differs


@pytest.mark.parametrize("prec", [32, 64])
def test_energy_noalloc_matches_diagnostics_twice(lib, prec):
    import torch
    g = W.GridSpec(64, 48, 40, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, g.Nz, g.Ny, g.Nx), seed=21 + prec)
    L = lib.lib()
    with lib.Context(g, None, 0.1, prec) as ctx:
        ctx.set_fields(f)
        want = ctx.diagnostics()
        ptr = C.c_void_p(ctx.fields.data_ptr())
        stream = C.c_void_p(ctx.stream.cuda_stream)
        for call in range(2):                                  # two calls in a row
            host = (C.c_double * 2)()
            st = L.psatd_energy_noalloc(ptr, prec, g.cells, host, 0, stream)
            assert st == lib.OK, call
            assert abs(host[0] - want["energy_E"]) <= TOL * want["energy_E"]
            assert abs(host[1] - want["energy_B"]) <= TOL * want["energy_B"]
            dev = torch.zeros(2, dtype=torch.float64, device=ctx.fields.device)
            st = L.psatd_energy_noalloc(ptr, prec, g.cells, C.cast(C.c_void_p(dev.data_ptr()), C.POINTER(C.c_double)),
                                        1, stream)
            assert st == lib.OK, call
            ctx.synchronize()
            got = dev.cpu().numpy()
            assert abs(got[0] - want["energy_E"]) <= TOL * want["energy_E"]
            assert abs(got[1] - want["energy_B"]) <= TOL * want["energy_B"]


def test_energy_noalloc_rejects_sizes_beyond_its_array(lib):
    L = lib.lib()
    host = (C.c_double * 2)()
    assert L.psatd_energy_noalloc(C.c_void_p(256), 32, (1 << 30) + 1, host, 0, None) == lib.ERR_SIZE
    assert L.psatd_energy_noalloc(C.c_void_p(256), 32, 0, host, 0, None) == lib.ERR_SIZE
    assert L.psatd_energy_noalloc(C.c_void_p(256), 16, 10, host, 0, None) == lib.ERR_ARG


def test_energy_noalloc_allocates_nothing_after_its_first_call(lib):
    """After one call (of either precision) on a device, calls of both
    precisions leave the device's free memory unchanged: the first call loads
    every kernel of the entry point."""
    import torch
    L = lib.lib()
    dev = torch.device("cuda", torch.cuda.current_device())
    n = 40 * 48 * 64
    f32 = torch.ones((6, n), dtype=torch.complex64, device=dev)
    f64 = torch.ones((6, n), dtype=torch.complex128, device=dev)
    out = torch.zeros(2, dtype=torch.float64, device=dev)
    pout = C.cast(C.c_void_p(out.data_ptr()), C.POINTER(C.c_double))
    s = C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    host = (C.c_double * 2)()
    assert L.psatd_energy_noalloc(C.c_void_p(f32.data_ptr()), 32, n, host, 0, s) == lib.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(2):
        for prec, f in ((64, f64), (32, f32)):
            assert L.psatd_energy_noalloc(C.c_void_p(f.data_ptr()), prec, n, pout, 1, s) == lib.OK
            torch.cuda.synchronize()
            assert out.cpu().numpy().tolist() == [3.0 * n, 3.0 * n]
            assert L.psatd_energy_noalloc(C.c_void_p(f.data_ptr()), prec, n, host, 0, s) == lib.OK
            assert [host[0], host[1]] == [3.0 * n, 3.0 * n]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
