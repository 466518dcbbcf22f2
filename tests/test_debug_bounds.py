"""The bounds-checked build (-DPSATD_DEBUG, libpsatd_debug.so): every
instrumented global index of the step, init, sampling, diagnostics and batched
kernels is checked against its buffer.  The parity shapes run through it with
no index out of range, and with the same results as the oracle."""
import ctypes as C

import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

TOL = {64: 1e-12, 32: 1e-5}


def ogrid(g):
    return O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_release_library_reports_no_checks():
    from paper_2010_00409_gb300 import psatd
    fi, fb = C.c_longlong(), C.c_longlong()
    assert psatd.lib().psatd_debug_bounds_report(C.byref(fi), C.byref(fb)) == -2


@pytest.fixture(scope="module")
def dbg():
    """The package's binding switched to the debug library for this module."""
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2010_00409_gb300 import build, psatd
    path = build.build_library(debug=True)
    saved = psatd._lib
    psatd._lib = psatd.load_library(path)
    yield psatd
    psatd._lib = saved


def report(psatd):
    fi, fb = C.c_longlong(), C.c_longlong()
    n = psatd.lib().psatd_debug_bounds_report(C.byref(fi), C.byref(fb))
    return n, fi.value, fb.value


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("shape", [(8, 6, 10), (30, 18, 20), (64, 64, 64), (1024, 2, 4), (256, 256, 16)])
@pytest.mark.parametrize("path", ["auto", "generic"])
def test_steps_stay_in_bounds(dbg, prec, shape, path):
    Nx, Ny, Nz = shape
    g = W.GridSpec(Nx, Ny, Nz, 0.5, 0.7, 0.3, -1.0, -2.0, 0.5, 1.0)
    f = W.random_complex_field((6, Nz, Ny, Nx), seed=9)
    assert report(dbg)[0] == 0
    with dbg.Context(g, None, 0.37, prec) as ctx:
        if path == "generic":
            ctx.set_kernel_path(dbg.PATH_GENERIC)
        ctx.set_fields(f)
        ctx.fft(dbg.FORWARD)
        ctx.fft(dbg.INVERSE)
        ctx.set_fields(f)
        ctx.advance(2)
        got = ctx.get_field(-1)
        ctx.diagnostics()
    assert report(dbg) == (0, 0, 0)
    assert rel(got, O.advance(f, ogrid(g), 0.37, 2)) <= 2 * TOL[prec]


@pytest.mark.gpu
def test_real_storage_job_stays_in_bounds(dbg):
    lam, R0, L = 1.0, 16.0, 2.0
    g = W.GridSpec(256, 256, 64, 7.0 / 256, 30.0 / 256, 30.0 / 64, -(R0 - L / 2) - 7.0, -15.0, -15.0, 1.0)
    m = W.MappingSpec(R0, L)
    p = W.PulseSpec(kind=W.FLAT_TOP, lam=lam, theta=np.arctan(1 / 0.6), eps=0.1, P0=1.0, div_project=1)
    args = (-6.5, 24, 20, -1.5, 1.5, -1.2, 1.2)
    with dbg.Context(g, m, 0.9, 32, real=True) as ctx:
        ctx.init_pulse(p)
        ctx.advance(2)
        ctx.sample_focal_plane(*args)
        ctx.diagnostics()
        ctx.focal_one_shot(p, 9.0, *args)
        ctx.sample_focal_plane(*args)
    assert report(dbg) == (0, 0, 0)


@pytest.mark.gpu
def test_pulse_sampling_and_one_shot_stay_in_bounds(dbg):
    g, m, p, n_steps, plane = W.tight_focus_workload(N=48)
    T = m.R0 / g.c
    args = (plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
    for prec in (64, 32):
        with dbg.Context(g, m, T / n_steps, prec) as ctx:
            ctx.init_pulse(p)
            ctx.advance(3)
            ctx.sample_focal_plane(*args)
            ctx.focal_one_shot(p, T, *args)
    assert report(dbg) == (0, 0, 0)


@pytest.mark.gpu
def test_batched_advance_stays_in_bounds(dbg):
    import torch
    stream = torch.cuda.Stream()
    shapes = [(30, 18, 20), (45, 27, 50), (8, 6, 10), (1, 8, 12)]
    ctxs, refs = [], []
    for i, (nx, ny, nz) in enumerate(shapes):
        g = W.GridSpec(nx, ny, nz, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
        f = W.random_complex_field((6, nz, ny, nx), seed=30 + i)
        c = dbg.Context(g, None, 0.3, 32, stream=stream)
        c.set_fields(f)
        ctxs.append(c)
        refs.append(O.advance(f, ogrid(g), 0.3, 2))
    dbg.multi_advance(ctxs, [2, 2, 1, 2])
    dbg.multi_advance(ctxs, [0, 0, 1, 0])
    for c, ref in zip(ctxs, refs):
        assert rel(c.get_field(-1), ref) <= 2 * TOL[32]
        c.close()
    assert report(dbg) == (0, 0, 0)
