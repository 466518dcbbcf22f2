"""Persistent batched advance (psatd_multi_advance): many boxes on uneven grids
stepped in one cooperative launch, against the oracle; its autotuner; capture
into a batch; the bounded grid-barrier wait."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}     # relative L2 per step; n steps allow n x TOL


def ogrid(g):
    return O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


SHAPES = [(30, 18, 20), (45, 27, 50), (96, 100, 108), (8, 6, 10), (1, 8, 12)]


def _boxes(lib, prec, stream, shapes=SHAPES, seed0=40):
    boxes = []
    for i, (nx, ny, nz) in enumerate(shapes):
        g = W.GridSpec(nx, ny, nz, 0.5 + 0.1 * i, 0.7, 0.3 + 0.05 * i, -1.0, -2.0, 0.5, 1.0)
        f = W.random_complex_field((6, nz, ny, nx), seed=seed0 + i)
        dt = 0.21 + 0.07 * i
        ctx = lib.Context(g, None, dt, prec, stream=stream)
        ctx.set_fields(f)
        boxes.append((ctx, g, f, dt))
    return boxes


@pytest.mark.parametrize("prec", [64, 32])
def test_multi_advance_matches_oracle_on_uneven_grids(lib, prec):
    import torch
    stream = torch.cuda.Stream()
    boxes = _boxes(lib, prec, stream)
    ctxs = [b[0] for b in boxes]
    n0 = ctxs[0].launch_count
    lib.multi_advance(ctxs, 3)
    assert ctxs[0].launch_count == n0 + 1                   # one launch for all boxes and steps
    for ctx, g, f, dt in boxes:
        got = ctx.get_field(-1)
        assert abs(ctx.time - 3 * dt) < 1e-14
        assert rel(got, O.advance(f, ogrid(g), dt, 3)) <= 3 * TOL[prec], (g.Nx, g.Ny, g.Nz)
    ctxs[0].synchronize()                                   # no barrier wait expired
    for c in ctxs:
        c.close()


def test_multi_advance_single_box_single_step_equals_eager(lib):
    import torch
    stream = torch.cuda.Stream()
    (ctx, g, f, dt), = _boxes(lib, 64, stream, shapes=[(48, 40, 36)])
    lib.multi_advance([ctx], 1)
    got = ctx.get_field(-1)
    with lib.Context(g, None, dt, 64, stream=stream) as ref:
        ref.set_fields(f)
        ref.advance(1)
        want = ref.get_field(-1)
    assert rel(got, want) <= 2 * TOL[64]
    ctx.close()


def test_multi_autotune_keeps_fields_and_caches(lib):
    import torch
    stream = torch.cuda.Stream()
    boxes = _boxes(lib, 32, stream, shapes=[(30, 18, 20), (45, 27, 50)], seed0=60)
    ctxs = [b[0] for b in boxes]
    ms = lib.multi_autotune(ctxs, 1)
    assert ms > 0
    for ctx, g, f, dt in boxes:
        assert np.array_equal(ctx.get_field(-1), f.astype(np.complex64))     # trials ran on copies
        assert ctx.time == 0.0
    lib.multi_advance(ctxs, 2)                              # with the tuned schedules
    for ctx, g, f, dt in boxes:
        assert rel(ctx.get_field(-1), O.advance(f, ogrid(g), dt, 2)) <= 2 * TOL[32]
    for c in ctxs:
        c.close()


def test_multi_advance_recorded_in_a_batch(lib):
    import torch
    stream = torch.cuda.Stream()
    boxes = _boxes(lib, 32, stream, shapes=[(30, 18, 20), (96, 100, 108), (8, 6, 10)], seed0=70)
    ctxs = [b[0] for b in boxes]
    steps = [2, 1, 3]                                       # a step count per box
    lib.multi_advance(ctxs, steps)                          # uploads the boxes outside the capture
    b = lib.Batch(stream)
    with b:
        lib.multi_advance(ctxs, steps)
    for (ctx, g, f, dt), k in zip(boxes, steps):
        assert abs(ctx.time - k * dt) < 1e-14               # recording does not move the time
    b.launch()
    b.launch()
    for (ctx, g, f, dt), k in zip(boxes, steps):
        assert abs(ctx.time - 3 * k * dt) < 1e-14
        assert rel(ctx.get_field(-1), O.advance(f, ogrid(g), dt, 3 * k)) <= 3 * k * TOL[32]
    b.close()
    for c in ctxs:
        c.close()


def test_grid_barrier_timeout_is_reported_and_context_survives(lib):
    import torch
    stream = torch.cuda.Stream()
    (ctx, g, f, dt), = _boxes(lib, 32, stream, shapes=[(30, 18, 20)], seed0=80)
    assert ctx.selftest_grid_barrier_timeout() == lib.ERR_TIMEOUT
    ctx.synchronize()                                       # the error word was cleared
    ctx.set_fields(f)
    ctx.set_time(0.0)
    lib.multi_advance([ctx], 2)
    assert rel(ctx.get_field(-1), O.advance(f, ogrid(g), dt, 2)) <= 2 * TOL[32]
    ctx.close()


def test_multi_advance_argument_errors(lib):
    import torch
    stream = torch.cuda.Stream()
    a = lib.Context(W.GridSpec(8, 8, 8, 1, 1, 1, 0, 0, 0, 1.0), None, 0.1, 32, stream=stream)
    b = lib.Context(W.GridSpec(8, 8, 8, 1, 1, 1, 0, 0, 0, 1.0), None, 0.1, 64, stream=stream)
    with pytest.raises(lib.PsatdError) as e:
        lib.multi_advance([a, b], 1)                        # mixed precision
    assert e.value.status == lib.ERR_ARG
    with pytest.raises(lib.PsatdError) as e:
        lib.multi_advance([a, a], 1)                        # the same storage twice
    assert e.value.status == lib.ERR_ARG
    r = lib.Context(W.GridSpec(256, 256, 64, 1, 1, 1, 0, 0, 0, 1.0), None, 0.1, 32, stream=stream, real=True)
    with pytest.raises(lib.PsatdError) as e:
        lib.multi_advance([r], 1)                           # real storage
    assert e.value.status == lib.ERR_STATE
    for c in (a, b, r):
        c.close()
