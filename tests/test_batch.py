"""Batches (CUDA graphs of library calls) and the autotuner."""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def ogrid(g):
    return O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def test_batched_advance_replays_the_eager_calls_exactly(lib):
    import torch
    stream = torch.cuda.Stream()
    shapes = [(32, 32, 32), (48, 40, 36), (64, 64, 64)]
    fields = [W.random_complex_field((6, nz, ny, nx), seed=i) for i, (nx, ny, nz) in enumerate(shapes)]
    grids = [W.GridSpec(nx, ny, nz, 0.5, 0.6, 0.7, 0.0, 0.0, 0.0, 1.0) for nx, ny, nz in shapes]
    dt = 0.3
    eager = []
    for g, f in zip(grids, fields):
        with lib.Context(g, None, dt, 32, stream=stream) as ctx:
            ctx.set_fields(f)
            ctx.advance(3)
            eager.append(ctx.get_field(-1))
    ctxs = [lib.Context(g, None, dt, 32, stream=stream) for g in grids]
    for c, f in zip(ctxs, fields):
        c.set_fields(f)
        c.advance(0)
    b = lib.Batch(stream)
    with b:
        for c in ctxs:
            c.advance(3)
        with pytest.raises(lib.PsatdError):
            ctxs[0].get_field(-1)                    # host copy refused while recording
    assert b.nodes >= 3 * 3 * 3
    for c in ctxs:
        assert c.time == 0.0
    b.launch()
    for c, want in zip(ctxs, eager):
        assert np.array_equal(c.get_field(-1), want)
        assert abs(c.time - 3 * dt) < 1e-15
    b.launch()                                       # a second replay advances again
    for c, g, f in zip(ctxs, grids, fields):
        ref = O.advance(f, ogrid(g), dt, 6)
        assert np.linalg.norm(c.get_field(-1) - ref) / np.linalg.norm(ref) <= 2e-5
    b.close()
    for c in ctxs:
        c.close()


def test_batched_one_shot_sweep_matches_eager(lib):
    import torch
    stream = torch.cuda.Stream()
    sweep = W.batched_sweep(n=3, seed=5)
    outs, ctxs, eager = [], [], []
    for g, m, p, T, plane in sweep:
        c = lib.Context(g, m, T / 100, 32, stream=stream)
        o = torch.empty((3, plane["nz"], plane["ny"]), dtype=torch.complex64, device="cuda")
        args = (plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"], plane["z0"], plane["z1"])
        c.focal_one_shot(p, T, *args, out=o)          # prepares tables and buffers
        c.synchronize()
        eager.append(o.cpu().numpy())
        o.zero_()
        ctxs.append((c, p, T, args))
        outs.append(o)
    b = lib.Batch(stream)
    with b:
        for (c, p, T, args), o in zip(ctxs, outs):
            c.focal_one_shot(p, T, *args, out=o)
    b.launch()
    stream.synchronize()
    for o, want in zip(outs, eager):
        assert np.max(np.abs(want)) > 0
        assert np.array_equal(o.cpu().numpy(), want)
    b.close()
    for c, *_ in ctxs:
        c.close()


def test_autotune_keeps_results_and_caches(lib):
    g = W.GridSpec(48, 40, 36, 0.5, 0.6, 0.7, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, g.Nz, g.Ny, g.Nx), seed=2)
    with lib.Context(g, None, 0.3, 64) as ctx:
        ctx.set_fields(f)
        path, shift, ms = ctx.autotune(2)
        assert path in (lib.PATH_AUTO, lib.PATH_REGISTER, lib.PATH_GENERIC) and shift in (-1, 0, 1) and ms > 0
        assert np.array_equal(ctx.get_field(-1), f.astype(np.complex128))   # trials ran on a copy
        ctx.advance(2)
        got = ctx.get_field(-1)
    ref = O.advance(f, ogrid(g), 0.3, 2)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 2e-12
    with lib.Context(g, None, 0.3, 64) as ctx:
        assert ctx.autotune(2) == (path, shift, -1.0)
