"""Real-field storage (PSATD_FLAG_REAL_FIELDS) against the float64 oracle.

A real-field step is the real part of the complex step (reading R20 of the
oracle; the mean update on Nyquist planes).  Random fields with a full
spectrum exercise every Nyquist plane, the packed k_x = 0 / Nyquist slot and
the mirrored y pencils.  Tolerance: float32 relative L2 1e-5, as for the
complex path.
"""
import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def ogrid(g):
    return O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def real_field(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("Nz,n", [(64, 3), (128, 1)])
def test_real_steps_match_oracle(lib, Nz, n):
    g = W.GridSpec(256, 256, Nz, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    f = real_field((6, Nz, 256, 256), seed=Nz)
    dt = 0.29
    with lib.Context(g, None, dt, 32, real=True) as ctx:
        ctx.set_fields(f)
        ctx.advance(n)
        got = ctx.get_field(-1)
    assert got.dtype == np.float32
    want = O.advance_real(f, ogrid(g), dt, n)
    assert rel(got, want) <= 1e-5


def test_real_step_of_single_modes_on_every_special_plane(lib):
    """One mode at a time on k_x = 0, the x Nyquist plane, k_y = 0, the y and z
    Nyquist planes and a generic mode: each lands in a different branch of the
    slot-0 / mirrored-pencil / mean-update logic."""
    Nz = 64
    g = W.GridSpec(256, 256, Nz, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    x = np.arange(256)
    z = np.arange(Nz)
    modes = [(0, 5, 7), (128, 5, 7), (3, 0, 7), (3, 128, 7), (3, 5, 32), (128, 128, 32), (0, 0, 0), (37, 200, 50)]
    rng = np.random.default_rng(1)
    for (mx, my, mz) in modes:
        ph = (2 * np.pi * (mx * x[None, None, :] / 256 + my * x[None, :, None] / 256 + mz * z[:, None, None] / Nz))
        f = np.stack([a * np.cos(ph) + b * np.sin(ph) for a, b in rng.standard_normal((6, 2))])
        f = f.astype(np.float32).astype(np.float64)
        with lib.Context(g, None, 0.41, 32, real=True) as ctx:
            ctx.set_fields(f)
            ctx.advance(1)
            got = ctx.get_field(-1)
        want = O.psatd_step_real(f, ogrid(g), 0.41)
        assert rel(got, want) <= 1e-5, (mx, my, mz)


def test_real_init_projection_sampling_diagnostics(lib):
    # flat-top f = 0.3 shell on a 256 x 256 x 64 layer (coarse in z, same on both sides)
    lam, R0, L = 1.0, 16.0, 2.0
    g = W.GridSpec(256, 256, 64, 7.0 / 256, 30.0 / 256, 30.0 / 64, -(R0 - L / 2) - 7.0, -15.0, -15.0, 1.0)
    m = W.MappingSpec(R0, L)
    p = W.PulseSpec(kind=W.FLAT_TOP, lam=lam, theta=np.arctan(1 / 0.6), eps=0.1, P0=1.0, div_project=1)
    og, om = ogrid(g), O.Mapping(R0, L)
    op = O.Pulse(p.kind, p.lam, p.theta, p.eps, p.P0, p.n_cycles, p.cep, p.ellipticity, p.pol_angle, 1)
    f0 = O.project_transverse(O.init_fields(og, om, op), og).real
    T = 2.0
    with lib.Context(g, m, T, 32, real=True) as ctx:
        ctx.init_pulse(p)
        got0 = ctx.get_field(-1)
        d0 = ctx.diagnostics()
        ctx.advance(1)
        # a plane through the converging shell (R ~ R0 - c T on the -x axis)
        s = ctx.sample_focal_plane(-14.0, 24, 20, -1.0, 1.0, -0.8, 0.8, comps=(0, 1, 2, 4))
    assert rel(got0, f0) <= 1e-5
    od = O.diagnostics(f0.astype(np.complex128), og)
    assert abs(d0["energy"] / od["energy"] - 1) <= 1e-5
    f1 = O.psatd_step_real(f0, og, T)
    ys, zs = np.linspace(-1.0, 1.0, 24, endpoint=False), np.linspace(-0.8, 0.8, 20, endpoint=False)
    ref = O.sample_plane(f1.astype(np.complex128), og, om, -14.0, ys, zs, T, comps=(0, 1, 2, 4))
    assert np.max(np.abs(ref)) > 1e-3 * np.max(np.abs(f0))
    assert rel(s, ref) <= 1e-5


def test_real_diagnostics_match_oracle(lib):
    # a random real field with longitudinal content: energy from the real
    # storage, divergence maxima from the half spectrum (slots and x-Nyquist array)
    g = W.GridSpec(256, 256, 64, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    rng = np.random.Generator(np.random.PCG64(17))
    f = rng.standard_normal((6, 64, 256, 256)).astype(np.float32)
    f[1] *= 0.5                                      # uneven components
    with lib.Context(g, None, 0.2, 32, real=True) as ctx:
        ctx.set_fields(f)
        d = ctx.diagnostics()
        assert np.array_equal(ctx.get_field(-1), f)     # the diagnostics leave the storage unchanged
    od = O.diagnostics(f.astype(np.complex128), ogrid(g))
    for k in ("energy", "energy_E", "energy_B"):
        assert abs(d[k] / od[k] - 1) <= 1e-6, k
    for k in ("max_div_E", "max_E_hat", "max_div_B", "max_B_hat"):
        assert abs(d[k] / od[k] - 1) <= 1e-5, (k, d[k], od[k])


def test_real_fields_argument_and_state_errors(lib):
    g = W.GridSpec(256, 256, 64, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 1.0)
    with pytest.raises(lib.PsatdError):
        lib.Context(g, None, 0.1, 64, real=True)
    with pytest.raises(lib.PsatdError):
        lib.Context(W.GridSpec(128, 256, 64, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 1.0), None, 0.1, 32, real=True)
    with pytest.raises(lib.PsatdError):
        lib.Context(W.GridSpec(256, 256, 60, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 1.0), None, 0.1, 32, real=True)
    with lib.Context(g, W.MappingSpec(4.0, 1.0), 0.1, 32, real=True) as ctx:
        with pytest.raises(lib.PsatdError):
            ctx.fft(lib.FORWARD)
        p = W.PulseSpec(kind=W.GAUSSIAN, lam=1.0, theta=0.4, eps=0.1, P0=1.0, n_cycles=2.0)
        ctx.focal_one_shot(p, 1.0, 0.0, 4, 4, -1, 1, -1, 1)
        with pytest.raises(lib.PsatdError):
            ctx.advance(1)                          # the storage holds the half spectrum now
        ctx.set_fields(np.zeros((6, 64, 256, 256), np.float32))
        assert ctx.autotune()[0] == lib.PATH_AUTO
        ctx.advance(0)
        assert np.all(ctx.get_field(0) == 0)


def _flat_top_layer():
    lam, R0, L = 1.0, 16.0, 2.0
    g = W.GridSpec(256, 256, 64, 7.0 / 256, 30.0 / 256, 30.0 / 64, -(R0 - L / 2) - 7.0, -15.0, -15.0, 1.0)
    return g, W.MappingSpec(R0, L), lam


@pytest.mark.parametrize("project", [1, 0])
def test_real_one_shot_matches_oracle_without_complex_scratch(lib, project):
    """One exact step of T on real storage (the half spectrum, the real-field
    update with the projection of B folded in), sampled from that spectrum,
    against the oracle's real-field exact step and sampling; no complex copy of
    the field is allocated on the way."""
    g, m, lam = _flat_top_layer()
    p = W.PulseSpec(kind=W.FLAT_TOP, lam=lam, theta=np.arctan(1 / 0.6), eps=0.1, P0=1.0, div_project=project)
    og, om = ogrid(g), O.Mapping(m.R0, m.L)
    op = O.Pulse(p.kind, p.lam, p.theta, p.eps, p.P0, p.n_cycles, p.cep, p.ellipticity, p.pol_angle, project)
    f0 = O.init_fields(og, om, op)
    if project:
        f0 = O.project_transverse(f0, og)
    f0 = f0.real
    T = 9.0
    ys, zs = np.linspace(-1.5, 1.5, 24, endpoint=False), np.linspace(-1.2, 1.2, 20, endpoint=False)
    args = (-6.5, 24, 20, -1.5, 1.5, -1.2, 1.2)
    L = lib.lib()
    with lib.Context(g, m, T / 10, 32, real=True) as ctx:
        live0 = L.psatd_debug_alloc_live()
        got = ctx.focal_one_shot(p, T, *args, comps=(0, 1, 2, 4))
        grown = L.psatd_debug_alloc_live() - live0
        assert grown < 6 * g.cells * 8 // 4               # far below a complex copy (48 B per cell)
        assert abs(ctx.time - T) == 0.0
        again = ctx.sample_focal_plane(*args, comps=(0, 1, 2, 4))
        assert np.array_equal(again, got)                  # sampled from the held half spectrum
    f1 = O.psatd_step_real(f0, og, T)
    ref = O.sample_plane(f1.astype(np.complex128), og, om, args[0], ys, zs, T, comps=(0, 1, 2, 4))
    assert np.max(np.abs(ref)) > 1e-2 * np.max(np.abs(f0))
    assert rel(got, ref) <= 1e-5
