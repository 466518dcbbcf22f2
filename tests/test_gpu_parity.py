"""Parity of the CUDA path (through the C ABI) with the float64 CPU oracle.

Tolerances (relative L2 over all compared values): float64 1e-12, float32 1e-5
for the solver; the focal-plane field of the full tight-focus run in float32
1e-4.  Sizes span several tiles and ragged tails; the full 256^3 workload is
checked on the sampled focal plane and on invariants.
"""
import math

import numpy as np
import pytest

from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {64: 1e-12, 32: 1e-5}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def ogrid(g):
    return O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, g.x_min, g.y_min, g.z_min, g.c)


def opulse(p):
    return O.Pulse(p.kind, p.lam, p.theta, p.eps, p.P0, p.n_cycles, p.cep, p.ellipticity,
                   p.pol_angle, p.div_project)


SHAPES = [(4, 4, 4), (8, 6, 10), (12, 10, 6), (1, 8, 12), (5, 3, 15), (30, 18, 20),
          (64, 64, 64), (96, 100, 108), (45, 81, 125), (2048, 2, 3)]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("shape", SHAPES)
def test_fft_forward_inverse_parity(lib, prec, shape):
    Nx, Ny, Nz = shape
    g = W.GridSpec(Nx, Ny, Nz, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, Nz, Ny, Nx), seed=Nx + Ny + Nz)
    with lib.Context(g, None, 0.1, prec) as ctx:
        ctx.set_fields(f)
        ctx.fft(lib.FORWARD)
        F = ctx.get_field(-1)
        assert rel(F, O.fft3(f)) <= TOL[prec]
        ctx.fft(lib.INVERSE)
        back = ctx.get_field(-1) / (Nx * Ny * Nz)
        assert rel(back, f) <= TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("shape", [(8, 6, 10), (12, 10, 6), (1, 8, 12), (30, 18, 20), (96, 100, 108), (45, 27, 50)])
def test_step_parity_ragged(lib, prec, shape, metrics_log):
    Nx, Ny, Nz = shape
    g = W.GridSpec(Nx, Ny, Nz, 0.5, 0.7, 0.3, -1.0, -2.0, 0.5, 1.0)
    f = W.random_complex_field((6, Nz, Ny, Nx), seed=7)
    dt = 0.37
    with lib.Context(g, None, dt, prec) as ctx:
        ctx.set_fields(f)
        ctx.advance(3)
        got = ctx.get_field(-1)
        assert abs(ctx.time - 3 * dt) < 1e-15
    err = rel(got, O.advance(f, ogrid(g), dt, 3))
    metrics_log("3 random-field steps %dx%dx%d" % shape, prec, err, TOL[prec] * 3)
    assert err <= TOL[prec] * 3


@pytest.mark.parametrize("prec", [64, 32])
def test_plain_method_64cubed_20_steps(lib, prec):
    """The 64^3 plain-method workload: x-polarised plane wave (4 periods along
    z) plus a seeded divergence-free random field (amplitude 1e-3), 20 steps
    at the Courant step; parity, exact phase, energy and divergence."""
    g = W.plain_grid(64)
    dt = g.courant_dt()
    pw = W.plane_wave_mode(g, periods=4)
    for seed in (0, 1, 2):
        f0 = pw + W.random_divfree_field(g, seed)
        with lib.Context(g, None, dt, prec) as ctx:
            ctx.set_fields(f0)
            d0 = ctx.diagnostics()
            ctx.advance(20)
            got = ctx.get_field(-1)
            d1 = ctx.diagnostics()
        want = O.advance(f0, ogrid(g), dt, 20)
        assert rel(got, want) <= TOL[prec]
        # |E'|^2 - |E|^2 is bounded by twice the relative L2 error of the state
        assert abs(d1["energy"] / d0["energy"] - 1) <= (1e-13 if prec == 64 else 2 * TOL[32])
        assert d1["max_div_E"] <= (1e-13 if prec == 64 else 1e-6) * d1["max_E_hat"]
        assert d1["max_div_B"] <= (1e-13 if prec == 64 else 1e-6) * d1["max_B_hat"]
    # the plane wave alone: exact phase exp(-i n c k0 dt), zero dispersion
    k0 = 2 * np.pi * 4 / (g.Nz * g.dz)
    with lib.Context(g, None, dt, prec) as ctx:
        ctx.set_fields(pw)
        ctx.advance(20)
        got = ctx.get_field(-1)
    expect = np.exp(-1j * 20 * g.c * k0 * dt) * pw
    assert np.max(np.abs(got - expect)) <= (1e-12 if prec == 64 else 2e-5)


def test_nyquist_corner_and_static_modes(lib):
    g = W.GridSpec(8, 8, 8, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    dt = g.courant_dt()
    x = np.arange(8)
    ph = np.exp(1j * np.pi * -(x[:, None, None] + x[None, :, None] + x[None, None, :]))
    e = np.array([1.0, -1.0, 0.0]) / math.sqrt(2)
    kh = -np.ones(3) / math.sqrt(3)
    b = np.cross(kh, e)
    f0 = np.zeros((6, 8, 8, 8), dtype=np.complex128)
    for a in range(3):
        f0[a] = e[a] * ph
        f0[3 + a] = b[a] * ph
    f0 += np.array([1.0, 2.0, 3.0, -1.0, 0.5, 0.25])[:, None, None, None]   # uniform (k = 0) part
    with lib.Context(g, None, dt, 64) as ctx:
        ctx.set_fields(f0)
        ctx.advance(1)
        got = ctx.get_field(-1)
    want = O.advance(f0, ogrid(g), dt, 1)
    assert rel(got, want) <= 1e-13
    static = np.array([1.0, 2.0, 3.0, -1.0, 0.5, 0.25])[:, None, None, None]
    assert np.max(np.abs(got - (static - (f0 - static)))) < 1e-12


def test_reversibility_and_semigroup(lib):
    g = W.plain_grid(32)
    dt = g.courant_dt()
    f0 = W.random_divfree_field(g, 4)
    with lib.Context(g, None, dt, 64) as ctx:
        ctx.set_fields(f0)
        ctx.advance(12)
        a = ctx.get_field(-1)
        ctx.set_dt(-dt)
        ctx.advance(12)
        back = ctx.get_field(-1)
        ctx.set_fields(f0)
        ctx.set_dt(12 * dt)
        ctx.advance(1)
        b = ctx.get_field(-1)
    assert rel(back, f0) <= 1e-12
    assert rel(a, b) <= 1e-12


def test_zero_steps_and_degenerate_grid(lib):
    g = W.GridSpec(1, 1, 1, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1.0)
    f0 = W.random_complex_field((6, 1, 1, 1), 3)
    with lib.Context(g, None, 0.5, 64) as ctx:
        ctx.set_fields(f0)
        ctx.advance(0)
        assert np.array_equal(ctx.get_field(-1), f0)
        ctx.advance(5)
        assert np.max(np.abs(ctx.get_field(-1) - f0)) < 1e-15


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", ["flat", "gauss", "gauss_ellip"])
def test_pulse_init_parity(lib, prec, kind):
    if kind == "flat":
        g, m, p = W.flat_top_workload(N=40)
    else:
        g, m, p, _, _ = W.tight_focus_workload(N=40)
        p.div_project = 0
        if kind == "gauss_ellip":
            p.ellipticity, p.cep, p.pol_angle = 0.6, 1.1, 0.4
    with lib.Context(g, m, 1e-17, prec) as ctx:
        ctx.init_pulse(p)
        got = ctx.get_field(-1)
    want = O.init_fields(ogrid(g), O.Mapping(m.R0, m.L), opulse(p))
    assert np.max(np.abs(want)) > 0
    assert rel(got, want) <= (1e-13 if prec == 64 else 1e-6)


@pytest.mark.parametrize("prec", [64, 32])
def test_pulse_init_with_projection(lib, prec):
    g, m, p, _, _ = W.tight_focus_workload(N=32)
    p.div_project = 1
    with lib.Context(g, m, 1e-17, prec) as ctx:
        ctx.init_pulse(p)
        got = ctx.get_field(-1)
        d = ctx.diagnostics()
    want = O.init_fields(ogrid(g), O.Mapping(m.R0, m.L), opulse(p))
    assert rel(got, want) <= TOL[prec]
    assert d["max_div_E"] <= (1e-13 if prec == 64 else 1e-6) * d["max_E_hat"]


@pytest.mark.parametrize("prec", [64, 32])
def test_sampling_parity(lib, prec):
    g = W.GridSpec(24, 20, 18, 0.5, 0.7, 0.4, -7.0, -7.0, -3.6, 1.0)
    m = W.MappingSpec(R0=10.0, L=4.0)
    f = W.random_complex_field((6, g.Nz, g.Ny, g.Nx), 11)
    with lib.Context(g, m, 0.1, prec) as ctx:
        ctx.set_fields(f)
        for t, xp in ((10.0, 0.3), (10.0, -1.2), (4.0, -5.1), (13.5, 2.2)):
            ctx.set_time(t)
            got = ctx.sample_focal_plane(xp, 13, 11, -3.0, 3.0, -2.5, 2.9, comps=(0, 2, 4))
            want = O.sample_plane(f, ogrid(g), O.Mapping(m.R0, m.L), xp,
                                  *W.plane_points(dict(ny=13, nz=11, y0=-3.0, y1=3.0, z0=-2.5, z1=2.9)),
                                  t, comps=(0, 2, 4))
            if np.linalg.norm(want) == 0:
                assert np.max(np.abs(got)) == 0
            else:
                assert rel(got, want) <= TOL[prec]


def test_sampling_at_nodes_returns_grid_values(lib):
    g = W.GridSpec(16, 12, 10, 0.5, 0.5, 0.5, -4.0, -3.0, -2.5, 1.0)
    m = W.MappingSpec(R0=1e6, L=1e6)
    f = W.random_complex_field((6, g.Nz, g.Ny, g.Nx), 5)
    with lib.Context(g, m, 0.1, 64) as ctx:
        ctx.set_fields(f)
        ctx.set_time(1e6)
        x_i = g.x_min + 5 * g.dx
        got = ctx.sample_focal_plane(x_i, 12, 10, g.y_min, g.y_min + 12 * g.dy, g.z_min,
                                     g.z_min + 10 * g.dz, comps=(1, 5))
    assert np.max(np.abs(got - f[[1, 5], :, :, 5])) < 1e-12


def test_diagnostics_parity_with_longitudinal_part(lib):
    g = W.GridSpec(12, 10, 8, 0.5, 0.7, 0.4, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, g.Nz, g.Ny, g.Nx), 9)
    with lib.Context(g, None, 0.1, 64) as ctx:
        ctx.set_fields(f)
        d = ctx.diagnostics()
    w = O.diagnostics(f, ogrid(g))
    for k in ("energy", "energy_E", "energy_B", "max_div_E", "max_div_B", "max_E_hat", "max_B_hat"):
        assert abs(d[k] - w[k]) <= 1e-12 * abs(w[k]), k


def test_invalid_state_and_arguments(lib):
    g = W.plain_grid(8)
    with lib.Context(g, None, 0.1, 64) as ctx:
        with pytest.raises(lib.PsatdError):
            ctx.advance(-1)
        with pytest.raises(lib.PsatdError):
            ctx.set_field(6, np.zeros((8, 8, 8)))
        with pytest.raises(lib.PsatdError):
            ctx.sample_focal_plane(0.0, 0, 4, 0, 1, 0, 1)
        with pytest.raises(lib.PsatdError):
            ctx.init_pulse(W.PulseSpec(lam=-1.0))   # no mapping and a bad wavelength


# ---------------------------------------------------------------------------
# Full-size tight-focus workload (256^3, the benchmarked launch sequence):
# init + 378 steps to the focus t = R0/c + focal-plane sampling, against the
# oracle's single exact step of 378 dt (the solver is exact in time).
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def focus_reference():
    g, m, p, n_steps, plane = W.tight_focus_workload(N=256)
    dt = (m.R0 / g.c) / n_steps
    og, om = ogrid(g), O.Mapping(m.R0, m.L)
    f0 = O.init_fields(og, om, opulse(p))
    f1 = O.advance_exact(f0, og, n_steps * dt)
    ys, zs = W.plane_points(plane)
    ref = O.sample_plane(f1, og, om, plane["x_p"], ys, zs, n_steps * dt, comps=(0, 1, 2))
    e0 = O.diagnostics(f0, og)["energy"]
    return g, m, p, n_steps, plane, dt, ref, e0


@pytest.mark.parametrize("prec", [64, 32])
def test_tight_focus_256_full_size(lib, focus_reference, prec):
    g, m, p, n_steps, plane, dt, ref, e0 = focus_reference
    with lib.Context(g, m, dt, prec) as ctx:
        ctx.init_pulse(p)
        ctx.advance(n_steps)
        got = ctx.sample_focal_plane(plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"],
                                     plane["z0"], plane["z1"], comps=(0, 1, 2))
        d = ctx.diagnostics()
    assert np.max(np.abs(ref)) > 0
    assert rel(got, ref) <= (1e-10 if prec == 64 else 1e-4)
    # The per-mode coefficients (C, S, k^) are rounded once to the storage type
    # and the same rounding repeats every step, so the energy drift grows
    # linearly: at most 2 * c0 * u per step with u the unit roundoff and c0 ~ 4
    # (C, S and the k^ products), i.e. 8 u n after n steps.
    u = 2.0 ** -53 if prec == 64 else 2.0 ** -24
    assert abs(d["energy"] / e0 - 1) <= max(8 * u * n_steps, 1e-12)
    assert d["max_div_E"] <= (1e-12 if prec == 64 else 1e-5) * d["max_E_hat"]


def test_tight_focus_256_full_size_real_fields(lib, focus_reference):
    """The same job with real float32 field storage (half the bytes per step)."""
    g, m, p, n_steps, plane, dt, ref, e0 = focus_reference
    with lib.Context(g, m, dt, 32, real=True) as ctx:
        ctx.init_pulse(p)
        ctx.advance(n_steps)
        got = ctx.sample_focal_plane(plane["x_p"], plane["ny"], plane["nz"], plane["y0"], plane["y1"],
                                     plane["z0"], plane["z1"], comps=(0, 1, 2))
        d = ctx.diagnostics()
    assert rel(got, ref) <= 1e-4
    assert abs(d["energy"] / e0 - 1) <= 8 * 2.0 ** -24 * n_steps
    assert d["max_div_E"] <= 1e-5 * d["max_E_hat"]


# ---------------------------------------------------------------------------
# Register-resident kernels (axis lengths 64, 128, 256, 512, 1024; z lengths
# without a fused kernel take forward z, the per-mode update and inverse z as
# three launches) against the oracle
# and against the generic shared-memory kernels on the same inputs.
# ---------------------------------------------------------------------------
FAST_SHAPES = [(64, 64, 64), (256, 64, 128), (128, 256, 64), (64, 128, 256), (512, 16, 64), (48, 64, 128),
               (1024, 4, 8), (8, 1024, 4), (8, 4, 1024), (4, 8, 512), (16, 512, 4), (32, 1024, 2)]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("shape", FAST_SHAPES)
def test_fast_kernels_match_oracle_and_generic(lib, prec, shape):
    Nx, Ny, Nz = shape
    g = W.GridSpec(Nx, Ny, Nz, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, Nz, Ny, Nx), seed=Nx * 3 + Ny + Nz)
    dt = 0.41
    out = {}
    for path in (lib.PATH_AUTO, lib.PATH_REGISTER, lib.PATH_GENERIC):
        with lib.Context(g, None, dt, prec) as ctx:
            ctx.set_kernel_path(path)
            ctx.set_fields(f)
            ctx.fft(lib.FORWARD)
            F = ctx.get_field(-1)
            ctx.set_fields(f)
            ctx.advance(2)
            out[path] = (F, ctx.get_field(-1))
    F_ref = O.fft3(f)
    step_ref = O.advance(f, ogrid(g), dt, 2)
    for path in out:
        assert rel(out[path][0], F_ref) <= TOL[prec]
        assert rel(out[path][1], step_ref) <= 2 * TOL[prec]
    assert rel(out[lib.PATH_AUTO][1], out[lib.PATH_GENERIC][1]) <= 2 * TOL[prec]
    assert rel(out[lib.PATH_REGISTER][1], out[lib.PATH_GENERIC][1]) <= 2 * TOL[prec]


# x lengths 512 / 1024 in float32 with a z length that has no fused z kernel:
# the step takes z, y, then the x pass with the update fused into it, then y, z.
@pytest.mark.parametrize("shape", [(1024, 6, 36), (512, 10, 300), (1024, 1, 2), (1024, 16, 1), (512, 3, 5)])
def test_row_fused_kspace_step_matches_oracle(lib, shape):
    Nx, Ny, Nz = shape
    g = W.GridSpec(Nx, Ny, Nz, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, Nz, Ny, Nx), seed=Nx + 5 * Ny + Nz)
    dt = 0.37
    with lib.Context(g, None, dt, 32) as ctx:
        ctx.set_fields(f)
        ctx.profile_enable(True)
        ctx.advance(3)
        prof = ctx.profile_read()
        got = ctx.get_field(-1)
    assert prof["kspace_z"][1] == 3                     # one fused launch per step
    assert "plane_xy" not in prof and prof.get("fft_x", (0, 0))[1] == 0
    assert rel(got, O.advance(f, ogrid(g), dt, 3)) <= 3 * TOL[32]


def test_bounded_wait_reports_timeout_and_context_survives(lib):
    import ctypes as C
    g = W.plain_grid(64)
    f0 = W.random_divfree_field(g, 5)
    with lib.Context(g, None, g.courant_dt(), 32) as ctx:
        st = lib.lib().psatd_selftest_wait_timeout(ctx._ptr)
        assert st == lib.ERR_TIMEOUT
        assert b"bounded device wait" in lib.lib().psatd_last_error(ctx._ptr)
        ctx.synchronize()                       # error word was cleared
        ctx.set_fields(f0)
        ctx.advance(2)
        got = ctx.get_field(-1)
    assert rel(got, O.advance(f0, ogrid(g), g.courant_dt(), 2)) <= TOL[32]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("Nz", [6, 64])
def test_plane_cluster_kernel_256_planes(lib, prec, Nz):
    """256 x 256 planes (the cluster x+y kernel in FP32) against the oracle and
    the per-axis kernels, for a thin, a fast-z and the full-size z extent."""
    g = W.GridSpec(256, 256, Nz, 0.5, 0.7, 0.3, 0.0, 0.0, 0.0, 1.0)
    f = W.random_complex_field((6, Nz, 256, 256), seed=Nz)
    dt = 0.29
    res = {}
    for path in (lib.PATH_AUTO, lib.PATH_REGISTER):
        with lib.Context(g, None, dt, prec) as ctx:
            ctx.set_kernel_path(path)
            ctx.set_fields(f)
            ctx.fft(lib.FORWARD)
            F = ctx.get_field(-1)
            ctx.fft(lib.INVERSE)
            back = ctx.get_field(-1) / g.cells
            ctx.set_fields(f)
            ctx.advance(1)
            res[path] = (F, back, ctx.get_field(-1))
    F_ref = O.fft3(f)
    step_ref = O.advance(f, ogrid(g), dt, 1)
    for path, (F, back, st) in res.items():
        assert rel(F, F_ref) <= TOL[prec]
        assert rel(back, f) <= TOL[prec]
        assert rel(st, step_ref) <= TOL[prec]
