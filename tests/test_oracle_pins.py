"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each check compares the oracle with something other than itself: a brute-force
sum, a closed-form solution of the vacuum Maxwell equations, an invariant, a
geometric brute force, or a number printed in the paper (tests/golden/).
The last test plants plausible mistakes in the oracle's update and shows that
these pins catch every one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import psatd_oracle as O
from paper_2010_00409_gb300 import workloads as W

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def small_grid(Nx=8, Ny=6, Nz=10, c=1.0):
    return O.Grid(Nx, Ny, Nz, 0.5, 0.7, 0.4, 0.0, 0.0, 0.0, c)


# --------------------------------------------------------------------------- FFT
# lengths above 32 take the recursive split (64 = 8 x 8, 40 = 5 x 8, 35 = 5 x 7,
# 96 = 8 x 12 then 12 directly); 37 is prime and summed directly
@pytest.mark.parametrize("shape", [(4, 4, 4), (6, 6, 6), (10, 6, 8), (6, 10, 12), (1, 3, 5),
                                   (2, 3, 64), (1, 40, 3), (35, 2, 1), (1, 1, 96), (1, 2, 37)])
def test_fft3_equals_bruteforce_sum(shape):
    f = W.random_complex_field((2,) + shape, seed=1)
    F = O.fft3(f)
    Fb = O.dft3_naive(f, -1)
    assert np.max(np.abs(F - Fb)) <= 1e-12 * np.max(np.abs(Fb))
    back = O.ifft3(F)
    assert np.max(np.abs(back - f)) <= 1e-14 * np.max(np.abs(f)) * 10
    assert np.max(np.abs(O.idft3_naive(Fb) - f)) <= 1e-12 * np.max(np.abs(f))


def test_fft3_split_catches_a_planted_twiddle_mistake(monkeypatch):
    """A twiddle of the split with the wrong index (r*k2 instead of r*k1) is
    caught by the brute-force comparison."""
    good = O._unit_roots
    calls = {"n": 0}

    def bad(e, N, sign):
        calls["n"] += 1
        return good(e.T if e.shape[0] != e.shape[1] else e + 1, N, sign)

    f = W.random_complex_field((1, 1, 2, 64), seed=4)
    Fb = O.dft3_naive(f, -1)
    monkeypatch.setattr(O, "_unit_roots", bad)
    F = O.fft3(f)
    assert calls["n"] > 0
    assert np.max(np.abs(F - Fb)) > 1e-3 * np.max(np.abs(Fb))


def test_fft_sign_convention_puts_plane_wave_at_plus_m():
    # R1: forward kernel exp(-i k x), so exp(+i k_m x) lands on bin +m
    N = 8
    x = np.arange(N)
    f = np.exp(2j * np.pi * 3 * x / N)[None, None, :] * np.ones((1, 1, 1))
    F = O.fft3(f)
    assert abs(F[0, 0, 3] - N) < 1e-12 and np.sum(np.abs(F)) - N < 1e-10


def test_wavenumbers_nyquist_negative():
    # R2: even N puts the Nyquist bin at m = -N/2
    k = O.wavenumbers(6, 1.0)
    assert np.allclose(k / (2 * np.pi / 6), [0, 1, 2, -3, -2, -1])
    k = O.wavenumbers(5, 2.0)
    assert np.allclose(k / (2 * np.pi / 10), [0, 1, 2, -2, -1])


# ----------------------------------------------------- closed forms of Maxwell
def eigenmode(grid, m, sign=+1, pol=None):
    """Single Fourier mode with B = sign * k^ x E (sign=+1 travels along +k)."""
    kx = 2 * np.pi * m[0] / (grid.Nx * grid.dx)
    ky = 2 * np.pi * m[1] / (grid.Ny * grid.dy)
    kz = 2 * np.pi * m[2] / (grid.Nz * grid.dz)
    k = np.array([kx, ky, kz])
    kh = k / np.linalg.norm(k)
    if pol is None:
        pol = np.cross(kh, [0.3, -0.5, 0.8])
    e = np.asarray(pol, dtype=float) - kh * np.dot(kh, pol)
    e /= np.linalg.norm(e)
    b = sign * np.cross(kh, e)
    x, y, z = grid.coords()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ph = np.exp(1j * (kx * (X - grid.x_min) + ky * (Y - grid.y_min) + kz * (Z - grid.z_min)))
    f = np.zeros((6,) + ph.shape, dtype=np.complex128)
    for a in range(3):
        f[a] = e[a] * ph
        f[3 + a] = b[a] * ph
    return f, np.linalg.norm(k)


def test_plane_wave_exact_phase_c1_geometry():
    """x-polarised mode along z, 4 periods in a 64^3 box at dt_C: after n steps the
    field is exp(-i n c k0 dt) times the start (zero dispersion, Sec. 2.1)."""
    g = W.plain_grid(64)
    grid = O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, c=g.c)
    f0 = W.plane_wave_mode(g, periods=4)
    dt = O.courant_dt(grid)
    k0 = 2 * np.pi * 4 / (g.Nz * g.dz)
    assert abs(g.c * k0 * dt - 0.2267249) < 1e-6      # 2 pi / (16 sqrt 3)
    f = O.advance(f0, grid, dt, 20)
    expect = np.exp(-1j * 20 * g.c * k0 * dt) * f0
    assert np.max(np.abs(f - expect)) < 1e-13


@pytest.mark.parametrize("sign", [+1, -1])
def test_oblique_eigenmodes_rotate_with_exact_frequency(sign):
    grid = small_grid()
    f0, kmag = eigenmode(grid, (1, -2, 3), sign)
    dt = 0.37
    f = O.advance(f0, grid, dt, 5)
    expect = np.exp(-1j * sign * 5 * grid.c * kmag * dt) * f0
    assert np.max(np.abs(f - expect)) < 1e-13


def test_zero_dispersion_phase_depends_only_on_kmag():
    grid = O.Grid(8, 8, 8, 1.0, 1.0, 1.0, c=1.0)
    fa, ka = eigenmode(grid, (3, 0, 0))
    fb, kb = eigenmode(grid, (0, 0, 3))
    assert abs(ka - kb) < 1e-15
    a = O.advance(fa, grid, 0.9, 3)
    b = O.advance(fb, grid, 0.9, 3)
    ra = a[1][0, 0, 1] / fa[1][0, 0, 1]
    rb = b[0][1, 0, 0] / fb[0][1, 0, 0]
    assert abs(ra - rb) < 1e-13 and abs(ra - np.exp(-3j * 0.9 * ka)) < 1e-13


def test_nyquist_corner_flips_sign_each_step():
    # |k| = sqrt(3) pi / d with dt_C gives c|k|dt = pi: C = -1, S = 0
    grid = O.Grid(8, 8, 8, 1.0, 1.0, 1.0, c=1.0)
    dt = O.courant_dt(grid)
    f0, kmag = eigenmode(grid, (-4, -4, -4))
    assert abs(kmag * dt - np.pi) < 1e-14
    f1 = O.advance(f0, grid, dt, 1)
    assert np.max(np.abs(f1 + f0)) < 1e-13


def test_uniform_fields_are_static():
    # R3: k = 0 keeps uniform E and B unchanged
    grid = small_grid()
    f0 = np.zeros((6, grid.Nz, grid.Ny, grid.Nx), dtype=np.complex128)
    for a, v in enumerate([1.0, -2.0, 0.5, 3.0, 0.25, -1.0]):
        f0[a] = v
    f = O.advance(f0, grid, 1.3, 4)
    assert np.max(np.abs(f - f0)) < 1e-14


def test_longitudinal_E_removed_and_longitudinal_B_scaled():
    # Eq. 3 removes k^(k^.E) every step; Eq. 4 (R4) gives B_par -> C B_par
    grid = small_grid()
    m = (1, 1, 2)
    k = np.array([2 * np.pi * m[0] / (grid.Nx * grid.dx), 2 * np.pi * m[1] / (grid.Ny * grid.dy),
                  2 * np.pi * m[2] / (grid.Nz * grid.dz)])
    kh = k / np.linalg.norm(k)
    x, y, z = grid.coords()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    ph = np.exp(1j * (k[0] * X + k[1] * Y + k[2] * Z))
    f0 = np.zeros((6,) + ph.shape, dtype=np.complex128)
    for a in range(3):
        f0[a] = kh[a] * ph
        f0[3 + a] = kh[a] * ph
    dt = 0.21
    f = O.advance(f0, grid, dt, 1)
    C = math.cos(grid.c * np.linalg.norm(k) * dt)
    assert np.max(np.abs(f[0:3])) < 1e-14
    assert np.max(np.abs(f[3:6] - C * f0[3:6])) < 1e-14


# ------------------------------------------------------------------- invariants
def c1_random_state(seed=0, N=16):
    g = W.plain_grid(N)
    grid = O.Grid(g.Nx, g.Ny, g.Nz, g.dx, g.dy, g.dz, c=g.c)
    f = W.random_divfree_field(g, seed) + 0.3 * W.plane_wave_mode(g, periods=2)
    return grid, f, O.courant_dt(grid)


def test_energy_conserved_parseval():
    grid, f0, dt = c1_random_state(0)
    e0 = O.diagnostics(f0, grid)["energy"]
    f = f0
    for _ in range(20):
        f = O.psatd_step(f, grid, dt)
        assert abs(O.diagnostics(f, grid)["energy"] / e0 - 1) < 1e-13


def test_divergence_free_preserved():
    grid, f0, dt = c1_random_state(1)
    d0 = O.diagnostics(f0, grid)
    assert d0["max_div_E"] <= 1e-13 * d0["max_E_hat"]
    f = O.advance(f0, grid, dt, 10)
    d = O.diagnostics(f, grid)
    assert d["max_div_E"] <= 1e-13 * d["max_E_hat"]
    assert d["max_div_B"] <= 1e-13 * d["max_B_hat"]


def test_reversibility():
    grid, f0, dt = c1_random_state(2)
    f = O.advance(O.advance(f0, grid, dt, 10), grid, -dt, 10)
    assert np.max(np.abs(f - f0)) <= 1e-13 * np.max(np.abs(f0))


def test_semigroup_n_steps_equal_one_long_step():
    grid, f0, dt = c1_random_state(0)
    a = O.advance(f0, grid, dt, 12)
    b = O.advance_exact(f0, grid, 12 * dt)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(f0))


# ------------------------------------------------------------- pulse models
def test_theta_from_fnumber_matches_paper():
    th = O.theta_from_fnumber(GOLD["fig1_fnumber"]["value"])
    assert abs(th - GOLD["fig1_theta_rad_approx"]["value"]) < GOLD["fig1_theta_rad_approx"]["tol"]


def test_F_series_close_to_integral_below_two():
    lim = GOLD["sec321_F_series_valid_below"]["value"]
    for t in np.linspace(0.05, lim, 12):
        rel = abs(O.F_series(t) / O.F_exact(t) - 1)
        assert rel < (2e-3 if t <= 1.5 else 1.2e-2)
    # small-angle limit: F ~ theta0^2/4 (Laplace)
    assert abs(O.F_exact(0.01) / (0.01 ** 2 / 4) - 1) < 1e-4


def test_u_ts_and_u_l_shapes():
    th, eps = 1.0, 0.1
    assert O.u_ts_flat(0.0, th, eps) == 1.0
    assert O.u_ts_flat(th - eps / 2, th, eps) == 1.0
    assert abs(O.u_ts_flat(th, th, eps) - 0.5) < 1e-15
    assert O.u_ts_flat(th + eps / 2 + 1e-9, th, eps) == 0.0
    lam, L = 1.0, 2.0
    assert abs(O.u_l_flat(lam / 4, lam, L) - math.cos(math.pi / 8) ** 2) < 1e-15
    assert O.u_l_flat(L / 2 + 1e-9, lam, L) == 0.0


def _pulse_points(pulse, mapping, c=1.0, n=4000, seed=0):
    rng = np.random.default_rng(seed)
    R = mapping.R0 + (rng.random(n) - 0.5) * mapping.L
    a = rng.random(n) * 1.1
    ph = rng.random(n) * 2 * np.pi
    X = -R * np.cos(a)
    Y = R * np.sin(a) * np.cos(ph)
    Z = R * np.sin(a) * np.sin(ph)
    E, B = O._pulse_fields_at(X, Y, Z, pulse, mapping, c)
    return X, Y, Z, E, B


@pytest.mark.parametrize("kind,ell", [(O.FLAT_TOP, 0.0), (O.GAUSSIAN, 0.0), (O.GAUSSIAN, 0.7), (O.FLAT_TOP, 1.0)])
def test_pulse_fields_transverse_equal_and_converging(kind, ell):
    m = O.Mapping(R0=16.0, L=2.0)
    p = O.Pulse(kind=kind, lam=1.0, theta=0.5, eps=0.1, P0=1.0, n_cycles=1.0,
                cep=0.3, ellipticity=ell, pol_angle=0.4)
    X, Y, Z, E, B = _pulse_points(p, m)
    Rv = np.stack([X, Y, Z])
    scale = np.max(np.abs(E)) + 1e-300
    assert np.max(np.abs(np.sum(E * Rv, 0))) / np.max(np.linalg.norm(Rv, axis=0)) < 1e-13 * scale
    assert np.max(np.abs(np.sum(E * B, 0))) < 1e-13 * scale ** 2
    assert np.max(np.abs(np.linalg.norm(E, axis=0) - np.linalg.norm(B, axis=0))) < 1e-13 * scale
    S = np.cross(E.T, B.T).T
    inward = -np.sum(S * Rv, 0)
    assert np.all(inward >= -1e-12 * scale ** 2) and np.max(inward) > 0


def _eq7_table(lam, L, dz):
    """Samples of Eq. 7's analytic waveform a = -i e^{i k zeta} cos^2(pi zeta / L)
    on |zeta| <= L/2 (its real part with a carrier phase phi is sin(k zeta + phi) cos^2)."""
    z = np.arange(-L / 2, L / 2 + dz / 2, dz)
    return -1j * np.exp(2j * np.pi * z / lam) * np.cos(np.pi * z / L) ** 2, float(z[0])


@pytest.mark.parametrize("cep,ell", [(0.0, 0.0), (1.1, 0.0), (0.4, 0.6)])
def test_profile_pulse_reproduces_flat_top_from_tabulated_eq7(cep, ell):
    # R21: the tabulated kind with Eq. 7's waveform as its table is the flat-top
    # pulse of Eq. 8, up to the linear-interpolation error (k dz)^2 / 8 ~ 1e-6
    m = O.Mapping(R0=16.0, L=2.0)
    dz = 1.0 / 2000
    a, z0 = _eq7_table(1.0, m.L, dz)
    flat = O.Pulse(kind=O.FLAT_TOP, lam=1.0, theta=0.5, eps=0.1, P0=1.0, cep=cep, ellipticity=ell, pol_angle=0.3)
    prof = O.Pulse(kind=O.PROFILE, lam=1.0, theta=0.5, eps=0.1, P0=1.0, cep=cep, ellipticity=ell, pol_angle=0.3,
                   profile=a, profile_z0=z0, profile_dz=dz)
    Xf, Yf, Zf, Ef, Bf = _pulse_points(flat, m)
    Xp, Yp, Zp, Ep, Bp = _pulse_points(prof, m)
    assert np.array_equal(Xf, Xp)
    scale = np.max(np.abs(Ef))
    assert scale > 0
    assert np.max(np.abs(Ep - Ef)) < 5e-6 * scale
    assert np.max(np.abs(Bp - Bf)) < 5e-6 * scale


def test_profile_pulse_is_zero_outside_its_table_and_the_shell():
    m = O.Mapping(R0=16.0, L=2.0)
    a = np.ones(11, dtype=np.complex128)
    p = O.Pulse(kind=O.PROFILE, lam=1.0, theta=0.5, eps=0.1, P0=1.0, profile=a, profile_z0=-0.5, profile_dz=0.1)
    zeta = np.array([-0.9, -0.51, -0.5, 0.0, 0.5, 0.51, 0.99, 1.2])
    R = m.R0 + zeta
    u = O.pulse_scalar(-R, 0 * R, 0 * R, p, m, 1.0, 0.0)
    A = O.flat_top_A(1.0, 1.0, 0.5)
    want = np.where(np.abs(zeta) <= 0.5, A / R, 0.0)
    assert np.allclose(u, want, rtol=1e-15, atol=0)


def _cycle_averaged_power(pulse, mapping, c, n_alpha=4000, n_s=64):
    """c/(8 pi) * R0^2 * integral of 2<u^2> over the sphere R = R0 (one carrier period)."""
    amax = min(math.pi, 3.0 * pulse.theta)
    a = (np.arange(n_alpha) + 0.5) * amax / n_alpha
    s = (np.arange(n_s) + 0.5) / n_s * pulse.lam - pulse.lam / 2
    A, S = np.meshgrid(a, s, indexing="ij")
    R = mapping.R0 + S
    X = -R * np.cos(A)
    Y = R * np.sin(A)
    u = O.pulse_scalar(X, Y, 0 * X, pulse, mapping, c, 0.0)
    mean_u2 = np.mean((u * R) ** 2, axis=1) / mapping.R0 ** 2       # <u^2> on R0
    integrand = 2 * mean_u2 * np.sin(a)
    return c / (8 * math.pi) * mapping.R0 ** 2 * 2 * math.pi * np.sum(integrand) * amax / n_alpha


def test_flat_top_amplitude_carries_P0():
    # Eq. 9: with a sharp edge and a long envelope, the cycle-averaged power
    # through the sphere R = R0 equals P0
    c = 3.0
    m = O.Mapping(R0=50.0, L=400.0)
    p = O.Pulse(kind=O.FLAT_TOP, lam=1.0, theta=0.8, eps=1e-4, P0=2.5)
    P = _cycle_averaged_power(p, m, c)
    assert abs(P / p.P0 - 1) < 2e-3


def test_gaussian_amplitude_carries_P0():
    # Sec. 3.2.1: E0 normalises the power at the pulse peak to P0 (series F)
    c = 3.0
    m = O.Mapping(R0=50.0, L=4000.0)
    p = O.Pulse(kind=O.GAUSSIAN, lam=1.0, theta=0.3, eps=1e-4, P0=2.5, n_cycles=400.0)
    P = _cycle_averaged_power(p, m, c)
    assert abs(P / p.P0 - 1) < 2e-3


# ------------------------------------------------------------------ mapping
def _overlap_bruteforce(R0, L, theta, n=300):
    """Smallest shift D along +x such that the sector and its copy do not meet,
    found by bisection over a dense sampling of the sector in the x-rho plane."""
    Rmin, Rmax = R0 - L / 2, R0 + L / 2
    R = np.linspace(Rmin, Rmax, n)
    a = np.linspace(0, theta, n)
    RR, AA = np.meshgrid(R, a, indexing="ij")
    xs = (-RR * np.cos(AA)).ravel()
    rs = (RR * np.sin(AA)).ravel()

    def overlaps(D):
        x2 = xs + D
        R2 = np.sqrt(x2 ** 2 + rs ** 2)
        a2 = np.arctan2(rs, -x2)
        return np.any((R2 >= Rmin) & (R2 <= Rmax) & (a2 <= theta))

    lo, hi = 0.0, 2 * Rmax
    for _ in range(50):
        mid = (lo + hi) / 2
        if overlaps(mid):
            lo = mid
        else:
            hi = mid
    return hi


@pytest.mark.parametrize("theta", [0.3, 0.8, 1.0, 1.3])
def test_d_min_matches_geometric_bruteforce(theta):
    R0, L = 16.0, 2.0
    assert abs(O.d_min(R0, L, theta) - _overlap_bruteforce(R0, L, theta)) < 0.06


def test_d_min_printed_value():
    # Fig. 4a quotes D_min/L ~ 1.9 for f = 0.3, R0 = 16 lam, L = 2 lam, eps = 0.1;
    # it is matched by Eq. 12 evaluated at theta + eps (R11)
    g = GOLD
    R0, L = g["sec31_R0_over_lambda"]["value"], g["sec31_L_over_lambda"]["value"]
    th = O.theta_from_fnumber(g["fig1_fnumber"]["value"]) + g["sec31_eps_rad"]["value"]
    assert abs(O.d_min(R0, L, th) / L - g["fig4a_Dmin_over_L_approx"]["value"]) < g["fig4a_Dmin_over_L_approx"]["tol"]


def test_mapping_T_properties():
    x_min, D = -23.0, 7.0
    x = np.linspace(-80, 40, 1001)
    t = O.mapping_T(x, x_min, D)
    assert np.all(t >= x_min) and np.all(t < x_min + D)
    assert np.allclose(O.mapping_T(t, x_min, D), t)
    assert np.allclose(O.mapping_T(x + 3 * D, x_min, D), t, atol=1e-12)
    assert np.allclose((x - t) / D, np.round((x - t) / D), atol=1e-9)


def test_indicator_S_branches():
    m = O.Mapping(R0=16.0, L=2.0)       # R_min 15, R_max 17
    c = 1.0
    I = lambda x, y, z, t: float(O.indicator_S(x, y, z, t, m, c))
    # converging phase (r < 0): keep R in [-r, -l), x <= 0
    t = 5.0                              # l = -12, r = -10
    assert I(-11.0, 0, 0, t) == 1.0
    assert I(-12.0, 0, 0, t) == 0.0      # R >= -l
    assert I(-9.0, 0, 0, t) == 0.0       # R < -r
    assert I(0.5, 10.9, 0, t) == 0.0     # x > 0
    # straddling (l <= 0 <= r): x < 0 keeps R <= L; x >= 0 keeps R <= r (R8)
    t = 16.0                             # l = -1, r = 1
    assert I(-1.5, 0, 0, t) == 1.0
    assert I(-2.5, 0, 0, t) == 0.0
    assert I(0.5, 0, 0, t) == 1.0
    assert I(1.5, 0, 0, t) == 0.0
    assert I(0.0, 0, 0, t) == 1.0
    # diverging (l > 0): keep l < R <= r and x >= 0
    t = 20.0                             # l = 3, r = 5
    assert I(4.0, 0, 0, t) == 1.0
    assert I(3.0, 0, 0, t) == 0.0
    assert I(5.5, 0, 0, t) == 0.0
    assert I(-4.0, 0, 0, t) == 0.0


def test_init_single_replica_equals_pulse_when_D_ge_Dmin():
    lam = 1.0
    m = O.Mapping(R0=8.0, L=2.0)
    p = O.Pulse(kind=O.FLAT_TOP, lam=lam, theta=0.6, eps=0.1, P0=1.0)
    D = 1.05 * O.d_min(m.R0, m.L, p.theta + p.eps / 2)
    N = 24
    grid = O.Grid(N, 20, 20, D / N, 1.0, 1.0, -m.R_min - D, -10.0, -10.0, 1.0)
    f = O.init_fields(grid, m, p)
    x, y, z = grid.coords()
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    best = np.zeros((6,) + X.shape)
    for k in range(-3, 4):
        E, B = O._pulse_fields_at(X + k * D, Y, Z, p, m, 1.0)
        nz = np.abs(E).sum(0) > 0
        assert not np.any(nz & (np.abs(best[:3]).sum(0) > 0)), "replicas overlap"
        best[:3] += E
        best[3:] += B
    assert np.max(np.abs(f.real - best)) < 1e-14 and np.max(np.abs(best)) > 0


# ------------------------------------------------------------------ sampling
def test_sampling_at_nodes_returns_grid_values():
    grid = O.Grid(8, 6, 10, 0.5, 0.7, 0.4, -2.0, -2.1, -2.0, 1.0)
    m = O.Mapping(R0=1e6, L=1e6)             # at t = R0/c, I_S = 1 for R < 5e5
    f = W.random_complex_field((6, grid.Nz, grid.Ny, grid.Nx), 3)
    x, y, z = grid.coords()
    i = 5
    out = O.sample_plane(f, grid, m, x[i], y[[0, 2, 5]], z[[1, 9]], 1e6, comps=(0, 4))
    assert np.max(np.abs(out - f[[0, 4]][:, [1, 9]][:, :, [0, 2, 5], i])) < 1e-13


def test_sampling_single_mode_off_grid_closed_form():
    grid = O.Grid(8, 6, 10, 0.5, 0.7, 0.4, -2.0, -2.1, -2.0, 1.0)
    m = O.Mapping(R0=1e6, L=1e6)
    f0, _ = eigenmode(grid, (2, -1, 3))
    kx = 2 * np.pi * 2 / (grid.Nx * grid.dx)
    ky = 2 * np.pi * -1 / (grid.Ny * grid.dy)
    kz = 2 * np.pi * 3 / (grid.Nz * grid.dz)
    ys = np.array([-1.234, 0.1, 0.77])
    zs = np.array([-0.3, 1.9])
    xp = 5.3                                  # maps back into the layer by T
    out = O.sample_plane(f0, grid, m, xp, ys, zs, 1e6, comps=(0, 1, 2))
    xt = O.mapping_T(xp, grid.x_min, grid.D)
    Zs, Ys = np.meshgrid(zs, ys, indexing="ij")
    ph = np.exp(1j * (kx * (xt - grid.x_min) + ky * (Ys - grid.y_min) + kz * (Zs - grid.z_min)))
    e = f0[0:3, 0, 0, 0]
    for a in range(3):
        assert np.max(np.abs(out[a] - e[a] * ph)) < 1e-13


# ------------------------------------------------------ planted mistakes
def _pins_pass(monkeypatch, update):
    monkeypatch.setattr(O, "psatd_update", update)
    results = []
    for fn in (test_plane_wave_exact_phase_c1_geometry,
               lambda: test_oblique_eigenmodes_rotate_with_exact_frequency(+1),
               test_longitudinal_E_removed_and_longitudinal_B_scaled,
               test_energy_conserved_parseval):
        try:
            fn()
            results.append(True)
        except AssertionError:
            results.append(False)
    return all(results)


def test_pins_catch_planted_mistakes(monkeypatch):
    good = O.psatd_update
    assert _pins_pass(monkeypatch, good)

    def flipped_i(Fk, grid, dt):          # wrong sign of i S
        return good(Fk, grid, -dt)

    def no_projection(Fk, grid, dt):      # dropped k^(k^.E) term
        out = good(Fk, grid, dt)
        kx, ky, kz = O._k_grids(grid)
        kx, ky, kz = np.broadcast_arrays(kx, ky, kz)
        km = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
        n = [np.where(km > 0, k / np.where(km > 0, km, 1), 0) for k in (kx, ky, kz)]
        C = np.cos(grid.c * km * dt)
        kE = n[0] * Fk[0] + n[1] * Fk[1] + n[2] * Fk[2]
        for a in range(3):
            out[a] = out[a] + C * n[a] * kE
        return out

    def swapped_components(Fk, grid, dt):  # transposed operand in a cross product
        G = Fk.copy()
        G[[3, 4]] = G[[4, 3]]
        return good(G, grid, dt)

    def sin_for_cos(Fk, grid, dt):         # wrong rotation angle (2 c|k| dt)
        return good(good(Fk, grid, dt), grid, dt)

    for bad in (flipped_i, no_projection, swapped_components, sin_for_cos):
        assert not _pins_pass(monkeypatch, bad), bad.__name__
    monkeypatch.setattr(O, "psatd_update", good)


# ------------------------------------------------------------ real fields (R20)
def _real_field(grid, seed, nyquist=True):
    """Random real fields; with nyquist=False every Nyquist plane of the
    spectrum is zeroed (the field stays real: those planes are self-mirrored)."""
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((6, grid.Nz, grid.Ny, grid.Nx))
    if not nyquist:
        F = np.fft.fftn(f, axes=(1, 2, 3))
        for ax, N in ((3, grid.Nx), (2, grid.Ny), (1, grid.Nz)):
            if N % 2 == 0:
                idx = [slice(None)] * 4
                idx[ax] = N // 2
                F[tuple(idx)] = 0
        f = np.fft.ifftn(F, axes=(1, 2, 3))
        assert np.max(np.abs(f.imag)) < 1e-12
        f = f.real
    return f


def test_complex_step_keeps_band_limited_real_fields_real():
    g = small_grid(8, 6, 10)
    f = _real_field(g, 3, nyquist=False)
    out = O.psatd_step(f.astype(np.complex128), g, 0.37)
    assert np.max(np.abs(out.imag)) <= 1e-13 * np.max(np.abs(out.real))
    assert np.allclose(O.psatd_step_real(f, g, 0.37), out.real, rtol=0, atol=1e-14 * np.max(np.abs(f)))


def _rotate_one_mode(E, B, kvec, c, dt):
    """Eq. 3-4 for one mode, written with vector products."""
    kn = float(np.linalg.norm(kvec))
    if kn == 0.0:
        return E.copy(), B.copy()
    n = kvec / kn
    C, S = math.cos(c * kn * dt), math.sin(c * kn * dt)
    return C * (E - n * np.dot(n, E)) + 1j * S * np.cross(n, B), C * B - 1j * S * np.cross(n, E)


def test_real_step_is_mean_update_at_mirrored_nyquist_wavevectors():
    # brute force over every mode of a grid with Nyquist planes on all axes
    g = small_grid(4, 4, 6)
    dt = 0.41
    f = _real_field(g, 5, nyquist=True)
    Fk = np.fft.fftn(f, axes=(1, 2, 3))
    kx, ky, kz = (O.wavenumbers(g.Nx, g.dx), O.wavenumbers(g.Ny, g.dy), O.wavenumbers(g.Nz, g.dz))
    out = np.zeros_like(Fk)
    for iz in range(g.Nz):
        for iy in range(g.Ny):
            for ix in range(g.Nx):
                kap = np.array([kx[ix], ky[iy], kz[iz]])
                flip = np.array([ix == g.Nx // 2, iy == g.Ny // 2, iz == g.Nz // 2])
                kap2 = np.where(flip, -kap, kap)
                E, B = Fk[0:3, iz, iy, ix], Fk[3:6, iz, iy, ix]
                E1, B1 = _rotate_one_mode(E, B, kap, g.c, dt)
                E2, B2 = _rotate_one_mode(E, B, kap2, g.c, dt)
                out[0:3, iz, iy, ix] = 0.5 * (E1 + E2)
                out[3:6, iz, iy, ix] = 0.5 * (B1 + B2)
    want = np.fft.ifftn(out, axes=(1, 2, 3))
    assert np.max(np.abs(want.imag)) <= 1e-13 * np.max(np.abs(want.real))
    got = O.psatd_step_real(f, g, dt)
    assert np.max(np.abs(got - want.real)) <= 1e-13 * np.max(np.abs(want.real))
    # the Nyquist planes matter here: the plain update leaves an imaginary part
    assert np.max(np.abs(O.psatd_step(f.astype(np.complex128), g, dt).imag)) > 1e-3 * np.max(np.abs(f))


def test_real_step_does_not_increase_energy():
    g = small_grid(8, 6, 10)
    f = _real_field(g, 7, nyquist=True)
    e0 = np.sum(f * f)
    f1 = O.advance_real(f, g, 0.29, 5)
    assert np.sum(f1 * f1) <= e0 * (1 + 1e-13)
    # transverse band-limited fields keep their energy (Parseval, Eq. 3-4 unitary)
    fb = O.project_transverse(_real_field(g, 7, nyquist=False).astype(np.complex128), g)
    assert np.max(np.abs(fb.imag)) <= 1e-13 * np.max(np.abs(fb.real))
    fb = fb.real
    eb = np.sum(fb * fb)
    fb1 = O.advance_real(fb, g, 0.29, 5)
    assert abs(np.sum(fb1 * fb1) / eb - 1) <= 1e-13
