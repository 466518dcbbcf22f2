"""A physical pin of the oracle's whole focusing chain: Gaussian pulse amplitude
(Sec. 3.2.1), transverse profile, initialisation on the mapped periodic layer
with its replicas (Sec. 2.3), the exact PSATD propagation (Sec. 2.1) and the
focal sampling (Eq. 14-16), against the diffraction integral of a converging
spherical wave and against the paper's paraxial limit.

Debye's integral: a spherical wave converging from the sphere R = R0 with
carrier amplitude E0 A(alpha) and polarisation s0(alpha, phi) has, at the
focus and in the short-wavelength limit (k R0 >> 1), the carrier amplitude

    E(0) = (k R0 / 2 pi) * integral of E0 A(alpha) s0 dOmega.

With d = y, s0 = (d - (d.R^) R^) / |...| has y component sqrt(1 - R^_y^2) and
its x and z components integrate to zero, so

    |E_y(0)| = k R0 E0 int_0^pi A(alpha) <sqrt(1 - sin^2 alpha cos^2 phi)>_phi
                   sin alpha dalpha.

For a pulse of any duration the time-domain form of the same integral gives
the field at the focus at t = R0/c from the slope of the longitudinal profile at
its centre: u_l(s) = sin(k s) cos^2(pi s / L) of Eq. 7 has slope k there, so the
flat-top pulse of Eq. 8-9 reaches |E_y(0)| = k A int u_ts sqrt(...) sin alpha.
B = u s1 with s1 = d x R^ / |d x R^| has z component cos alpha / sqrt(1 - R^_y^2),
so B_z(0) = k A int u_ts <cos alpha / sqrt(1 - sin^2 alpha cos^2 phi)>_phi
sin alpha, with the sign of E_y for a converging pulse (E x B along +x there).

For the untruncated Gaussian A = exp(-alpha^2/theta0^2) and small theta0 this
tends to the paraxial focus I0 = 2 P0 / (pi w0^2), w0 = 2 f lambda / pi, that
the paper uses to validate its solver in the weak-focusing limit (Sec. 3.2.1;
cycle-averaged CGS intensity c E^2 / (8 pi)).  The oracle's profile also has
the Eq. 5 edge at 2 theta0, which lowers the focal field by a few per cent.
"""
import math

import numpy as np

from oracle import psatd_oracle as O

LAM, R0, C, P0, EPS, N_CYCLES = 1.0, 20.0, 1.0, 1.0, 0.1, 4.0


def smooth235(n):
    while True:
        k = n
        for p in (2, 3, 5):
            while k % p == 0:
                k //= p
        if k == 1:
            return n
        n += 1


def edge_window(alpha, theta, eps):
    """1 up to theta - eps/2, a cos^2 ramp to 0 at theta + eps/2 (Eq. 5)."""
    ramp = np.cos(np.pi * (alpha - theta + eps / 2) / (2 * eps)) ** 2
    return np.where(alpha <= theta - eps / 2, 1.0, np.where(alpha <= theta + eps / 2, ramp, 0.0))


def polarisation_average(a, component="E"):
    """Over phi: <sqrt(1 - sin^2 a cos^2 phi)> (y component of s0, "E") or
    <cos a / sqrt(1 - sin^2 a cos^2 phi)> (z component of s1, "B"; a < pi/2)."""
    phi = np.linspace(0.0, 2 * math.pi, 721)[:-1]
    coarse = a[::400]
    q = np.sqrt(1.0 - np.outer(np.sin(coarse) ** 2, np.cos(phi) ** 2))
    pol = (q if component == "E" else np.cos(coarse)[:, None] / q).mean(axis=1)
    return np.interp(a, coarse, pol)


def layer_grid(theta_support, R0, L, ppl=6):
    """Mapped layer for a shell whose profile ends at the angle theta_support:
    period D = D_min (Eq. 12) + lambda, transverse half width R_max sin + lambda."""
    m = O.Mapping(R0, L)
    D = O.d_min(R0, L, theta_support) + LAM
    H = m.R_max * math.sin(theta_support) + LAM
    d = LAM / ppl
    Nx, Nt = smooth235(int(math.ceil(D / d))), smooth235(int(math.ceil(2 * H / d)))
    return O.Grid(Nx, Nt, Nt, d, d, d, -(R0 - L / 2) - Nx * d, -Nt * d / 2, -Nt * d / 2, C), m


def debye_focal_field(theta0, truncated):
    """|E_y| at the focus from Debye's integral, with E0 from the printed
    normalisation (power P0 through the sphere) and F by quadrature."""
    a = np.linspace(0.0, math.pi, 400001)
    F = np.trapezoid(np.sin(a) * np.exp(-2 * a * a / theta0 ** 2), a)
    E0 = math.sqrt(4 * P0 / (C * R0 * R0 * F))          # SI E0 of Sec. 3.2.1 with eps0 -> 1/(4 pi)
    A = np.exp(-a * a / theta0 ** 2)
    if truncated:
        A = A * edge_window(a, 2 * theta0, EPS)
    k = 2 * math.pi / LAM
    return k * R0 * E0 * np.trapezoid(A * polarisation_average(a) * np.sin(a), a)


def oracle_focal_field(fnum, ppl=6):
    """Amplitude of E at the focus at t = R0/c from the oracle: init on the
    mapped layer, one exact step, sampling at the origin; the carrier amplitude
    from two samples a quarter period apart."""
    theta0 = O.theta_from_fnumber(fnum)
    g, m = layer_grid(2 * theta0 + EPS / 2, R0, 4.5 * N_CYCLES * LAM, ppl)
    p = O.Pulse(kind=O.GAUSSIAN, lam=LAM, theta=theta0, eps=EPS, P0=P0, n_cycles=N_CYCLES)
    f0 = O.init_fields(g, m, p)
    T = R0 / C
    samples = []
    for t in (T, T + LAM / (4 * C)):
        s = O.sample_plane(O.advance_exact(f0, g, t), g, m, 0.0, np.array([0.0]), np.array([0.0]), t)
        samples.append(s[:, 0, 0].real)
    return np.sqrt(samples[0] ** 2 + samples[1] ** 2)


def test_gaussian_focus_matches_debye_integral_and_paraxial_limit():
    fnum = 4.0
    theta0 = math.atan(1.0 / (2 * fnum))
    E = oracle_focal_field(fnum)
    Ed = debye_focal_field(theta0, truncated=True)
    # the y-polarised pulse focuses to E_y; E_x and E_z vanish on the axis
    assert E[0] < 1e-6 * E[1] and E[2] < 1e-6 * E[1]
    assert abs(E[1] / Ed - 1.0) < 1e-3
    # the untruncated Gaussian reaches the paraxial focus up to O(theta0^2)
    w0 = 2 * fnum * LAM / math.pi
    E_par = math.sqrt(16 * P0 / (C * w0 * w0))
    assert abs(debye_focal_field(theta0, truncated=False) / E_par - 1.0) < 0.02
    # and the oracle's intensity sits just below I0, by the edge at 2 theta0
    ratio = (E[1] / E_par) ** 2
    assert 0.9 < ratio < 1.0


def flat_top_focus_checks():
    """The paper's tight-focusing case (Sec. 3.1: f = 0.3, theta ~ 1 rad,
    R0 = 16 lambda, L = 2 lambda, eps = 0.1), far from the paraxial regime:
    each check of the focal E and B against the Debye integrals, by name."""
    fnum, R0f, L = 0.3, 16.0, 2.0
    theta = math.atan(1.0 / (2 * fnum))
    g, m = layer_grid(theta + EPS / 2, R0f, L)
    p = O.Pulse(kind=O.FLAT_TOP, lam=LAM, theta=theta, eps=EPS, P0=P0)
    T = R0f / C
    EB = O.sample_plane(O.advance_exact(O.init_fields(g, m, p), g, T), g, m, 0.0, np.array([0.0]),
                        np.array([0.0]), T, comps=(0, 1, 2, 3, 4, 5))[:, 0, 0].real
    E, B = EB[:3], EB[3:]
    a = np.linspace(0.0, theta + EPS / 2, 400001)                 # the support of u_ts
    A = math.sqrt(4 * P0 / (C * (1 - math.cos(theta))))          # Eq. 9
    w = edge_window(a, theta, EPS) * np.sin(a)
    Ed = 2 * math.pi / LAM * A * np.trapezoid(w * polarisation_average(a, "E"), a)
    Bd = 2 * math.pi / LAM * A * np.trapezoid(w * polarisation_average(a, "B"), a)
    return {
        "E along y": abs(E[0]) < 1e-5 * abs(E[1]) and abs(E[2]) < 1e-5 * abs(E[1]),
        "E_y = Debye": abs(abs(E[1]) / Ed - 1.0) < 2e-3,
        # B is along z with E_y's sign, and smaller than E_y at this focusing (Bd / Ed = 0.97)
        "B along z": abs(B[0]) < 1e-5 * abs(B[2]) and abs(B[1]) < 1e-5 * abs(B[2]),
        "B_z = Debye, sign of E_y": bool(B[2] * E[1] > 0) and abs(B[2] / Bd - 1.0) < 2e-3,
    }


def test_flat_top_tight_focus_matches_debye_integral():
    checks = flat_top_focus_checks()
    assert all(checks.values()), checks


def test_focus_checks_catch_planted_mistakes(monkeypatch):
    """Plausible mistakes in the amplitude, the polarisation and the mapping
    each fail at least one of the focus checks."""
    good_A, good_pol, good_T = O.flat_top_A, O.polarisation_vectors, O.mapping_T

    def A_wrong_sign(P0_, c, theta):           # 1 + cos theta in Eq. 9
        return math.sqrt(4.0 * P0_ / (c * (1.0 + math.cos(theta))))

    def B_reversed(X, Y, Z, d):                # s1 = R x d: a diverging pulse
        s0, s1 = good_pol(X, Y, Z, d)
        return s0, -s1

    def T_half_period(x, x_min, D):            # Eq. 13 off by half a period
        return good_T(np.asarray(x) + D / 2, x_min, D)

    for name, plant in (("flat_top_A", A_wrong_sign), ("polarisation_vectors", B_reversed),
                        ("mapping_T", T_half_period)):
        monkeypatch.setattr(O, name, plant)
        assert not all(flat_top_focus_checks().values()), name
        monkeypatch.setattr(O, name, {"flat_top_A": good_A, "polarisation_vectors": good_pol,
                                      "mapping_T": good_T}[name])
