"""Seeded synthetic inputs and workload parameters.

This module holds no step of the method: only sizes, physical parameters and
seeded random input fields.  Both the CUDA path and the CPU oracle receive
their inputs from here (the oracle is never imported by this module).

Units are CGS (Sec. 2.1 of the paper): lengths in cm, times in s,
c = 2.99792458e10 cm/s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

C_CGS = 2.99792458e10          # cm/s
LAMBDA0 = 800e-7               # 800 nm in cm

FLAT_TOP = 0
GAUSSIAN = 1


@dataclass
class GridSpec:
    Nx: int
    Ny: int
    Nz: int
    dx: float
    dy: float
    dz: float
    x_min: float = 0.0
    y_min: float = 0.0
    z_min: float = 0.0
    c: float = C_CGS

    @property
    def D(self) -> float:
        return self.Nx * self.dx

    @property
    def cells(self) -> int:
        return self.Nx * self.Ny * self.Nz

    def courant_dt(self) -> float:
        """Yee 3D Courant value, used only as a reference step size."""
        return 1.0 / (self.c * math.sqrt(1 / self.dx ** 2 + 1 / self.dy ** 2 + 1 / self.dz ** 2))


@dataclass
class MappingSpec:
    R0: float
    L: float


@dataclass
class PulseSpec:
    kind: int = FLAT_TOP
    lam: float = LAMBDA0
    theta: float = 1.0
    eps: float = 0.1
    P0: float = 1e7            # 1 W in erg/s
    n_cycles: float = 2.0
    cep: float = 0.0
    ellipticity: float = 0.0
    pol_angle: float = 0.0
    div_project: int = 0


# --------------------------------------------------------------------------
# Plain-method workload: 64^3 periodic box, dx = lambda/16
# --------------------------------------------------------------------------
def plain_grid(N: int = 64, lam: float = LAMBDA0, ppw: int = 16) -> GridSpec:
    d = lam / ppw
    return GridSpec(N, N, N, d, d, d, 0.0, 0.0, 0.0, C_CGS)


def plane_wave_mode(g: GridSpec, periods: int = 4, amplitude: float = 1.0) -> np.ndarray:
    """x-polarised complex plane wave along +z: E = x^ a e^{i k0 z}, B = y^ a e^{i k0 z},
    k0 = 2 pi * periods / (Nz dz).  Returns complex128 [6, Nz, Ny, Nx]."""
    z = g.dz * np.arange(g.Nz)
    k0 = 2 * np.pi * periods / (g.Nz * g.dz)
    ph = amplitude * np.exp(1j * k0 * z)[:, None, None] * np.ones((1, g.Ny, g.Nx))
    f = np.zeros((6, g.Nz, g.Ny, g.Nx), dtype=np.complex128)
    f[0] = ph
    f[4] = ph
    return f


def random_divfree_field(g: GridSpec, seed: int, k0: float | None = None,
                         rms: float = 1e-3) -> np.ndarray:
    """Seeded random divergence-free E and B (real-valued, complex dtype).

    Each of E and B is the curl of an independent random vector potential with a
    Gaussian spectrum exp(-|k|^2 / (2 k0^2)); the curl makes it solenoidal by
    construction.  Each is scaled to the given RMS per component.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    if k0 is None:
        k0 = 2 * np.pi / (16 * g.dx)
    kx = 2 * np.pi * np.fft.fftfreq(g.Nx, g.dx)[None, None, :]
    ky = 2 * np.pi * np.fft.fftfreq(g.Ny, g.dy)[None, :, None]
    kz = 2 * np.pi * np.fft.fftfreq(g.Nz, g.dz)[:, None, None]
    k2 = kx * kx + ky * ky + kz * kz
    env = np.exp(-k2 / (2 * k0 * k0))
    out = np.zeros((6, g.Nz, g.Ny, g.Nx), dtype=np.complex128)
    for base in (0, 3):
        a = rng.standard_normal((3, g.Nz, g.Ny, g.Nx))
        A = np.fft.fftn(a, axes=(-3, -2, -1)) * env
        cx = 1j * (ky * A[2] - kz * A[1])
        cy = 1j * (kz * A[0] - kx * A[2])
        cz = 1j * (kx * A[1] - ky * A[0])
        v = np.real(np.fft.ifftn(np.stack([cx, cy, cz]), axes=(-3, -2, -1)))
        s = math.sqrt(float(np.mean(v * v)))
        out[base:base + 3] = v * (rms / s if s > 0 else 0.0)
    return out


def random_complex_field(shape, seed: int) -> np.ndarray:
    """Unstructured complex normal field (for FFT / linear-map parity checks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# --------------------------------------------------------------------------
# Tight-focus workload: f = 1, 2-cycle Gaussian pulse at 800 nm, R0 = 20 lambda
# on a 256^3 mapped grid (dx = lambda/16 over D = 16 lambda, y,z in [-18, 18) lambda)
# --------------------------------------------------------------------------
def tight_focus_workload(N: int = 256, lam: float = LAMBDA0):
    """Returns (grid, mapping, pulse, n_steps, plane) for the f = 1 Gaussian focus.

    Geometry: R0 = 20 lam, L = 4.5 * n * lam = 9 lam, D = 16 lam (D_min = 12.6 lam
    for the pulse's angular support 2*theta0 + 0.1).  x_min = -(R0 - L/2) - D.
    Time: dt = (R0/c) / n_steps with n_steps = 378 (the Courant value of the
    256^3 grid), so the last step lands on the focus t = R0/c.
    Scaled sizes keep the physical box and change the resolution.
    """
    R0 = 20 * lam
    ncyc = 2.0
    L = 4.5 * ncyc * lam
    D = 16 * lam
    W = 36 * lam
    dx = D / N
    dyz = W / N
    R_min = R0 - L / 2
    g = GridSpec(N, N, N, dx, dyz, dyz, -R_min - D, -W / 2, -W / 2, C_CGS)
    m = MappingSpec(R0, L)
    theta0 = math.atan(1.0 / (2.0 * 1.0))
    p = PulseSpec(kind=GAUSSIAN, lam=lam, theta=theta0, eps=0.2, P0=1e7,
                  n_cycles=ncyc, cep=0.0, ellipticity=0.0, pol_angle=0.0, div_project=1)
    n_steps = max(1, int(round(378 * N / 256)))
    plane = dict(x_p=0.0, ny=128, nz=128, y0=-1.5 * lam, y1=1.5 * lam,
                 z0=-1.5 * lam, z1=1.5 * lam)
    return g, m, p, n_steps, plane


def flat_top_workload(N: int = 64, lam: float = 1e-4):
    """The Sec. 3.1 flat-top case (f = 0.3, R0 = 16 lam, L = 2 lam, eps = 0.1,
    P0 = 1 W) on a small mapped grid with D = 3.5 L (Sec. 3.1)."""
    R0 = 16 * lam
    L = 2 * lam
    D = 3.5 * L
    W = 40 * lam
    theta = math.atan(1.0 / (2.0 * 0.3))
    g = GridSpec(N, N, N, D / N, W / N, W / N, -(R0 - L / 2) - D, -W / 2, -W / 2, C_CGS)
    m = MappingSpec(R0, L)
    p = PulseSpec(kind=FLAT_TOP, lam=lam, theta=theta, eps=0.1, P0=1e7, div_project=0)
    return g, m, p


def plane_points(plane: dict):
    """Sample coordinates of a focal-plane lattice: half-open [y0, y1), [z0, z1)."""
    ys = plane["y0"] + (plane["y1"] - plane["y0"]) * np.arange(plane["ny"]) / plane["ny"]
    zs = plane["z0"] + (plane["z1"] - plane["z0"]) * np.arange(plane["nz"]) / plane["nz"]
    return ys, zs


# --------------------------------------------------------------------------
# Batched sweep: seeded pulse realisations on uneven mapped grids
# --------------------------------------------------------------------------
SWEEP_SIZES = (96, 100, 108, 120, 128, 135, 144, 150, 160, 162, 180, 192)


def _sweep_size(n_needed: int) -> int:
    for n in SWEEP_SIZES:
        if n >= n_needed:
            return n
    return SWEEP_SIZES[-1]


def batched_sweep(n: int = 64, seed: int = 0, lam: float = LAMBDA0):
    """n seeded 2-cycle Gaussian realisations: f-number ~ U[0.5, 2], CEP ~
    U[0, 2 pi), ellipticity ~ U[0, 1], R0 = max(20, 10 f^2) lam, L = 9 lam.

    Each gets its own periodic layer: D is 5 % above the x-extent of the shell
    sector (R_max - R_min cos(support angle)), so replicas never overlap; the
    transverse half-width is R_max sin(support) + lam.  Grid sizes are the
    smallest of SWEEP_SIZES reaching 8 points per wavelength along x and, across,
    a step 30 % below the Nyquist limit lam / (2 sin(support)) of the pulse's
    largest transverse wavenumber (capped at 192).  Returns a list of
    (grid, mapping, pulse, T, plane) with T = R0/c and a 64 x 64 focal plane.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        f = rng.uniform(0.5, 2.0)
        cep = rng.uniform(0.0, 2 * np.pi)
        ell = rng.uniform(0.0, 1.0)
        theta0 = math.atan(1.0 / (2.0 * f))
        R0 = max(20.0, 10.0 * f * f) * lam
        L = 9.0 * lam
        support = 2 * theta0 + 0.1
        r_min, r_max = R0 - L / 2, R0 + L / 2
        D = 1.05 * (r_max - r_min * math.cos(support))
        Nx = _sweep_size(math.ceil(D / (lam / 8)))
        s_max = math.sin(min(support, math.pi / 2))
        H = r_max * s_max + lam
        Nt = _sweep_size(math.ceil(2 * H / (lam / (2.6 * s_max))))
        g = GridSpec(Nx, Nt, Nt, D / Nx, 2 * H / Nt, 2 * H / Nt, -r_min - D, -H, -H, C_CGS)
        p = PulseSpec(kind=GAUSSIAN, lam=lam, theta=theta0, eps=0.2, P0=1e7, n_cycles=2.0, cep=cep,
                      ellipticity=ell, pol_angle=0.0, div_project=1)
        plane = dict(x_p=0.0, ny=64, nz=64, y0=-1.5 * lam, y1=1.5 * lam, z0=-1.5 * lam, z1=1.5 * lam)
        out.append((g, MappingSpec(R0, L), p, R0 / C_CGS, plane))
    return out


# --------------------------------------------------------------------------
# Multi-octave workload: 400-3200 nm spectrum, seeded GDD / TOD, f = 0.5,
# tabulated longitudinal profile on a mapped grid (1024^3 at full size)
# --------------------------------------------------------------------------
PROFILE = 2
MO_LAM_MIN = 400e-7            # cm
MO_LAM_MAX = 3200e-7           # cm
MO_GDD_FS2 = 2.0               # |GDD| bound, fs^2
MO_TOD_FS3 = 4.0               # |TOD| bound, fs^3


def multi_octave_phase(seed: int):
    """Seeded spectral phase coefficients (GDD in fs^2, TOD in fs^3), uniform in
    [-MO_GDD_FS2, MO_GDD_FS2] x [-MO_TOD_FS3, MO_TOD_FS3]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.uniform(-MO_GDD_FS2, MO_GDD_FS2), rng.uniform(-MO_TOD_FS3, MO_TOD_FS3)


def multi_octave_profile(gdd_fs2: float, tod_fs3: float, L: float, dzeta: float = 2e-7,
                         lam_min: float = MO_LAM_MIN, lam_max: float = MO_LAM_MAX, edge: float = 0.2,
                         taper: float = 1e-4, n_fft: int = 1 << 16):
    """Longitudinal waveform of the multi-octave pulse as samples of a complex
    (analytic) profile a(zeta), zeta = R - R0, for the tabulated pulse kind.

    Spectrum: amplitude flat in angular frequency over [2 pi c/lam_max, 2 pi c/lam_min]
    with sin^2 ramps over `edge` of the band at both ends; spectral phase
    GDD (w - w0)^2 / 2 + TOD (w - w0)^3 / 6 about the mean frequency w0.
    a(zeta) = -i sum_w S(w) e^{i phase(w)} e^{i w zeta / c} (one-sided, so the real
    part is the waveform and the imaginary part its quadrature; the factor -i
    makes the unchirped pulse sine-like at zeta = 0, as Eq. 7), normalised to
    max |a| = 1, cut to |zeta| <= L/2 with a cos^2 taper over the outer `taper`.
    Returns (a, zeta0, dzeta, lambda0) with lambda0 = 2 pi c / w0.
    """
    c = C_CGS
    w_lo, w_hi = 2 * math.pi * c / lam_max, 2 * math.pi * c / lam_min
    w0 = 0.5 * (w_lo + w_hi)
    dw = 2 * math.pi * c / (n_fft * dzeta)
    w = dw * np.arange(n_fft)
    e = edge * (w_hi - w_lo)
    S = np.zeros(n_fft)
    S[(w >= w_lo + e) & (w <= w_hi - e)] = 1.0
    m = (w >= w_lo) & (w < w_lo + e)
    S[m] = np.sin(0.5 * math.pi * (w[m] - w_lo) / e) ** 2
    m = (w > w_hi - e) & (w <= w_hi)
    S[m] = np.sin(0.5 * math.pi * (w_hi - w[m]) / e) ** 2
    psi = 0.5 * gdd_fs2 * 1e-30 * (w - w0) ** 2 + tod_fs3 * 1e-45 / 6.0 * (w - w0) ** 3
    # zeta_j = (j - n/2) dzeta: e^{i w_k zeta_j / c} = e^{2 pi i j k / n} (-1)^k
    a = -1j * n_fft * np.fft.ifft(S * np.exp(1j * psi) * (-1.0) ** np.arange(n_fft))
    a /= np.abs(a).max()
    zeta = (np.arange(n_fft) - n_fft // 2) * dzeta
    sel = np.abs(zeta) <= L / 2
    a, zeta = a[sel], zeta[sel]
    edge_dist = L / 2 - np.abs(zeta)
    tap = np.where(edge_dist < taper, np.sin(0.5 * math.pi * np.clip(edge_dist, 0.0, None) / taper) ** 2, 1.0)
    return a * tap, float(zeta[0]), dzeta, 2 * math.pi * c / w0


def multi_octave_workload(N: int = 1024, seed: int = 0):
    """Returns (grid, mapping, pulse, profile, n_steps, plane) for the f = 0.5
    multi-octave focus; profile = (a, zeta0, dzeta).

    Pulse: tabulated kind (flat-top transverse shape, theta = 45 deg, eps = 0.1),
    waveform of multi_octave_profile with the seed's GDD / TOD, L = 12 um,
    R0 = 32 um (10 lambda_max).  Layer: D = 50 um along x (D_min = 15.3 um),
    y, z in [-H, H) with H = R_max sin(theta + eps/2) + 1 um; N cells per axis.
    dt = (R0/c) / n_steps with n_steps = ceil((R0/c) / Courant value), so the last
    step lands on the focus.  Focal plane x = 0, 128 x 128 over +-1.5 lambda0.
    """
    R0 = 32e-4
    L = 12e-4
    D = 50e-4
    theta = math.atan(1.0 / (2.0 * 0.5))
    eps = 0.1
    H = (R0 + L / 2) * math.sin(theta + eps / 2) + 1e-4
    g = GridSpec(N, N, N, D / N, 2 * H / N, 2 * H / N, -(R0 - L / 2) - D, -H, -H, C_CGS)
    gdd, tod = multi_octave_phase(seed)
    a, z0, dz, lam0 = multi_octave_profile(gdd, tod, L)
    p = PulseSpec(kind=PROFILE, lam=lam0, theta=theta, eps=eps, P0=1e7, n_cycles=1.0, cep=0.0,
                  ellipticity=0.0, pol_angle=0.0, div_project=1)
    T = R0 / C_CGS
    n_steps = int(math.ceil(T / g.courant_dt()))
    plane = dict(x_p=0.0, ny=128, nz=128, y0=-1.5 * lam0, y1=1.5 * lam0, z0=-1.5 * lam0, z1=1.5 * lam0)
    return g, MappingSpec(R0, L), p, (a, z0, dz), n_steps, plane
