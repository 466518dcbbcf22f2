"""PSATD oracle: vacuum spectral Maxwell step, pulse models, mapping and sampling.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, __graft_entry__.smoke() and the
CPU legs of bench.py; never by the product path.

Everything here is float64 numpy, written from the paper (arXiv:2010.00409,
"Tight focusing of short pulses by mapping to periodic space"), each function
citing the section / equation it follows.  The 3D DFT is this module's own
recursive decimation-in-time transform (one split near sqrt(N) per level,
direct sums of length <= 32 at the leaves), pinned against the brute-force
sum; library primitives used as single steps: matrix products.

Field layout: ``fields[6, Nz, Ny, Nx]`` complex128, components
(Ex, Ey, Ez, Bx, By, Bz), x fastest.  Node (i, j, l) sits at
(x_min + i*dx, y_min + j*dy, z_min + l*dz).

Readings of places where the paper is silent or garbled (numbered as in the
design notes):
  R1  forward DFT kernel exp(-i k.x), unnormalised; inverse carries 1/N
      (then the curl is +ik and Eq. 3-4 hold as printed).
  R2  even-N Nyquist index is m = -N/2 (numpy fftfreq order).
  R3  at k = 0 the unit vector k^ is taken as 0 and C = 1, S = 0.
  R4  Eq. 3-4 are applied literally every step; an optional one-time
      projection of E and B after initialisation.
  R5  Eq. 5: the edge window is half-open so u_ts is continuous.
  R6  alpha = atan2(sqrt(y^2+z^2), -x), the angle from the -x axis.
  R7  s0 = normalise(R x (d x R)), s1 = normalise(d x R).
  R8  I_S case 3 reads "R > r(t)".
  R9  y_min = -Ny*dy/2, z_min = -Nz*dz/2 by default; x_min = -R_min - D.
  R10 overlapping replicas are summed (linearity).
  R12 Gaussian pulse: u_ts = exp(-a^2/t0^2) times the Eq. 5 edge with
      theta = 2*t0; u_l windowed to |zeta| <= L/2; CGS amplitude.
  R13 CEP phi, ellipticity e and polarisation angle psi.
  R20 real fields: one step of real E, B is the real part of the complex
      step.  Eq. 3-4 keep a Hermitian spectrum Hermitian except on Nyquist
      planes, where the wave number -pi/d is its own mirror index; the real
      part there is the mean of the update at kappa and at kappa with its
      Nyquist components negated.
  R21 tabulated longitudinal profile (Sec. 2.2 allows any profile along the
      radial direction): Eq. 8 with the flat-top transverse shape of Eq. 5 and
      the amplitude A of Eq. 9, u_l(zeta) = Re(a(zeta) e^{i phi}) with a the
      analytic waveform linearly interpolated between given samples.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Grid", "Mapping", "Pulse", "FLAT_TOP", "GAUSSIAN", "PROFILE", "profile_ul",
    "wavenumbers", "fft3", "ifft3", "dft3_naive", "idft3_naive",
    "psatd_update", "psatd_step", "advance", "advance_exact",
    "psatd_step_real", "advance_real",
    "theta_from_fnumber", "d_min", "mapping_T", "indicator_S",
    "omega", "u_ts_flat", "u_l_flat", "flat_top_A", "F_series", "F_exact",
    "gaussian_E0", "pulse_scalar", "polarisation_vectors",
    "init_fields", "project_transverse", "sample_plane", "diagnostics",
    "courant_dt",
]

FLAT_TOP = 0
GAUSSIAN = 1
PROFILE = 2


# ----------------------------------------------------------------------------
# Parameters
# ----------------------------------------------------------------------------
@dataclass
class Grid:
    """Periodic box: Nx*Ny*Nz nodes with steps dx, dy, dz and origin r_min."""
    Nx: int
    Ny: int
    Nz: int
    dx: float
    dy: float
    dz: float
    x_min: float = 0.0
    y_min: float = 0.0
    z_min: float = 0.0
    c: float = 1.0

    @property
    def D(self) -> float:
        """Period of the mapped layer along x (Sec. 2.3)."""
        return self.Nx * self.dx

    def coords(self):
        x = self.x_min + self.dx * np.arange(self.Nx)
        y = self.y_min + self.dy * np.arange(self.Ny)
        z = self.z_min + self.dz * np.arange(self.Nz)
        return x, y, z


@dataclass
class Mapping:
    """Geometry of the initial spherical shell R0-L/2 <= R <= R0+L/2 (Sec. 2.2-2.3)."""
    R0: float
    L: float

    @property
    def R_min(self) -> float:
        return self.R0 - self.L / 2

    @property
    def R_max(self) -> float:
        return self.R0 + self.L / 2


@dataclass
class Pulse:
    """Pulse model parameters (Sec. 2.2 flat-top, Sec. 3.2.1 Gaussian)."""
    kind: int = FLAT_TOP
    lam: float = 1.0          # carrier wavelength
    theta: float = 1.0        # flat-top half angle theta; Gaussian theta0
    eps: float = 0.1          # edge smoothing angle of Eq. 5
    P0: float = 1.0           # power
    n_cycles: float = 2.0     # Gaussian FWHM duration in wavelengths
    cep: float = 0.0          # carrier phase phi (R13)
    ellipticity: float = 0.0  # e (R13)
    pol_angle: float = 0.0    # psi (R13): d1 = (0, cos psi, sin psi)
    div_project: int = 0      # one-time transverse projection after init (R4)
    # PROFILE (R21): complex samples a_k = a(profile_z0 + k profile_dz) of the
    # longitudinal waveform
    profile: np.ndarray | None = None
    profile_z0: float = 0.0
    profile_dz: float = 1.0


# ----------------------------------------------------------------------------
# Spectral solver (Sec. 2.1)
# ----------------------------------------------------------------------------
def wavenumbers(N: int, d: float) -> np.ndarray:
    """k_m = 2*pi*m/(N*d) with m = i for i < (N+1)/2 and m = i - N above (R2:
    the even-N Nyquist index is -N/2)."""
    i = np.arange(N)
    m = np.where(i < (N + 1) // 2, i, i - N)
    return 2.0 * np.pi * m / (N * d)


def _split(N: int) -> int:
    """Factor p split off at one level of the recursive DFT: the largest divisor
    of N not above sqrt(N); 1 (sum directly) for N <= 32 or N prime."""
    if N <= 32:
        return 1
    for p in range(int(math.isqrt(N)), 1, -1):
        if N % p == 0:
            return p
    return 1


def _unit_roots(e: np.ndarray, N: int, sign: int) -> np.ndarray:
    """exp(sign*2*pi*i*e/N) for integer exponents e, reduced modulo N first."""
    return np.exp(sign * 2j * np.pi * (np.mod(e, N) / N))


def _dft_last(x: np.ndarray, sign: int) -> np.ndarray:
    """DFT along the last axis, X[k] = sum_n x[n] exp(sign*2*pi*i*n*k/N), by
    decimation in time.  With N = p*M, n = p*m + r and k = k1 + M*k2:
        X[k1 + M*k2] = sum_r exp(sign*2*pi*i*r*k2/p) exp(sign*2*pi*i*r*k1/N) Y_r[k1],
    Y_r the M-point DFT of the subsequence x[r::p] (computed by recursion).
    Short or prime lengths are summed directly (a product with the DFT
    matrix)."""
    N = x.shape[-1]
    p = _split(N)
    if p == 1:
        n = np.arange(N)
        return x @ _unit_roots(np.outer(n, n), N, sign)
    M = N // p
    r, k1 = np.arange(p), np.arange(M)
    xr = x.reshape(x.shape[:-1] + (M, p))                       # xr[..., m, r] = x[p*m + r]
    Y = _dft_last(np.swapaxes(xr, -1, -2), sign)                 # Y[..., r, k1]
    Y = np.swapaxes(Y, -1, -2) * _unit_roots(np.outer(k1, r), N, sign)   # twiddled, [..., k1, r]
    Z = Y @ _unit_roots(np.outer(r, r), p, sign)                 # Z[..., k1, k2]
    return np.swapaxes(Z, -1, -2).reshape(x.shape)               # k = k1 + M*k2


def _dft3(f: np.ndarray, sign: int) -> np.ndarray:
    out = np.asarray(f, dtype=np.complex128)
    for axis in (-1, -2, -3):
        out = np.moveaxis(_dft_last(np.moveaxis(out, axis, -1), sign), -1, axis)
    return out


def fft3(f: np.ndarray) -> np.ndarray:
    """Unnormalised forward 3D DFT over the last three axes, kernel exp(-i k.x) (R1)."""
    return _dft3(f, -1)


def ifft3(F: np.ndarray) -> np.ndarray:
    """Inverse 3D DFT with the 1/(Nx*Ny*Nz) factor (R1)."""
    N = F.shape[-1] * F.shape[-2] * F.shape[-3]
    return _dft3(F, +1) / N


def _dft_matrix(N: int, sign: int) -> np.ndarray:
    n = np.arange(N)
    return np.exp(sign * 2j * np.pi * np.outer(n, n) / N)


def dft3_naive(f: np.ndarray, sign: int = -1) -> np.ndarray:
    """Brute-force 3D DFT: F[kz,ky,kx] = sum_{z,y,x} f exp(sign*2*pi*i*(k.n)/N).

    Written as an explicit sum over every node for each output mode; only for
    tiny grids (it is O(N^2) in the number of nodes).
    """
    Nz, Ny, Nx = f.shape[-3:]
    out = np.zeros(f.shape, dtype=np.complex128)
    z = np.arange(Nz)[:, None, None]
    y = np.arange(Ny)[None, :, None]
    x = np.arange(Nx)[None, None, :]
    for kz in range(Nz):
        for ky in range(Ny):
            for kx in range(Nx):
                ph = np.exp(sign * 2j * np.pi * (kz * z / Nz + ky * y / Ny + kx * x / Nx))
                out[..., kz, ky, kx] = np.sum(f * ph, axis=(-3, -2, -1))
    return out


def idft3_naive(F: np.ndarray) -> np.ndarray:
    """Brute-force inverse of :func:`dft3_naive` (kernel exp(+i k.x), 1/N)."""
    N = F.shape[-1] * F.shape[-2] * F.shape[-3]
    return dft3_naive(F, +1) / N


def _k_grids(grid: Grid):
    kx = wavenumbers(grid.Nx, grid.dx)[None, None, :]
    ky = wavenumbers(grid.Ny, grid.dy)[None, :, None]
    kz = wavenumbers(grid.Nz, grid.dz)[:, None, None]
    return kx, ky, kz


def psatd_update(Fk: np.ndarray, grid: Grid, dt: float) -> np.ndarray:
    """Per-mode vacuum PSATD update with Poisson correction, Eq. 3-4 (Sec. 2.1).

    E^{n+1} = C (E - k^(k^.E)) + i S k^ x B
    B^{n+1} = C B - i S k^ x E
    with C = cos(c|k|dt), S = sin(c|k|dt), both right-hand sides from step n.
    At k = 0: k^ = 0, C = 1, S = 0 (R3).
    """
    kx, ky, kz = _k_grids(grid)
    kx, ky, kz = np.broadcast_arrays(kx, ky, kz)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    safe = np.where(kmag > 0, kmag, 1.0)
    nx = np.where(kmag > 0, kx / safe, 0.0)
    ny = np.where(kmag > 0, ky / safe, 0.0)
    nz = np.where(kmag > 0, kz / safe, 0.0)
    C = np.cos(grid.c * kmag * dt)
    S = np.sin(grid.c * kmag * dt)

    Ex, Ey, Ez, Bx, By, Bz = (Fk[i] for i in range(6))
    kE = nx * Ex + ny * Ey + nz * Ez
    # k^ x B and k^ x E
    cBx = ny * Bz - nz * By
    cBy = nz * Bx - nx * Bz
    cBz = nx * By - ny * Bx
    cEx = ny * Ez - nz * Ey
    cEy = nz * Ex - nx * Ez
    cEz = nx * Ey - ny * Ex
    out = np.empty_like(Fk)
    out[0] = C * (Ex - nx * kE) + 1j * S * cBx
    out[1] = C * (Ey - ny * kE) + 1j * S * cBy
    out[2] = C * (Ez - nz * kE) + 1j * S * cBz
    out[3] = C * Bx - 1j * S * cEx
    out[4] = C * By - 1j * S * cEy
    out[5] = C * Bz - 1j * S * cEz
    return out


def psatd_step(fields: np.ndarray, grid: Grid, dt: float) -> np.ndarray:
    """One step: forward 3D DFT of the six components, Eq. 3-4, inverse DFT (Sec. 2.1)."""
    return ifft3(psatd_update(fft3(fields), grid, dt))


def advance(fields: np.ndarray, grid: Grid, dt: float, n: int) -> np.ndarray:
    """n consecutive PSATD steps of size dt."""
    f = np.array(fields, dtype=np.complex128, copy=True)
    for _ in range(n):
        f = psatd_step(f, grid, dt)
    return f


def advance_exact(fields: np.ndarray, grid: Grid, T: float) -> np.ndarray:
    """A single step of size T.  In vacuum the solver is exact in time, so this
    equals any number of steps summing to T up to rounding (Sec. 2.1, Sec. 3.1)."""
    return psatd_step(np.asarray(fields, dtype=np.complex128), grid, T)


def psatd_step_real(fields: np.ndarray, grid: Grid, dt: float) -> np.ndarray:
    """One step of real fields [6, Nz, Ny, Nx] (float64): the real part of the
    complex step of Sec. 2.1 applied to them (R20)."""
    return psatd_step(np.asarray(fields, dtype=np.float64).astype(np.complex128), grid, dt).real


def advance_real(fields: np.ndarray, grid: Grid, dt: float, n: int) -> np.ndarray:
    """n consecutive real-field steps of size dt (R20)."""
    f = np.array(fields, dtype=np.float64, copy=True)
    for _ in range(n):
        f = psatd_step_real(f, grid, dt)
    return f


def courant_dt(grid: Grid) -> float:
    """The Yee 3D Courant value 1/(c*sqrt(1/dx^2+1/dy^2+1/dz^2)) used as the
    reference step (PSATD itself has no stability limit, Sec. 2.1)."""
    return 1.0 / (grid.c * math.sqrt(1 / grid.dx ** 2 + 1 / grid.dy ** 2 + 1 / grid.dz ** 2))


# ----------------------------------------------------------------------------
# Problem statement: pulse models (Sec. 2.2, Sec. 3.2.1)
# ----------------------------------------------------------------------------
def theta_from_fnumber(f: float) -> float:
    """theta = arctan(1/(2f)) (Sec. 2.2)."""
    return math.atan(1.0 / (2.0 * f))


def omega(x, a, b):
    """Rectangular window of Eq. 6: 1 on the closed interval [a, b], else 0."""
    x = np.asarray(x, dtype=np.float64)
    return ((x >= a) & (x <= b)).astype(np.float64)


def u_ts_flat(alpha, theta: float, eps: float):
    """Flat-top transverse shape with a cos^2 edge of width eps, Eq. 5.

    Both windows of Eq. 5 are printed closed, so at alpha = theta - eps/2 the
    sum would be 2; the edge window is taken half-open, (theta - eps/2,
    theta + eps/2], which keeps the profile continuous (R5).
    """
    alpha = np.asarray(alpha, dtype=np.float64)
    edge = np.cos(np.pi * (alpha - theta + eps / 2) / (2 * eps)) ** 2
    in_edge = ((alpha > theta - eps / 2) & (alpha <= theta + eps / 2)).astype(np.float64)
    return omega(alpha, 0.0, theta - eps / 2) + edge * in_edge


def u_l_flat(s, lam: float, L: float, phase: float = 0.0):
    """Longitudinal shape of Eq. 7 (carrier phase added per R13)."""
    s = np.asarray(s, dtype=np.float64)
    return np.sin(2 * np.pi * s / lam + phase) * np.cos(np.pi * s / L) ** 2 * omega(s, -L / 2, L / 2)


def profile_ul(s, a, z0: float, dz: float, phase: float = 0.0):
    """Tabulated longitudinal factor Re(a(s) e^{i phase}) (R21): the samples
    a_k = a(z0 + k dz) joined by straight lines, zero outside [z0, z0 + (n-1) dz]."""
    s = np.asarray(s, dtype=np.float64)
    a = np.asarray(a, dtype=np.complex128)
    zk = z0 + dz * np.arange(a.size)
    inside = (s >= z0) & (s <= zk[-1])
    ar = np.interp(s, zk, a.real)
    ai = np.interp(s, zk, a.imag)
    return np.where(inside, ar * math.cos(phase) - ai * math.sin(phase), 0.0)


def flat_top_A(P0: float, c: float, theta: float) -> float:
    """Amplitude of Eq. 9, A = sqrt(4 P0 / (c (1 - cos theta)))."""
    return math.sqrt(4.0 * P0 / (c * (1.0 - math.cos(theta))))


def F_series(theta0: float) -> float:
    """The series theta0^2/4 - theta0^4/48 + theta0^6/960 for F (Sec. 3.2.1)."""
    t2 = theta0 * theta0
    return t2 / 4 - t2 * t2 / 48 + t2 * t2 * t2 / 960


def F_exact(theta0: float, n: int = 200001) -> float:
    """F(theta0) = int_0^pi sin(t) exp(-2 t^2/theta0^2) dt by composite Simpson."""
    t = np.linspace(0.0, np.pi, n)
    g = np.sin(t) * np.exp(-2 * t * t / theta0 ** 2)
    h = t[1] - t[0]
    return float(h / 3 * (g[0] + g[-1] + 4 * g[1:-1:2].sum() + 2 * g[2:-1:2].sum()))


def gaussian_E0(P0: float, c: float, R0: float, theta0: float) -> float:
    """Gaussian-pulse amplitude (Sec. 3.2.1) in CGS.

    The paper prints E0 = sqrt(P0 / (pi eps0 c R0^2 F(theta0))) in SI units; with
    eps0 -> 1/(4 pi) this is sqrt(4 P0 / (c R0^2 F(theta0))), the same
    cycle-averaged-power normalisation as the flat-top A of Eq. 9.
    """
    return math.sqrt(4.0 * P0 / (c * R0 * R0 * F_series(theta0)))


def _alpha(X, Y, Z):
    """Angle between R and the -x axis (R6)."""
    return np.arctan2(np.sqrt(Y * Y + Z * Z), -X)


def pulse_scalar(X, Y, Z, pulse: Pulse, mapping: Mapping, c: float, phase: float):
    """Scalar amplitude u(R) with carrier phase `phase`.

    FLAT_TOP: Eq. 8, u = A/R * u_l(R - R0) * u_ts(alpha).
    GAUSSIAN: Sec. 3.2.1 with R12, u = E0 R0 sin(k(R-R0)+phase) u_l u_ts / R.
    PROFILE: Eq. 8 with the tabulated u_l of R21 on |R - R0| <= L/2.
    """
    R = np.sqrt(X * X + Y * Y + Z * Z)
    Rs = np.where(R > 0, R, 1.0)
    alpha = _alpha(X, Y, Z)
    zeta = R - mapping.R0
    if pulse.kind == FLAT_TOP:
        A = flat_top_A(pulse.P0, c, pulse.theta)
        u = A / Rs * u_l_flat(zeta, pulse.lam, mapping.L, phase) * u_ts_flat(alpha, pulse.theta, pulse.eps)
    elif pulse.kind == PROFILE:
        A = flat_top_A(pulse.P0, c, pulse.theta)
        ul = profile_ul(zeta, pulse.profile, pulse.profile_z0, pulse.profile_dz, phase) \
            * omega(zeta, -mapping.L / 2, mapping.L / 2)
        u = A / Rs * ul * u_ts_flat(alpha, pulse.theta, pulse.eps)
    elif pulse.kind == GAUSSIAN:
        E0 = gaussian_E0(pulse.P0, c, mapping.R0, pulse.theta)
        k = 2 * np.pi / pulse.lam
        ul = np.exp(-zeta * zeta * math.log(4.0) / (pulse.n_cycles * pulse.lam) ** 2) \
            * omega(zeta, -mapping.L / 2, mapping.L / 2)
        uts = np.exp(-alpha * alpha / pulse.theta ** 2) * u_ts_flat(alpha, 2 * pulse.theta, pulse.eps)
        u = E0 * mapping.R0 * np.sin(k * zeta + phase) * ul * uts / Rs
    else:
        raise ValueError("unknown pulse kind")
    return np.where(R > 0, u, 0.0)


def polarisation_vectors(X, Y, Z, d):
    """s0 = normalise(R x (d x R)), s1 = normalise(d x R)  (Eq. 10-11 with R7)."""
    d = np.asarray(d, dtype=np.float64)
    R = np.stack(np.broadcast_arrays(X, Y, Z))
    dxR = np.stack([d[1] * R[2] - d[2] * R[1],
                    d[2] * R[0] - d[0] * R[2],
                    d[0] * R[1] - d[1] * R[0]])
    Rx_dxR = np.stack([R[1] * dxR[2] - R[2] * dxR[1],
                       R[2] * dxR[0] - R[0] * dxR[2],
                       R[0] * dxR[1] - R[1] * dxR[0]])
    n0 = np.sqrt(np.sum(Rx_dxR ** 2, axis=0))
    n1 = np.sqrt(np.sum(dxR ** 2, axis=0))
    s0 = np.where(n0 > 0, Rx_dxR / np.where(n0 > 0, n0, 1.0), 0.0)
    s1 = np.where(n1 > 0, dxR / np.where(n1 > 0, n1, 1.0), 0.0)
    return s0, s1


def _pulse_fields_at(X, Y, Z, pulse: Pulse, mapping: Mapping, c: float):
    """E and B of the pulse at physical points (Eq. 10-11, R13)."""
    psi = pulse.pol_angle
    d1 = (0.0, math.cos(psi), math.sin(psi))
    d2 = (0.0, -math.sin(psi), math.cos(psi))
    u1 = pulse_scalar(X, Y, Z, pulse, mapping, c, pulse.cep)
    s0, s1 = polarisation_vectors(X, Y, Z, d1)
    E = u1 * s0
    B = u1 * s1
    if pulse.ellipticity != 0.0:
        u2 = pulse_scalar(X, Y, Z, pulse, mapping, c, pulse.cep + np.pi / 2)
        t0, t1 = polarisation_vectors(X, Y, Z, d2)
        E = E + pulse.ellipticity * u2 * t0
        B = B + pulse.ellipticity * u2 * t1
    return E, B


# ----------------------------------------------------------------------------
# Mapping to and from the periodic layer (Sec. 2.3)
# ----------------------------------------------------------------------------
def d_min(R0: float, L: float, theta: float) -> float:
    """Smallest replica period without overlap, Eq. 12."""
    Rmin, Rmax = R0 - L / 2, R0 + L / 2
    return -Rmin * math.cos(theta) + math.sqrt(Rmax * Rmax - (Rmin * math.sin(theta)) ** 2)


def mapping_T(x, x_min: float, D: float):
    """Eq. 13: x~ = x_min + D * frac((x - x_min)/D); y, z unchanged."""
    s = (np.asarray(x, dtype=np.float64) - x_min) / D
    return x_min + D * (s - np.floor(s))


def indicator_S(X, Y, Z, t: float, mapping: Mapping, c: float):
    """Cut-out indicator I_S(t)(R) of Eq. 15 with l, r of Eq. 16 (case 3 per R8)."""
    X, Y, Z = np.broadcast_arrays(np.asarray(X, dtype=np.float64),
                                  np.asarray(Y, dtype=np.float64),
                                  np.asarray(Z, dtype=np.float64))
    R = np.sqrt(X * X + Y * Y + Z * Z)
    l = -mapping.R_max + c * t
    r = -mapping.R_min + c * t
    zero = np.zeros(R.shape, dtype=bool)
    if r < 0:
        zero |= (R >= -l) | (R < -r) | (X > 0)
    if l <= 0 <= r:
        zero |= (X < 0) & (R > mapping.L)
        zero |= (X >= 0) & (R > r)
    if l > 0:
        zero |= (R <= l) | (R > r) | (X < 0)
    return np.where(zero, 0.0, 1.0)


def _replica_range(grid: Grid, mapping: Mapping):
    """Replica indices m whose copy x~ + m D can meet the shell (with margin)."""
    D = grid.D
    lo = -mapping.R_max
    hi = mapping.R_max
    m_lo = math.floor((lo - (grid.x_min + D)) / D) - 1
    m_hi = math.ceil((hi - grid.x_min) / D) + 1
    return range(m_lo, m_hi + 1)


def init_fields(grid: Grid, mapping: Mapping, pulse: Pulse, z_chunk: int = 8) -> np.ndarray:
    """Initial E, B on the periodic layer: each node takes the sum over replicas
    m of the pulse at x~ + m D (Eq. 13 inverted per node, with R10).

    Returns complex128 fields[6, Nz, Ny, Nx] (imaginary part 0).  If
    pulse.div_project is set the result is projected transverse once (R4).
    """
    x, y, z = grid.coords()
    out = np.zeros((6, grid.Nz, grid.Ny, grid.Nx), dtype=np.complex128)
    reps = list(_replica_range(grid, mapping))
    for z0 in range(0, grid.Nz, z_chunk):
        zs = z[z0:z0 + z_chunk]
        Z, Y, X0 = np.meshgrid(zs, y, x, indexing="ij")
        accE = np.zeros((3,) + X0.shape)
        accB = np.zeros((3,) + X0.shape)
        for m in reps:
            E, B = _pulse_fields_at(X0 + m * grid.D, Y, Z, pulse, mapping, grid.c)
            accE += E
            accB += B
        out[0:3, z0:z0 + len(zs)] = accE
        out[3:6, z0:z0 + len(zs)] = accB
    if pulse.div_project:
        out = project_transverse(out, grid)
    return out


def project_transverse(fields: np.ndarray, grid: Grid) -> np.ndarray:
    """Remove k^(k^.E) and k^(k^.B) once in Fourier space (Sec. 2.1, R4)."""
    F = fft3(fields)
    kx, ky, kz = _k_grids(grid)
    kx, ky, kz = np.broadcast_arrays(kx, ky, kz)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    safe = np.where(kmag > 0, kmag, 1.0)
    n = [np.where(kmag > 0, kk / safe, 0.0) for kk in (kx, ky, kz)]
    for base in (0, 3):
        dot = n[0] * F[base] + n[1] * F[base + 1] + n[2] * F[base + 2]
        for a in range(3):
            F[base + a] = F[base + a] - n[a] * dot
    return ifft3(F)


def sample_plane(fields: np.ndarray, grid: Grid, mapping: Mapping, x_p: float,
                 ys: np.ndarray, zs: np.ndarray, t: float, comps=(0, 1, 2)) -> np.ndarray:
    """Field on the physical plane x = x_p at points (ys[p], zs[q]) (Eq. 14).

    u(R, t) = u~(T(R)) * I_S(t)(R), with u~ the exact trigonometric interpolant
    of the periodic grid field, u~(r) = (1/N) sum_m F(m) exp(i k_m.(r - r_min))
    (R16).  Returns complex128 out[len(comps), len(zs), len(ys)].
    """
    ys = np.asarray(ys, dtype=np.float64)
    zs = np.asarray(zs, dtype=np.float64)
    xt = float(mapping_T(x_p, grid.x_min, grid.D))
    kx = wavenumbers(grid.Nx, grid.dx)
    ky = wavenumbers(grid.Ny, grid.dy)
    kz = wavenumbers(grid.Nz, grid.dz)
    ex = np.exp(1j * kx * (xt - grid.x_min))                       # [Nx]
    ey = np.exp(1j * np.outer(ys - grid.y_min, ky))                # [ny, Ny]
    ez = np.exp(1j * np.outer(zs - grid.z_min, kz))                # [nz, Nz]
    N = grid.Nx * grid.Ny * grid.Nz
    Zg, Yg = np.meshgrid(zs, ys, indexing="ij")
    mask = indicator_S(np.full(Zg.shape, x_p), Yg, Zg, t, mapping, grid.c)
    out = np.empty((len(comps), len(zs), len(ys)), dtype=np.complex128)
    for a, ci in enumerate(comps):
        F = fft3(fields[ci])                                       # [Nz, Ny, Nx]
        G = F @ ex                                                 # [Nz, Ny]
        H = ez @ G                                                 # [nz, Ny]
        out[a] = (H @ ey.T) / N * mask                             # [nz, ny]
    return out


def diagnostics(fields: np.ndarray, grid: Grid) -> dict:
    """Energy sum_cells |E|^2 + |B|^2 and the spectral divergence
    max_k |k^.E^(k)|, max_k |k^.B^(k)| with the unnormalised forward DFT."""
    eE = float(np.sum(np.abs(fields[0:3]) ** 2))
    eB = float(np.sum(np.abs(fields[3:6]) ** 2))
    kx, ky, kz = _k_grids(grid)
    kx, ky, kz = np.broadcast_arrays(kx, ky, kz)
    kmag = np.sqrt(kx * kx + ky * ky + kz * kz)
    safe = np.where(kmag > 0, kmag, 1.0)
    n = [np.where(kmag > 0, kk / safe, 0.0) for kk in (kx, ky, kz)]
    res = {"energy": eE + eB, "energy_E": eE, "energy_B": eB}
    for name, base in (("E", 0), ("B", 3)):
        F = fft3(fields[base:base + 3])
        div = n[0] * F[0] + n[1] * F[1] + n[2] * F[2]
        res["max_div_" + name] = float(np.max(np.abs(div)))
        res["max_" + name + "_hat"] = float(np.max(np.sqrt(np.sum(np.abs(F) ** 2, axis=0))))
    return res
