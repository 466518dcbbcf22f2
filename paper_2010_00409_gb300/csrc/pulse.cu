// Pulse initialisation on the mapped periodic layer (Sec. 2.2, 2.3, 3.2.1).
//
// Each node (x~_i, y_j, z_l) of the layer is the image under the mapping T of
// Eq. 13 of the physical points x~_i + m D, y_j, z_l; its field is the sum of the
// pulse over those replicas m (replicas that do not overlap contribute at most
// one nonzero term).  float64 storage: coordinates, angles and the pulse are
// evaluated in float64 and rounded once.  float32 storage: the offset
// zeta = R - R0 and the carrier phase (reduced to [-pi, pi]) to float64
// accuracy — the phase 2 pi zeta / lambda needs ~1e-7 rad at R ~ 20 lambda — and
// the rest (angle, windows, amplitude 1/R, polarisation vectors) in float32,
// adding ~1e-7 relative error to the rounding to float32.  float64 arithmetic
// is the scarce unit on GB300, so zeta takes the float32 root of R^2 refined by
// one Newton step whose residual R^2 - R_f^2 is formed in float64 (about ten
// float64 operations a replica, no float64 division, square root or
// transcendental), and the two carriers of an elliptical pulse (phases cep and
// cep + pi/2) share one evaluation of the geometry.
#include "common.cuh"

namespace psatd {

namespace {

constexpr double kPi = 3.14159265358979323846;

// Eq. 5 (edge window half-open so the profile is continuous)
__device__ __forceinline__ double u_ts_flat(double a, double th, double eps) {
    if (a <= th - 0.5 * eps) return 1.0;
    if (a <= th + 0.5 * eps) {
        const double c = cos(kPi * (a - th + 0.5 * eps) / (2.0 * eps));
        return c * c;
    }
    return 0.0;
}

// Tabulated longitudinal factor Re(a(zeta) e^{i phase}), a linearly
// interpolated between the samples; 0 outside the table.
__device__ __forceinline__ double profile_ul(double zeta, const PulseParams& p, double phase) {
    const double s = (zeta - p.prof_z0) / p.prof_dz;
    if (!(s >= 0.0) || s > (double)(p.prof_n - 1)) return 0.0;
    int k = (int)s;
    if (k > p.prof_n - 2) k = p.prof_n - 2;
    const double t = s - k;
    const double2 a0 = p.prof[PSATD_IX(k, p.prof_n)], a1 = p.prof[PSATD_IX(k + 1, p.prof_n)];
    const double ar = a0.x + t * (a1.x - a0.x), ai = a0.y + t * (a1.y - a0.y);
    return ar * cos(phase) - ai * sin(phase);
}

// Scalar amplitude u(R) with carrier phase `phase`; 0 outside the support.
__device__ __forceinline__ double pulse_u(double X, double Y, double Z, const PulseParams& p,
                                          const ShellGeom& sh, double phase) {
    const double R = sqrt(X * X + Y * Y + Z * Z);
    if (!(R > 0.0)) return 0.0;
    const double zeta = R - sh.R0;
    if (zeta < -0.5 * sh.L || zeta > 0.5 * sh.L) return 0.0;
    const double alpha = atan2(sqrt(Y * Y + Z * Z), -X);   // angle from the -x axis
    if (p.kind == 0) {
        // flat-top, Eq. 7-8
        const double uts = u_ts_flat(alpha, p.theta, p.eps);
        if (uts == 0.0) return 0.0;
        const double cl = cos(kPi * zeta / sh.L);
        const double ul = sin(2.0 * kPi * zeta / p.lambda + phase) * cl * cl;
        return p.amp / R * ul * uts;
    }
    if (p.kind == 2) {
        // flat-top transverse shape (Eq. 5), tabulated longitudinal profile
        const double uts = u_ts_flat(alpha, p.theta, p.eps);
        if (uts == 0.0) return 0.0;
        return p.amp / R * profile_ul(zeta, p, phase) * uts;
    }
    // Gaussian, Sec. 3.2.1
    double uts = u_ts_flat(alpha, 2.0 * p.theta, p.eps);
    if (uts == 0.0) return 0.0;
    uts *= exp(-alpha * alpha / (p.theta * p.theta));
    const double w = p.n_cycles * p.lambda;
    const double ul = exp(-zeta * zeta * 1.38629436111989061883 / (w * w));   // ln 4
    return p.amp * sh.R0 * sin(2.0 * kPi / p.lambda * zeta + phase) * ul * uts / R;
}

// s0 = R x (d x R) / |.|, s1 = d x R / |.|  (Eq. 10-11)
__device__ __forceinline__ void pol_vectors(double X, double Y, double Z, double d0, double d1,
                                            double d2, double s0[3], double s1[3]) {
    const double a0 = d1 * Z - d2 * Y, a1 = d2 * X - d0 * Z, a2 = d0 * Y - d1 * X;   // d x R
    const double b0 = Y * a2 - Z * a1, b1 = Z * a0 - X * a2, b2 = X * a1 - Y * a0;   // R x (d x R)
    const double n1 = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
    const double n0 = sqrt(b0 * b0 + b1 * b1 + b2 * b2);
    const double i1 = n1 > 0.0 ? 1.0 / n1 : 0.0, i0 = n0 > 0.0 ? 1.0 / n0 : 0.0;
    s0[0] = b0 * i0; s0[1] = b1 * i0; s0[2] = b2 * i0;
    s1[0] = a0 * i1; s1[1] = a1 * i1; s1[2] = a2 * i1;
}

// float32-storage variants of u_ts_flat, pulse_u and pol_vectors
__device__ __forceinline__ float u_ts_flat_f(float a, float th, float eps) {
    if (a <= th - 0.5f * eps) return 1.f;
    if (a <= th + 0.5f * eps) {
        const float c = cosf((float)kPi * (a - th + 0.5f * eps) / (2.f * eps));
        return c * c;
    }
    return 0.f;
}

// Per-launch constants of the float32-storage evaluation (built on the host).
struct PulseF32 {
    double R0, halfL, k0, inv2pi, two_pi, phase, prof_z0, prof_inv_dz;
    double cps, sps;        // cos, sin of the polarisation angle (float64 storage)
    float lo2, hi2, pi_over_L, th, eps, inv_th2, g4, amp, amp_R0, ell;
    float cp[2], sp[2];     // cos, sin of the carrier phases cep and cep + pi/2 (profile kind)
    float cf, sf;           // cos, sin of the polarisation angle
    float x0, y0, z0, dx, dy, dz, D;   // the grid in float32 (rejection tests)
};

// Geometry of one replica point given in float32 (xf, yf, zf; rejection) and
// float64 (X, Y, Z; formed only for points near the shell): false outside the
// shell; else R (float32), zeta = R - R0 (float64 accuracy) and the angle alpha
// from the -x axis.
template <typename XYZ>
__device__ __forceinline__ bool shell_point(float xf, float yf, float zf, XYZ xyz, const PulseF32& k, float& Rf,
                                            double& zeta, float& alpha) {
    const float r2 = xf * xf + yf * yf + zf * zf;
    if (r2 < k.lo2 || r2 > k.hi2) return false;        // well outside the shell (margin 1e-4 in R^2)
    double X, Y, Z;
    xyz(X, Y, Z);
    xf = (float)X; yf = (float)Y; zf = (float)Z;
    Rf = sqrtf(xf * xf + yf * yf + zf * zf);
    if (!(Rf > 0.f)) return false;
    // one Newton step on R^2 = S: R = R_f + (S - R_f^2) / (2 R_f), the residual
    // exact in float64 (R_f^2 has 48 bits), the correction (~1e-7 R) in float32
    const double S = fma(X, X, fma(Y, Y, Z * Z));
    const float corr = (float)(S - (double)Rf * (double)Rf) / (2.f * Rf);
    zeta = ((double)Rf - k.R0) + (double)corr;
    if (zeta < -k.halfL || zeta > k.halfL) return false;
    alpha = atan2f(sqrtf(yf * yf + zf * zf), -xf);
    return true;
}

// Both carrier amplitudes of one replica point (u1 at phase cep, u2 at
// cep + pi/2, the latter to be scaled by the ellipticity); false if zero.
template <typename XYZ>
__device__ __forceinline__ bool pulse_u_f2(float xf, float yf, float zf, XYZ xyz, const PulseParams& p,
                                           const PulseF32& k, float& u1, float& u2) {
    float Rf, alpha;
    double zeta;
    if (!shell_point(xf, yf, zf, xyz, k, Rf, zeta, alpha)) return false;
    const float inv_R = 1.f / Rf;
    if (p.kind == 2) {
        // tabulated profile: the sample index in float64 (a spacing of a few nm
        // against |zeta| of tens of um), the interpolation weights in float32
        const float uts = u_ts_flat_f(alpha, k.th, k.eps);
        if (uts == 0.f) return false;
        const double s = (zeta - k.prof_z0) * k.prof_inv_dz;
        if (!(s >= 0.0) || s > (double)(p.prof_n - 1)) return false;
        int ik = (int)s;
        if (ik > p.prof_n - 2) ik = p.prof_n - 2;
        const float t = (float)(s - ik);
        const double2 a0 = p.prof[PSATD_IX(ik, p.prof_n)], a1 = p.prof[PSATD_IX(ik + 1, p.prof_n)];
        const float ar = (float)a0.x + t * (float)(a1.x - a0.x), ai = (float)a0.y + t * (float)(a1.y - a0.y);
        const float A = k.amp * inv_R * uts;
        u1 = A * (ar * k.cp[0] - ai * k.sp[0]);
        u2 = A * (ar * k.cp[1] - ai * k.sp[1]);
        return true;
    }
    // carrier: the phase k0 zeta + cep reduced to [-pi, pi] in float64
    const double arg = fma(k.k0, zeta, k.phase);
    float sn, cs;
    sincosf((float)fma(-k.two_pi, rint(arg * k.inv2pi), arg), &sn, &cs);
    const float zeta_f = (float)zeta;
    float A;
    if (p.kind == 0) {
        // flat-top, Eq. 7-8
        const float uts = u_ts_flat_f(alpha, k.th, k.eps);
        if (uts == 0.f) return false;
        const float cl = cosf(k.pi_over_L * zeta_f);
        A = k.amp * inv_R * cl * cl * uts;
    } else {
        // Gaussian, Sec. 3.2.1
        float uts = u_ts_flat_f(alpha, 2.f * k.th, k.eps);
        if (uts == 0.f) return false;
        uts *= expf(-alpha * alpha * k.inv_th2);
        A = k.amp_R0 * inv_R * expf(-zeta_f * zeta_f * k.g4) * uts;
    }
    u1 = A * sn;                                       // sin(phase)
    u2 = A * cs;                                       // sin(phase + pi/2)
    return true;
}

__device__ __forceinline__ void pol_vectors_f(float X, float Y, float Z, float d0, float d1, float d2, float s0[3],
                                              float s1[3]) {
    const float a0 = d1 * Z - d2 * Y, a1 = d2 * X - d0 * Z, a2 = d0 * Y - d1 * X;   // d x R
    const float b0 = Y * a2 - Z * a1, b1 = Z * a0 - X * a2, b2 = X * a1 - Y * a0;   // R x (d x R)
    const float n1 = sqrtf(a0 * a0 + a1 * a1 + a2 * a2);
    const float n0 = sqrtf(b0 * b0 + b1 * b1 + b2 * b2);
    const float i1 = n1 > 0.f ? 1.f / n1 : 0.f, i0 = n0 > 0.f ? 1.f / n0 : 0.f;
    s0[0] = b0 * i0; s0[1] = b1 * i0; s0[2] = b2 * i0;
    s1[0] = a0 * i1; s1[1] = a1 * i1; s1[2] = a2 * i1;
}

// One field value: complex storage takes (v, 0), real float32 storage v.
template <typename T, bool REAL>
__device__ __forceinline__ void store_value(void* data, size_t i, size_t n, T v) {
    if constexpr (REAL) static_cast<float*>(data)[PSATD_IX(i, n)] = (float)v;
    else static_cast<cplx<T>*>(data)[PSATD_IX(i, n)] = mk<T>(v, (T)0);
}

template <typename T, bool REAL>
__global__ void init_pulse_kernel(void* __restrict__ data, GridGeom g, ShellGeom sh, PulseParams p, PulseF32 kf,
                                  int m_lo, int m_hi) {
    const size_t n_cells = (size_t)g.Nx * g.Ny * g.Nz;
    const double D = g.Nx * g.dx;
    const double cps = kf.cps, sps = kf.sps;
    const bool small = n_cells <= 0xFFFFFFFFull;          // 32-bit index arithmetic
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n_cells;
         idx += (size_t)gridDim.x * blockDim.x) {
        int i, j, l;
        if (small) {
            const unsigned u = (unsigned)idx, r = u / (unsigned)g.Nx;
            i = (int)(u - r * (unsigned)g.Nx);
            l = (int)(r / (unsigned)g.Ny);
            j = (int)(r - (unsigned)l * (unsigned)g.Ny);
        } else {
            i = (int)(idx % g.Nx);
            const size_t r = idx / g.Nx;
            j = (int)(r % g.Ny);
            l = (int)(r / g.Ny);
        }
        if constexpr (sizeof(T) == 4) {
            // float32 coordinates for the rejection test; float64 ones only near the shell
            const float cf = kf.cf, sf = kf.sf;
            const float xtf = kf.x0 + (float)i * kf.dx, yf = kf.y0 + (float)j * kf.dy, zf = kf.z0 + (float)l * kf.dz;
            float E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
            for (int m = m_lo; m <= m_hi; ++m) {
                float u1, u2;
                auto xyz = [&](double& X, double& Y, double& Z) {
                    X = (g.x_min + i * g.dx) + m * D;
                    Y = g.y_min + j * g.dy;
                    Z = g.z_min + l * g.dz;
                };
                if (!pulse_u_f2(xtf + (float)m * kf.D, yf, zf, xyz, p, kf, u1, u2)) continue;
                double X, Y, Z;
                xyz(X, Y, Z);
                const float xs = (float)X, ys = (float)Y, zs = (float)Z;
                float s0[3], s1[3];
                if (u1 != 0.f) {
                    pol_vectors_f(xs, ys, zs, 0.f, cf, sf, s0, s1);
                    for (int a = 0; a < 3; ++a) { E[a] += u1 * s0[a]; B[a] += u1 * s1[a]; }
                }
                u2 *= kf.ell;
                if (u2 != 0.f) {
                    pol_vectors_f(xs, ys, zs, 0.f, -sf, cf, s0, s1);
                    for (int a = 0; a < 3; ++a) { E[a] += u2 * s0[a]; B[a] += u2 * s1[a]; }
                }
            }
            for (int a = 0; a < 3; ++a) {
                store_value<T, REAL>(data, a * n_cells + idx, 6 * n_cells, (T)E[a]);
                store_value<T, REAL>(data, (3 + a) * n_cells + idx, 6 * n_cells, (T)B[a]);
            }
            continue;
        }
        const double xt = g.x_min + i * g.dx;
        const double y = g.y_min + j * g.dy;
        const double z = g.z_min + l * g.dz;
        double E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
        for (int m = m_lo; m <= m_hi; ++m) {
            const double x = xt + m * D;
            const double u1 = pulse_u(x, y, z, p, sh, p.cep);
            if (u1 != 0.0) {
                double s0[3], s1[3];
                pol_vectors(x, y, z, 0.0, cps, sps, s0, s1);
                for (int a = 0; a < 3; ++a) { E[a] += u1 * s0[a]; B[a] += u1 * s1[a]; }
            }
            if (p.ellipticity != 0.0) {
                const double u2 = p.ellipticity * pulse_u(x, y, z, p, sh, p.cep + 0.5 * kPi);
                if (u2 != 0.0) {
                    double s0[3], s1[3];
                    pol_vectors(x, y, z, 0.0, -sps, cps, s0, s1);
                    for (int a = 0; a < 3; ++a) { E[a] += u2 * s0[a]; B[a] += u2 * s1[a]; }
                }
            }
        }
        for (int a = 0; a < 3; ++a) {
            store_value<T, REAL>(data, a * n_cells + idx, 6 * n_cells, (T)E[a]);
            store_value<T, REAL>(data, (3 + a) * n_cells + idx, 6 * n_cells, (T)B[a]);
        }
    }
}

PulseF32 pulse_f32(const PulseParams& p, const ShellGeom& sh, const GridGeom& g) {
    PulseF32 k;
    k.cps = cos(p.pol_angle);
    k.sps = sin(p.pol_angle);
    k.cf = (float)k.cps;
    k.sf = (float)k.sps;
    k.x0 = (float)g.x_min; k.y0 = (float)g.y_min; k.z0 = (float)g.z_min;
    k.dx = (float)g.dx; k.dy = (float)g.dy; k.dz = (float)g.dz;
    k.D = (float)(g.Nx * g.dx);
    k.R0 = sh.R0;
    k.halfL = 0.5 * sh.L;
    k.k0 = 2.0 * kPi / p.lambda;
    k.inv2pi = 1.0 / (2.0 * kPi);
    k.two_pi = 2.0 * kPi;
    k.phase = p.cep;
    k.prof_z0 = p.prof_z0;
    k.prof_inv_dz = p.prof_dz != 0.0 ? 1.0 / p.prof_dz : 0.0;
    const float lo = (float)(sh.R0 - 0.5 * sh.L), hi = (float)(sh.R0 + 0.5 * sh.L);
    k.lo2 = lo * lo * 0.9999f;
    k.hi2 = hi * hi * 1.0001f;
    k.pi_over_L = (float)(kPi / sh.L);
    k.th = (float)p.theta;
    k.eps = (float)p.eps;
    k.inv_th2 = (float)(1.0 / (p.theta * p.theta));
    const double w = p.n_cycles * p.lambda;
    k.g4 = (float)(1.38629436111989061883 / (w * w));   // ln 4 / w^2
    k.amp = (float)p.amp;
    k.amp_R0 = (float)(p.amp * sh.R0);
    k.ell = (float)p.ellipticity;
    k.cp[0] = (float)cos(p.cep); k.sp[0] = (float)sin(p.cep);
    k.cp[1] = (float)cos(p.cep + 0.5 * kPi); k.sp[1] = (float)sin(p.cep + 0.5 * kPi);
    return k;
}

}  // namespace

template <typename T>
cudaError_t launch_init_pulse(cplx<T>* data, const GridGeom& g, const ShellGeom& sh,
                              const PulseParams& p, int m_lo, int m_hi, cudaStream_t s,
                              long long* nlaunch) {
    const size_t n_cells = (size_t)g.Nx * g.Ny * g.Nz;
    const int threads = 256;
    long long blocks = (long long)((n_cells + threads - 1) / threads);
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    init_pulse_kernel<T, false><<<(unsigned)blocks, threads, 0, s>>>(data, g, sh, p, pulse_f32(p, sh, g), m_lo, m_hi);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_init_pulse_real(float* data, const GridGeom& g, const ShellGeom& sh, const PulseParams& p,
                                   int m_lo, int m_hi, cudaStream_t s, long long* nlaunch) {
    const size_t n_cells = (size_t)g.Nx * g.Ny * g.Nz;
    const int threads = 256;
    long long blocks = (long long)((n_cells + threads - 1) / threads);
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    init_pulse_kernel<float, true><<<(unsigned)blocks, threads, 0, s>>>(data, g, sh, p, pulse_f32(p, sh, g), m_lo, m_hi);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

template cudaError_t launch_init_pulse<float>(cplx<float>*, const GridGeom&, const ShellGeom&, const PulseParams&, int, int, cudaStream_t, long long*);
template cudaError_t launch_init_pulse<double>(cplx<double>*, const GridGeom&, const ShellGeom&, const PulseParams&, int, int, cudaStream_t, long long*);

}  // namespace psatd
