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
#include "ff.cuh"

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

// The closed support |R - R0| <= L/2 (and R > 0) in float64.
__device__ __forceinline__ bool edge_inside(double X, double Y, double Z, const ShellGeom& sh) {
    const double R = sqrt(X * X + Y * Y + Z * Z);
    if (!(R > 0.0)) return false;
    const double zeta = R - sh.R0;
    return !(zeta < -0.5 * sh.L || zeta > 0.5 * sh.L);
}

// Scalar amplitude u(R) with carrier phase `phase`; 0 outside the support.
__device__ __forceinline__ double pulse_u(double X, double Y, double Z, const PulseParams& p,
                                          const ShellGeom& sh, double phase) {
    if (!edge_inside(X, Y, Z, sh)) return 0.0;
    const double R = sqrt(X * X + Y * Y + Z * Z);
    const double zeta = R - sh.R0;
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
    double cps, sps;        // cos, sin of the polarisation angle (float64 storage)
    FF x0, y0, z0, dx, dy, dz, D;      // the grid
    FF R0, k0, phase, two_pi, prof_z0, prof_inv_dz;
    float halfL, inv2pi, lo2, hi2, pi_over_L, th, eps, inv_th2, g4, amp, amp_R0, ell;
    float cp[2], sp[2];     // cos, sin of the carrier phases cep and cep + pi/2 (profile kind)
    float cf, sf;           // cos, sin of the polarisation angle
};

// Geometry of the replica point X = x0 + i dx + m D, Y = y0 + j dy, Z = z0 + l dz:
// false outside the shell; else the point (X, Y, Z rounded to float32), R
// (float32), zeta = R - R0 (double-float, float64-level accuracy) and the angle
// alpha from the -x axis.  A float32 test rejects points well outside the shell
// first; for the rest the float32 root of R^2 is refined by one Newton step
// whose residual R^2 - R_f^2 is formed in double-float.  A point within a
// relative 1e-6 of the support's edge |zeta| = L/2 (grid points can lie on it
// exactly, and the closed window then depends on rounding) takes the float64
// test of the float64 initialiser, so that both storages keep the same points.
__device__ __forceinline__ bool shell_point(int i, int j, int l, int m, const GridGeom& g, const ShellGeom& sh,
                                            const PulseF32& k, float3& P, float& Rf, FF& zeta, float& alpha) {
    const float xf = fmaf((float)i, k.dx.h, k.x0.h) + (float)m * k.D.h;
    const float yf = fmaf((float)j, k.dy.h, k.y0.h), zf = fmaf((float)l, k.dz.h, k.z0.h);
    const float r2 = xf * xf + yf * yf + zf * zf;
    if (r2 < k.lo2 || r2 > k.hi2) return false;        // well outside the shell (margin 1e-4 in R^2)
    const FF X = ff_add(ff_add(k.x0, ff_mul_f(k.dx, (float)i)), ff_mul_f(k.D, (float)m));
    const FF Y = ff_add(k.y0, ff_mul_f(k.dy, (float)j)), Z = ff_add(k.z0, ff_mul_f(k.dz, (float)l));
    const FF S = ff_add(ff_add(ff_sqr(X), ff_sqr(Y)), ff_sqr(Z));
    Rf = sqrtf(S.h);
    if (!(Rf > 0.f)) return false;
    const float corr = ff_add(S, ff_neg(two_prod(Rf, Rf))).h / (2.f * Rf);
    zeta = ff_add(two_sum(Rf, -k.R0.h), two_sum(corr, -k.R0.l));
    if (fabsf(fabsf(zeta.h) - k.halfL) < 1e-6f * k.halfL) {
        const double X = (g.x_min + i * g.dx) + m * (g.Nx * g.dx), Y = g.y_min + j * g.dy, Z = g.z_min + l * g.dz;
        if (!edge_inside(X, Y, Z, sh)) return false;
    } else if (zeta.h < -k.halfL || zeta.h > k.halfL) {
        return false;
    }
    P = make_float3(X.h, Y.h, Z.h);
    alpha = atan2f(sqrtf(Y.h * Y.h + Z.h * Z.h), -X.h);
    return true;
}

// Both carrier amplitudes of one replica point (u1 at phase cep, u2 at
// cep + pi/2, the latter to be scaled by the ellipticity); false if zero.
__device__ __forceinline__ bool pulse_u_f2(int i, int j, int l, int m, const GridGeom& g, const ShellGeom& sh,
                                           const PulseParams& p, const PulseF32& k, float3& P, float& u1, float& u2) {
    float Rf, alpha;
    FF zeta;
    if (!shell_point(i, j, l, m, g, sh, k, P, Rf, zeta, alpha)) return false;
    const float inv_R = 1.f / Rf;
    if (p.kind == 2) {
        // tabulated profile: the sample index in double-float (a spacing of a few
        // nm against |zeta| of tens of um), the interpolation weights in float32
        const float uts = u_ts_flat_f(alpha, k.th, k.eps);
        if (uts == 0.f) return false;
        const FF s = ff_mul(ff_add(zeta, ff_neg(k.prof_z0)), k.prof_inv_dz);
        if (!(s.h >= 0.f) || s.h > (float)(p.prof_n - 1)) return false;
        int ik = (int)floorf(s.h);
        float t = (s.h - (float)ik) + s.l;
        if (t < 0.f) { --ik; t += 1.f; }
        if (ik < 0) { ik = 0; t = 0.f; }
        if (ik > p.prof_n - 2) { ik = p.prof_n - 2; t = 1.f; }
        const double2 a0 = p.prof[PSATD_IX(ik, p.prof_n)], a1 = p.prof[PSATD_IX(ik + 1, p.prof_n)];
        const float ar = (float)a0.x + t * (float)(a1.x - a0.x), ai = (float)a0.y + t * (float)(a1.y - a0.y);
        const float A = k.amp * inv_R * uts;
        u1 = A * (ar * k.cp[0] - ai * k.sp[0]);
        u2 = A * (ar * k.cp[1] - ai * k.sp[1]);
        return true;
    }
    // carrier: the phase k0 zeta + cep reduced to [-pi, pi] in double-float
    const FF arg = ff_add(ff_mul(k.k0, zeta), k.phase);
    const FF red = ff_add(arg, ff_neg(ff_mul_f(k.two_pi, rintf(arg.h * k.inv2pi))));
    float sn, cs;
    sincosf(red.h + red.l, &sn, &cs);
    const float zeta_f = zeta.h;
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
            const float cf = kf.cf, sf = kf.sf;
            float E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
            for (int m = m_lo; m <= m_hi; ++m) {
                float u1, u2;
                float3 P;
                if (!pulse_u_f2(i, j, l, m, g, sh, p, kf, P, u1, u2)) continue;
                const float xs = P.x, ys = P.y, zs = P.z;
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
    k.x0 = ff_from(g.x_min); k.y0 = ff_from(g.y_min); k.z0 = ff_from(g.z_min);
    k.dx = ff_from(g.dx); k.dy = ff_from(g.dy); k.dz = ff_from(g.dz);
    k.D = ff_from(g.Nx * g.dx);
    k.R0 = ff_from(sh.R0);
    k.halfL = (float)(0.5 * sh.L);
    k.k0 = ff_from(2.0 * kPi / p.lambda);
    k.inv2pi = (float)(1.0 / (2.0 * kPi));
    k.two_pi = ff_from(2.0 * kPi);
    k.phase = ff_from(p.cep);
    k.prof_z0 = ff_from(p.prof_z0);
    k.prof_inv_dz = ff_from(p.prof_dz != 0.0 ? 1.0 / p.prof_dz : 0.0);
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
