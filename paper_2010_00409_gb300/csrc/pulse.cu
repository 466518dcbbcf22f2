// Pulse initialisation on the mapped periodic layer (Sec. 2.2, 2.3, 3.2.1).
//
// Each node (x~_i, y_j, z_l) of the layer is the image under the mapping T of
// Eq. 13 of the physical points x~_i + m D, y_j, z_l; its field is the sum of the
// pulse over those replicas m (replicas that do not overlap contribute at most
// one nonzero term).  float64 storage: coordinates, angles and the pulse are
// evaluated in float64 and rounded once.  float32 storage: the distance R, the
// offset zeta = R - R0 and the carrier phase (reduced to [-pi, pi]) in float64 —
// the phase 2 pi zeta / lambda needs ~1e-7 rad at R ~ 20 lambda — and the rest
// (angle, windows, polarisation vectors) in float32, adding ~1e-7 relative error
// to the rounding to float32 (float64 arithmetic is the scarce unit on GB300).
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

__device__ __forceinline__ float pulse_u_f(double X, double Y, double Z, const PulseParams& p, const ShellGeom& sh,
                                           double phase) {
    // cheap rejection of points well outside the shell (float32 R^2, margin 1e-4)
    const float xf = (float)X, yf = (float)Y, zf2 = (float)Z;
    const float r2 = xf * xf + yf * yf + zf2 * zf2;
    const float lo = (float)(sh.R0 - 0.5 * sh.L), hi = (float)(sh.R0 + 0.5 * sh.L);
    if (r2 < lo * lo * 0.9999f || r2 > hi * hi * 1.0001f) return 0.f;
    const double R = sqrt(X * X + Y * Y + Z * Z);
    if (!(R > 0.0)) return 0.f;
    const double zeta = R - sh.R0;
    if (zeta < -0.5 * sh.L || zeta > 0.5 * sh.L) return 0.f;
    const float alpha = atan2f(sqrtf((float)(Y * Y + Z * Z)), (float)(-X));
    if (p.kind == 2) {
        // tabulated profile: the interpolation in float64 (a sample spacing of a
        // few nm against |zeta| of tens of um), the transverse shape in float32
        const float uts = u_ts_flat_f(alpha, (float)p.theta, (float)p.eps);
        if (uts == 0.f) return 0.f;
        return (float)(p.amp / R * profile_ul(zeta, p, phase)) * uts;
    }
    const double arg = 2.0 * kPi * zeta / p.lambda + phase;
    const float carrier = sinf((float)(arg - 2.0 * kPi * rint(arg / (2.0 * kPi))));
    const float zf = (float)zeta;
    if (p.kind == 0) {
        const float uts = u_ts_flat_f(alpha, (float)p.theta, (float)p.eps);
        if (uts == 0.f) return 0.f;
        const float cl = cosf((float)kPi * zf / (float)sh.L);
        return (float)(p.amp / R) * carrier * cl * cl * uts;
    }
    float uts = u_ts_flat_f(alpha, (float)(2.0 * p.theta), (float)p.eps);
    if (uts == 0.f) return 0.f;
    const float th = (float)p.theta;
    uts *= expf(-alpha * alpha / (th * th));
    const float w = (float)(p.n_cycles * p.lambda);
    const float ul = expf(-zf * zf * 1.38629436111989061883f / (w * w));   // ln 4
    return (float)(p.amp * sh.R0 / R) * carrier * ul * uts;
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
__global__ void init_pulse_kernel(void* __restrict__ data, GridGeom g, ShellGeom sh, PulseParams p,
                                  int m_lo, int m_hi) {
    const size_t n_cells = (size_t)g.Nx * g.Ny * g.Nz;
    const double D = g.Nx * g.dx;
    const double cps = cos(p.pol_angle), sps = sin(p.pol_angle);
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n_cells;
         idx += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(idx % g.Nx);
        const size_t r = idx / g.Nx;
        const int j = (int)(r % g.Ny);
        const int l = (int)(r / g.Ny);
        const double xt = g.x_min + i * g.dx;
        const double y = g.y_min + j * g.dy;
        const double z = g.z_min + l * g.dz;
        if constexpr (sizeof(T) == 4) {
            const float cf = (float)cps, sf = (float)sps;
            float E[3] = {0, 0, 0}, B[3] = {0, 0, 0};
            for (int m = m_lo; m <= m_hi; ++m) {
                const double x = xt + m * D;
                const float u1 = pulse_u_f(x, y, z, p, sh, p.cep);
                if (u1 != 0.f) {
                    float s0[3], s1[3];
                    pol_vectors_f((float)x, (float)y, (float)z, 0.f, cf, sf, s0, s1);
                    for (int a = 0; a < 3; ++a) { E[a] += u1 * s0[a]; B[a] += u1 * s1[a]; }
                }
                if (p.ellipticity != 0.0) {
                    const float u2 = (float)p.ellipticity * pulse_u_f(x, y, z, p, sh, p.cep + 0.5 * kPi);
                    if (u2 != 0.f) {
                        float s0[3], s1[3];
                        pol_vectors_f((float)x, (float)y, (float)z, 0.f, -sf, cf, s0, s1);
                        for (int a = 0; a < 3; ++a) { E[a] += u2 * s0[a]; B[a] += u2 * s1[a]; }
                    }
                }
            }
            for (int a = 0; a < 3; ++a) {
                store_value<T, REAL>(data, a * n_cells + idx, 6 * n_cells, (T)E[a]);
                store_value<T, REAL>(data, (3 + a) * n_cells + idx, 6 * n_cells, (T)B[a]);
            }
            continue;
        }
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

}  // namespace

template <typename T>
cudaError_t launch_init_pulse(cplx<T>* data, const GridGeom& g, const ShellGeom& sh,
                              const PulseParams& p, int m_lo, int m_hi, cudaStream_t s,
                              long long* nlaunch) {
    const size_t n_cells = (size_t)g.Nx * g.Ny * g.Nz;
    const int threads = 256;
    long long blocks = (long long)((n_cells + threads - 1) / threads);
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    init_pulse_kernel<T, false><<<(unsigned)blocks, threads, 0, s>>>(data, g, sh, p, m_lo, m_hi);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_init_pulse_real(float* data, const GridGeom& g, const ShellGeom& sh, const PulseParams& p,
                                   int m_lo, int m_hi, cudaStream_t s, long long* nlaunch) {
    const size_t n_cells = (size_t)g.Nx * g.Ny * g.Nz;
    const int threads = 256;
    long long blocks = (long long)((n_cells + threads - 1) / threads);
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    init_pulse_kernel<float, true><<<(unsigned)blocks, threads, 0, s>>>(data, g, sh, p, m_lo, m_hi);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

template cudaError_t launch_init_pulse<float>(cplx<float>*, const GridGeom&, const ShellGeom&, const PulseParams&, int, int, cudaStream_t, long long*);
template cudaError_t launch_init_pulse<double>(cplx<double>*, const GridGeom&, const ShellGeom&, const PulseParams&, int, int, cudaStream_t, long long*);

}  // namespace psatd
