// Focal-plane sampling (Sec. 2.3, Eq. 13-16).
//
// The field at a physical point R = (x_p, y, z) is u~(T(R)) * I_S(t)(R), with T
// of Eq. 13 and u~ the exact trigonometric interpolant of the periodic grid
// field: u~(r) = (1/N) sum_m F(m) exp(i k_m . (r - r_min)).  Substituting the
// forward DFT gives the separable form
//     u~(r) = sum_{i,j,l} w_x(x - x_i) w_y(y - y_j) w_z(z - z_l) f_{l j i},
//     w_N(s) = (1/N) sum_m exp(i 2 pi m s / (N d)),  m = -floor(N/2) .. ceil(N/2)-1,
// and the geometric sum closes to
//     w_N(s) = exp(i (m_lo + (N-1)/2) phi) sin(N phi / 2) / (N sin(phi / 2)),
//     phi = 2 pi s / (N d)   (w = 1 at phi = 0; w is N d-periodic in s).
// The three contractions (x, then y, then z) run in float64 for float64
// storage and in double-float arithmetic (ff.cuh: float32 pairs, ~48 bits) for
// float32 storage, whose inputs are float32: the same sums to ~1e-14 without
// float64 instructions, which GB300 issues at 1/64 of the float32 rate.  The
// weights and the partial sums g, h then live in the scratch buffers as float4
// {re.h, re.l, im.h, im.l} (the size of a double2).
#include "common.cuh"
#include "ff.cuh"

namespace psatd {

namespace {

constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double2 dirichlet_weight(double s, int N, double d) {
    double u = s / (N * d);
    u -= floor(u + 0.5);                       // u in [-1/2, 1/2)
    if (u == 0.0) return make_double2(1.0, 0.0);
    const double phi = 2.0 * kPi * u;
    const double m_c = (double)(-(N / 2)) + 0.5 * (N - 1);
    const double ratio = sin(0.5 * N * phi) / (N * sin(0.5 * phi));
    return make_double2(ratio * cos(m_c * phi), ratio * sin(m_c * phi));
}

__device__ __forceinline__ double cut_out_indicator(double x, double y, double z, double t,
                                                    const ShellGeom& sh, double c) {
    // Eq. 15-16; the third case reads "R > r(t)" (the printed "R > l(t)" would
    // remove the focus itself, since l(t) <= 0 there).
    const double R = sqrt(x * x + y * y + z * z);
    const double Rmin = sh.R0 - 0.5 * sh.L, Rmax = sh.R0 + 0.5 * sh.L;
    const double l = -Rmax + c * t, r = -Rmin + c * t;
    bool zero = false;
    if (r < 0) zero = zero || (R >= -l) || (R < -r) || (x > 0);
    if (l <= 0 && r >= 0) {
        zero = zero || ((x < 0) && (R > sh.L));
        zero = zero || ((x >= 0) && (R > r));
    }
    if (l > 0) zero = zero || (R <= l) || (R > r) || (x < 0);
    return zero ? 0.0 : 1.0;
}

// a weight in float64 (double2) or double-float (float4) form
template <bool FFW>
__device__ __forceinline__ void put_w(double2* w, int i, int n, double2 v) {
    if constexpr (FFW) reinterpret_cast<float4*>(w)[PSATD_IX(i, n)] = cff_from(v.x, v.y);
    else w[PSATD_IX(i, n)] = v;
}

template <bool FFW>
__global__ void weights_kernel(GridGeom g, double x_phys, int ny, int nz, double y0, double y1,
                               double z0, double z1, double2* wx, double2* wy, double2* wz) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nwx = g.Nx, nwy = ny * g.Ny, nwz = nz * g.Nz;
    const double D = g.Nx * g.dx;
    if (tid < nwx) {
        double q = (x_phys - g.x_min) / D;
        const double xt = g.x_min + D * (q - floor(q));              // Eq. 13
        put_w<FFW>(wx, tid, nwx, dirichlet_weight(xt - (g.x_min + tid * g.dx), g.Nx, g.dx));
    } else if (tid < nwx + nwy) {
        const int e = tid - nwx, p = e / g.Ny, j = e - p * g.Ny;
        const double y = y0 + (y1 - y0) * p / ny;
        put_w<FFW>(wy, e, nwy, dirichlet_weight(y - (g.y_min + j * g.dy), g.Ny, g.dy));
    } else if (tid < nwx + nwy + nwz) {
        const int e = tid - nwx - nwy, q = e / g.Nz, l = e - q * g.Nz;
        const double z = z0 + (z1 - z0) * q / nz;
        put_w<FFW>(wz, e, nwz, dirichlet_weight(z - (g.z_min + l * g.dz), g.Nz, g.dz));
    }
}

// Weights that evaluate the interpolant straight from a spectrum that already
// carries the 1/N of the inverse DFT (as the k-space pass leaves it):
// u~(r) = sum_m G(m) prod_a exp(i k_{a,m} (r_a - r_min,a)),  G = F / N.
__device__ __forceinline__ double2 mode_phase(int i, int N, double d, double s) {
    const int m = i <= (N - 1) / 2 ? i : i - N;
    const double ph = 2.0 * kPi * (double)m / (N * d) * s;
    return make_double2(cos(ph), sin(ph));
}

template <bool FFW>
__global__ void spectral_weights_kernel(GridGeom g, double x_phys, int ny, int nz, double y0, double y1,
                                        double z0, double z1, double2* wx, double2* wy, double2* wz) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nwx = g.Nx, nwy = ny * g.Ny, nwz = nz * g.Nz;
    const double D = g.Nx * g.dx;
    if (tid < nwx) {
        double q = (x_phys - g.x_min) / D;
        const double xt = g.x_min + D * (q - floor(q));              // Eq. 13
        put_w<FFW>(wx, tid, nwx, mode_phase(tid, g.Nx, g.dx, xt - g.x_min));
    } else if (tid < nwx + nwy) {
        const int e = tid - nwx, p = e / g.Ny, j = e - p * g.Ny;
        put_w<FFW>(wy, e, nwy, mode_phase(j, g.Ny, g.dy, y0 + (y1 - y0) * p / ny - g.y_min));
    } else if (tid < nwx + nwy + nwz) {
        const int e = tid - nwx - nwy, q = e / g.Nz, l = e - q * g.Nz;
        put_w<FFW>(wz, e, nwz, mode_phase(l, g.Nz, g.dz, z0 + (z1 - z0) * q / nz - g.z_min));
    }
}

struct CompList { int c[6]; };

// g[a][l][j] = sum_i wx[i] f[c_a][l][j][i]; one warp per (a, l, j) row.
template <typename T>
__global__ void contract_x_kernel(const cplx<T>* __restrict__ f, GridGeom g, CompList cl, int ncomp,
                                  const double2* __restrict__ wx, double2* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long rows = (long long)ncomp * g.Nz * g.Ny;
    if (warp >= rows) return;
    const int a = (int)(warp / ((long long)g.Nz * g.Ny));
    const long long rl = warp - (long long)a * g.Nz * g.Ny;
    const cplx<T>* row = f + (size_t)cl.c[a] * g.Nx * g.Ny * g.Nz + (size_t)rl * g.Nx;
    const GBuf<const cplx<T>> F{f, 6LL * g.Nx * g.Ny * g.Nz};
    double re = 0.0, im = 0.0;
    for (int i = lane; i < g.Nx; i += 32) {
        const cplx<T> v = F.at(row, i);
        const double2 w = wx[PSATD_IX(i, g.Nx)];
        re += w.x * (double)v.x - w.y * (double)v.y;
        im += w.x * (double)v.y + w.y * (double)v.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) out[PSATD_IX(warp, rows)] = make_double2(re, im);
}

// h[a][l][p] = sum_j wy[p][j] g[a][l][j]
__global__ void contract_y_kernel(const double2* __restrict__ gin, GridGeom g, int ncomp, int ny,
                                  const double2* __restrict__ wy, double2* __restrict__ h) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)ncomp * g.Nz * ny) return;
    const int p = (int)(tid % ny);
    const long long al = tid / ny;                 // a * Nz + l
    const double2* gr = gin + (size_t)al * g.Ny;
    const double2* w = wy + (size_t)p * g.Ny;
    double re = 0.0, im = 0.0;
    const GBuf<const double2> Gi{gin, (long long)ncomp * g.Nz * g.Ny}, Wy{wy, (long long)ny * g.Ny};
    for (int j = 0; j < g.Ny; ++j) {
        const double2 a = Gi.at(gr, j), b = Wy.at(w, j);
        re += b.x * a.x - b.y * a.y;
        im += b.x * a.y + b.y * a.x;
    }
    h[PSATD_IX(tid, (long long)ncomp * g.Nz * ny)] = make_double2(re, im);
}

// out[a][q][p] = I_S(x_p, y_p, z_q, t) * sum_l wz[q][l] h[a][l][p]
template <typename T>
__global__ void contract_z_kernel(const double2* __restrict__ h, GridGeom g, ShellGeom sh, int ncomp,
                                  int ny, int nz, double x_phys, double y0, double y1, double z0,
                                  double z1, double t, const double2* __restrict__ wz,
                                  cplx<T>* __restrict__ out) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)ncomp * nz * ny) return;
    const int p = (int)(tid % ny);
    const long long r = tid / ny;
    const int q = (int)(r % nz);
    const int a = (int)(r / nz);
    const double2* w = wz + (size_t)q * g.Nz;
    const double2* hc = h + (size_t)a * g.Nz * ny + p;
    double re = 0.0, im = 0.0;
    const GBuf<const double2> Hb{h, (long long)ncomp * g.Nz * ny}, Wz{wz, (long long)nz * g.Nz};
    for (int l = 0; l < g.Nz; ++l) {
        const double2 v = Hb.at(hc, (long long)l * ny), b = Wz.at(w, l);
        re += b.x * v.x - b.y * v.y;
        im += b.x * v.y + b.y * v.x;
    }
    const double y = y0 + (y1 - y0) * p / ny;
    const double z = z0 + (z1 - z0) * q / nz;
    const double m = cut_out_indicator(x_phys, y, z, t, sh, g.c);
    out[PSATD_IX(tid, (long long)ncomp * nz * ny)] = mk<T>((T)(re * m), (T)(im * m));
}

// ---------------------------------------------------------------------------
// float32 storage: the same three contractions in double-float arithmetic
// (weights, g and h as float4 double-float complex values).

// g[a][l][j] = sum_i wx[i] f[c_a][l][j][i] for complex float32 f; one warp per row.
__global__ void contract_x_ff_kernel(const float2* __restrict__ f, GridGeom g, CompList cl, int ncomp,
                                     const float4* __restrict__ wx, float4* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long rows = (long long)ncomp * g.Nz * g.Ny;
    if (warp >= rows) return;
    const int a = (int)(warp / ((long long)g.Nz * g.Ny));
    const long long rl = warp - (long long)a * g.Nz * g.Ny;
    const float2* row = f + (size_t)cl.c[a] * g.Nx * g.Ny * g.Nz + (size_t)rl * g.Nx;
    const GBuf<const float2> F{f, 6LL * g.Nx * g.Ny * g.Nz};
    CFF acc{{0.f, 0.f}, {0.f, 0.f}};
    for (int i = lane; i < g.Nx; i += 32) cff_mac(acc, cff_load(wx[PSATD_IX(i, g.Nx)]), F.at(row, i));
    acc = cff_warp_sum(acc);
    if (lane == 0) out[PSATD_IX(warp, rows)] = cff_store(acc);
}

// the same for real float32 f
__global__ void contract_x_real_ff_kernel(const float* __restrict__ f, GridGeom g, CompList cl, int ncomp,
                                          const float4* __restrict__ wx, float4* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long rows = (long long)ncomp * g.Nz * g.Ny;
    if (warp >= rows) return;
    const int a = (int)(warp / ((long long)g.Nz * g.Ny));
    const long long rl = warp - (long long)a * g.Nz * g.Ny;
    const float* row = f + (size_t)cl.c[a] * g.Nx * g.Ny * g.Nz + (size_t)rl * g.Nx;
    const GBuf<const float> F{f, 6LL * g.Nx * g.Ny * g.Nz};
    CFF acc{{0.f, 0.f}, {0.f, 0.f}};
    for (int i = lane; i < g.Nx; i += 32) cff_mac_real(acc, cff_load(wx[PSATD_IX(i, g.Nx)]), F.at(row, i));
    acc = cff_warp_sum(acc);
    if (lane == 0) out[PSATD_IX(warp, rows)] = cff_store(acc);
}

// Half spectrum of real fields (slots p < Nx/2 holding x mode mode[p], the x
// Nyquist mode in Q), with the 1/N of the inverse DFT folded in.  The modes with
// negative k_x are the conjugates F(-k) = conj F(k) of the stored ones, so
//   g[a][l][j] = A[l][j] + conj(A'[-l][-j]),
//   A  = sum_p S[p] wx[mode[p]] + Q wx[Nx/2]   (k_x >= 0 and the Nyquist mode),
//   A' = A without the k_x = 0 and Nyquist terms  (their mirrors are themselves),
// using conj(F) wx[-k_x] = conj(F wx[k_x]); -l, -j are the mirrored indices
// (N - l) mod N.  One warp per (a, l, j).
__global__ void contract_x_half_ff_kernel(const float2* __restrict__ S, const float2* __restrict__ Q, GridGeom g,
                                          CompList cl, int ncomp, const int* __restrict__ mode,
                                          const float4* __restrict__ wx, float4* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long rows = (long long)ncomp * g.Nz * g.Ny;
    if (warp >= rows) return;
    const int a = (int)(warp / ((long long)g.Nz * g.Ny));
    const long long rl = warp - (long long)a * g.Nz * g.Ny;
    const int l = (int)(rl / g.Ny), j = (int)(rl - (long long)l * g.Ny);
    const int lm = (g.Nz - l) % g.Nz, jm = (g.Ny - j) % g.Ny;
    const int nh = g.Nx / 2;
    const size_t cbase = (size_t)cl.c[a] * g.Nz * g.Ny;
    const float2* row = S + (cbase + (size_t)l * g.Ny + j) * nh;
    const float2* rowm = S + (cbase + (size_t)lm * g.Ny + jm) * nh;
    const GBuf<const float2> SF{S, 6LL * g.Nz * g.Ny * nh};
    CFF A{{0.f, 0.f}, {0.f, 0.f}}, Bm{{0.f, 0.f}, {0.f, 0.f}};
    for (int p = lane; p < nh; p += 32) {
        const int m = mode[PSATD_IX(p, nh)];
        const CFF w = cff_load(wx[PSATD_IX(m, g.Nx)]);
        cff_mac(A, w, SF.at(row, p));
        if (m != 0) cff_mac(Bm, w, SF.at(rowm, p));
    }
    A = cff_warp_sum(A);
    Bm = cff_warp_sum(Bm);
    if (lane == 0) {
        const CFF w = cff_load(wx[PSATD_IX(nh, g.Nx)]);
        cff_mac(A, w, Q[PSATD_IX(cbase + (size_t)l * g.Ny + j, 6LL * g.Nz * g.Ny)]);
        const CFF r{ff_add(A.re, Bm.re), ff_sub(A.im, Bm.im)};
        out[PSATD_IX(warp, rows)] = cff_store(r);
    }
}

// h[a][l][p] = sum_j wy[p][j] g[a][l][j]
__global__ void contract_y_ff_kernel(const float4* __restrict__ gin, GridGeom g, int ncomp, int ny,
                                     const float4* __restrict__ wy, float4* __restrict__ h) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)ncomp * g.Nz * ny) return;
    const int p = (int)(tid % ny);
    const long long al = tid / ny;                 // a * Nz + l
    const float4* gr = gin + (size_t)al * g.Ny;
    const float4* w = wy + (size_t)p * g.Ny;
    const GBuf<const float4> Gi{gin, (long long)ncomp * g.Nz * g.Ny}, Wy{wy, (long long)ny * g.Ny};
    CFF acc{{0.f, 0.f}, {0.f, 0.f}};
    for (int j = 0; j < g.Ny; ++j) cff_mac_cff(acc, cff_load(Wy.at(w, j)), cff_load(Gi.at(gr, j)));
    h[PSATD_IX(tid, (long long)ncomp * g.Nz * ny)] = cff_store(acc);
}

// out[a][q][p] = I_S(x_p, y_p, z_q, t) * sum_l wz[q][l] h[a][l][p], rounded to float32
__global__ void contract_z_ff_kernel(const float4* __restrict__ h, GridGeom g, ShellGeom sh, int ncomp, int ny,
                                     int nz, double x_phys, double y0, double y1, double z0, double z1, double t,
                                     const float4* __restrict__ wz, float2* __restrict__ out) {
    const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (tid >= (long long)ncomp * nz * ny) return;
    const int p = (int)(tid % ny);
    const long long r = tid / ny;
    const int q = (int)(r % nz);
    const int a = (int)(r / nz);
    const float4* w = wz + (size_t)q * g.Nz;
    const float4* hc = h + (size_t)a * g.Nz * ny + p;
    const GBuf<const float4> Hb{h, (long long)ncomp * g.Nz * ny}, Wz{wz, (long long)nz * g.Nz};
    CFF acc{{0.f, 0.f}, {0.f, 0.f}};
    for (int l = 0; l < g.Nz; ++l) cff_mac_cff(acc, cff_load(Wz.at(w, l)), cff_load(Hb.at(hc, (long long)l * ny)));
    const double y = y0 + (y1 - y0) * p / ny;
    const double z = z0 + (z1 - z0) * q / nz;
    const float m = (float)cut_out_indicator(x_phys, y, z, t, sh, g.c);
    out[PSATD_IX(tid, (long long)ncomp * nz * ny)] = make_float2(ff_float(acc.re) * m, ff_float(acc.im) * m);
}

}  // namespace

template <typename T>
cudaError_t launch_sample_plane(const cplx<T>* data, const GridGeom& g, const ShellGeom& sh,
                                double x_phys, int ny, int nz, double y0, double y1, double z0,
                                double z1, double t, const int* comps, int ncomp,
                                const SampleScratch& sc, cplx<T>* out, cudaStream_t s,
                                long long* nlaunch, bool from_spectrum) {
    CompList cl;
    for (int a = 0; a < 6; ++a) cl.c[a] = a < ncomp ? comps[a] : 0;
    const int nw = g.Nx + ny * g.Ny + nz * g.Nz;
    constexpr bool ffw = sizeof(T) == 4;               // float32 storage: double-float sums
    if (from_spectrum)
        spectral_weights_kernel<ffw><<<(nw + 255) / 256, 256, 0, s>>>(g, x_phys, ny, nz, y0, y1, z0, z1, sc.wx, sc.wy, sc.wz);
    else
        weights_kernel<ffw><<<(nw + 255) / 256, 256, 0, s>>>(g, x_phys, ny, nz, y0, y1, z0, z1, sc.wx, sc.wy, sc.wz);
    const long long rows = (long long)ncomp * g.Nz * g.Ny;
    const long long nh = (long long)ncomp * g.Nz * ny;
    const long long no = (long long)ncomp * nz * ny;
    if constexpr (ffw) {
        float4 *wx = reinterpret_cast<float4*>(sc.wx), *wy = reinterpret_cast<float4*>(sc.wy);
        float4 *wz = reinterpret_cast<float4*>(sc.wz), *gg = reinterpret_cast<float4*>(sc.g);
        float4* hh = reinterpret_cast<float4*>(sc.h);
        contract_x_ff_kernel<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(
            reinterpret_cast<const float2*>(data), g, cl, ncomp, wx, gg);
        contract_y_ff_kernel<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(gg, g, ncomp, ny, wy, hh);
        contract_z_ff_kernel<<<(unsigned)((no + 255) / 256), 256, 0, s>>>(hh, g, sh, ncomp, ny, nz, x_phys, y0, y1, z0,
                                                                          z1, t, wz, reinterpret_cast<float2*>(out));
        if (nlaunch) *nlaunch += 4;
        return cudaGetLastError();
    }
    contract_x_kernel<T><<<(unsigned)((rows * 32 + 255) / 256), 256, 0, s>>>(data, g, cl, ncomp, sc.wx, sc.g);
    contract_y_kernel<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(sc.g, g, ncomp, ny, sc.wy, sc.h);
    contract_z_kernel<T><<<(unsigned)((no + 255) / 256), 256, 0, s>>>(sc.h, g, sh, ncomp, ny, nz, x_phys,
                                                                      y0, y1, z0, z1, t, sc.wz, out);
    if (nlaunch) *nlaunch += 4;
    return cudaGetLastError();
}

cudaError_t launch_sample_plane_real(const float* data, const float2* nyq, const int* slot_mode, const GridGeom& g,
                                     const ShellGeom& sh, double x_phys, int ny, int nz, double y0, double y1,
                                     double z0, double z1, double t, const int* comps, int ncomp,
                                     const SampleScratch& sc, float2* out, cudaStream_t s, long long* nlaunch,
                                     bool from_spectrum) {
    CompList cl;
    for (int a = 0; a < 6; ++a) cl.c[a] = a < ncomp ? comps[a] : 0;
    const int nw = g.Nx + ny * g.Ny + nz * g.Nz;
    if (from_spectrum)
        spectral_weights_kernel<true><<<(nw + 255) / 256, 256, 0, s>>>(g, x_phys, ny, nz, y0, y1, z0, z1, sc.wx, sc.wy, sc.wz);
    else
        weights_kernel<true><<<(nw + 255) / 256, 256, 0, s>>>(g, x_phys, ny, nz, y0, y1, z0, z1, sc.wx, sc.wy, sc.wz);
    float4 *wx = reinterpret_cast<float4*>(sc.wx), *wy = reinterpret_cast<float4*>(sc.wy);
    float4 *wz = reinterpret_cast<float4*>(sc.wz), *gg = reinterpret_cast<float4*>(sc.g);
    float4* hh = reinterpret_cast<float4*>(sc.h);
    const long long rows = (long long)ncomp * g.Nz * g.Ny;
    const unsigned xb = (unsigned)((rows * 32 + 255) / 256);
    if (from_spectrum)
        contract_x_half_ff_kernel<<<xb, 256, 0, s>>>(reinterpret_cast<const float2*>(data), nyq, g, cl, ncomp,
                                                     slot_mode, wx, gg);
    else
        contract_x_real_ff_kernel<<<xb, 256, 0, s>>>(data, g, cl, ncomp, wx, gg);
    const long long nh = (long long)ncomp * g.Nz * ny;
    contract_y_ff_kernel<<<(unsigned)((nh + 255) / 256), 256, 0, s>>>(gg, g, ncomp, ny, wy, hh);
    const long long no = (long long)ncomp * nz * ny;
    contract_z_ff_kernel<<<(unsigned)((no + 255) / 256), 256, 0, s>>>(hh, g, sh, ncomp, ny, nz, x_phys, y0, y1, z0, z1,
                                                                      t, wz, out);
    if (nlaunch) *nlaunch += 4;
    return cudaGetLastError();
}

template cudaError_t launch_sample_plane<float>(const cplx<float>*, const GridGeom&, const ShellGeom&, double, int, int, double, double, double, double, double, const int*, int, const SampleScratch&, cplx<float>*, cudaStream_t, long long*, bool);
template cudaError_t launch_sample_plane<double>(const cplx<double>*, const GridGeom&, const ShellGeom&, double, int, int, double, double, double, double, double, const int*, int, const SampleScratch&, cplx<double>*, cudaStream_t, long long*, bool);

}  // namespace psatd
