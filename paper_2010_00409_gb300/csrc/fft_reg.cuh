// Register-resident FFT pieces for the fast kernels.
//
// A pencil of length N = N1 * N2 (N2 divides N1) is spread over N2 threads that
// hold N1 complex values each.  Forward transform (Cooley-Tukey, n = j + N2 n1,
// k = k1 + N1 k2):
//   1. thread j holds x[j + N2 n1] (n1 < N1), takes an N1-point DFT over n1 in
//      registers and multiplies output k1 by W_N^{j k1};
//   2. the values are exchanged through shared memory so that thread t gathers,
//      for each k1 = t + N2 q (q < N1/N2), the N2 values of all threads;
//   3. an N2-point DFT over j gives X[k1 + N1 k2]; thread t then holds
//      X[(t + N2 q) + N1 k2] in register q*N2 + k2.
// The inverse runs the same steps mirrored and returns to the input layout.
// In both layouts a fixed register index maps consecutive threads to
// consecutive elements, so global loads and stores of a pencil coalesce.
//
// The small DFTs run the Stockham passes of fft_core.cuh on register arrays
// with every index and twiddle fixed at compile time (static_for); twiddles are
// exp(S 2 pi i p/q) evaluated at compile time by ct_cos2pi / ct_sin2pi below.
#pragma once

#include <type_traits>
#include <utility>

#include "fft_core.cuh"

namespace psatd {

// ---------------------------------------------------------------------------
// compile-time cos / sin of 2 pi p / q: reduce to [-pi/4, pi/4] with the
// quadrant symmetries, then the Taylor series (|x| <= pi/4: 13 terms reach
// well below double rounding).
// ---------------------------------------------------------------------------
constexpr double kCtPi = 3.14159265358979323846264338327950288;

constexpr double ct_sin_taylor(double x) {
    double x2 = x * x, term = x, sum = x;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / ((2.0 * n) * (2.0 * n + 1.0));
        sum += term;
    }
    return sum;
}
constexpr double ct_cos_taylor(double x) {
    double x2 = x * x, term = 1.0, sum = 1.0;
    for (int n = 1; n < 14; ++n) {
        term *= -x2 / ((2.0 * n - 1.0) * (2.0 * n));
        sum += term;
    }
    return sum;
}
// angle 2 pi p/q with the octant chosen by integer arithmetic on 8p mod 8q
constexpr void ct_sincos2pi(long long p, long long q, double* s, double* c) {
    p %= q;
    if (p < 0) p += q;
    // octant o = floor(8 p / q), remainder r/q in [0, 1/8)
    long long o = (8 * p) / q;
    long long r8 = 8 * p - o * q;               // 2 pi p/q = o pi/4 + 2 pi r8/(8q)
    double x = 2.0 * kCtPi * (double)r8 / (8.0 * (double)q);   // in [0, pi/4)
    // for odd octants use the complement angle pi/4 - x to stay small
    double sx = ct_sin_taylor(x), cx = ct_cos_taylor(x);
    double y = kCtPi / 4.0 - x;
    double sy = ct_sin_taylor(y), cy = ct_cos_taylor(y);
    // angle = o*pi/4 + x ; write it as multiple of pi/2 plus a small angle
    double S = 0, C = 0;
    switch (o) {
        case 0: S = sx; C = cx; break;                       // x
        case 1: S = cy; C = sy; break;                       // pi/2 - y
        case 2: S = cx; C = -sx; break;                      // pi/2 + x
        case 3: S = sy; C = -cy; break;                      // pi - y
        case 4: S = -sx; C = -cx; break;                     // pi + x
        case 5: S = -cy; C = -sy; break;                     // 3pi/2 - y
        case 6: S = -cx; C = sx; break;                      // 3pi/2 + x
        default: S = -sy; C = cy; break;                     // 2pi - y
    }
    *s = S;
    *c = C;
}
constexpr double ct_cos2pi(long long p, long long q) { double s = 0, c = 0; ct_sincos2pi(p, q, &s, &c); return c; }
constexpr double ct_sin2pi(long long p, long long q) { double s = 0, c = 0; ct_sincos2pi(p, q, &s, &c); return s; }

// ---------------------------------------------------------------------------
// static_for: f(integral_constant<int, i>) for i in [B, E)
// ---------------------------------------------------------------------------
template <int B, int E, typename F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// radix plan of a register DFT: largest radices first
template <int N> struct RegPlanFirst {
    static constexpr int value = (N % 8 == 0 && N != 16) ? 8 : (N % 4 == 0) ? 4 : (N % 5 == 0) ? 5
                                 : (N % 3 == 0) ? 3 : (N % 2 == 0) ? 2 : N;
};

// one Stockham pass of radix R over a register array of length N (product of
// earlier radices Ns)
template <typename T, int S, int N, int R, int Ns>
__host__ __device__ __forceinline__ void reg_pass(const cplx<T> (&in)[N], cplx<T> (&out)[N]) {
    static_for<0, N / R>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        constexpr int k = j % Ns;
        cplx<T> v[R];
        static_for<0, R>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            v[r] = in[j + r * (N / R)];
            if constexpr (Ns > 1 && r > 0 && k > 0) {
                constexpr double c = ct_cos2pi((long long)r * k, (long long)Ns * R);
                constexpr double s = (double)S * ct_sin2pi((long long)r * k, (long long)Ns * R);
                constexpr bool diag = (c > 0.7 || c < -0.7) && (s > 0.7 || s < -0.7);   // odd multiple of 45 deg
                if constexpr (sizeof(T) == 4 && diag) {
                    // (c, s) = (sc, ss) / sqrt 2: exact sign flips, then the compensated 1/sqrt 2
                    constexpr T sc = c > 0 ? T(1) : T(-1), ss = s > 0 ? T(1) : T(-1);
                    const cplx<T> u = v[r];
                    v[r] = mk<T>(mul_rsqrt2<T>(sc * u.x - ss * u.y), mul_rsqrt2<T>(ss * u.x + sc * u.y));
                } else if constexpr (sizeof(T) == 4) {
                    constexpr UnitF w = unit_f32(c, s);
                    v[r] = cmul(v[r], mk<T>(w.c, w.s));
                } else {
                    v[r] = cmul(v[r], mk<T>((T)c, (T)s));
                }
            }
        });
        dft_r<T, R, S>(v);
        constexpr int idx = (j / Ns) * Ns * R + k;
        static_for<0, R>([&](auto rc) {
            constexpr int r = decltype(rc)::value;
            out[idx + r * Ns] = v[r];
        });
    });
}

template <typename T, int S, int N, int Ns>
__host__ __device__ __forceinline__ void reg_dft_rec(cplx<T> (&v)[N]) {
    if constexpr (Ns < N) {
        constexpr int R = RegPlanFirst<N / Ns>::value;
        cplx<T> t[N];
        reg_pass<T, S, N, R, Ns>(v, t);
        static_for<0, N>([&](auto ic) { v[decltype(ic)::value] = t[decltype(ic)::value]; });
        reg_dft_rec<T, S, N, Ns * R>(v);
    }
}

// In-place N-point DFT of a register array, natural order in and out.
template <typename T, int S, int N>
__host__ __device__ __forceinline__ void reg_dft(cplx<T> (&v)[N]) {
    if constexpr (N == 16) {
        // 16 = 4 x 4 keeps the butterflies multiplication-free except 9 twiddles
        cplx<T> t[16];
        reg_pass<T, S, 16, 4, 1>(v, t);
        reg_pass<T, S, 16, 4, 4>(t, v);
    } else {
        reg_dft_rec<T, S, N, 1>(v);
    }
}

// ---------------------------------------------------------------------------
// Pencil stages.  tw[t] = exp(-2 pi i t / N) (inverse uses the conjugate).
// ---------------------------------------------------------------------------
template <typename T, int S>
__host__ __device__ __forceinline__ cplx<T> twiddle(const cplx<T>* __restrict__ tw, int idx, int n) {
#ifdef __CUDA_ARCH__
    const cplx<T> w = tw[PSATD_IX(idx, n)];          // the table holds n = N entries
#else
    (void)n;
    const cplx<T> w = tw[idx];
#endif
    return S < 0 ? w : mk<T>(w.x, -w.y);
}

// Forward stage 1 (input layout): DFT_N1 over n1, then multiply by W_N^{j k1}.
template <typename T, int S, int N1, int N2>
__host__ __device__ __forceinline__ void stage_a_fwd(cplx<T> (&v)[N1], int j, const cplx<T>* __restrict__ tw) {
    reg_dft<T, S, N1>(v);
    static_for<1, N1>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        if (j) v[k1] = cmul(v[k1], twiddle<T, S>(tw, j * k1, N1 * N2));
    });
}

// scratch layout [k1][j], row stride N2 + 1
template <typename T, int N1, int N2>
__host__ __device__ __forceinline__ void scatter_a(const cplx<T> (&v)[N1], cplx<T>* sc, int j) {
    static_for<0, N1>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        sc[k1 * (N2 + 1) + j] = v[k1];
    });
}

// Forward stage 2: thread t gathers rows k1 = t + N2 q and takes DFT_N2 over j;
// register q*N2 + k2 ends holding X[(t + N2 q) + N1 k2].
template <typename T, int S, int N1, int N2>
__host__ __device__ __forceinline__ void gather_b_fwd(cplx<T> (&v)[N1], const cplx<T>* sc, int t) {
    static_for<0, N1 / N2>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        cplx<T> w[N2];
        const cplx<T>* row = sc + (t + N2 * q) * (N2 + 1);
        static_for<0, N2>([&](auto jc) { w[decltype(jc)::value] = row[decltype(jc)::value]; });
        reg_dft<T, S, N2>(w);
        static_for<0, N2>([&](auto kc) { v[q * N2 + decltype(kc)::value] = w[decltype(kc)::value]; });
    });
}

// Inverse stage 1 (spectral layout): for each held k1 = t + N2 q, DFT_N2 over
// k2, then multiply output n2 by W_N^{S n2 k1}; scatter to [k1][n2].
template <typename T, int S, int N1, int N2>
__host__ __device__ __forceinline__ void stage_a_inv_scatter(cplx<T> (&v)[N1], cplx<T>* sc, int t,
                                                     const cplx<T>* __restrict__ tw) {
    static_for<0, N1 / N2>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        cplx<T> w[N2];
        static_for<0, N2>([&](auto kc) { w[decltype(kc)::value] = v[q * N2 + decltype(kc)::value]; });
        reg_dft<T, S, N2>(w);
        const int k1 = t + N2 * q;
        cplx<T>* row = sc + k1 * (N2 + 1);
        static_for<0, N2>([&](auto nc) {
            constexpr int n2 = decltype(nc)::value;
            row[n2] = (n2 == 0 || k1 == 0) ? w[n2] : cmul(w[n2], twiddle<T, S>(tw, n2 * k1, N1 * N2));
        });
    });
}

// Inverse stage 2: thread j gathers column j of every row k1 and takes DFT_N1
// over k1, giving x[j + N2 n1] in register n1.
template <typename T, int S, int N1, int N2>
__host__ __device__ __forceinline__ void gather_b_inv(cplx<T> (&v)[N1], const cplx<T>* sc, int j) {
    static_for<0, N1>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        v[k1] = sc[k1 * (N2 + 1) + j];
    });
    reg_dft<T, S, N1>(v);
}

// ---------------------------------------------------------------------------
// 16 x 16 transpose across the 16 lanes of a group by four XOR-shuffle stages:
// on entry lane j holds a_j[i] in v[i]; on exit lane t holds a_n[t] in v[n].
// Register indices are compile-time; the lane bit only selects values.
template <typename T>
__device__ __forceinline__ void lane_transpose16(cplx<T> (&v)[16], int lane) {
    static_for<0, 4>([&](auto sc) {
        constexpr int sbit = 8 >> decltype(sc)::value;
        const bool up = (lane & sbit) != 0;
        static_for<0, 16>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            if constexpr ((i & sbit) == 0) {
                constexpr int ip = i | sbit;
                const cplx<T> send = up ? v[i] : v[ip];
                cplx<T> recv;
                recv.x = __shfl_xor_sync(0xffffffffu, send.x, sbit, 16);
                recv.y = __shfl_xor_sync(0xffffffffu, send.y, sbit, 16);
                if (up) v[i] = recv;
                else v[ip] = recv;
            }
        });
    });
}

// ---------------------------------------------------------------------------
// exchange helpers with an explicit layout: element (k1, j) at k1*RS + j*ES
template <typename T, int N1, int N2, int RS, int ES>
__device__ __forceinline__ void xscatter(const cplx<T> (&v)[N1], cplx<T>* sc, int j) {
    static_for<0, N1>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        sc[k1 * RS + j * ES] = v[k1];
    });
}

template <typename T, int S, int N1, int N2, int RS, int ES>
__device__ __forceinline__ void xgather_fwd(cplx<T> (&v)[N1], const cplx<T>* sc, int t) {
    static_for<0, N1 / N2>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        cplx<T> w[N2];
        const cplx<T>* row = sc + (t + N2 * q) * RS;
        static_for<0, N2>([&](auto jc) { w[decltype(jc)::value] = row[decltype(jc)::value * ES]; });
        reg_dft<T, S, N2>(w);
        static_for<0, N2>([&](auto kc) { v[q * N2 + decltype(kc)::value] = w[decltype(kc)::value]; });
    });
}

template <typename T, int S, int N1, int N2, int RS, int ES>
__device__ __forceinline__ void xscatter_inv(cplx<T> (&v)[N1], cplx<T>* sc, int t,
                                             const cplx<T>* __restrict__ tw) {
    static_for<0, N1 / N2>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        cplx<T> w[N2];
        static_for<0, N2>([&](auto kc) { w[decltype(kc)::value] = v[q * N2 + decltype(kc)::value]; });
        reg_dft<T, S, N2>(w);
        const int k1 = t + N2 * q;
        cplx<T>* row = sc + k1 * RS;
        static_for<0, N2>([&](auto nc) {
            constexpr int n2 = decltype(nc)::value;
            row[n2 * ES] = (n2 == 0) ? w[n2] : (k1 == 0 ? w[n2] : cmul(w[n2], twiddle<T, S>(tw, n2 * k1, N1 * N2)));
        });
    });
}

template <typename T, int S, int N1, int N2, int RS, int ES>
__device__ __forceinline__ void xgather_inv(cplx<T> (&v)[N1], const cplx<T>* sc, int j) {
    static_for<0, N1>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        v[k1] = sc[k1 * RS + j * ES];
    });
    reg_dft<T, S, N1>(v);
}

// ---------------------------------------------------------------------------
// Per mode (kx, ky, kz) with C' = cos(c|k|dt)/Ntot, S' = sin(c|k|dt)/Ntot and
// n = k/|k| (0 at k = 0):  E <- C'(E - n(n.E)) + i S' n x B,  B <- C' B - i S' n x E.
template <typename T>
__device__ __forceinline__ void rotate_mode(cplx<T>& Ex, cplx<T>& Ey, cplx<T>& Ez, cplx<T>& Bx,
                                            cplx<T>& By, cplx<T>& Bz, T nx, T ny, T nz, T C, T S,
                                            bool project_b = false) {
    if (project_b) {
        const T kBr = nx * Bx.x + ny * By.x + nz * Bz.x, kBi = nx * Bx.y + ny * By.y + nz * Bz.y;
        Bx = mk<T>(Bx.x - nx * kBr, Bx.y - nx * kBi);
        By = mk<T>(By.x - ny * kBr, By.y - ny * kBi);
        Bz = mk<T>(Bz.x - nz * kBr, Bz.y - nz * kBi);
    }
    const T kEr = nx * Ex.x + ny * Ey.x + nz * Ez.x, kEi = nx * Ex.y + ny * Ey.y + nz * Ez.y;
    const T cBxr = ny * Bz.x - nz * By.x, cBxi = ny * Bz.y - nz * By.y;
    const T cByr = nz * Bx.x - nx * Bz.x, cByi = nz * Bx.y - nx * Bz.y;
    const T cBzr = nx * By.x - ny * Bx.x, cBzi = nx * By.y - ny * Bx.y;
    const T cExr = ny * Ez.x - nz * Ey.x, cExi = ny * Ez.y - nz * Ey.y;
    const T cEyr = nz * Ex.x - nx * Ez.x, cEyi = nz * Ex.y - nx * Ez.y;
    const T cEzr = nx * Ey.x - ny * Ex.x, cEzi = nx * Ey.y - ny * Ex.y;
    const cplx<T> nEx = mk<T>(C * (Ex.x - nx * kEr) - S * cBxi, C * (Ex.y - nx * kEi) + S * cBxr);
    const cplx<T> nEy = mk<T>(C * (Ey.x - ny * kEr) - S * cByi, C * (Ey.y - ny * kEi) + S * cByr);
    const cplx<T> nEz = mk<T>(C * (Ez.x - nz * kEr) - S * cBzi, C * (Ez.y - nz * kEi) + S * cBzr);
    Bx = mk<T>(C * Bx.x + S * cExi, C * Bx.y - S * cExr);
    By = mk<T>(C * By.x + S * cEyi, C * By.y - S * cEyr);
    Bz = mk<T>(C * Bz.x + S * cEzi, C * Bz.y - S * cEzr);
    Ex = nEx; Ey = nEy; Ez = nEz;
}

// Real fields: the transverse projection of B that keeps the field real, on a
// Nyquist plane the mean of the projections along n and along m (n with its
// Nyquist components negated): B <- B - (n(n.B) + m(m.B))/2; off the Nyquist
// planes m = n and this is B - n(n.B).
template <typename T>
__device__ __forceinline__ void project_b_mean(cplx<T>& Bx, cplx<T>& By, cplx<T>& Bz, T nx, T ny, T nz, bool fx,
                                               bool fy, bool fz) {
    const T mx = fx ? -nx : nx, my = fy ? -ny : ny, mz = fz ? -nz : nz;
    const T nBr = nx * Bx.x + ny * By.x + nz * Bz.x, nBi = nx * Bx.y + ny * By.y + nz * Bz.y;
    const T mBr = mx * Bx.x + my * By.x + mz * Bz.x, mBi = mx * Bx.y + my * By.y + mz * Bz.y;
    const T h = T(0.5);
    Bx = mk<T>(Bx.x - h * (nx * nBr + mx * mBr), Bx.y - h * (nx * nBi + mx * mBi));
    By = mk<T>(By.x - h * (ny * nBr + my * mBr), By.y - h * (ny * nBi + my * mBi));
    Bz = mk<T>(Bz.x - h * (nz * nBr + mz * mBr), Bz.y - h * (nz * nBi + mz * mBi));
}

// Real fields: on a Nyquist plane the wave number -pi/d is its own mirror, so the
// update that keeps the field real is the mean of the update at n and at m = n
// with the Nyquist components (flags fx, fy, fz) negated:
//   E <- C'(E - (n(n.E) + m(m.E))/2) + i S' a x B,  B <- C' B - i S' a x E,
// with a = (n + m)/2 (the Nyquist components of n removed).  Off the Nyquist
// planes m = n and this is rotate_mode.
template <typename T>
__device__ __forceinline__ void rotate_mode_mean(cplx<T>& Ex, cplx<T>& Ey, cplx<T>& Ez, cplx<T>& Bx,
                                                 cplx<T>& By, cplx<T>& Bz, T nx, T ny, T nz, bool fx, bool fy,
                                                 bool fz, T C, T S) {
    if (!(fx || fy || fz)) {
        rotate_mode<T>(Ex, Ey, Ez, Bx, By, Bz, nx, ny, nz, C, S);
        return;
    }
    const T mx = fx ? -nx : nx, my = fy ? -ny : ny, mz = fz ? -nz : nz;
    const T ax = fx ? T(0) : nx, ay = fy ? T(0) : ny, az = fz ? T(0) : nz;
    const T nEr = nx * Ex.x + ny * Ey.x + nz * Ez.x, nEi = nx * Ex.y + ny * Ey.y + nz * Ez.y;
    const T mEr = mx * Ex.x + my * Ey.x + mz * Ez.x, mEi = mx * Ex.y + my * Ey.y + mz * Ez.y;
    const T h = T(0.5);
    const T cBxr = ay * Bz.x - az * By.x, cBxi = ay * Bz.y - az * By.y;
    const T cByr = az * Bx.x - ax * Bz.x, cByi = az * Bx.y - ax * Bz.y;
    const T cBzr = ax * By.x - ay * Bx.x, cBzi = ax * By.y - ay * Bx.y;
    const T cExr = ay * Ez.x - az * Ey.x, cExi = ay * Ez.y - az * Ey.y;
    const T cEyr = az * Ex.x - ax * Ez.x, cEyi = az * Ex.y - ax * Ez.y;
    const T cEzr = ax * Ey.x - ay * Ex.x, cEzi = ax * Ey.y - ay * Ex.y;
    const cplx<T> nEx = mk<T>(C * (Ex.x - h * (nx * nEr + mx * mEr)) - S * cBxi,
                              C * (Ex.y - h * (nx * nEi + mx * mEi)) + S * cBxr);
    const cplx<T> nEy = mk<T>(C * (Ey.x - h * (ny * nEr + my * mEr)) - S * cByi,
                              C * (Ey.y - h * (ny * nEi + my * mEi)) + S * cByr);
    const cplx<T> nEz = mk<T>(C * (Ez.x - h * (nz * nEr + mz * mEr)) - S * cBzi,
                              C * (Ez.y - h * (nz * nEi + mz * mEi)) + S * cBzr);
    Bx = mk<T>(C * Bx.x + S * cExi, C * Bx.y - S * cExr);
    By = mk<T>(C * By.x + S * cEyi, C * By.y - S * cEyr);
    Bz = mk<T>(C * Bz.x + S * cEzi, C * Bz.y - S * cEzr);
    Ex = nEx; Ey = nEy; Ez = nEz;
}

}  // namespace psatd
