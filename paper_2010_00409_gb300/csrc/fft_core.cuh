// Device FFT building blocks: radix-2/3/4/5/8 butterflies and a Stockham
// (self-sorting) pass over a tile of pencils held in shared memory.
//
// Sign convention: S = -1 is the forward transform (kernel exp(-2 pi i nk/N)),
// S = +1 the inverse; neither is normalised.
//
// Stockham decimation-in-time, mixed radix: after the passes with radices
// R_1..R_{p-1} (product Ns), pass p with radix R reads element j + r*N/R of the
// input (r < R, j < N/R), multiplies it by exp(S 2 pi i r (j mod Ns)/(Ns R)),
// applies the R-point DFT and writes the outputs to
// (j div Ns)*Ns*R + (j mod Ns) + r*Ns.  After the last pass the data are in
// natural order.
#pragma once

#include "common.cuh"

namespace psatd {

// Complex sum and difference of butterfly operands.  float32 pairs on the GPU
// use the packed two-lane adds of sm_100-class SMs (add/sub.rn.f32x2: one
// instruction per complex add, the same round-to-nearest result as two scalar
// adds); double pairs and host code use cadd / csub.
template <typename V> __host__ __device__ __forceinline__ V badd(V a, V b) { return cadd(a, b); }
template <typename V> __host__ __device__ __forceinline__ V bsub(V a, V b) { return csub(a, b); }
__host__ __device__ __forceinline__ float2 badd(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    float2 r;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
#else
    return cadd(a, b);
#endif
}
__host__ __device__ __forceinline__ float2 bsub(float2 a, float2 b) {
#ifdef __CUDA_ARCH__
    float2 r;
    asm("{.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;}"
        : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
#else
    return csub(a, b);
#endif
}

// t + S i u and t - S i u in scalar form: the lane swap of i u does not pack.
template <typename V, int S>
__host__ __device__ __forceinline__ void add_sub_si(const V& t, const V& u, V& plus, V& minus) {
    if constexpr (S > 0) {
        plus.x = t.x - u.y; plus.y = t.y + u.x;
        minus.x = t.x + u.y; minus.y = t.y - u.x;
    } else {
        plus.x = t.x + u.y; plus.y = t.y - u.x;
        minus.x = t.x - u.y; minus.y = t.y + u.x;
    }
}

template <typename V, int S>
__host__ __device__ __forceinline__ void bfly2(V& a0, V& a1) {
    V t = a0; a0 = badd(t, a1); a1 = bsub(t, a1);
}

template <typename V, int S>
__host__ __device__ __forceinline__ void bfly4(V& a0, V& a1, V& a2, V& a3) {
    V t0 = badd(a0, a2), t1 = bsub(a0, a2), t2 = badd(a1, a3), u = bsub(a1, a3);
    a0 = badd(t0, t2); a2 = bsub(t0, t2);
    add_sub_si<V, S>(t1, u, a1, a3);                 // t1 +- S i (a1 - a3)
}

// x / sqrt 2.  In float32 the rounded 1/sqrt 2 makes |(1 + i)/sqrt 2|^2 =
// 1 - 3.4e-8, an energy loss that every 45-degree rotation of every transform
// would repeat each step; the product is therefore formed with the rounding
// residue of 1/sqrt 2 added in (one more multiply), which leaves only the
// unbiased rounding of the result.
template <typename T> __host__ __device__ __forceinline__ T mul_rsqrt2(T x) {
    if constexpr (sizeof(T) == 4) {
        constexpr float hi = (float)0.70710678118654752440;
        constexpr float lo = (float)(0.70710678118654752440 - (double)hi);
        return fmaf(x, hi, x * lo);
    } else {
        return x * (T)0.70710678118654752440;
    }
}

template <typename T, int S>
__host__ __device__ __forceinline__ void bfly8(cplx<T>* v) {
    // even / odd 4-point DFTs, then combine with exp(S 2 pi i k / 8)
    bfly4<cplx<T>, S>(v[0], v[2], v[4], v[6]);
    bfly4<cplx<T>, S>(v[1], v[3], v[5], v[7]);
    cplx<T> o1 = v[3], o2 = v[5], o3 = v[7];
    // W^1 = (1 + S i)/sqrt2
    cplx<T> w1 = mk<T>(mul_rsqrt2<T>(o1.x - S * o1.y), mul_rsqrt2<T>(o1.y + S * o1.x));
    // W^3 = (-1 + S i)/sqrt2
    cplx<T> w3 = mk<T>(-mul_rsqrt2<T>(o3.x + S * o3.y), mul_rsqrt2<T>(S * o3.x - o3.y));
    cplx<T> e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = badd(e0, o0); v[4] = bsub(e0, o0);
    v[1] = badd(e1, w1); v[5] = bsub(e1, w1);
    add_sub_si<cplx<T>, S>(e2, o2, v[2], v[6]);     // W^2 = S i
    v[3] = badd(e3, w3); v[7] = bsub(e3, w3);
}

template <typename T, int S>
__host__ __device__ __forceinline__ void bfly3(cplx<T>& a0, cplx<T>& a1, cplx<T>& a2) {
    const T h = (T)0.86602540378443864676;   // sin(2 pi / 3)
    cplx<T> t = cadd(a1, a2), u = csub(a1, a2);
    cplx<T> m = mk<T>(a0.x - (T)0.5 * t.x, a0.y - (T)0.5 * t.y);
    cplx<T> v = cmul_si(cscale(u, h), S);
    a0 = cadd(a0, t);
    a1 = cadd(m, v);
    a2 = csub(m, v);
}

template <typename T, int S>
__host__ __device__ __forceinline__ void bfly5(cplx<T>* a) {
    const T c1 = (T)0.30901699437494742410;    // cos(2 pi / 5)
    const T c2 = (T)-0.80901699437494742410;   // cos(4 pi / 5)
    const T s1 = (T)0.95105651629515357212;    // sin(2 pi / 5)
    const T s2 = (T)0.58778525229247312917;    // sin(4 pi / 5)
    cplx<T> t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
    cplx<T> u1 = csub(a[1], a[4]), u2 = csub(a[2], a[3]);
    cplx<T> a0 = a[0];
    cplx<T> p1 = mk<T>(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
    cplx<T> p2 = mk<T>(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
    cplx<T> q1 = cmul_si(mk<T>(s1 * u1.x + s2 * u2.x, s1 * u1.y + s2 * u2.y), S);
    cplx<T> q2 = cmul_si(mk<T>(s2 * u1.x - s1 * u2.x, s2 * u1.y - s1 * u2.y), S);
    a[0] = cadd(a0, cadd(t1, t2));
    a[1] = cadd(p1, q1);
    a[4] = csub(p1, q1);
    a[2] = cadd(p2, q2);
    a[3] = csub(p2, q2);
}

template <typename T, int R, int S>
__host__ __device__ __forceinline__ void dft_r(cplx<T>* v) {
    if constexpr (R == 2) bfly2<cplx<T>, S>(v[0], v[1]);
    else if constexpr (R == 3) bfly3<T, S>(v[0], v[1], v[2]);
    else if constexpr (R == 4) bfly4<cplx<T>, S>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) bfly5<T, S>(v);
    else if constexpr (R == 8) bfly8<T, S>(v);
}

// Shared-memory layout of a tile of W pencils: element i of pencil w sits at
// w * P + pad32(i), pad32(i) = i + i / 32.  The one unused slot per 32 elements
// spreads the stride-R stores of the early Stockham passes (R consecutive
// outputs per thread) over the banks, and the pencil stride P (odd, at least
// pad32(N - 1) + 1) keeps the row-by-row tile loads of strided axes on
// distinct banks.
__host__ __device__ __forceinline__ int pad32(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ int pencil_stride(int N) { return (N + ((N - 1) >> 5)) | 1; }

// Division by a per-pass constant d as a multiply-high: q = umulhi(n, m) with
// m = ceil(2^32 / d) equals n / d for 0 <= n < 2^16 and 1 <= d < 2^16 (the
// error term n (m - 2^32/d) / 2^32 < 2^-16 stays below the gap 1/d to the next
// integer); d = 1 is taken apart.  For d >= 2, ceil(2^32 / d) = (2^32 - 1) / d
// + 1 (a 32-bit division, once per pass).
struct FastDiv {
    unsigned m;
    int d;
};
__host__ __device__ __forceinline__ FastDiv fast_div(int d) {
    FastDiv f;
    f.d = d;
    f.m = d <= 1 ? 0u : 0xFFFFFFFFu / (unsigned)d + 1u;
    return f;
}
#ifdef __CUDACC__
__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
    return f.d <= 1 ? n : (int)__umulhi((unsigned)n, f.m);
}

// One Stockham pass over `W` pencils of length N (layout above) in `in`,
// written to `out`.  Work items b = tid, tid + nthr, ... < W*N/R (fewer than
// 2^16).  tw[t] = exp(-2 pi i t / N); the inverse uses its conjugate.
template <typename T, int R, int S>
__device__ __forceinline__ void stockham_pass(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, int N,
                                              int Ns, int W, int P, const cplx<T>* __restrict__ tw, int tid,
                                              int nthr) {
    const int nb = N / R;
    const int tstride = N / (Ns * R);
    const FastDiv dnb = fast_div(nb), dns = fast_div(Ns);
    for (int b = tid; b < W * nb; b += nthr) {
        const int w = fdiv(b, dnb);
        const int j = b - w * nb;
        const cplx<T>* src = in + (size_t)w * P;
        cplx<T>* dst = out + (size_t)w * P;
        cplx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[pad32(j + r * nb)];
        const int jq = fdiv(j, dns);
        const int k = j - jq * Ns;
        if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const cplx<T> wv = tw[PSATD_IX((r * k) * tstride, N)];
                v[r] = (S < 0) ? cmul(v[r], wv) : cmulc(v[r], wv);
            }
        }
        dft_r<T, R, S>(v);
        const int idx = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[pad32(idx + r * Ns)] = v[r];
    }
}

template <typename T, int S>
__device__ __forceinline__ void stockham_dispatch(int R, const cplx<T>* in, cplx<T>* out, int N, int Ns, int W,
                                                  int P, const cplx<T>* tw, int tid, int nthr) {
    switch (R) {
        case 2: stockham_pass<T, 2, S>(in, out, N, Ns, W, P, tw, tid, nthr); break;
        case 3: stockham_pass<T, 3, S>(in, out, N, Ns, W, P, tw, tid, nthr); break;
        case 4: stockham_pass<T, 4, S>(in, out, N, Ns, W, P, tw, tid, nthr); break;
        case 5: stockham_pass<T, 5, S>(in, out, N, Ns, W, P, tw, tid, nthr); break;
        default: stockham_pass<T, 8, S>(in, out, N, Ns, W, P, tw, tid, nthr); break;
    }
}
#endif

#ifdef __CUDACC__
// Full transform of a shared-memory tile, ping-ponging between a and b.
// Returns the buffer that holds the result.  Must be called by the whole block.
template <typename T, int S>
__device__ __forceinline__ cplx<T>* fft_tile(cplx<T>* a, cplx<T>* b, const AxisPlan& pl, int W,
                                             int P, const cplx<T>* tw) {
    int Ns = 1;
    for (int p = 0; p < pl.npass; ++p) {
        const int R = pl.radix[p];
        stockham_dispatch<T, S>(R, a, b, pl.N, Ns, W, P, tw, threadIdx.x, blockDim.x);
        __syncthreads();
        cplx<T>* t = a; a = b; b = t;
        Ns *= R;
    }
    return a;
}
#endif

}  // namespace psatd
