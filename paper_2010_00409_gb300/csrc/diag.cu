// Diagnostics: field energy sum |E|^2 + |B|^2 over the cells, and the spectral
// divergence max_k |k^ . F(k)| of an already-transformed 3-component field
// (Poisson's equation k^ . E^ = 0 is the constraint of Sec. 2.1).  Block
// partials are written to a scratch array and reduced by one block in a fixed
// order, so results are deterministic.  Per-cell and per-mode values are formed
// in the storage precision (float32 storage: float32 arithmetic, relative error
// ~1e-7, far below the float32 solver's own); sums over cells are float64.
#include "common.cuh"

namespace psatd {

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
    return r;
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
    return r;
}

// partial[b][0] = sum |E|^2, partial[b][1] = sum |B|^2 over this block's cells
template <typename T>
__global__ void __launch_bounds__(kThreads)
energy_kernel(const cplx<T>* __restrict__ f, size_t n, double* __restrict__ partial) {
    __shared__ double sh[kThreads / 32];
    double eE = 0.0, eB = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const GBuf<const cplx<T>> F{f, 6LL * (long long)n};
        eE += cell_energy3<T>(F[i], F[n + i], F[2 * n + i]);
        eB += cell_energy3<T>(F[3 * n + i], F[4 * n + i], F[5 * n + i]);
    }
    const double sE = block_sum(eE, sh);
    const double sB = block_sum(eB, sh);
    const GBuf<double> Pt{partial, 2LL * gridDim.x};
    if (threadIdx.x == 0) { Pt[2 * blockIdx.x] = sE; Pt[2 * blockIdx.x + 1] = sB; }
}

// partial[b][0] = max |k^ . F|, partial[b][1] = max |F| over this block's modes
template <typename T>
__global__ void __launch_bounds__(kThreads)
divergence_kernel(const cplx<T>* __restrict__ F, GridGeom g, const T* __restrict__ kx,
                  const T* __restrict__ ky, const T* __restrict__ kz, double* __restrict__ partial) {
    __shared__ double sh[kThreads / 32];
    const size_t n = (size_t)g.Nx * g.Ny * g.Nz;
    const int rows = g.Ny * g.Nz;
    T md2 = 0, mf2 = 0;                                // squared maxima
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int iy = row % g.Ny, iz = row / g.Ny;
        const T b = ky[PSATD_IX(iy, g.Ny)], c = kz[PSATD_IX(iz, g.Nz)];
        const size_t base = (size_t)row * g.Nx;
        for (int ix = threadIdx.x; ix < g.Nx; ix += blockDim.x) {
            const T a = kx[PSATD_IX(ix, g.Nx)];
            const T k2 = a * a + b * b + c * c;
            const size_t i = base + ix;
            const GBuf<const cplx<T>> S3{F, 3LL * (long long)n};
            const cplx<T> X = S3[i], Y = S3[n + i], Z = S3[2 * n + i];
            const T dr = a * X.x + b * Y.x + c * Z.x;
            const T di = a * X.y + b * Y.y + c * Z.y;
            if (k2 > T(0)) md2 = max(md2, (dr * dr + di * di) / k2);
            mf2 = max(mf2, (T)cell_energy3<T>(X, Y, Z));
        }
    }
    const double bd = block_max(sqrt((double)md2), sh);
    const double bf = block_max(sqrt((double)mf2), sh);
    const GBuf<double> Pt{partial, 2LL * gridDim.x};
    if (threadIdx.x == 0) { Pt[2 * blockIdx.x] = bd; Pt[2 * blockIdx.x + 1] = bf; }
}

// Real float32 storage [6][n]: partial[b][0] = sum E^2, partial[b][1] = sum B^2.
__global__ void __launch_bounds__(kThreads)
energy_real_kernel(const float* __restrict__ f, size_t n, double* __restrict__ partial) {
    __shared__ double sh[kThreads / 32];
    double eE = 0.0, eB = 0.0;
    const GBuf<const float> F{f, 6LL * (long long)n};
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        float a = F[i], b = F[n + i], c = F[2 * n + i];
        eE += (double)fmaf(c, c, fmaf(b, b, a * a));
        a = F[3 * n + i]; b = F[4 * n + i]; c = F[5 * n + i];
        eB += (double)fmaf(c, c, fmaf(b, b, a * a));
    }
    const double sE = block_sum(eE, sh);
    const double sB = block_sum(eB, sh);
    const GBuf<double> Pt{partial, 2LL * gridDim.x};
    if (threadIdx.x == 0) { Pt[2 * blockIdx.x] = sE; Pt[2 * blockIdx.x + 1] = sB; }
}

// The spectrum of three real components as the real-field plane kernels leave
// it: the half spectrum S [3][Nz][Ny][Nx/2] in slot order (slot p has wave
// number kxs[p]) and the x-Nyquist array Q [3][Nz][Ny] (wave number kx_nyq).
// The modes with negative k_x mirror the stored ones (F(-k) = conj F(k)), so
// the maxima over the stored modes are the maxima over the whole spectrum.
__global__ void __launch_bounds__(kThreads)
divergence_half_kernel(const float2* __restrict__ S, const float2* __restrict__ Q, GridGeom g,
                       const float* __restrict__ kxs, float kx_nyq, const float* __restrict__ ky,
                       const float* __restrict__ kz, double* __restrict__ partial) {
    __shared__ double sh[kThreads / 32];
    const int nh = g.Nx / 2, rows = g.Ny * g.Nz;
    const GBuf<const float2> SF{S, 3LL * rows * nh}, QF{Q, 3LL * rows};
    float md2 = 0.f, mf2 = 0.f;
    for (int row = blockIdx.x; row < rows; row += gridDim.x) {
        const int iy = row % g.Ny, iz = row / g.Ny;
        const float b = ky[PSATD_IX(iy, g.Ny)], c = kz[PSATD_IX(iz, g.Nz)];
        for (int p = threadIdx.x; p <= nh; p += blockDim.x) {
            const float a = p < nh ? kxs[PSATD_IX(p, nh)] : kx_nyq;
            float2 X, Y, Z;
            if (p < nh) {
                const size_t i = (size_t)row * nh + p, st = (size_t)rows * nh;
                X = SF[i]; Y = SF[st + i]; Z = SF[2 * st + i];
            } else {
                X = QF[row]; Y = QF[rows + row]; Z = QF[2 * rows + row];
            }
            const float k2 = a * a + b * b + c * c;
            const float dr = a * X.x + b * Y.x + c * Z.x;
            const float di = a * X.y + b * Y.y + c * Z.y;
            if (k2 > 0.f) md2 = fmaxf(md2, (dr * dr + di * di) / k2);
            mf2 = fmaxf(mf2, (float)cell_energy3<float>(X, Y, Z));
        }
    }
    const double bd = block_max(sqrt((double)md2), sh);
    const double bf = block_max(sqrt((double)mf2), sh);
    const GBuf<double> Pt{partial, 2LL * gridDim.x};
    if (threadIdx.x == 0) { Pt[2 * blockIdx.x] = bd; Pt[2 * blockIdx.x + 1] = bf; }
}

__global__ void reduce_final_kernel(const double* __restrict__ partial, int nblocks, int width, int nsum,
                                    double* __restrict__ out) {
    __shared__ double sh[kThreads / 32];
    for (int col = 0; col < width; ++col) {
        const bool is_sum = col < nsum;
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double x = partial[PSATD_IX((size_t)b * width + col, (long long)nblocks * width)];
            v = is_sum ? v + x : fmax(v, x);
        }
        const double r = is_sum ? block_sum(v, sh) : block_max(v, sh);
        if (threadIdx.x == 0) out[PSATD_IX(col, width)] = r;
        __syncthreads();
    }
}

}  // namespace

template <typename T>
cudaError_t launch_energy(const cplx<T>* data, size_t n_per_comp, double* partial, int nblocks,
                          cudaStream_t s, long long* nlaunch) {
    energy_kernel<T><<<nblocks, kThreads, 0, s>>>(data, n_per_comp, partial);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_divergence(const cplx<T>* spec3, const GridGeom& g, const Tables<T>& tb,
                              double* partial, int nblocks, cudaStream_t s, long long* nlaunch) {
    divergence_kernel<T><<<nblocks, kThreads, 0, s>>>(spec3, g, tb.k[0], tb.k[1], tb.k[2], partial);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_energy_real(const float* data, size_t n_per_comp, double* partial, int nblocks, cudaStream_t s,
                               long long* nlaunch) {
    energy_real_kernel<<<nblocks, kThreads, 0, s>>>(data, n_per_comp, partial);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_divergence_half(const float2* spec, const float2* nyq, const GridGeom& g, const float* slot_k,
                                   float kx_nyq, const Tables<float>& tb, double* partial, int nblocks,
                                   cudaStream_t s, long long* nlaunch) {
    divergence_half_kernel<<<nblocks, kThreads, 0, s>>>(spec, nyq, g, slot_k, kx_nyq, tb.k[1], tb.k[2], partial);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

cudaError_t launch_reduce_final(const double* partial, int nblocks, int width, int nsum, double* out,
                                cudaStream_t s, long long* nlaunch) {
    reduce_final_kernel<<<1, kThreads, 0, s>>>(partial, nblocks, width, nsum, out);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

template cudaError_t launch_energy<float>(const cplx<float>*, size_t, double*, int, cudaStream_t, long long*);
template cudaError_t launch_energy<double>(const cplx<double>*, size_t, double*, int, cudaStream_t, long long*);
template cudaError_t launch_divergence<float>(const cplx<float>*, const GridGeom&, const Tables<float>&, double*, int, cudaStream_t, long long*);
template cudaError_t launch_divergence<double>(const cplx<double>*, const GridGeom&, const Tables<double>&, double*, int, cudaStream_t, long long*);

}  // namespace psatd
