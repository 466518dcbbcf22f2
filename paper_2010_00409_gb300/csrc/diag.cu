// Diagnostics: field energy sum |E|^2 + |B|^2 over the cells, and the spectral
// divergence max_k |k^ . F(k)| of an already-transformed 3-component field
// (Poisson's equation k^ . E^ = 0 is the constraint of Sec. 2.1).  Block
// partials are written to a scratch array and reduced by one block in a fixed
// order, so results are deterministic; accumulation is float64.
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
        for (int c = 0; c < 3; ++c) {
            const cplx<T> v = f[c * n + i];
            eE += (double)v.x * v.x + (double)v.y * v.y;
            const cplx<T> w = f[(3 + c) * n + i];
            eB += (double)w.x * w.x + (double)w.y * w.y;
        }
    }
    const double sE = block_sum(eE, sh);
    const double sB = block_sum(eB, sh);
    if (threadIdx.x == 0) { partial[2 * blockIdx.x] = sE; partial[2 * blockIdx.x + 1] = sB; }
}

// partial[b][0] = max |k^ . F|, partial[b][1] = max |F| over this block's modes
template <typename T>
__global__ void __launch_bounds__(kThreads)
divergence_kernel(const cplx<T>* __restrict__ F, GridGeom g, const T* __restrict__ kx,
                  const T* __restrict__ ky, const T* __restrict__ kz, double* __restrict__ partial) {
    __shared__ double sh[kThreads / 32];
    const size_t n = (size_t)g.Nx * g.Ny * g.Nz;
    double md = 0.0, mf = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(i % g.Nx);
        const size_t r = i / g.Nx;
        const int iy = (int)(r % g.Ny), iz = (int)(r / g.Ny);
        const double a = kx[ix], b = ky[iy], c = kz[iz];
        const double km = sqrt(a * a + b * b + c * c);
        const double inv = km > 0.0 ? 1.0 / km : 0.0;
        const cplx<T> X = F[i], Y = F[n + i], Z = F[2 * n + i];
        const double dr = (a * X.x + b * Y.x + c * Z.x) * inv;
        const double di = (a * X.y + b * Y.y + c * Z.y) * inv;
        md = fmax(md, sqrt(dr * dr + di * di));
        mf = fmax(mf, sqrt((double)X.x * X.x + (double)X.y * X.y + (double)Y.x * Y.x +
                           (double)Y.y * Y.y + (double)Z.x * Z.x + (double)Z.y * Z.y));
    }
    const double bd = block_max(md, sh);
    const double bf = block_max(mf, sh);
    if (threadIdx.x == 0) { partial[2 * blockIdx.x] = bd; partial[2 * blockIdx.x + 1] = bf; }
}

__global__ void reduce_final_kernel(const double* __restrict__ partial, int nblocks, int width, int nsum,
                                    double* __restrict__ out) {
    __shared__ double sh[kThreads / 32];
    for (int col = 0; col < width; ++col) {
        const bool is_sum = col < nsum;
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
            const double x = partial[(size_t)b * width + col];
            v = is_sum ? v + x : fmax(v, x);
        }
        const double r = is_sum ? block_sum(v, sh) : block_max(v, sh);
        if (threadIdx.x == 0) out[col] = r;
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
