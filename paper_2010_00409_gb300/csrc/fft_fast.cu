// Fast FFT kernels for axis lengths N = N1 * N2 with a register plan
// (see fft_reg.cuh): each pencil lives in the registers of N2 threads, goes
// through one shared-memory exchange per transform, and is loaded and stored
// straight from/to global memory with coalesced accesses.
//
//  fft_rows_kernel     x axis: one row per group of N2 threads.
//  fft_cols_kernel     y or z axis: W consecutive x-columns x N2 threads.
//  kspace_cols_kernel  the fused k-space pass of one PSATD step (Sec. 2.1,
//                      Eq. 3-4): forward z transform of all six components of
//                      W columns, the per-mode update in registers, inverse z
//                      transform, one read and one write of the field.
#include "fft_reg.cuh"

namespace psatd {

namespace {

// --------------------------------------------------------------------------- x
// S = -1: natural order in (input layout), natural order out (spectral layout).
// S = +1: the mirror.  Both unnormalised.
// groups of N2 threads per block for the row kernel: at most 256 threads and
// 48 KB of static shared memory
template <typename T, int N1, int N2> struct RowsCfg {
    static constexpr int by_threads = 256 / N2;
    static constexpr int by_smem = (48 * 1024) / (N1 * (N2 + 1) * (int)sizeof(cplx<T>));
    static constexpr int G = by_threads < by_smem ? by_threads : by_smem;
    static constexpr int threads = G * N2;
};

// columns per block for the strided kernel: 128 contiguous bytes per row of the
// tile, halved until the exchange buffer fits the shared-memory budget.  Along
// z, whose rows lie a whole plane apart, 128 KB (at 1024^2 planes, 32-byte runs
// 8 MB apart used the DRAM bursts poorly: the z transforms took 2.3 times as
// long as with 128-byte runs, and 64-byte runs at two blocks per SM 1.16
// times).  Along y (rows one plane row apart) 48 KB, or 64 KB for 1024-point
// columns: eight columns, 256 threads held to 128 registers so that two blocks
// share an SM (at 1024^3, 47.1 against 51.4 ms per step in one process for four
// columns at 166 registers, three blocks per SM).
#ifndef PSATD_COLS_Y_BUDGET
#define PSATD_COLS_Y_BUDGET (48 * 1024)
#endif
template <typename T, int N, bool ZAXIS> constexpr int cols_width() {
    const int budget = ZAXIS ? 128 * 1024 : (N >= 1024 ? 64 * 1024 : PSATD_COLS_Y_BUDGET);
    int w = 128 / (int)sizeof(cplx<T>);
    while (w > 1 && N * w * (int)sizeof(cplx<T>) > budget) w /= 2;
    return w;
}
// 1024-point columns: blocks per SM for the launch bounds, so that 512 threads
// share the register file (at most 128 registers a thread)
template <int N, int THREADS> constexpr int cols_min_blocks() {
    return (N >= 1024 && THREADS < 512) ? 512 / THREADS : 1;
}

template <typename T, int N1, int N2, int S>
__global__ void __launch_bounds__(RowsCfg<T, N1, N2>::threads)
fft_rows_kernel(cplx<T>* __restrict__ data, long long rows, const cplx<T>* __restrict__ tw) {
    constexpr int N = N1 * N2;
    constexpr int G = RowsCfg<T, N1, N2>::G;
    constexpr int RS = N2 + 1;
    __shared__ cplx<T> scratch[G * N1 * RS];
    const int g = threadIdx.x / N2, j = threadIdx.x % N2;
    const long long row = (long long)blockIdx.x * G + g;
    if (row >= rows) return;          // whole groups exit together; groups never straddle warps
    // barrier mask of this group's N2 lanes only (other groups of the warp may have exited)
    const unsigned lane0 = (threadIdx.x & 31u) & ~(unsigned)(N2 - 1);
    const unsigned gmask = N2 >= 32 ? 0xffffffffu : (((1u << N2) - 1u) << lane0);
    cplx<T>* p = data + row * N;
    const GBuf<cplx<T>> F{data, rows * N};
    cplx<T>* sc = scratch + g * N1 * RS;
    cplx<T> v[N1];
    if constexpr (S < 0) {
        static_for<0, N1>([&](auto nc) { v[decltype(nc)::value] = F.at(p, j + N2 * decltype(nc)::value); });
        stage_a_fwd<T, S, N1, N2>(v, j, tw);
        xscatter<T, N1, N2, RS, 1>(v, sc, j);
        __syncwarp(gmask);
        xgather_fwd<T, S, N1, N2, RS, 1>(v, sc, j);
        static_for<0, N1 / N2>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            static_for<0, N2>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                F.at(p, (j + N2 * q) + N1 * k2) = v[q * N2 + k2];
            });
        });
    } else {
        static_for<0, N1 / N2>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            static_for<0, N2>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                v[q * N2 + k2] = F.at(p, (j + N2 * q) + N1 * k2);
            });
        });
        xscatter_inv<T, S, N1, N2, RS, 1>(v, sc, j, tw);
        __syncwarp(gmask);
        xgather_inv<T, S, N1, N2, RS, 1>(v, sc, j);
        static_for<0, N1>([&](auto nc) { F.at(p, j + N2 * decltype(nc)::value) = v[decltype(nc)::value]; });
    }
}

// --------------------------------------------------------------------------- y / z
// Block = W columns x N2 threads (c fastest).  Tile g -> (comp, o, x-tile);
// element n of column c at base + n*stride + c.
template <typename T, int N1, int N2, int W, int S>
__global__ void __launch_bounds__(W * N2, cols_min_blocks<N1 * N2, W * N2>())
fft_cols_kernel(cplx<T>* __restrict__ data, int Nx, int Ny, int Nz, int axis, const cplx<T>* __restrict__ tw) {
    constexpr int RS = N2 * W, ES = W;
    extern __shared__ __align__(16) unsigned char cols_smem[];
    cplx<T>* scratch = reinterpret_cast<cplx<T>*>(cols_smem);     // [N1 * N2 * W]
    const int c = threadIdx.x % W, j = threadIdx.x / W;
    const size_t plane = (size_t)Nx * Ny;
    const int ntile = Nx / W;
    const int outerN = axis == 1 ? Nz : Ny;
    const int t = blockIdx.x % ntile;
    const long long rest = blockIdx.x / ntile;
    const int o = (int)(rest % outerN);
    const int comp = (int)(rest / outerN);
    const size_t stride = axis == 1 ? (size_t)Nx : plane;
    cplx<T>* base = data + (size_t)comp * plane * Nz + (axis == 1 ? (size_t)o * plane : (size_t)o * Nx) + (size_t)t * W + c;
    const GBuf<cplx<T>> F{data, (long long)(gridDim.x / (ntile * outerN)) * plane * Nz};
    cplx<T>* sc = scratch + c;
    cplx<T> v[N1];
    if constexpr (S < 0) {
        static_for<0, N1>([&](auto nc) { v[decltype(nc)::value] = F.at(base, (long long)(j + N2 * decltype(nc)::value) * stride); });
        stage_a_fwd<T, S, N1, N2>(v, j, tw);
        xscatter<T, N1, N2, RS, ES>(v, sc, j);
        __syncthreads();
        xgather_fwd<T, S, N1, N2, RS, ES>(v, sc, j);
        static_for<0, N1 / N2>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            static_for<0, N2>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                F.at(base, (long long)((j + N2 * q) + N1 * k2) * stride) = v[q * N2 + k2];
            });
        });
    } else {
        static_for<0, N1 / N2>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            static_for<0, N2>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                v[q * N2 + k2] = F.at(base, (long long)((j + N2 * q) + N1 * k2) * stride);
            });
        });
        xscatter_inv<T, S, N1, N2, RS, ES>(v, sc, j, tw);
        __syncthreads();
        xgather_inv<T, S, N1, N2, RS, ES>(v, sc, j);
        static_for<0, N1>([&](auto nc) { F.at(base, (long long)(j + N2 * decltype(nc)::value) * stride) = v[decltype(nc)::value]; });
    }
}

// --------------------------------------------------------------------------- k-space
// Block = W columns x N2 threads at one y; the six spectra of the W z-pencils are
// kept in shared memory, slot q in natural kz order (element (kz, c) at
// kz*W + c).  During each transform the slot of that component doubles as its
// exchange buffer, so the block needs 6 * Nz * W complex values in total.
template <typename T, int N1, int N2, int W>
__global__ void __launch_bounds__(W * N2)
kspace_cols_kernel(cplx<T>* __restrict__ data, int Nx, int Ny, const cplx<T>* __restrict__ tw,
                   const T* __restrict__ kxs, const T* __restrict__ kys, const T* __restrict__ kzs,
                   const ModeCoef<T>* __restrict__ coef) {
    constexpr int Nz = N1 * N2;
    constexpr int RS = N2 * W, ES = W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* spec = reinterpret_cast<cplx<T>*>(smem_raw);      // [6][Nz][W]
    const int c = threadIdx.x % W, j = threadIdx.x / W;
    const size_t plane = (size_t)Nx * Ny;
    const size_t cstride = plane * Nz;
    const int ntile = Nx / W;
    const int xt = blockIdx.x % ntile;
    const int y = blockIdx.x / ntile;
    const int ix = xt * W + c;
    cplx<T>* base = data + (size_t)y * Nx + ix;
    const GBuf<cplx<T>> F{data, 6LL * (long long)cstride};
    cplx<T> v[N1];

    // forward z transforms: spectrum of component q -> slot q
    for (int q = 0; q < 6; ++q) {
        cplx<T>* p = base + q * cstride;
        cplx<T>* sl = spec + q * (Nz * W) + c;
        static_for<0, N1>([&](auto nc) { v[decltype(nc)::value] = F.at(p, (long long)(j + N2 * decltype(nc)::value) * plane); });
        stage_a_fwd<T, -1, N1, N2>(v, j, tw);
        xscatter<T, N1, N2, RS, ES>(v, sl, j);
        __syncthreads();
        xgather_fwd<T, -1, N1, N2, RS, ES>(v, sl, j);
        __syncthreads();
        static_for<0, N1 / N2>([&](auto qc) {
            constexpr int qq = decltype(qc)::value;
            static_for<0, N2>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                sl[((j + N2 * qq) + N1 * k2) * W] = v[qq * N2 + k2];
            });
        });
    }
    __syncthreads();

    // per-mode update; thread (c, j) takes modes kz = j + N2 s, s < N1
    {
        const int Nxh = Nx / 2 + 1, Nyh = Ny / 2 + 1;
        const int ax = min(ix, Nx - ix), ay = min(y, Ny - y);
        const T kx = kxs[PSATD_IX(ix, Nx)], ky = kys[PSATD_IX(y, Ny)];
        const long long ncoef = (long long)(Nz / 2 + 1) * Nyh * Nxh;
        cplx<T>* sl = spec + c;
#pragma unroll 4
        for (int s = 0; s < N1; ++s) {
            const int iz = j + N2 * s;
            const int az = min(iz, Nz - iz);
            const ModeCoef<T> m = coef[PSATD_IX(((size_t)az * Nyh + ay) * Nxh + ax, ncoef)];
            const int o = iz * W;
            cplx<T> Ex = sl[o], Ey = sl[Nz * W + o], Ez = sl[2 * Nz * W + o];
            cplx<T> Bx = sl[3 * Nz * W + o], By = sl[4 * Nz * W + o], Bz = sl[5 * Nz * W + o];
            rotate_mode<T>(Ex, Ey, Ez, Bx, By, Bz, kx * m.kinv, ky * m.kinv, kzs[PSATD_IX(iz, Nz)] * m.kinv, m.C, m.S);
            sl[o] = Ex; sl[Nz * W + o] = Ey; sl[2 * Nz * W + o] = Ez;
            sl[3 * Nz * W + o] = Bx; sl[4 * Nz * W + o] = By; sl[5 * Nz * W + o] = Bz;
        }
    }
    __syncthreads();

    // inverse z transforms back to the field
    for (int q = 0; q < 6; ++q) {
        cplx<T>* sl = spec + q * (Nz * W) + c;
        static_for<0, N1 / N2>([&](auto qc) {
            constexpr int qq = decltype(qc)::value;
            static_for<0, N2>([&](auto kc) {
                constexpr int k2 = decltype(kc)::value;
                v[qq * N2 + k2] = sl[((j + N2 * qq) + N1 * k2) * W];
            });
        });
        __syncthreads();
        xscatter_inv<T, +1, N1, N2, RS, ES>(v, sl, j, tw);
        __syncthreads();
        xgather_inv<T, +1, N1, N2, RS, ES>(v, sl, j);
        cplx<T>* p = base + q * cstride;
        static_for<0, N1>([&](auto nc) { F.at(p, (long long)(j + N2 * decltype(nc)::value) * plane) = v[decltype(nc)::value]; });
    }
}

template <typename T, int N1, int N2, int W>
cudaError_t cols_launch(cplx<T>* data, int ncomp, const GridGeom& g, const cplx<T>* tw, int axis, int dir,
                        cudaStream_t s) {
    if (g.Nx % W != 0) return cudaErrorNotSupported;
    const long long blocks = (long long)ncomp * (axis == 1 ? g.Nz : g.Ny) * (g.Nx / W);
    const size_t smem = (size_t)N1 * N2 * W * sizeof(cplx<T>);
    auto k = dir < 0 ? fft_cols_kernel<T, N1, N2, W, -1> : fft_cols_kernel<T, N1, N2, W, +1>;
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)blocks, W * N2, smem, s>>>(data, g.Nx, g.Ny, g.Nz, axis, tw);
    return cudaGetLastError();
}

template <typename T, int N1, int N2>
cudaError_t axis_fast(cplx<T>* data, int ncomp, const GridGeom& g, const cplx<T>* tw, int axis, int dir,
                      cudaStream_t s) {
    constexpr int N = N1 * N2;
    if (axis == 0) {
        const long long rows = (long long)ncomp * g.Nz * g.Ny;
        using Cfg = RowsCfg<T, N1, N2>;
        const unsigned blocks = (unsigned)((rows + Cfg::G - 1) / Cfg::G);
        if (dir < 0) fft_rows_kernel<T, N1, N2, -1><<<blocks, Cfg::threads, 0, s>>>(data, rows, tw);
        else fft_rows_kernel<T, N1, N2, +1><<<blocks, Cfg::threads, 0, s>>>(data, rows, tw);
        return cudaGetLastError();
    }
    return axis == 2 ? cols_launch<T, N1, N2, cols_width<T, N, true>()>(data, ncomp, g, tw, axis, dir, s)
                     : cols_launch<T, N1, N2, cols_width<T, N, false>()>(data, ncomp, g, tw, axis, dir, s);
}

}  // namespace

// Returns cudaErrorNotSupported when the axis length has no register plan here.
template <typename T>
cudaError_t launch_fft_axis_fast(cplx<T>* data, int ncomp, const GridGeom& g, const Tables<T>& tb, int axis,
                                 int dir, cudaStream_t s) {
    const int N = tb.plan[axis].N;
    const cplx<T>* tw = tb.tw[axis];
    switch (N) {
        case 64: return axis_fast<T, 8, 8>(data, ncomp, g, tw, axis, dir, s);
        case 128: return axis_fast<T, 16, 8>(data, ncomp, g, tw, axis, dir, s);
        case 256: return axis_fast<T, 16, 16>(data, ncomp, g, tw, axis, dir, s);
        case 512:
            if constexpr (sizeof(T) == 4) return axis_fast<T, 32, 16>(data, ncomp, g, tw, axis, dir, s);
            return cudaErrorNotSupported;
        case 1024:
            if constexpr (sizeof(T) == 4) return axis_fast<T, 32, 32>(data, ncomp, g, tw, axis, dir, s);
            return cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
    }
}

template <typename T, int N1, int N2, int W>
cudaError_t kspace_fast_launch(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, cudaStream_t s) {
    const size_t smem = (size_t)6 * N1 * N2 * W * sizeof(cplx<T>);
    auto k = kspace_cols_kernel<T, N1, N2, W>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((long long)g.Ny * (g.Nx / W));
    k<<<blocks, W * N2, smem, s>>>(data, g.Nx, g.Ny, tb.tw[2], tb.k[0], tb.k[1], tb.k[2], tb.coef);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kspace_fast(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, cudaStream_t s) {
    // 64-byte rows of the tile: 8 complex64 or 4 complex128 columns
    constexpr int W = sizeof(T) == 4 ? 8 : 4;
    if (g.Nx % W != 0) return cudaErrorNotSupported;
    switch (g.Nz) {
        case 64: return kspace_fast_launch<T, 8, 8, W>(data, g, tb, s);
        case 128: return kspace_fast_launch<T, 16, 8, W>(data, g, tb, s);
        case 256: return kspace_fast_launch<T, 16, 16, W>(data, g, tb, s);
        default: return cudaErrorNotSupported;
    }
}

template cudaError_t launch_fft_axis_fast<float>(cplx<float>*, int, const GridGeom&, const Tables<float>&, int, int, cudaStream_t);
template cudaError_t launch_fft_axis_fast<double>(cplx<double>*, int, const GridGeom&, const Tables<double>&, int, int, cudaStream_t);
template cudaError_t launch_kspace_fast<float>(cplx<float>*, const GridGeom&, const Tables<float>&, cudaStream_t);
template cudaError_t launch_kspace_fast<double>(cplx<double>*, const GridGeom&, const Tables<double>&, cudaStream_t);

}  // namespace psatd
