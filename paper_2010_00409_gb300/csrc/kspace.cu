// Fused k-space pass (generic sizes): forward FFT along z, the per-mode PSATD
// update of Eq. 3-4 (Sec. 2.1), and the inverse FFT along z, for all six
// components of a tile of W x-columns at one y.  The x and y transforms of the
// step have already been applied, so after the forward z transform the tile
// holds Fourier amplitudes E^(k), B^(k) of the modes (kx[x0..x0+W), ky[y], kz[*]).
//
// Update per mode, with C' = cos(c|k|dt)/Ntot, S' = sin(c|k|dt)/Ntot (the 1/Ntot
// of the inverse DFT folded in) and n = k/|k| (0 at k = 0):
//   E <- C' (E - n (n.E)) + i S' n x B
//   B <- C' B - i S' n x E                (both right-hand sides from step n)
// KS_PROJECT instead removes the longitudinal part of E and B and scales by
// 1/Ntot (the one-time projection after initialisation).
#include "fft_core.cuh"

namespace psatd {

namespace {

constexpr int kThreads = 256;

template <typename T>
__device__ __forceinline__ void mode_update(cplx<T>* F0, cplx<T>* F1, cplx<T>* F2, cplx<T>* F3,
                                            cplx<T>* F4, cplx<T>* F5, T nx, T ny, T nz, T C, T S,
                                            int mode, T scale) {
    const cplx<T> Ex = *F0, Ey = *F1, Ez = *F2;
    cplx<T> Bx = *F3, By = *F4, Bz = *F5;
    if (mode == KS_ROTATE_SPECTRAL_PROJ) {
        const cplx<T> kB = mk<T>(nx * Bx.x + ny * By.x + nz * Bz.x, nx * Bx.y + ny * By.y + nz * Bz.y);
        Bx = csub(Bx, cscale(kB, nx));
        By = csub(By, cscale(kB, ny));
        Bz = csub(Bz, cscale(kB, nz));
    }
    if (mode == KS_PROJECT) {
        cplx<T> kE = mk<T>(nx * Ex.x + ny * Ey.x + nz * Ez.x, nx * Ex.y + ny * Ey.y + nz * Ez.y);
        cplx<T> kB = mk<T>(nx * Bx.x + ny * By.x + nz * Bz.x, nx * Bx.y + ny * By.y + nz * Bz.y);
        *F0 = cscale(csub(Ex, cscale(kE, nx)), scale);
        *F1 = cscale(csub(Ey, cscale(kE, ny)), scale);
        *F2 = cscale(csub(Ez, cscale(kE, nz)), scale);
        *F3 = cscale(csub(Bx, cscale(kB, nx)), scale);
        *F4 = cscale(csub(By, cscale(kB, ny)), scale);
        *F5 = cscale(csub(Bz, cscale(kB, nz)), scale);
        return;
    }
    const cplx<T> kE = mk<T>(nx * Ex.x + ny * Ey.x + nz * Ez.x, nx * Ex.y + ny * Ey.y + nz * Ez.y);
    // n x B and n x E
    const cplx<T> cBx = mk<T>(ny * Bz.x - nz * By.x, ny * Bz.y - nz * By.y);
    const cplx<T> cBy = mk<T>(nz * Bx.x - nx * Bz.x, nz * Bx.y - nx * Bz.y);
    const cplx<T> cBz = mk<T>(nx * By.x - ny * Bx.x, nx * By.y - ny * Bx.y);
    const cplx<T> cEx = mk<T>(ny * Ez.x - nz * Ey.x, ny * Ez.y - nz * Ey.y);
    const cplx<T> cEy = mk<T>(nz * Ex.x - nx * Ez.x, nz * Ex.y - nx * Ez.y);
    const cplx<T> cEz = mk<T>(nx * Ey.x - ny * Ex.x, nx * Ey.y - ny * Ex.y);
    // i S v = (-S v.y, S v.x)
    *F0 = mk<T>(C * (Ex.x - nx * kE.x) - S * cBx.y, C * (Ex.y - nx * kE.y) + S * cBx.x);
    *F1 = mk<T>(C * (Ey.x - ny * kE.x) - S * cBy.y, C * (Ey.y - ny * kE.y) + S * cBy.x);
    *F2 = mk<T>(C * (Ez.x - nz * kE.x) - S * cBz.y, C * (Ez.y - nz * kE.y) + S * cBz.x);
    *F3 = mk<T>(C * Bx.x + S * cEx.y, C * Bx.y - S * cEx.x);
    *F4 = mk<T>(C * By.x + S * cEy.y, C * By.y - S * cEy.x);
    *F5 = mk<T>(C * Bz.x + S * cEz.y, C * Bz.y - S * cEz.x);
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
kspace_z_kernel(cplx<T>* __restrict__ data, int Nx, int Ny, int Nz, int W, int P, AxisPlan pl,
                const cplx<T>* __restrict__ twz, const T* __restrict__ kx, const T* __restrict__ ky,
                const T* __restrict__ kz, const ModeCoef<T>* __restrict__ coef, int mode, T scale) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* F = reinterpret_cast<cplx<T>*>(smem_raw);        // [6][W][P]
    cplx<T>* scratch = F + (size_t)6 * W * P;                  // [W][P]
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ntile = (Nx + W - 1) / W;
    const int t = blockIdx.x % ntile;
    const int y = blockIdx.x / ntile;
    const int x0 = t * W;
    const int nw = min(W, Nx - x0);
    const size_t plane = (size_t)Nx * Ny;
    const size_t cstride = plane * Nz;
    const size_t comp_tile = (size_t)W * P;
    cplx<T>* base = data + (size_t)y * Nx + x0;
    const GBuf<cplx<T>> G{data, 6LL * (long long)cstride};

    const FastDiv dw = fast_div(nw), dz = fast_div(Nz);
    for (int c = 0; c < 6; ++c) {
        for (int e = tid; e < Nz * nw; e += nthr) {
            const int n = fdiv(e, dw), w = e - n * nw;
            F[c * comp_tile + w * P + pad32(n)] = G.at(base, c * cstride + (size_t)n * plane + w);
        }
    }
    __syncthreads();

    if (pl.N > 1) {
        for (int c = 0; c < 6; ++c) {
            cplx<T>* res = fft_tile<T, -1>(F + c * comp_tile, scratch, pl, nw, P, twz);
            if (res != F + c * comp_tile) {
                for (int e = tid; e < nw * P; e += nthr) F[c * comp_tile + e] = scratch[e];
                __syncthreads();
            }
        }
    }

    const int Nxh = Nx / 2 + 1, Nyh = Ny / 2 + 1;
    const int ay = min(y, Ny - y);
    for (int e = tid; e < nw * Nz; e += nthr) {
        const int w = fdiv(e, dz), n = e - w * Nz;
        const int ix = x0 + w;
        const int ax = min(ix, Nx - ix), az = min(n, Nz - n);
        const ModeCoef<T> m = coef[PSATD_IX(((size_t)az * Nyh + ay) * Nxh + ax, (long long)(Nz / 2 + 1) * Nyh * Nxh)];
        const T nxv = kx[PSATD_IX(ix, Nx)] * m.kinv, nyv = ky[PSATD_IX(y, Ny)] * m.kinv, nzv = kz[PSATD_IX(n, Nz)] * m.kinv;
        const size_t o = (size_t)w * P + pad32(n);
        mode_update<T>(F + o, F + comp_tile + o, F + 2 * comp_tile + o, F + 3 * comp_tile + o,
                       F + 4 * comp_tile + o, F + 5 * comp_tile + o, nxv, nyv, nzv, m.C, m.S, mode,
                       scale);
    }
    __syncthreads();

    if (pl.N > 1 && mode != KS_ROTATE_SPECTRAL && mode != KS_ROTATE_SPECTRAL_PROJ) {
        for (int c = 0; c < 6; ++c) {
            cplx<T>* res = fft_tile<T, +1>(F + c * comp_tile, scratch, pl, nw, P, twz);
            if (res != F + c * comp_tile) {
                for (int e = tid; e < nw * P; e += nthr) F[c * comp_tile + e] = scratch[e];
                __syncthreads();
            }
        }
    }

    for (int c = 0; c < 6; ++c) {
        for (int e = tid; e < Nz * nw; e += nthr) {
            const int n = fdiv(e, dw), w = e - n * nw;
            G.at(base, c * cstride + (size_t)n * plane + w) = F[c * comp_tile + w * P + pad32(n)];
        }
    }
}

// The per-mode update alone, on a spectrum already transformed along all three
// axes (the z transforms run as separate launches for axis lengths without a
// fused kernel): one thread per mode, x fastest, all six components.
template <typename T>
__global__ void __launch_bounds__(kThreads)
modes_kernel(cplx<T>* __restrict__ data, int Nx, int Ny, int Nz, const T* __restrict__ kx,
             const T* __restrict__ ky, const T* __restrict__ kz, const ModeCoef<T>* __restrict__ coef, int mode,
             T scale) {
    const size_t n = (size_t)Nx * Ny * Nz;
    const int Nxh = Nx / 2 + 1, Nyh = Ny / 2 + 1;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
        const int ix = (int)(e % Nx);
        const size_t r = e / Nx;
        const int iy = (int)(r % Ny), iz = (int)(r / Ny);
        const int ax = min(ix, Nx - ix), ay = min(iy, Ny - iy), az = min(iz, Nz - iz);
        const ModeCoef<T> m = coef[PSATD_IX(((size_t)az * Nyh + ay) * Nxh + ax, (long long)(Nz / 2 + 1) * Nyh * Nxh)];
        const GBuf<cplx<T>> G{data, 6LL * (long long)n};
        mode_update<T>(&G[e], &G[n + e], &G[2 * n + e], &G[3 * n + e], &G[4 * n + e], &G[5 * n + e],
                       kx[PSATD_IX(ix, Nx)] * m.kinv, ky[PSATD_IX(iy, Ny)] * m.kinv, kz[PSATD_IX(iz, Nz)] * m.kinv,
                       m.C, m.S, mode, scale);
    }
}

}  // namespace

template <typename T>
cudaError_t launch_modes(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, int mode, double scale,
                         cudaStream_t s) {
    const size_t n = (size_t)g.Nx * g.Ny * g.Nz;
    long long blocks = (long long)((n + kThreads - 1) / kThreads);
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    modes_kernel<T><<<(unsigned)blocks, kThreads, 0, s>>>(data, g.Nx, g.Ny, g.Nz, tb.k[0], tb.k[1], tb.k[2],
                                                          tb.coef, mode, (T)scale);
    return cudaGetLastError();
}

template cudaError_t launch_modes<float>(cplx<float>*, const GridGeom&, const Tables<float>&, int, double, cudaStream_t);
template cudaError_t launch_modes<double>(cplx<double>*, const GridGeom&, const Tables<double>&, int, double, cudaStream_t);

template <typename T>
cudaError_t launch_kspace_z(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, int mode,
                            double scale, cudaStream_t s, long long* nlaunch) {
    const int es = (int)sizeof(cplx<T>);
    const int P = pencil_stride(g.Nz);
    // 64 contiguous bytes per tile row; the tile capped at 56 KB (float32, four
    // blocks per SM) or 100 KB (float64, two)
    const size_t cap = es == 8 ? 56 * 1024 : 100 * 1024;
    int W = min(g.Nx, 64 / es);
    if (tb.tile_shift > 0) W = min(g.Nx, W << tb.tile_shift);
    if (tb.tile_shift < 0) W = max(1, W >> -tb.tile_shift);
    while (W > 1 && 7 * (size_t)W * P * es > cap) W /= 2;
    const size_t smem = 7 * (size_t)W * P * es;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const long long nblocks = (long long)g.Ny * ((g.Nx + W - 1) / W);
    auto k = kspace_z_kernel<T>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<(unsigned)nblocks, kThreads, smem, s>>>(data, g.Nx, g.Ny, g.Nz, W, P, tb.plan[2], tb.tw[2],
                                                tb.k[0], tb.k[1], tb.k[2], tb.coef, mode, (T)scale);
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

template cudaError_t launch_kspace_z<float>(cplx<float>*, const GridGeom&, const Tables<float>&, int, double, cudaStream_t, long long*);
template cudaError_t launch_kspace_z<double>(cplx<double>*, const GridGeom&, const Tables<double>&, int, double, cudaStream_t, long long*);

}  // namespace psatd
