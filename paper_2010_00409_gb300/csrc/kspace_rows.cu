// Fused k-space pass along x for grids whose z length has no fused kernel
// (complex storage, N_x = N1 * N2 with a register plan: 512 and 1024 in
// float32).  The step (Sec. 2.1, Eq. 3-4) then takes its transforms in the
// order z, y, x and fuses the per-mode update into the x pass: one block takes
// the six components of one (k_y, k_z) row, transforms each along x (one group
// of N2 threads per component, whose shared-memory slot doubles as its
// exchange buffer), applies the update to every mode of the row and transforms
// back.  The last forward transform, the update and the first inverse
// transform then cost one read and one write of the field; x rows are
// contiguous, so every load and store is a coalesced 256-byte (N2 = 32) run.
//
// Blocks walk the z index as 0, 1, N_z - 1, 2, N_z - 2, ... so that the rows
// k_z and N_z - k_z, which read the same rows of the coefficient table, run
// close together and the second read hits L2.
#include "fft_reg.cuh"
#include "tma.cuh"

namespace psatd {

namespace {

template <int N2>
__device__ __forceinline__ void group_sync() {
    if constexpr (N2 == 32) __syncwarp();       // a group is one warp
    else __syncthreads();
}

template <typename T, int N1, int N2>
constexpr int rows_slot() { return N1 * (N2 + 1); }   // >= N1 * N2: the padded exchange layout

// float32 at N2 = 32: four blocks of 192 threads per SM (at most 85 registers)
#ifndef PSATD_ROWS_MINB
#define PSATD_ROWS_MINB 4
#endif
template <typename T, int N1, int N2>
__global__ void __launch_bounds__(6 * N2, N2 == 32 ? PSATD_ROWS_MINB : 1)
kspace_rows_kernel(cplx<T>* __restrict__ data, int Ny, int Nz, const cplx<T>* __restrict__ tw2,
                   const T* __restrict__ kxs, const T* __restrict__ kys, const T* __restrict__ kzs,
                   const ModeCoef<T>* __restrict__ coef) {
    constexpr int N = N1 * N2;
    constexpr int RS = N2 + 1;                          // exchange row stride (bank spread)
    constexpr int SLOT = rows_slot<T, N1, N2>();
    extern __shared__ __align__(16) unsigned char rows_smem[];
    cplx<T>* slot = reinterpret_cast<cplx<T>*>(rows_smem);    // [6][SLOT]

    const int q = threadIdx.x / N2, j = threadIdx.x % N2;    // component q, lane j of its group
    const int pz = (int)(blockIdx.x / Ny), iy = (int)(blockIdx.x % Ny);
    const int iz = pz == 0 ? 0 : ((pz & 1) ? (pz + 1) / 2 : Nz - pz / 2);
    const size_t cells = (size_t)N * Ny * Nz;
    const size_t row = (size_t)iz * Ny + iy;
    const GBuf<cplx<T>> F{data, 6LL * (long long)cells};
    cplx<T>* p = data + (size_t)q * cells + row * N;
    cplx<T>* sc = slot + q * SLOT;
    cplx<T> v[N1];
    const int Nxh = N / 2 + 1, Nyh = Ny / 2 + 1;
    const int ay = min(iy, Ny - iy), az = min(iz, Nz - iz);
    const long long ncoef = (long long)(Nz / 2 + 1) * Nyh * Nxh;
    const long long crow = ((long long)az * Nyh + ay) * Nxh;
    if (threadIdx.x == 0) {
        // the row's Nx/2 + 1 table entries to L2 while the forward transforms run
        // (16-byte aligned range, clipped to whole 16-byte chunks of the table)
        const uintptr_t b = reinterpret_cast<uintptr_t>(coef);
        const uintptr_t lo = (reinterpret_cast<uintptr_t>(coef + crow)) & ~(uintptr_t)15;
        uintptr_t hi = (reinterpret_cast<uintptr_t>(coef + crow + Nxh) + 15) & ~(uintptr_t)15;
        const uintptr_t end = (b + (uintptr_t)ncoef * sizeof(ModeCoef<T>)) & ~(uintptr_t)15;
        if (hi > end) hi = end;
        if (hi > lo) prefetch_l2_bulk(reinterpret_cast<const void*>(lo), (uint32_t)(hi - lo));
    }

    // forward x transform of component q; its spectrum to the slot in natural order
    // (twiddles W^{j k1} from the [k1][j] table: a warp reads 32 consecutive entries)
    static_for<0, N1>([&](auto nc) { v[decltype(nc)::value] = F.at(p, j + N2 * decltype(nc)::value); });
    reg_dft<T, -1, N1>(v);
    static_for<1, N1>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        if (j) v[k1] = cmul(v[k1], tw2[PSATD_IX(k1 * 32 + j, 1024)]);
    });
    xscatter<T, N1, N2, RS, 1>(v, sc, j);
    group_sync<N2>();
    xgather_fwd<T, -1, N1, N2, RS, 1>(v, sc, j);        // v[qq N2 + k2] = X[(j + N2 qq) + N1 k2]
    group_sync<N2>();                                   // the exchange rows are read before the slot is reused
    static_for<0, N1 / N2>([&](auto qc) {
        constexpr int qq = decltype(qc)::value;
        static_for<0, N2>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            sc[(j + N2 * qq) + N1 * k2] = v[qq * N2 + k2];
        });
    });
    __syncthreads();

    // Eq. 3-4 on every mode of the row (C, S carry 1/(Nx Ny Nz))
    {
        const T ky = kys[PSATD_IX(iy, Ny)], kz = kzs[PSATD_IX(iz, Nz)];
        // this thread's modes k = tid + 6 N2 i: their table entries are loaded
        // together first (independent loads in flight at once), then updated
        constexpr int NI = (N + 6 * N2 - 1) / (6 * N2);
        ModeCoef<T> mc[NI];
        T kx[NI];
        static_for<0, NI>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const int k = (int)threadIdx.x + 6 * N2 * i;
            if (k < N) {
                mc[i] = coef[PSATD_IX(crow + min(k, N - k), ncoef)];
                kx[i] = kxs[PSATD_IX(k, N)];
            }
        });
        static_for<0, NI>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const int k = (int)threadIdx.x + 6 * N2 * i;
            if (k < N) {
                const ModeCoef<T> m = mc[i];
                cplx<T> Ex = slot[k], Ey = slot[SLOT + k], Ez = slot[2 * SLOT + k];
                cplx<T> Bx = slot[3 * SLOT + k], By = slot[4 * SLOT + k], Bz = slot[5 * SLOT + k];
                rotate_mode<T>(Ex, Ey, Ez, Bx, By, Bz, kx[i] * m.kinv, ky * m.kinv, kz * m.kinv, m.C, m.S);
                slot[k] = Ex; slot[SLOT + k] = Ey; slot[2 * SLOT + k] = Ez;
                slot[3 * SLOT + k] = Bx; slot[4 * SLOT + k] = By; slot[5 * SLOT + k] = Bz;
            }
        });
    }
    __syncthreads();

    // inverse x transform of component q, stored (the twiddle pointer passes
    // through an opaque move so that the inverse's twiddle loads are not hoisted
    // above the forward transform, where they would double the live registers)
    const cplx<T>* twi = tw2;
    asm volatile("" : "+l"(twi));
    static_for<0, N1 / N2>([&](auto qc) {
        constexpr int qq = decltype(qc)::value;
        static_for<0, N2>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            v[qq * N2 + k2] = sc[(j + N2 * qq) + N1 * k2];
        });
    });
    group_sync<N2>();                                   // the spectrum is read before the exchange overwrites it
    // inverse N2-point transforms, twiddles conj W^{n2 k1} from the [n2][k1] table
    static_for<0, N1 / N2>([&](auto qc) {
        constexpr int qq = decltype(qc)::value;
        cplx<T> w[N2];
        static_for<0, N2>([&](auto kc) { w[decltype(kc)::value] = v[qq * N2 + decltype(kc)::value]; });
        reg_dft<T, +1, N2>(w);
        const int k1 = j + N2 * qq;
        static_for<0, N2>([&](auto nc) {
            constexpr int n2 = decltype(nc)::value;
            sc[k1 * RS + n2] = (n2 == 0 || k1 == 0) ? w[n2] : cmulc(w[n2], twi[PSATD_IX(n2 * 32 + k1, 1024)]);
        });
    });
    group_sync<N2>();
    xgather_inv<T, +1, N1, N2, RS, 1>(v, sc, j);
    static_for<0, N1>([&](auto nc) { F.at(p, j + N2 * decltype(nc)::value) = v[decltype(nc)::value]; });
}

template <typename T, int N1, int N2>
cudaError_t rows_launch(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, cudaStream_t s) {
    const size_t smem = (size_t)6 * rows_slot<T, N1, N2>() * sizeof(cplx<T>);
    auto k = kspace_rows_kernel<T, N1, N2>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long blocks = (long long)g.Ny * g.Nz;
    if (blocks > 0x7FFFFFFFLL) return cudaErrorInvalidValue;
    k<<<(unsigned)blocks, 6 * N2, smem, s>>>(data, g.Ny, g.Nz, tb.tw2[0], tb.k[0], tb.k[1], tb.k[2], tb.coef);
    return cudaGetLastError();
}

}  // namespace

bool kspace_rows_supported(int prec, const GridGeom& g) {
    return prec == 32 && (g.Nx == 512 || g.Nx == 1024);
}

// Forward x, the per-mode update and inverse x of the six complex components
// (storage [6][Nz][Ny][Nx], natural order along every axis; y and z must
// already be in k-space), or cudaErrorNotSupported (nothing launched).
template <typename T>
cudaError_t launch_kspace_rows(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, cudaStream_t s) {
    if (!tb.tw2[0]) return cudaErrorNotSupported;
    if constexpr (sizeof(T) == 4) {
        if (g.Nx == 1024) return rows_launch<T, 32, 32>(data, g, tb, s);
        if (g.Nx == 512) return rows_launch<T, 32, 16>(data, g, tb, s);
    }
    return cudaErrorNotSupported;
}

template cudaError_t launch_kspace_rows<float>(cplx<float>*, const GridGeom&, const Tables<float>&, cudaStream_t);
template cudaError_t launch_kspace_rows<double>(cplx<double>*, const GridGeom&, const Tables<double>&, cudaStream_t);

}  // namespace psatd
