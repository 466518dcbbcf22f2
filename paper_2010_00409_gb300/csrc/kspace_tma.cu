// Fused k-space pass of one PSATD step (Sec. 2.1, Eq. 3-4), fed by the tensor
// copy engine: at block start one thread issues six tiled bulk-tensor loads
// (one per field component, box = W x-columns x 1 y x Nz z, 64 contiguous bytes
// per row) into the six shared-memory slots, all completing on one mbarrier.
// The whole tile (6 * Nz * W complex values) is then in flight at once, while
// the other resident block computes.  Per component: forward z transform in
// registers (the slot doubles as the exchange buffer), spectrum back to the
// slot; the per-mode update over all six slots; inverse z transforms stored
// straight from registers to the field.
//
// The wait on the copies is bounded: past the limit the block sets an error bit
// in the context's device error word and returns without touching the field.
#include "fft_reg.cuh"
#include "tma.cuh"

namespace psatd {

namespace {

template <typename T, int N1, int N2, int W>
__global__ void __launch_bounds__(W * N2)
kspace_tma_kernel(const __grid_constant__ CUtensorMap map, cplx<T>* __restrict__ data, int Nx, int Ny,
                  const cplx<T>* __restrict__ tw, const T* __restrict__ kxs, const T* __restrict__ kys,
                  const T* __restrict__ kzs, const ModeCoef<T>* __restrict__ coef, int* __restrict__ err) {
    constexpr int Nz = N1 * N2;
    constexpr int RS = N2 * W, ES = W;
    constexpr int SLOT = Nz * W;
    constexpr uint32_t kBytes = 6u * SLOT * sizeof(cplx<T>);
    static_assert(kBytes < (1u << 20), "mbarrier transaction count is 20 bits");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cplx<T>* spec = reinterpret_cast<cplx<T>*>(smem_raw);      // [6][Nz][W]
    __shared__ __align__(8) uint64_t bar;
    __shared__ int failed;

    const int c = threadIdx.x % W, j = threadIdx.x / W;
    const size_t plane = (size_t)Nx * Ny;
    const size_t cstride = plane * Nz;
    const int ntile = Nx / W;
    const int xt = blockIdx.x % ntile;
    const int y = blockIdx.x / ntile;
    const int ix = xt * W + c;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, kBytes);
        constexpr int xw = (int)(sizeof(cplx<T>) / 8);        // 8-byte elements per complex
        for (int q = 0; q < 6; ++q) tma_load_4d(spec + q * SLOT, &map, &bar, xt * W * xw, y, 0, q);
        bool ok = mbar_wait_bounded(&bar, 0);
        if (!ok) {
            atomicOr(err, DEV_ERR_TMA_TIMEOUT);
            mbar_wait_bounded(&bar, 0);                        // give copies in flight a second chance
        }
        failed = ok ? 0 : 1;
    }
    __syncthreads();
    if (failed) return;

    cplx<T>* base = data + (size_t)y * Nx + ix;
    cplx<T> v[N1];

    // forward z transforms; raw element (z, c) sits at z*W + c of its slot and
    // each thread's exchange writes land on exactly the positions it read
    for (int q = 0; q < 6; ++q) {
        cplx<T>* sl = spec + q * SLOT + c;
        static_for<0, N1>([&](auto nc) { v[decltype(nc)::value] = sl[(j + N2 * decltype(nc)::value) * W]; });
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

    {
        const int Nxh = Nx / 2 + 1, Nyh = Ny / 2 + 1;
        const int ax = min(ix, Nx - ix), ay = min(y, Ny - y);
        const T kx = kxs[ix], ky = kys[y];
        cplx<T>* sl = spec + c;
#pragma unroll 4
        for (int s = 0; s < N1; ++s) {
            const int iz = j + N2 * s;
            const int az = min(iz, Nz - iz);
            const ModeCoef<T> m = coef[((size_t)az * Nyh + ay) * Nxh + ax];
            const int o = iz * W;
            cplx<T> Ex = sl[o], Ey = sl[SLOT + o], Ez = sl[2 * SLOT + o];
            cplx<T> Bx = sl[3 * SLOT + o], By = sl[4 * SLOT + o], Bz = sl[5 * SLOT + o];
            rotate_mode<T>(Ex, Ey, Ez, Bx, By, Bz, kx * m.kinv, ky * m.kinv, kzs[iz] * m.kinv, m.C, m.S);
            sl[o] = Ex; sl[SLOT + o] = Ey; sl[2 * SLOT + o] = Ez;
            sl[3 * SLOT + o] = Bx; sl[4 * SLOT + o] = By; sl[5 * SLOT + o] = Bz;
        }
    }
    __syncthreads();

    for (int q = 0; q < 6; ++q) {
        cplx<T>* sl = spec + q * SLOT + c;
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
        static_for<0, N1>([&](auto nc) { p[(j + N2 * decltype(nc)::value) * plane] = v[decltype(nc)::value]; });
    }
}

template <typename T, int N1, int N2, int W>
cudaError_t kspace_tma_launch(const CUtensorMap& map, cplx<T>* data, const GridGeom& g, const Tables<T>& tb,
                              int* err, cudaStream_t s) {
    const size_t smem = (size_t)6 * N1 * N2 * W * sizeof(cplx<T>);
    auto k = kspace_tma_kernel<T, N1, N2, W>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((long long)g.Ny * (g.Nx / W));
    k<<<blocks, W * N2, smem, s>>>(map, data, g.Nx, g.Ny, tb.tw[2], tb.k[0], tb.k[1], tb.k[2], tb.coef, err);
    return cudaGetLastError();
}

// Self-test of the bounded-wait path: waits on an mbarrier whose 16 expected
// bytes no copy will ever deliver, gives up after `limit` polls and reports
// DEV_ERR_TMA_TIMEOUT.  No asynchronous copy is issued, so nothing is in flight
// when the block exits.
__global__ void wait_timeout_selftest_kernel(int* err, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, 16);
        bool ok = false;
        for (uint32_t it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(&bar, 0);
        if (!ok) atomicOr(err, DEV_ERR_TMA_TIMEOUT);
    }
}

}  // namespace

cudaError_t launch_wait_timeout_selftest(int* err, cudaStream_t s) {
    wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(err, 1024);
    return cudaGetLastError();
}

template <typename T> constexpr int kspace_tma_width() { return 64 / (int)sizeof(cplx<T>); }

template <typename T>
cudaError_t launch_kspace_tma(const CUtensorMap& map, cplx<T>* data, const GridGeom& g, const Tables<T>& tb,
                              int* err, cudaStream_t s) {
    constexpr int W = kspace_tma_width<T>();
    if (g.Nx % W != 0) return cudaErrorNotSupported;
    switch (g.Nz) {
        case 64: return kspace_tma_launch<T, 8, 8, W>(map, data, g, tb, err, s);
        case 128: return kspace_tma_launch<T, 16, 8, W>(map, data, g, tb, err, s);
        case 256: return kspace_tma_launch<T, 16, 16, W>(map, data, g, tb, err, s);
        default: return cudaErrorNotSupported;
    }
}

int kspace_tma_box_x(int prec) { return prec == 64 ? kspace_tma_width<double>() * 2 : kspace_tma_width<float>(); }

template cudaError_t launch_kspace_tma<float>(const CUtensorMap&, cplx<float>*, const GridGeom&, const Tables<float>&, int*, cudaStream_t);
template cudaError_t launch_kspace_tma<double>(const CUtensorMap&, cplx<double>*, const GridGeom&, const Tables<double>&, int*, cudaStream_t);

}  // namespace psatd
