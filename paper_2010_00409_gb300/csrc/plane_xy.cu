// Fused 2D FFT of x-y planes (one HBM read and one write per plane) using
// thread-block clusters and distributed shared memory.
//
// A cluster of C blocks owns one plane (component, z) of Ny rows x Nx columns.
// Block r of the cluster:
//   phase 1  FFTs the rows y in [r Ny/C, (r+1) Ny/C) along x (register plan,
//            groups of 16 lanes, exchange by a shuffle transpose) and writes
//            each output element x into the shared-memory slab of the block that
//            owns column x (slab = all Ny rows of Nx/C columns, x fastest);
//   cluster barrier (all remote writes complete and visible);
//   phase 2  FFTs its Nx/C columns along y in chunks of 16 columns straight
//            from its slab (block-wide exchange in place in the slab) and
//            stores them to HBM with 128-byte row segments.
// The slab is the block's only shared memory (64 KB for 256 x 256 in FP32 with
// C = 8), so three blocks fit on an SM.
// After the barrier no block touches another block's shared memory, so blocks
// may leave independently.
// Forward (S = -1) reads natural-order x rows and writes natural-order
// spectra; the inverse (S = +1) is the mirror.  Both are unnormalised.
#include <cooperative_groups.h>

#include "fft_reg.cuh"

namespace cg = cooperative_groups;

namespace psatd {

namespace {

constexpr int kPlaneThreads = 256;

template <typename T, int N1X, int N2X, int N1Y, int N2Y, int C, int S>
__global__ void __launch_bounds__(kPlaneThreads)
plane_xy_kernel(cplx<T>* __restrict__ data, const cplx<T>* __restrict__ twx, const cplx<T>* __restrict__ twy) {
    constexpr int NX = N1X * N2X, NY = N1Y * N2Y;
    constexpr int COLS = NX / C;                 // columns per block
    constexpr int ROWS = NY / C;                 // rows per block in phase 1
    constexpr int G = kPlaneThreads / N2X;       // row groups
    constexpr int WY = 16;                       // columns per phase-2 chunk
    static_assert(N1X == 16 && N2X == 16, "phase 1 uses the 16-lane register transpose");
    static_assert(COLS % WY == 0 && ROWS % G == 0 && WY * N2Y == kPlaneThreads, "plane tiling");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* slab = reinterpret_cast<cplx<T>*>(smem_raw);       // [NY][COLS]

    pdl_launch_dependents();
    cg::cluster_group cluster = cg::this_cluster();
    // every block of the cluster must have started before its shared memory is
    // written remotely: arrive now, wait just before the first remote store
    cluster.barrier_arrive();
    const int r = (int)cluster.block_rank();
    const long long plane_id = blockIdx.x / C;
    cplx<T>* plane = data + plane_id * (long long)(NX * NY);
    const GBuf<cplx<T>> F{data, (long long)(gridDim.x / C) * NX * NY};
    pdl_wait();                                        // the previous kernel's output is read below

    // ---------------- phase 1: rows along x, exchange by lane transpose
    {
        const int g = threadIdx.x / N2X, j = threadIdx.x % N2X;
        cplx<T> v[N1X];
#pragma unroll 1
        for (int rr = 0; rr < ROWS / G; ++rr) {
            const int y = r * ROWS + rr * G + g;
            const cplx<T>* p = plane + (long long)y * NX;
            if constexpr (S < 0) {
                static_for<0, N1X>([&](auto nc) { v[decltype(nc)::value] = F.at(p, j + N2X * decltype(nc)::value); });
                stage_a_fwd<T, S, N1X, N2X>(v, j, twx);
                lane_transpose16<T>(v, j);
                reg_dft<T, S, N2X>(v);                   // v[k2] = X[j + 16 k2]
                if (rr == 0) cluster.barrier_wait();
                static_for<0, N2X>([&](auto kc) {
                    constexpr int k2 = decltype(kc)::value;
                    const int x = j + N1X * k2;
                    cplx<T>* dst = cluster.map_shared_rank(slab, x / COLS);
                    dst[y * COLS + (x % COLS)] = v[k2];
                });
            } else {
                static_for<0, N2X>([&](auto kc) { v[decltype(kc)::value] = F.at(p, j + N1X * decltype(kc)::value); });
                reg_dft<T, S, N2X>(v);                   // over k2: v[n2] for k1 = j
                static_for<1, N2X>([&](auto nc) {
                    constexpr int n2 = decltype(nc)::value;
                    if (j) v[n2] = cmul(v[n2], twiddle<T, S>(twx, n2 * j, NX));
                });
                lane_transpose16<T>(v, j);
                reg_dft<T, S, N1X>(v);                   // v[n1] = x[j + 16 n1]
                if (rr == 0) cluster.barrier_wait();
                static_for<0, N1X>([&](auto nc) {
                    constexpr int n1 = decltype(nc)::value;
                    const int x = j + N2X * n1;
                    cplx<T>* dst = cluster.map_shared_rank(slab, x / COLS);
                    dst[y * COLS + (x % COLS)] = v[n1];
                });
            }
        }
    }
    cluster.sync();

    // ---------------- phase 2: columns along y, exchange in place in the slab
    {
        constexpr int RS = N2Y * COLS, ES = COLS;    // element (k1, j) at (k1 N2Y + j) * COLS
        const int c = threadIdx.x % WY, j = threadIdx.x / WY;
        cplx<T> v[N1Y];
#pragma unroll 1
        for (int h = 0; h < COLS / WY; ++h) {
            cplx<T>* col = slab + h * WY + c;
            cplx<T>* out = plane + (long long)r * COLS + h * WY + c;
            if constexpr (S < 0) {
                // reads and exchange writes of a thread hit the same positions
                static_for<0, N1Y>([&](auto nc) { v[decltype(nc)::value] = col[(j + N2Y * decltype(nc)::value) * COLS]; });
                stage_a_fwd<T, S, N1Y, N2Y>(v, j, twy);
                xscatter<T, N1Y, N2Y, RS, ES>(v, col, j);
                __syncthreads();
                xgather_fwd<T, S, N1Y, N2Y, RS, ES>(v, col, j);
                static_for<0, N1Y / N2Y>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    static_for<0, N2Y>([&](auto kc) {
                        constexpr int k2 = decltype(kc)::value;
                        F.at(out, (long long)((j + N2Y * q) + N1Y * k2) * NX) = v[q * N2Y + k2];
                    });
                });
            } else {
                static_for<0, N1Y / N2Y>([&](auto qc) {
                    constexpr int q = decltype(qc)::value;
                    static_for<0, N2Y>([&](auto kc) {
                        constexpr int k2 = decltype(kc)::value;
                        v[q * N2Y + k2] = col[((j + N2Y * q) + N1Y * k2) * COLS];
                    });
                });
                __syncthreads();
                xscatter_inv<T, S, N1Y, N2Y, RS, ES>(v, col, j, twy);
                __syncthreads();
                xgather_inv<T, S, N1Y, N2Y, RS, ES>(v, col, j);
                static_for<0, N1Y>([&](auto nc) {
                    F.at(out, (long long)(j + N2Y * decltype(nc)::value) * NX) = v[decltype(nc)::value];
                });
            }
        }
    }
}

template <typename T, int N1X, int N2X, int N1Y, int N2Y, int C>
cudaError_t plane_launch(cplx<T>* data, int ncomp, int Nz, const cplx<T>* twx, const cplx<T>* twy, int dir,
                         cudaStream_t s) {
    constexpr int NX = N1X * N2X, NY = N1Y * N2Y;
    const size_t smem = (size_t)NY * (NX / C) * sizeof(cplx<T>);
    auto k = dir < 0 ? plane_xy_kernel<T, N1X, N2X, N1Y, N2Y, C, -1> : plane_xy_kernel<T, N1X, N2X, N1Y, N2Y, C, +1>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (C > 8) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((long long)ncomp * Nz * C), 1, 1);
    cfg.blockDim = dim3(kPlaneThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;     // may overlap the previous kernel's tail
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, k, data, twx, twy);
}

}  // namespace

bool plane_xy_supported(int prec, const GridGeom& g) { return prec == 32 && g.Nx == 256 && g.Ny == 256; }

// Fused x+y FFT of ncomp components, or cudaErrorNotSupported (nothing
// launched) for plane shapes without a cluster plan.
template <typename T>
cudaError_t launch_plane_xy(cplx<T>* data, int ncomp, const GridGeom& g, const Tables<T>& tb, int dir,
                            cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (g.Nx == 256 && g.Ny == 256)
            return plane_launch<T, 16, 16, 16, 16, 8>(data, ncomp, g.Nz, tb.tw[0], tb.tw[1], dir, s);
    }
    return cudaErrorNotSupported;
}

template cudaError_t launch_plane_xy<float>(cplx<float>*, int, const GridGeom&, const Tables<float>&, int, cudaStream_t);
template cudaError_t launch_plane_xy<double>(cplx<double>*, int, const GridGeom&, const Tables<double>&, int, cudaStream_t);

}  // namespace psatd
