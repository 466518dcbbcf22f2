// Generic in-place FFT along one axis of a [ncomp][Nz][Ny][Nx] complex array
// (the 3D DFT of Sec. 2.1 is three of these; the kernel is exp(-ikx) forward).
//
// Each block stages a tile of W pencils in shared memory (the padded pencil
// layout of fft_core.cuh, odd pencil stride P, so the strided loads hit
// distinct banks), runs the Stockham passes between two shared buffers, and
// writes the pencils back.
//  - x (contiguous): W consecutive rows, loaded and stored as one run.
//  - y / z (strided): W consecutive x-columns at one (comp, z) or (comp, y),
//    loaded row by row so each warp touches W*sizeof(complex) contiguous bytes.
#include "fft_core.cuh"

namespace psatd {

namespace {

constexpr int kThreads = 256;

template <typename T, int S>
__global__ void __launch_bounds__(kThreads)
fft_axis_kernel(cplx<T>* __restrict__ data, int axis, int Nx, int Ny, int Nz, int ncomp, int W,
                int P, AxisPlan pl, const cplx<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* A = reinterpret_cast<cplx<T>*>(smem_raw);
    cplx<T>* B = A + (size_t)W * P;
    const int N = pl.N;
    const int tid = threadIdx.x, nthr = blockDim.x;

    if (axis == 0) {
        const long long rows = (long long)ncomp * Nz * Ny;
        const long long row0 = (long long)blockIdx.x * W;
        const int nrow = (int)min((long long)W, rows - row0);
        cplx<T>* base = data + row0 * Nx;
        const GBuf<cplx<T>> F{data, rows * Nx};
        const FastDiv dn = fast_div(Nx);
        for (int e = tid; e < nrow * Nx; e += nthr) {
            const int w = fdiv(e, dn), n = e - w * Nx;
            A[w * P + pad32(n)] = F.at(base, e);
        }
        __syncthreads();
        cplx<T>* res = fft_tile<T, S>(A, B, pl, nrow, P, tw);
        for (int e = tid; e < nrow * Nx; e += nthr) {
            const int w = fdiv(e, dn), n = e - w * Nx;
            F.at(base, e) = res[w * P + pad32(n)];
        }
        return;
    }

    const size_t plane = (size_t)Nx * Ny;
    const int ntile = (Nx + W - 1) / W;
    const int outerN = (axis == 1) ? Nz : Ny;
    const long long g = blockIdx.x;
    const int t = (int)(g % ntile);
    const long long rest = g / ntile;
    const int o = (int)(rest % outerN);
    const int comp = (int)(rest / outerN);
    const int x0 = t * W;
    const int nw = min(W, Nx - x0);
    const size_t stride = (axis == 1) ? (size_t)Nx : plane;
    cplx<T>* base = data + (size_t)comp * plane * Nz + (axis == 1 ? (size_t)o * plane : (size_t)o * Nx) + x0;
    const GBuf<cplx<T>> F{data, (long long)ncomp * plane * Nz};
    const FastDiv dw = fast_div(nw);
    for (int e = tid; e < N * nw; e += nthr) {
        const int n = fdiv(e, dw), w = e - n * nw;
        A[w * P + pad32(n)] = F.at(base, (long long)n * stride + w);
    }
    __syncthreads();
    cplx<T>* res = fft_tile<T, S>(A, B, pl, nw, P, tw);
    for (int e = tid; e < N * nw; e += nthr) {
        const int n = fdiv(e, dw), w = e - n * nw;
        F.at(base, (long long)n * stride + w) = res[w * P + pad32(n)];
    }
}

// Tile width for an axis: strided axes take up to 128 contiguous bytes per row
// of the tile; x takes enough rows for ~2048 elements.  Shared memory is
// capped at 56 KB (float32) / 96 KB (float64) so four / two blocks fit on an SM.
template <typename T>
void choose_tile(int axis, int N, int Nx, int shift, int* W, int* P) {
    const int es = (int)sizeof(cplx<T>);
    const size_t cap = es == 8 ? 56 * 1024 : 96 * 1024;
    *P = pencil_stride(N);
    int w;
    if (axis == 0) w = max(1, min(64, 2048 / max(N, 1)));
    else w = min(Nx, 128 / es);
    if (shift > 0) w = min(axis == 0 ? 128 : Nx, w << shift);
    if (shift < 0) w = max(1, w >> -shift);
    while (w > 1 && 2 * (size_t)w * (*P) * es > cap) w /= 2;
    *W = max(1, w);
}

}  // namespace

template <typename T>
cudaError_t launch_fft_axis(cplx<T>* data, int ncomp, const GridGeom& g, const Tables<T>& tb,
                            int axis, int dir, cudaStream_t s, long long* nlaunch) {
    const AxisPlan& pl = tb.plan[axis];
    if (pl.N <= 1) return cudaSuccess;
    int W, P;
    const int Nx = g.Nx;
    choose_tile<T>(axis, pl.N, Nx, tb.tile_shift, &W, &P);
    long long nblocks;
    if (axis == 0) nblocks = ((long long)ncomp * g.Nz * g.Ny + W - 1) / W;
    else nblocks = (long long)ncomp * (axis == 1 ? g.Nz : g.Ny) * ((Nx + W - 1) / W);
    const size_t smem = 2 * (size_t)W * P * sizeof(cplx<T>);
    if (dir < 0) {
        auto k = fft_axis_kernel<T, -1>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<(unsigned)nblocks, kThreads, smem, s>>>(data, axis, g.Nx, g.Ny, g.Nz, ncomp, W, P, pl, tb.tw[axis]);
    } else {
        auto k = fft_axis_kernel<T, +1>;
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k<<<(unsigned)nblocks, kThreads, smem, s>>>(data, axis, g.Nx, g.Ny, g.Nz, ncomp, W, P, pl, tb.tw[axis]);
    }
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
}

template cudaError_t launch_fft_axis<float>(cplx<float>*, int, const GridGeom&, const Tables<float>&, int, int, cudaStream_t, long long*);
template cudaError_t launch_fft_axis<double>(cplx<double>*, int, const GridGeom&, const Tables<double>&, int, int, cudaStream_t, long long*);

}  // namespace psatd
