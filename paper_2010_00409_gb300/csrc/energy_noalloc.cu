// Field energy without any device allocation (psatd_energy_noalloc).
//
// Some callers cannot allocate device memory at the moment they need this
// number: code that runs while a stream is being captured into a CUDA graph
// (an allocation there either fails or breaks the capture), frameworks whose
// caching allocator has already reserved the whole device, and tight loops
// that cannot afford cudaMalloc/cudaFree (both may synchronise the device).
// For them this entry point keeps its per-block partial sums in a file-scope
// __device__ array instead of a buffer it allocates; the caller passes the
// field and the place for the result.
//
// The array holds 2 doubles per partial for at most kMaxPartials partials plus
// 2 result slots (1 MB + 16 B); one partial covers kCellsPerPartial cells, so
// grids above kMaxPartials * kCellsPerPartial = 2^30 cells are rejected.  Every
// GPU that loads the library holds the array until the process exits.  All calls
// share it: each call overwrites every partial it reads, so nothing needs
// clearing, but two calls whose kernels overlap on a GPU (different streams)
// race on it and must be serialised by the caller.  The first call on a device
// also loads the three kernels, so that no later call allocates.
#include <mutex>

#include "../../include/psatd.h"
#include "common.cuh"

namespace psatd {

namespace {

constexpr int kThreads = 256;
constexpr long long kCellsPerPartial = 16384;
constexpr int kMaxPartials = 65536;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_scratch[2 * kMaxPartials + 2];

// Device address of g_energy_scratch per device, looked up once per device
// with that device current (in host code the symbol is only a stand-in).
double* g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// partial[2b], partial[2b+1] = sum |E|^2, sum |B|^2 over cells [b*K, (b+1)*K)
template <typename T>
__global__ void __launch_bounds__(kThreads)
energy_partials_kernel(const cplx<T>* __restrict__ f, long long n, double* __restrict__ partial) {
    __shared__ double sE[kThreads / 32], sB[kThreads / 32];
    const long long begin = blockIdx.x * kCellsPerPartial;
    const long long end = min(begin + kCellsPerPartial, n);
    double eE = 0.0, eB = 0.0;
    for (long long i = begin + threadIdx.x; i < end; i += kThreads) {
        eE += cell_energy3<T>(f[PSATD_IX(i, 6 * n)], f[PSATD_IX(n + i, 6 * n)], f[PSATD_IX(2 * n + i, 6 * n)]);
        eB += cell_energy3<T>(f[PSATD_IX(3 * n + i, 6 * n)], f[PSATD_IX(4 * n + i, 6 * n)],
                              f[PSATD_IX(5 * n + i, 6 * n)]);
    }
    eE = warp_sum(eE);
    eB = warp_sum(eB);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sE[wid] = eE; sB[wid] = eB; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tE = 0.0, tB = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) { tE += sE[w]; tB += sB[w]; }
        partial[PSATD_IX(2 * blockIdx.x, 2 * kMaxPartials)] = tE;
        partial[PSATD_IX(2 * blockIdx.x + 1, 2 * kMaxPartials)] = tB;
    }
}

// out[0..1] = column sums of partial[nparts][2], in a fixed order
__global__ void __launch_bounds__(kThreads)
energy_final_kernel(const double* __restrict__ partial, int nparts, double* __restrict__ out) {
    __shared__ double sE[kThreads / 32], sB[kThreads / 32];
    double eE = 0.0, eB = 0.0;
    for (int b = threadIdx.x; b < nparts; b += kThreads) {
        eE += partial[PSATD_IX(2 * b, 2 * kMaxPartials)];
        eB += partial[PSATD_IX(2 * b + 1, 2 * kMaxPartials)];
    }
    eE = warp_sum(eE);
    eB = warp_sum(eB);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sE[wid] = eE; sB[wid] = eB; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tE = 0.0, tB = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) { tE += sE[w]; tB += sB[w]; }
        out[0] = tE;
        out[1] = tB;
    }
}

}  // namespace

}  // namespace psatd

using namespace psatd;

extern "C" psatd_status psatd_energy_noalloc(const void* fields, int precision, long long n_cells,
                                             double* out, int out_on_device, void* cuda_stream) {
    if (!fields || !out) return PSATD_ERR_ARG;
    if (precision != 32 && precision != 64) return PSATD_ERR_ARG;
    if (n_cells < 1) return PSATD_ERR_SIZE;
    const long long nparts = (n_cells + kCellsPerPartial - 1) / kCellsPerPartial;
    if (nparts > kMaxPartials) return PSATD_ERR_SIZE;    // more than 2^30 cells
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PSATD_ERR_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_addr[dev]) {
            // The runtime loads kernels lazily, and loading one can allocate
            // device memory; load all three here so that no later call, of
            // either precision, does.
            cudaFuncAttributes fa;
            void* p = nullptr;
            if (cudaFuncGetAttributes(&fa, energy_partials_kernel<float>) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, energy_partials_kernel<double>) != cudaSuccess ||
                cudaFuncGetAttributes(&fa, energy_final_kernel) != cudaSuccess ||
                cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) {
                cudaGetLastError();                        // clear this call's own failure
                return PSATD_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double*>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    // cudaLaunchKernel returns this launch's own error: an error that the
    // caller left pending is neither consumed nor reported here
    int np = (int)nparts;
    double* result = out_on_device ? out : scratch + 2 * (size_t)kMaxPartials;
    void* args_p[] = {const_cast<void**>(&fields), &n_cells, &scratch};
    const void* kp = precision == 64 ? (const void*)energy_partials_kernel<double>
                                     : (const void*)energy_partials_kernel<float>;
    if (cudaLaunchKernel(kp, dim3((unsigned)nparts), dim3(kThreads), args_p, 0, s) != cudaSuccess)
        return PSATD_ERR_CUDA;
    void* args_f[] = {&scratch, &np, &result};
    if (cudaLaunchKernel((const void*)energy_final_kernel, dim3(1), dim3(kThreads), args_f, 0, s) != cudaSuccess)
        return PSATD_ERR_CUDA;
    if (!out_on_device) {
        if (cudaMemcpyAsync(out, result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return PSATD_ERR_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return PSATD_ERR_CUDA;
    }
    return PSATD_OK;
}
