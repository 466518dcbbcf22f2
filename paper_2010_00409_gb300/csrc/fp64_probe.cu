// FP64 arithmetic rate probe (psatd_fp64_fma_probe).
//
// The float64 solver is bound by the GPU's float64 arithmetic, not by memory,
// so its roofline needs the rate of float64 fused multiply-adds on this GPU.
// Each thread runs eight independent FMA chains (enough independent work per
// warp to keep the float64 pipe busy) and writes one sum, so nothing is dead
// code; 16 floating-point operations per thread and iteration.
#include "../../include/psatd.h"
#include "common.cuh"

namespace psatd {

namespace {

constexpr int kChains = 8;

__global__ void fp64_fma_kernel(double* __restrict__ out, int iters) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    // a contraction toward 1/(1 - b) * c = 2^-4 from distinct starting values
    const double b = 1.0 - 1.0 / 1048576.0, c = 1.0 / 16777216.0;
    double a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = 1e-6 * (double)(t & 1023) + (double)k;
#pragma unroll 4
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], b, c);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; ++k) s += a[k];
    out[t] = s;
}

}  // namespace

}  // namespace psatd

extern "C" psatd_status psatd_fp64_fma_probe(double* out, int blocks, int threads, int iters, void* cuda_stream) {
    if (!out || blocks < 1 || blocks > (1 << 20) || threads < 32 || threads > 1024 || threads % 32 != 0 || iters < 1)
        return PSATD_ERR_ARG;
    psatd::fp64_fma_kernel<<<(unsigned)blocks, (unsigned)threads, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
        out, iters);
    return cudaGetLastError() == cudaSuccess ? PSATD_OK : PSATD_ERR_CUDA;
}
