// Real-field storage helpers: real <-> complex copies for the operations that
// run on a complex scratch copy of real fields (init, sampling, diagnostics).
#include "common.cuh"

namespace psatd {

namespace {

__global__ void widen_kernel(const float* __restrict__ in, float2* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[PSATD_IX(i, n)] = make_float2(in[PSATD_IX(i, n)], 0.f);
}

__global__ void narrow_kernel(const float2* __restrict__ in, float* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[PSATD_IX(i, n)] = in[PSATD_IX(i, n)].x;
}

unsigned elementwise_blocks(size_t n) {
    const size_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_widen(const float* in, float2* out, size_t n, cudaStream_t s) {
    widen_kernel<<<elementwise_blocks(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const float2* in, float* out, size_t n, cudaStream_t s) {
    narrow_kernel<<<elementwise_blocks(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace psatd
