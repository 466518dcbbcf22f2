// Real-field storage helpers.
//
// kspace_x0_kernel: slot 0 of the half spectrum holds, per (k_y, k_z), the
// packed value P = S0 + i SN of the k_x = 0 spectrum S0 and the x Nyquist
// spectrum SN of the real fields (each Hermitian in (k_y, k_z)).  The k-space
// pass leaves the z spectra of slot 0 in side[component][y][k_z]; one block
// takes the pencil at y for all six components, reads its mirror at Ny - y,
// unpacks
//   S0(k) = (P(k) + conj P(-k)) / 2,   SN(k) = (P(k) - conj P(-k)) / (2i),
// applies the update of Sec. 2.1 (Eq. 3-4) to both, with the mean over the
// mirrored Nyquist wave vectors that keeps the fields real (k_x = -pi/dx is a
// Nyquist component of SN), repacks P' = S0' + i SN', transforms back along z
// and stores slot 0 at y.  The data is 1/128 of the field, so the inverse
// transform is the generic shared-memory Stockham one over the 6 pencils.
#include "fft_core.cuh"
#include "fft_reg.cuh"

namespace psatd {

namespace {

constexpr int kX0Threads = 256;

__global__ void __launch_bounds__(kX0Threads)
kspace_x0_kernel(float2* __restrict__ data, const float2* __restrict__ side, int Nh, int Ny, int Nz, AxisPlan pz,
                 const float2* __restrict__ twz,
                 float kx_nyq, const float* __restrict__ kys, const float* __restrict__ kzs,
                 const ModeCoef<float>* __restrict__ coef, int Nxh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* a = reinterpret_cast<float2*>(smem_raw);      // [6][Nz]: component q at q * Nz
    float2* b = a + 6 * Nz;
    const int y = blockIdx.x, ym = (Ny - y) % Ny;          // this pencil and its mirror
    const size_t plane = (size_t)Nh * Ny, cstride = plane * Nz;
    pdl_launch_dependents();
    pdl_wait();

    const int Nyh = Ny / 2 + 1, ax_nyq = Nxh - 1;
    for (int kz = threadIdx.x; kz < Nz; kz += blockDim.x) {
        const int kzm = (Nz - kz) % Nz;
        const int ay = min(y, Ny - y), az = min(kz, Nz - kz);
        const bool fy = (2 * y == Ny), fz = (2 * kz == Nz);
        float2 S0[6], SN[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const float2 P1 = side[((size_t)q * Ny + y) * Nz + kz], P2 = side[((size_t)q * Ny + ym) * Nz + kzm];
            S0[q] = make_float2(0.5f * (P1.x + P2.x), 0.5f * (P1.y - P2.y));
            SN[q] = make_float2(0.5f * (P1.y + P2.y), -0.5f * (P1.x - P2.x));
        }
        const float kyv = kys[y], kzv = kzs[kz];
        const ModeCoef<float> m0 = coef[((size_t)az * Nyh + ay) * Nxh];
        rotate_mode_mean<float>(S0[0], S0[1], S0[2], S0[3], S0[4], S0[5], 0.f, kyv * m0.kinv, kzv * m0.kinv,
                                false, fy, fz, m0.C, m0.S);
        const ModeCoef<float> mn = coef[((size_t)az * Nyh + ay) * Nxh + ax_nyq];
        rotate_mode_mean<float>(SN[0], SN[1], SN[2], SN[3], SN[4], SN[5], kx_nyq * mn.kinv, kyv * mn.kinv,
                                kzv * mn.kinv, true, fy, fz, mn.C, mn.S);
#pragma unroll
        for (int q = 0; q < 6; ++q) a[q * Nz + kz] = make_float2(S0[q].x - SN[q].y, S0[q].y + SN[q].x);
    }
    __syncthreads();
    float2* g = fft_tile<float, +1>(a, b, pz, 6, Nz, twz);
    for (int e = threadIdx.x; e < 6 * Nz; e += blockDim.x) {
        const int z = e % Nz, q = e / Nz;
        data[q * cstride + (size_t)z * plane + (size_t)y * Nh] = g[e];
    }
}

__global__ void widen_kernel(const float* __restrict__ in, float2* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2(in[i], 0.f);
}

__global__ void narrow_kernel(const float2* __restrict__ in, float* __restrict__ out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = in[i].x;
}

unsigned elementwise_blocks(size_t n) {
    const size_t b = (n + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_kspace_x0(float2* data, const GridGeom& g, const Tables<float>& tb, const HalfSlots<float>& hs,
                             cudaStream_t s) {
    const size_t smem = (size_t)2 * 6 * g.Nz * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(kspace_x0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.Ny, 1, 1);
    cfg.blockDim = dim3(kX0Threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;     // may overlap the previous kernel's tail
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kspace_x0_kernel, data, (const float2*)hs.side, g.Nx / 2, g.Ny, g.Nz, tb.plan[2],
                              tb.tw[2], (float)(-3.14159265358979323846 / g.dx), tb.k[1], tb.k[2], hs.coef,
                              g.Nx / 2 + 1);
}

cudaError_t launch_widen(const float* in, float2* out, size_t n, cudaStream_t s) {
    widen_kernel<<<elementwise_blocks(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_narrow(const float2* in, float* out, size_t n, cudaStream_t s) {
    narrow_kernel<<<elementwise_blocks(n), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

}  // namespace psatd
