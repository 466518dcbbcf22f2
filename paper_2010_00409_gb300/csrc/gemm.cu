// Strided, batched GEMM on the tensor cores for the surrogate network:
//   C[b] = alpha * A[b] * B[b] + beta * C[b]
// with A[b](m, k) = A[b0 * sAb0 + b1 * sAb1 + m * sAm + k * sAk] (any strides),
// B[b](k, n) and C[b](m, n) likewise, b = b0 * nb1 + b1.  Inputs and outputs are
// float32 in memory; tiles are rounded to bfloat16 when staged in shared memory
// and multiplied with mma.sync m16n8k16 (bf16 x bf16 -> f32 accumulate).
// Split-K (ksplit > 1) partitions K over blocks and adds partial tiles to C with
// float atomics (C must hold beta * C beforehand; the launcher scales it).
#include <cuda_bf16.h>

#include "common.cuh"

namespace psatd {


namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int PAD = 8;            // bf16 elements of padding per shared row
constexpr int kThreads = 128;     // 4 warps, each a 32 x 32 sub-tile

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__global__ void __launch_bounds__(kThreads) gemm_kernel(GemmArgs g) {
    __shared__ __align__(16) __nv_bfloat16 As[BM][BK + PAD];     // [m][k]
    __shared__ __align__(16) __nv_bfloat16 Bs[BN][BK + PAD];     // [n][k]
    const int bz = blockIdx.z;
    const int split = bz % g.ksplit;
    const int bidx = bz / g.ksplit;
    const int b0 = bidx / g.nb1, b1 = bidx % g.nb1;
    const float* A = g.A + b0 * g.sAb0 + b1 * g.sAb1;
    const float* B = g.B + b0 * g.sBb0 + b1 * g.sBb1;
    float* C = g.C + b0 * g.sCb0 + b1 * g.sCb1;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kchunk = ((g.K + g.ksplit - 1) / g.ksplit + BK - 1) / BK * BK;
    const int kbeg = split * kchunk, kend = min(g.K, kbeg + kchunk);

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int grp = lane >> 2, tig = lane & 3;
    float acc[2][4][4] = {};

    for (int k0 = kbeg; k0 < kend; k0 += BK) {
        // stage A (BM x BK) and B (BK x BN, stored transposed) as bf16
        for (int e = tid; e < BM * BK; e += kThreads) {
            int m, k;
            if (g.sAk == 1) { m = e / BK; k = e % BK; } else { k = e / BM; m = e % BM; }
            const int gm = m0 + m, gk = k0 + k;
            const float v = (gm < g.M && gk < kend) ? A[gm * g.sAm + gk * g.sAk] : 0.f;
            As[m][k] = __float2bfloat16_rn(v);
        }
        for (int e = tid; e < BN * BK; e += kThreads) {
            int n, k;
            if (g.sBn == 1) { k = e / BN; n = e % BN; } else { n = e / BK; k = e % BK; }
            const int gn = n0 + n, gk = k0 + k;
            const float v = (gn < g.N && gk < kend) ? B[gk * g.sBk + gn * g.sBn] : 0.f;
            Bs[n][k] = __float2bfloat16_rn(v);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + grp;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * tig]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * tig]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * tig + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * tig + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int cidx = wn + j * 8 + grp;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[cidx][kk + 2 * tig]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[cidx][kk + 2 * tig + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int m = m0 + wm + i * 16 + grp + (h >= 2 ? 8 : 0);
                const int n = n0 + wn + j * 8 + 2 * tig + (h & 1);
                if (m < g.M && n < g.N) {
                    float* dst = C + m * g.sCm + n * g.sCn;
                    const float v = g.alpha * acc[i][j][h];
                    if (g.ksplit > 1) atomicAdd(dst, v);
                    else *dst = (g.beta == 0.f) ? v : v + g.beta * *dst;
                }
            }
}

__global__ void scale_kernel(GemmArgs g) {
    const long long total = (long long)g.nb0 * g.nb1 * g.M * g.N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(e % g.N);
        const long long r = e / g.N;
        const int m = (int)(r % g.M);
        const long long b = r / g.M;
        const int b0 = (int)(b / g.nb1), b1 = (int)(b % g.nb1);
        float* dst = g.C + b0 * g.sCb0 + b1 * g.sCb1 + m * g.sCm + n * g.sCn;
        *dst = g.beta == 0.f ? 0.f : g.beta * *dst;
    }
}

}  // namespace

cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t s) {
    if (a.M <= 0 || a.N <= 0 || a.nb0 <= 0 || a.nb1 <= 0) return cudaSuccess;
    GemmArgs g = a;
    if (g.ksplit < 1) g.ksplit = 1;
    if (g.K <= 0) g.ksplit = 1;
    if (g.ksplit > 1) {
        scale_kernel<<<1024, 256, 0, s>>>(g);
    }
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.nb0 * g.nb1 * g.ksplit);
    if (grid.z > 65535) return cudaErrorInvalidValue;
    gemm_kernel<<<grid, kThreads, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace psatd
