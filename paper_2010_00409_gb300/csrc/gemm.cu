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

// ---------------------------------------------------------------------------
// 5th-generation tensor-core path: tcgen05.mma (kind::f16, bf16 x bf16 -> f32)
// with the accumulator tile in tensor memory.  Block = 128 threads, tile
// 128 (M) x BN (N) x 64 (K).  Per K block the threads round their A and B
// elements to bfloat16 and store them in the no-swizzle K-major layout of the
// tensor core's shared-memory descriptors: 8-row x 16-byte "core matrices"
// (8 rows x 8 bf16 along K, 128 contiguous bytes), core matrix (i, kc) of A at
// kc * (BM/8) * 128 + i * 128 bytes (B alike with BN rows), so the
// leading-dimension offset (between core matrices adjacent along K) is
// (rows/8) * 128 bytes and the stride-dimension offset (between adjacent 8-row
// groups) 128 bytes.  One thread issues the four K = 16 MMAs of the block and
// commits them to an mbarrier that all threads wait on (bounded) before the
// tile is overwritten; after the last block each warp reads its 32 accumulator
// rows from tensor memory (tcgen05.ld, lanes 32w .. 32w + 31).
constexpr int TBM = 128, TBK = 64, kTcThreads = 128;
// operand regions sized so that every descriptor read stays inside the
// block's shared memory whatever the offsets
constexpr int kTcARegion = 48 * 1024, kTcBRegion = 48 * 1024;
constexpr size_t kTcSmem = kTcARegion + kTcBRegion;
__device__ int g_gemm_error;        // set when a bounded wait of the tensor-core GEMM expires

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);           // bits 46-48: 0b001, no swizzle
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = tc_smem(bar);
    for (uint32_t it = 0; it < (1u << 24); ++it) {
        uint32_t ok;
        asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     " selp.u32 %0, 1, 0, p;\n}\n" : "=r"(ok) : "r"(a), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

template <int BN>
__global__ void __launch_bounds__(kTcThreads) gemm_tc_kernel(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    unsigned char* As = tc_raw;
    unsigned char* Bs = tc_raw + kTcARegion;
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mma_bar;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bz = blockIdx.z;
    const int split = bz % g.ksplit;
    const int bidx = bz / g.ksplit;
    const int b0 = bidx / g.nb1, b1 = bidx % g.nb1;
    const float* A = g.A + b0 * g.sAb0 + b1 * g.sAb1;
    const float* B = g.B + b0 * g.sBb0 + b1 * g.sBb1;
    float* C = g.C + b0 * g.sCb0 + b1 * g.sCb1;
    const int m0 = blockIdx.y * TBM, n0 = blockIdx.x * BN;
    const int kchunk = ((g.K + g.ksplit - 1) / g.ksplit + TBK - 1) / TBK * TBK;
    const int kbeg = split * kchunk, kend = min(g.K, kbeg + kchunk);
    const int nkb = kend > kbeg ? (kend - kbeg + TBK - 1) / TBK : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_base)),
                     "r"(BN < 32 ? 32 : BN) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&mma_bar)), "r"(1) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // instruction descriptor: D f32, A and B bf16, both K-major, N = BN, M = 128
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(TBM >> 4) << 24);
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
        if (kb > 0) ok = tc_wait(&mma_bar, (kb - 1) & 1) && ok;     // the previous MMAs have read the tile
        const int k0 = kbeg + kb * TBK;
        // A (TBM x TBK): element (m, k) -> core matrix (m/8, k/8), row m%8, column k%8
        for (int e = tid; e < TBM * TBK; e += kTcThreads) {
            int m, k;
            if (g.sAk == 1) { m = e / TBK; k = e % TBK; } else { k = e / TBM; m = e % TBM; }
            const int gm = m0 + m, gk = k0 + k;
            const float v = (gm < g.M && gk < kend) ? A[gm * g.sAm + gk * g.sAk] : 0.f;
            const int off = (k >> 3) * (TBM / 8) * 128 + (m >> 3) * 128 + (m & 7) * 16 + (k & 7) * 2;
            *reinterpret_cast<__nv_bfloat16*>(As + off) = __float2bfloat16_rn(v);
        }
        // B (TBK x BN) stored as the N x K operand
        for (int e = tid; e < BN * TBK; e += kTcThreads) {
            int n, k;
            if (g.sBn == 1) { k = e / BN; n = e % BN; } else { n = e / TBK; k = e % TBK; }
            const int gn = n0 + n, gk = k0 + k;
            const float v = (gn < g.N && gk < kend) ? B[gk * g.sBk + gn * g.sBn] : 0.f;
            const int off = (k >> 3) * (BN / 8) * 128 + (n >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2;
            *reinterpret_cast<__nv_bfloat16*>(Bs + off) = __float2bfloat16_rn(v);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor-core reads
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < TBK / 16; ++kk) {
                const uint64_t ad = tc_desc(tc_smem(As) + kk * 2 * (TBM / 8) * 128, (TBM / 8) * 128, 128);
                const uint64_t bd = tc_desc(tc_smem(Bs) + kk * 2 * (BN / 8) * 128, (BN / 8) * 128, 128);
                const uint32_t acc = (kb > 0 || kk > 0) ? 1u : 0u;
                asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                             " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                             "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             tc_smem(&mma_bar))
                         : "memory");
        }
    }
    if (nkb > 0) {
        ok = tc_wait(&mma_bar, (nkb - 1) & 1) && ok;
        if (!ok) tc_wait(&mma_bar, (nkb - 1) & 1);     // a second bounded wait for MMAs still in flight
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    // epilogue: row m = 32 warp + lane, 16 columns per tensor-memory load
    const int m = m0 + 32 * warp + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t r[16];
        if (nkb > 0) {
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) r[i] = 0u;
        }
        if (m < g.M) {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int n = n0 + c0 + i;
                if (n < g.N) {
                    float* dst = C + m * g.sCm + n * g.sCn;
                    const float v = g.alpha * __uint_as_float(r[i]);
                    if (g.ksplit > 1) atomicAdd(dst, v);
                    else *dst = (g.beta == 0.f) ? v : v + g.beta * *dst;
                }
            }
        }
    }
    if (!ok && tid == 0) atomicExch(&g_gemm_error, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN < 32 ? 32 : BN)
                     : "memory");
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
#ifdef PSATD_GEMM_TC
    {
        const int bn = g.N <= 32 ? 32 : (g.N <= 64 ? 64 : 128);
        dim3 grid((g.N + bn - 1) / bn, (g.M + TBM - 1) / TBM, g.nb0 * g.nb1 * g.ksplit);
        if (grid.z > 65535) return cudaErrorInvalidValue;
        auto k = bn == 32 ? gemm_tc_kernel<32> : (bn == 64 ? gemm_tc_kernel<64> : gemm_tc_kernel<128>);
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (e != cudaSuccess) return e;
        k<<<grid, kTcThreads, kTcSmem, s>>>(g);
        return cudaGetLastError();
    }
#endif
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.nb0 * g.nb1 * g.ksplit);
    if (grid.z > 65535) return cudaErrorInvalidValue;
    gemm_kernel<<<grid, kThreads, 0, s>>>(g);
    return cudaGetLastError();
}

}  // namespace psatd
