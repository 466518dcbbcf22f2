// Strided, batched GEMM on the 5th-generation tensor cores for the surrogate
// network:
//   C[b] = alpha * A[b] * B[b] + beta * C[b]
// with A[b](m, k) = A[b0 * sAb0 + b1 * sAb1 + m * sAm + k * sAk] (any strides),
// B[b](k, n) and C[b](m, n) likewise, b = b0 * nb1 + b1.  Inputs and outputs are
// float32 in memory; operands are rounded to bfloat16 when staged in shared
// memory and multiplied by tcgen05.mma (kind::f16, float32 accumulators in
// tensor memory).  Split-K (ksplit > 1) partitions K over tiles and adds partial
// tiles to C with float atomics (C must hold beta * C beforehand; the launcher
// scales it).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace psatd {


namespace {

// ---------------------------------------------------------------------------
// tcgen05.mma (kind::f16, bf16 x bf16 -> f32) with the accumulators in tensor
// memory.  A kernel that allocates tensor memory runs one block per SM, so the
// grid is one persistent block of 512 threads per SM; tile 128 (M) x BN (N), K
// in blocks of 64.  Two-stage pipeline: while the tensor core multiplies the
// operands of one K block, the threads stage the next one, and while the MMAs
// of tile t run, the threads read tile t-1's accumulators (two accumulators of
// BN columns in tensor memory).
//
// Staging: each thread takes 8 consecutive k of one row, rounds them to
// bfloat16 and writes them as one 16-byte row of a "core matrix" (8 rows x 8
// bf16, 128 contiguous bytes) of the no-swizzle K-major layout that the
// shared-memory descriptors describe: core matrix (i, kc) at kc * (rows/8) *
// 128 + i * 128 bytes, so the leading-dimension offset (core matrices adjacent
// along K) is (rows/8) * 128 bytes and the stride-dimension offset (adjacent
// 8-row groups) 128 bytes.  One thread issues the K = 16 MMAs of a K block (as
// many as hold data) and commits them to the stage's mbarrier (the stage may be
// refilled) and, after a tile's last K block, to the accumulator's mbarrier
// (the tile may be read).  All waits are bounded; an expired wait sets
// g_gemm_error (gemm_take_error reads and clears it).
constexpr int TBM = 128, TBK = 64, kTcThreads = 512;
__device__ int g_gemm_error;

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

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_smem(bar))
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

template <int BN> struct TcCfg {
    static constexpr int kStageA = TBM * TBK * 2;             // bytes of one A stage
    static constexpr int kStageB = BN * TBK * 2;
    static constexpr int kSmem = 2 * (kStageA + kStageB);
    static constexpr int kCols = 2 * BN;                      // two accumulators
};

struct TcTile {
    int m0, n0, kbeg, kend, nkb;
    const float* A;
    const float* B;
    float* C;
};

__device__ __forceinline__ TcTile tc_tile(const GemmArgs& g, int tile, int ntm, int ntn, int BN) {
    TcTile t;
    const int mt = tile % ntm;
    const int rest = tile / ntm;
    const int nt = rest % ntn;
    const int bz = rest / ntn;
    const int split = bz % g.ksplit;
    const int bidx = bz / g.ksplit;
    const int b0 = bidx / g.nb1, b1 = bidx % g.nb1;
    t.A = g.A + b0 * g.sAb0 + b1 * g.sAb1;
    t.B = g.B + b0 * g.sBb0 + b1 * g.sBb1;
    t.C = g.C + b0 * g.sCb0 + b1 * g.sCb1;
    t.m0 = mt * TBM;
    t.n0 = nt * BN;
    const int kchunk = ((g.K + g.ksplit - 1) / g.ksplit + TBK - 1) / TBK * TBK;
    t.kbeg = split * kchunk;
    t.kend = min(g.K, t.kbeg + kchunk);
    t.nkb = t.kend > t.kbeg ? (t.kend - t.kbeg + TBK - 1) / TBK : 0;
    return t;
}

// rows x TBK operand block -> bf16 core matrices; element (r, k) of the block is
// src[(r0 + r) * s_r + (k0 + k) * s_k], zero outside rows < nrows, k < kend
// vec: k is the unit-stride axis and every row starts on a 16-byte boundary
// (then 8 consecutive k from a multiple of 8 are two aligned float4 loads)
// Only the first kcs 8-column chunks are staged (the MMAs of a short last K
// block read no further).
template <int ROWS>
__device__ __forceinline__ void tc_stage(unsigned char* dst, const float* __restrict__ src, long long s_r,
                                         long long s_k, int r0, int nrows, int k0, int kend, bool vec, int kcs) {
    const int items = ROWS * kcs;
#pragma unroll 4
    for (int i = threadIdx.x; i < items; i += kTcThreads) {
        const int r = i % ROWS, kc = i / ROWS;
        const int gr = r0 + r, gk = k0 + kc * 8;
        float v[8];
        if (vec && gr < nrows && gk + 8 <= kend) {
            const float4* q4 = reinterpret_cast<const float4*>(src + gr * s_r + gk);
            const float4 a = __ldg(q4), b = __ldg(q4 + 1);
            v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
            v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = (gr < nrows && gk + q < kend) ? src[gr * s_r + (gk + q) * s_k] : 0.f;
        }
        uint4 w;
        w.x = pack_bf16x2(v[0], v[1]);
        w.y = pack_bf16x2(v[2], v[3]);
        w.z = pack_bf16x2(v[4], v[5]);
        w.w = pack_bf16x2(v[6], v[7]);
        *reinterpret_cast<uint4*>(dst + kc * (ROWS / 8) * 128 + (r >> 3) * 128 + (r & 7) * 16) = w;
    }
}

// Epilogue.  Warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (the rows of
// its lane quarter); the kTcThreads / 128 warps of one quarter split the
// columns (cols each), read in loads of 8.  With beta != 0 the thread's C
// values are loaded first (tc_epilogue_c, issued before the wait on the
// accumulator, so their latency overlaps the MMAs).
template <int BN> struct TcEpi {
    static constexpr int parts = kTcThreads / 128, cols = BN / parts;
    static_assert(cols % 8 == 0, "column split");
};

template <int BN>
__device__ __forceinline__ void tc_epilogue_c(const GemmArgs& g, const TcTile& t, float (&cv)[TcEpi<BN>::cols]) {
    constexpr int cols = TcEpi<BN>::cols;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m = t.m0 + 32 * (warp & 3) + lane, c0 = (warp >> 2) * cols;
    const bool need = g.ksplit == 1 && g.beta != 0.f && m < g.M;
#pragma unroll
    for (int i = 0; i < cols; ++i) {
        const int n = t.n0 + c0 + i;
        cv[i] = (need && n < g.N) ? t.C[m * g.sCm + n * g.sCn] : 0.f;
    }
}

template <int BN>
__device__ __forceinline__ void tc_epilogue(const GemmArgs& g, const TcTile& t, uint32_t acc_addr, bool have,
                                            const float (&cv)[TcEpi<BN>::cols]) {
    constexpr int cols = TcEpi<BN>::cols;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int quarter = warp & 3;
    const int m = t.m0 + 32 * quarter + lane, c0 = (warp >> 2) * cols;
#pragma unroll
    for (int cc = 0; cc < cols; cc += 8) {
        uint32_t r[8];
        if (have) {
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7])
                         : "r"(acc_addr + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(c0 + cc)));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) r[i] = 0u;
        }
        if (m < g.M) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int n = t.n0 + c0 + cc + i;
                if (n < g.N) {
                    float* dst = t.C + m * g.sCm + n * g.sCn;
                    const float v = g.alpha * __uint_as_float(r[i]);
                    if (g.ksplit > 1) atomicAdd(dst, v);
                    else *dst = (g.beta == 0.f) ? v : v + g.beta * cv[cc + i];
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

template <int BN>
__global__ void __launch_bounds__(kTcThreads) gemm_tc_kernel(GemmArgs g, int ntm, int ntn, int ntiles) {
    using Cfg = TcCfg<BN>;
    extern __shared__ __align__(1024) unsigned char tc_raw[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t sbar[2], abar[2];
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_base)),
                     "r"(Cfg::kCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&sbar[i])), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&abar[i])), "r"(1) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    // instruction descriptor: D f32, A and B bf16, both K-major, N = BN, M = 128
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                               ((uint32_t)(TBM >> 4) << 24);
    const bool vecA = g.sAk == 1 && (g.sAm & 3) == 0 && (g.sAb0 & 3) == 0 && (g.sAb1 & 3) == 0 &&
                      (reinterpret_cast<uintptr_t>(g.A) & 15) == 0;
    const bool vecB = g.sBk == 1 && (g.sBn & 3) == 0 && (g.sBb0 & 3) == 0 && (g.sBb1 & 3) == 0 &&
                      (reinterpret_cast<uintptr_t>(g.B) & 15) == 0;
    bool ok = true;
    uint32_t it = 0, tl = 0;
    TcTile prev{};
#pragma unroll 1
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tl) {
        // every thread has finished waiting on the accumulator barriers before
        // thread 0 commits to them again (also when a tile has no K block)
        __syncthreads();
        const TcTile t = tc_tile(g, tile, ntm, ntn, BN);
        const uint32_t acc = tmem + (tl & 1) * BN;
#pragma unroll 1
        for (int kb = 0; kb < t.nkb; ++kb, ++it) {
            const int s = it & 1;
            if (it >= 2) ok = tc_wait(&sbar[s], ((it - 2) >> 1) & 1) && ok;     // stage s read by the MMAs
            unsigned char* As = tc_raw + s * (Cfg::kStageA + Cfg::kStageB);
            unsigned char* Bs = As + Cfg::kStageA;
            const int k0 = t.kbeg + kb * TBK;
            const int nkk = min(TBK / 16, (t.kend - k0 + 15) / 16);         // K = 16 MMAs with data
            tc_stage<TBM>(As, t.A, g.sAm, g.sAk, t.m0, g.M, k0, t.kend, vecA, 2 * nkk);
            tc_stage<BN>(Bs, t.B, g.sBn, g.sBk, t.n0, g.N, k0, t.kend, vecB, 2 * nkk);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> tensor-core reads
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                for (int kk = 0; kk < nkk; ++kk) {
                    const uint64_t ad = tc_desc(tc_smem(As) + kk * 2 * (TBM / 8) * 128, (TBM / 8) * 128, 128);
                    const uint64_t bd = tc_desc(tc_smem(Bs) + kk * 2 * (BN / 8) * 128, (BN / 8) * 128, 128);
                    const uint32_t accum = (kb > 0 || kk > 0) ? 1u : 0u;
                    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                                 "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                                 : "memory");
                }
                tc_commit(&sbar[s]);
            }
        }
        if (tid == 0) tc_commit(&abar[tl & 1]);          // this tile's accumulator (immediate when nkb = 0)
        if (tl > 0) {                                     // read the previous tile while these MMAs run
            float cv[TcEpi<BN>::cols];
            tc_epilogue_c<BN>(g, prev, cv);
            ok = tc_wait(&abar[(tl - 1) & 1], ((tl - 1) >> 1) & 1) && ok;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            tc_epilogue<BN>(g, prev, tmem + ((tl - 1) & 1) * BN, prev.nkb > 0, cv);
        }
        prev = t;
    }
    if (tl > 0) {
        float cv[TcEpi<BN>::cols];
        tc_epilogue_c<BN>(g, prev, cv);
        ok = tc_wait(&abar[(tl - 1) & 1], ((tl - 1) >> 1) & 1) && ok;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        tc_epilogue<BN>(g, prev, tmem + ((tl - 1) & 1) * BN, prev.nkb > 0, cv);
    }
    if (!ok) {
        if (tid == 0) atomicExch(&g_gemm_error, 1);
        // second bounded waits: no MMA may still write the accumulators at dealloc
        for (int i = 0; i < 2; ++i) tc_wait(&abar[i], 0), tc_wait(&abar[i], 1);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Cfg::kCols) : "memory");
}

// ---------------------------------------------------------------------------
// bf16 operands in memory, fed by the tensor copy engine: C = A B^T with A (M x
// K) and B (N x K) both K-major bf16, C (M x N) row-major float32.  Tile 128 x
// 256, K in blocks of 64 (128 bytes of bf16 per row, one 128-byte swizzle
// atom), four stages of 48 KB.  Warp 0 (one lane) issues the tensor copies of
// a stage once the MMAs have released it; warp 1 (one lane) issues the four
// K = 16 MMAs of each stage into one of two accumulators of 256 columns in
// tensor memory and commits the stage back to the producer and, after a tile's
// last stage, the accumulator to the epilogue; warps 2-5 read the accumulator
// (warp w reads lanes 32 (w % 4) .. + 31, i.e. rows of its quarter) and store
// the rows, then hand the accumulator back.  Tiles are visited in groups of 16
// along M so that the tiles in flight share operand rows in L2.
//
// Shared-memory operands are in the canonical K-major 128-byte-swizzle layout
// that the copy engine writes with CU_TENSOR_MAP_SWIZZLE_128B: row r of a
// block at r * 128 bytes, 8-row atoms of 1024 bytes (the descriptor's stride
// offset), 16-byte chunks permuted within a row by the copy engine; the K = 16
// steps inside the atom advance the descriptor's start address by 32 bytes.
#ifndef PSATD_GT_GROUP_M
#define PSATD_GT_GROUP_M 16
#endif
constexpr int GT_BM = 128, GT_BN = 256, GT_BK = 64, GT_STAGES = 4, GT_THREADS = 192, GT_GROUP_M = PSATD_GT_GROUP_M;
constexpr int GT_STAGE_A = GT_BM * GT_BK * 2, GT_STAGE_B = GT_BN * GT_BK * 2;
constexpr int GT_STAGE = GT_STAGE_A + GT_STAGE_B;
constexpr int GT_SMEM = GT_STAGES * GT_STAGE + 1024;           // + alignment slack
constexpr int GT_TMEM_COLS = 2 * GT_BN;

__device__ __forceinline__ uint64_t gt_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);                       // version 1, 128-byte swizzle
}

__device__ __forceinline__ void gt_arrive_expect(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void gt_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(bar)) : "memory");
}

__device__ __forceinline__ void gt_load(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(tc_smem(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(tc_smem(bar))
        : "memory");
}

__device__ __forceinline__ void gt_tile(int tile, int ntm, int ntn, int* mt, int* nt) {
    const int per_group = GT_GROUP_M * ntn;
    const int gi = tile / per_group, in = tile - gi * per_group;
    const int m_first = gi * GT_GROUP_M;
    const int gm = min(GT_GROUP_M, ntm - m_first);
    *mt = m_first + in % gm;
    *nt = in / gm;
}

__global__ void __launch_bounds__(GT_THREADS, 1)
gemm_tma_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_b,
                float* __restrict__ C, int M, int N, int K, int ntm, int ntn) {
    extern __shared__ __align__(1024) unsigned char gt_raw[];
    __shared__ __align__(8) uint64_t full[GT_STAGES], empty[GT_STAGES], afull[2], aempty[2];
    __shared__ uint32_t tmem_base;
    __shared__ int any_err;
    unsigned char* smem = gt_raw + ((1024 - (tc_smem(gt_raw) & 1023)) & 1023);   // 1024-byte aligned stages
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = ntm * ntn, nkb = K / GT_BK;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&tmem_base)),
                     "r"(GT_TMEM_COLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 32) {
        for (int i = 0; i < GT_STAGES; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&full[i])), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&empty[i])), "r"(1) : "memory");
        }
        for (int i = 0; i < 2; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&afull[i])), "r"(1) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(&aempty[i])), "r"(4) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        any_err = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    bool ok = true;

    if (warp == 0) {
        if (lane == 0) {                                   // producer: tensor copies
            uint32_t it = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
                int mt, nt;
                gt_tile(tile, ntm, ntn, &mt, &nt);
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % GT_STAGES;
                    ok = tc_wait(&empty[s], ((it / GT_STAGES) & 1) ^ 1) && ok;
                    unsigned char* sa = smem + s * GT_STAGE;
                    gt_arrive_expect(&full[s], GT_STAGE);
                    gt_load(sa, &map_a, &full[s], kb * GT_BK, mt * GT_BM);
                    gt_load(sa + GT_STAGE_A, &map_b, &full[s], kb * GT_BK, nt * GT_BN);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {                                   // MMA issue
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GT_BN >> 3) << 17) |
                                       ((uint32_t)(GT_BM >> 4) << 24);
            uint32_t it = 0, tl = 0;
            for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tl) {
                const int acc = tl & 1;
                ok = tc_wait(&aempty[acc], ((tl >> 1) & 1) ^ 1) && ok;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + acc * GT_BN;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int s = it % GT_STAGES;
                    ok = tc_wait(&full[s], (it / GT_STAGES) & 1) && ok;
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = tc_smem(smem + s * GT_STAGE), sb = sa + GT_STAGE_A;
#pragma unroll
                    for (int kk = 0; kk < GT_BK / 16; ++kk) {
                        const uint64_t ad = gt_desc(sa + kk * 32), bd = gt_desc(sb + kk * 32);
                        const uint32_t accum = (kb > 0 || kk > 0) ? 1u : 0u;
                        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                                     " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
                                     "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                                     : "memory");
                    }
                    tc_commit(&empty[s]);                  // the stage is free once these MMAs have read it
                }
                tc_commit(&afull[acc]);                    // the tile's accumulator is complete
            }
        }
    } else {                                               // epilogue: warps 2-5
        const int q = warp & 3;
        uint32_t tl = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++tl) {
            int mt, nt;
            gt_tile(tile, ntm, ntn, &mt, &nt);
            const int acc = tl & 1;
            ok = tc_wait(&afull[acc], (tl >> 1) & 1) && ok;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m = mt * GT_BM + 32 * q + lane;
            float* row = C + (size_t)m * N + (size_t)nt * GT_BN;
            const uint32_t base = tmem + ((uint32_t)(32 * q) << 16) + acc * GT_BN;
#pragma unroll 1
            for (int c = 0; c < GT_BN; c += 16) {
                uint32_t r[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15])
                    : "r"(base + (uint32_t)c));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float4* dst = reinterpret_cast<float4*>(row + c);
#pragma unroll
                for (int v = 0; v < 4; ++v)
                    dst[v] = make_float4(__uint_as_float(r[4 * v]), __uint_as_float(r[4 * v + 1]),
                                         __uint_as_float(r[4 * v + 2]), __uint_as_float(r[4 * v + 3]));
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) gt_arrive(&aempty[acc]);        // the MMAs may write this accumulator again
        }
    }
    if (!ok) {
        atomicExch(&g_gemm_error, 1);
        any_err = 1;
    }
    __syncthreads();
    if (any_err && threadIdx.x == 0) {
        // an expired wait left the pipeline out of step: second bounded waits so
        // that no copy or MMA is still in flight when the block leaves
        for (int i = 0; i < 2; ++i) tc_wait(&afull[i], 0), tc_wait(&afull[i], 1);
        for (int i = 0; i < GT_STAGES; ++i) tc_wait(&full[i], 0), tc_wait(&full[i], 1);
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(GT_TMEM_COLS)
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
    // The epilogue writes one row per lane, so it coalesces when C is
    // column-major; a row-major C (or, for other layouts, M < N: the tile is 128
    // rows by at most 128 columns) is handled as C^T = B^T A^T, a relabelling
    // of the same products.
    if (g.sCm != 1 && (g.sCn == 1 || g.M < g.N)) {
        GemmArgs t = g;
        t.M = g.N; t.N = g.M;
        t.A = g.B; t.sAb0 = g.sBb0; t.sAb1 = g.sBb1; t.sAm = g.sBn; t.sAk = g.sBk;
        t.B = g.A; t.sBb0 = g.sAb0; t.sBb1 = g.sAb1; t.sBk = g.sAk; t.sBn = g.sAm;
        t.sCm = g.sCn; t.sCn = g.sCm;
        g = t;
    }
    {
        const int bn = g.N <= 32 ? 32 : (g.N <= 64 ? 64 : 128);
        const int bi = bn == 32 ? 0 : (bn == 64 ? 1 : 2);
        const long long ntm = (g.M + TBM - 1) / TBM, ntn = (g.N + bn - 1) / bn;
        const long long ntiles = ntm * ntn * (long long)g.nb0 * g.nb1 * g.ksplit;
        if (ntiles > 0x7fffffffLL) return cudaErrorInvalidValue;
        auto k = bi == 0 ? gemm_tc_kernel<32> : (bi == 1 ? gemm_tc_kernel<64> : gemm_tc_kernel<128>);
        const int smem = bi == 0 ? TcCfg<32>::kSmem : (bi == 1 ? TcCfg<64>::kSmem : TcCfg<128>::kSmem);
        // one resident block per SM (a kernel that allocates tensor memory runs
        // one block per SM), persistent over the tiles
        static int sms = 0, per_sm[3] = {0, 0, 0}, smem_launch[3] = {0, 0, 0};
        if (!per_sm[bi]) {
            int dev = 0;
            cudaGetDevice(&dev);
            if (!sms) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (sms < 1) sms = 1;
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
            int occ = 0;
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, kTcThreads, smem);
            if (e != cudaSuccess) return e;
            if (occ < 1) return cudaErrorInvalidConfiguration;
            per_sm[bi] = occ;
            smem_launch[bi] = smem;
        }
        const long long cap = (long long)sms * per_sm[bi];
        const long long grid = ntiles < cap ? ntiles : cap;
        k<<<(unsigned)grid, kTcThreads, smem_launch[bi], s>>>(g, (int)ntm, (int)ntn, (int)ntiles);
        return cudaGetLastError();
    }
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 gemm_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2D map of a K-major bf16 matrix (rows x K), box 64 (K) x box_rows, 128-byte swizzle
bool gemm_map(CUtensorMap* map, const void* ptr, int rows, int K, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = gemm_map_encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)GT_BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}
}  // namespace

cudaError_t launch_gemm_tma(const void* A, const void* B, float* C, int M, int N, int K, cudaStream_t s) {
    if (M % GT_BM || N % GT_BN || K % GT_BK || M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) | reinterpret_cast<uintptr_t>(C)) & 15)
        return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!gemm_map(&ma, A, M, K, GT_BM) || !gemm_map(&mb, B, N, K, GT_BN)) return cudaErrorInvalidValue;
    static int sms = 0;
    static bool attr = false;
    if (!attr) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms < 1) sms = 1;
        const cudaError_t e = cudaFuncSetAttribute(gemm_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   GT_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int ntm = M / GT_BM, ntn = N / GT_BN;
    const long long ntiles = (long long)ntm * ntn;
    const int grid = (int)(ntiles < sms ? ntiles : sms);
    gemm_tma_kernel<<<grid, GT_THREADS, GT_SMEM, s>>>(ma, mb, C, M, N, K, ntm, ntn);
    return cudaGetLastError();
}

// Read and clear the flag of an expired bounded wait in the GEMM kernel
// (synchronises the device).
bool gemm_take_error() {
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, g_gemm_error, sizeof(int)) != cudaSuccess) return false;
    if (h) {
        const int zero = 0;
        cudaMemcpyToSymbol(g_gemm_error, &zero, sizeof(int));
    }
    return h != 0;
}

}  // namespace psatd
