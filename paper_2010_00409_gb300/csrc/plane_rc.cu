// Plane transforms of REAL fields (FP32, 256 x 256 planes) for the real-storage
// step: one HBM read and one write per x-y plane, in place.
//
// A real row x[0..256) is read as 128 complex z[n] = x[2n] + i x[2n+1].  Its
// 128-point transform is split as n = j + 8 n1, k = k1 + 16 k2 (j < 8, n1 < 16,
// k1 < 16, k2 < 8):  stage A = 16-point DFT over n1 and twiddle W_128^{j k1}
// (in the registers of lane j), stage B = 8-point DFT over j.  The real-to-
// complex step pairs Z[k] with Z[128-k]:
//   X[k] = (Z[k] + conj Z[128-k])/2 + W_256^k (Z[k] - conj Z[128-k])/(2i),
// and X[0], X[128] (both real) share slot 0 as X[0] + i X[128] through the y
// transform; block 0 then unpacks the column with its mirror k_y
//   S0 = (P(k_y) + conj P(-k_y)) / 2,   SN = (P(k_y) - conj P(-k_y)) / (2i)
// and stores S0 (the k_x = 0 spectrum) in slot 0 and SN (the x Nyquist spectrum)
// in a separate array nyq[plane][k_y]; the inverse repacks S0 + i SN pointwise.
//
// A cluster of 8 blocks owns one plane.  Block r owns the stage-A outputs with
// k1 in {r, 16-r} (block 0: {0, 8}); those are exactly the k that pair with each
// other, so the exchange between the blocks (distributed shared memory) is also
// the transpose of the 128-point transform.  Block r stores its 16 spectral
// columns at slots 16 r .. 16 r + 15: slot p = 16 r + 8 s + k2 holds
// X[k1(r, s) + 16 k2] with k1(r, 0) = r, k1(r, 1) = 16 - r (k1(0, 1) = 8).
// The spectrum between the plane kernels is kept in this slot order; the
// k-space kernels read the slot's wave number from a table.
//
// Forward (r2c):   phase 1  rows of block r (32 per block): stage A, scatter to
//                           the owners of k1;  cluster barrier;
//                  phase 2a one thread per row: stage B and the r2c pairing,
//                           in place;
//                  phase 2b the 16 columns along y (256 points), in place
//                           exchange, stores of 128-byte row segments.
// Inverse (c2r) is the mirror: inverse y on the block's 16 columns, the c2r
// pairing and inverse stage B per row, scatter to the owners of the rows,
// cluster barrier, inverse stage A per row, stores.
//
// Shared memory: one 32 KB tile per block of 16-byte pairs.  In the row
// layout, row y holds its 16 columns as 8 pairs, column c = 2 p + s in half s of
// pair p, pair p at y * 8 + (p ^ (y & 7)): the two values a thread sends to one
// owner, or reads back for one stage-B input, move as one 16-byte access, and
// every access pattern above runs at the minimum number of wavefronts (rows of
// a warp spread over the eight bank groups).  The inverse's exchange target is
// [j][sender q][row] with the pair of row yl at (j * 8 + q) * 32 + (yl ^ j): the
// 32 lanes of one remote store write one contiguous 512-byte block (remote
// stores scattered over 32 rows cost about twice the kernel's time).
#include <cooperative_groups.h>

#include "fft_reg.cuh"
#include "tma.cuh"

namespace cg = cooperative_groups;

namespace psatd {

namespace {

constexpr int kRcThreads = 256;
constexpr int kRcC = 8;               // blocks per plane (cluster size)
constexpr int kM = 128;               // complex elements per row
constexpr int kNy = 256;
// row layout: pair p of row y (float4 index), element (y, c = 2 p + s) (float2 index)
__device__ __forceinline__ int pr8(int row, int p) { return row * 8 + (p ^ (row & 7)); }
__device__ __forceinline__ int el16(int row, int c) { return 2 * pr8(row, c >> 1) + (c & 1); }
// the slot (column of the stored spectrum, within the block's 16) of tile column c
__device__ __forceinline__ int slot_of_col(int c) { return 8 * (c & 1) + (c >> 1); }

// the two stage-A outputs k1 owned by block o (half s of its pairs)
constexpr int k1_of(int o, int s) { return o == 0 ? 8 * s : (s ? 16 - o : o); }

__device__ __forceinline__ float4 pack2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// Field loads and stores of the plane kernels.  Each field value is read once
// and written once per launch.
#ifndef PSATD_RC_LD
#define PSATD_RC_LD 0
#endif
__device__ __forceinline__ float2 ld_field(const float2* p) {
#if PSATD_RC_LD == 1
    return __ldcs(p);
#elif PSATD_RC_LD == 2
    float2 v;
    asm volatile("ld.global.nc.L1::no_allocate.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
#else
    return *p;
#endif
}
__device__ __forceinline__ void st_field(float2* p, float2 v) {
#if PSATD_RC_LD >= 1
    __stcs(p, v);
#else
    *p = v;
#endif
}

// W_256^k for compile-time k
template <int K> __device__ __forceinline__ float2 w256() {
    constexpr UnitF w = unit_f32(ct_cos2pi(K, 256), -ct_sin2pi(K, 256));
    return make_float2(w.c, w.s);
}

// r2c pairing of Z = Z[k] and P = Z[128-k] with w = W_256^k: returns X[k] in *a
// and X[128-k] in *b.
__device__ __forceinline__ void r2c_pair(float2 Z, float2 P, float2 w, float2* a, float2* b) {
    const float2 A = make_float2(0.5f * (Z.x + P.x), 0.5f * (Z.y - P.y));
    const float2 Bv = make_float2(0.5f * (Z.y + P.y), -0.5f * (Z.x - P.x));
    const float2 T = cmul(w, Bv);
    *a = make_float2(A.x + T.x, A.y + T.y);
    *b = make_float2(A.x - T.x, T.y - A.y);           // conj(A - T)
}

// c2r pairing of X = X[k] and P = X[128-k] with w = W_256^k (the inverse uses
// W_256^{-k} = conj w): Z2[k] in *a, Z2[128-k] in *b, where
//   Z2[k] = (X + conj P) + i W^{-k} (X - conj P)
__device__ __forceinline__ void c2r_pair(float2 X, float2 P, float2 w, float2* a, float2* b) {
    const float2 Pp = make_float2(X.x + P.x, X.y - P.y);
    const float2 Q = make_float2(X.x - P.x, X.y + P.y);
    const float2 U = cmulc(Q, w);
    *a = make_float2(Pp.x - U.y, Pp.y + U.x);
    *b = make_float2(Pp.x + U.y, U.x - Pp.y);         // conj(Pp - i U)
}

// ---------------------------------------------------------------------------
// Phases of one plane.

// r2c phase 1 compute: stage A over n1 of the row segment in v (lane j holds
// z[j + 8 n1]) and the twiddles W_128^{j k1}.
__device__ __forceinline__ void r2c_stage_a(float2 (&v)[16], int j, const float2* __restrict__ twx) {
    const GBuf<const float2> TX{twx, 256};
    reg_dft<float, -1, 16>(v);
    static_for<1, 16>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value;
        if (j) v[k1] = cmul(v[k1], TX[2 * j * k1]);
    });
}

// r2c phase 1 exchange: row y's outputs k1 to the block that owns k1, the two
// outputs of one owner as one 16-byte store (pair j of row y).
__device__ __forceinline__ void r2c_scatter(const float2 (&v)[16], cg::cluster_group& cluster, float4* tile4, int y,
                                            int j) {
    static_for<0, 8>([&](auto oc) {
        constexpr int o = decltype(oc)::value;
        float4* dst = cluster.map_shared_rank(tile4, o);
        dst[pr8(y, j)] = pack2(v[k1_of(o, 0)], v[k1_of(o, 1)]);
    });
}

// r2c phases 2a and 2b on the block's 16 columns (the tile holds the
// exchanged stage-A outputs), spectra stored to `plane`, block 0's x Nyquist
// column to nq.
__device__ __forceinline__ void r2c_columns(float4* tile4, float2* col0, int r, int tid, const float2* __restrict__ twx,
                                            const float2* __restrict__ twy, float2* __restrict__ plane,
                                            float2* __restrict__ nq, const GBuf<float2>& F,
                                            const GBuf<float2>& NQ) {
    const GBuf<const float2> TX{twx, 256};
    float2* tile = reinterpret_cast<float2*>(tile4);
    // ---------------- phase 2a: stage B and the r2c pairing, one row per thread
    {
        const int y = tid;
        float2 a[2][8];
        static_for<0, 8>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            const float4 q = tile4[pr8(y, j)];
            a[0][j] = make_float2(q.x, q.y);
            a[1][j] = make_float2(q.z, q.w);
        });
        static_for<0, 2>([&](auto sc) { reg_dft<float, -1, 8>(a[decltype(sc)::value]); });   // a[s][k2] = Z[k1(r, s) + 16 k2]
        // the pairing is done in place: each pair (k, 128 - k) is read and
        // written at the same two registers
        if (r == 0) {
            a[0][0] = make_float2(a[0][0].x + a[0][0].y, a[0][0].x - a[0][0].y);   // X[0] + i X[128]
            static_for<1, 5>([&](auto kc) {            // k = 16 k2 pairs with 16 (8 - k2)
                constexpr int k2 = decltype(kc)::value;
                r2c_pair(a[0][k2], a[0][8 - k2], w256<16 * k2>(), &a[0][k2], &a[0][8 - k2]);
            });
            static_for<0, 4>([&](auto kc) {            // k = 8 + 16 k2 pairs with 8 + 16 (7 - k2)
                constexpr int k2 = decltype(kc)::value;
                r2c_pair(a[1][k2], a[1][7 - k2], w256<8 + 16 * k2>(), &a[1][k2], &a[1][7 - k2]);
            });
        } else {
            static_for<0, 8>([&](auto kc) {            // k = r + 16 k2 pairs with (16 - r) + 16 (7 - k2)
                constexpr int k2 = decltype(kc)::value;
                r2c_pair(a[0][k2], a[1][7 - k2], TX[r + 16 * k2], &a[0][k2], &a[1][7 - k2]);
            });
        }
        static_for<0, 8>([&](auto kc) {               // column 2 k2 + s: slot 8 s + k2
            constexpr int k2 = decltype(kc)::value;
            tile4[pr8(y, k2)] = pack2(a[0][k2], a[1][k2]);
        });
    }
    __syncthreads();

    // ---------------- phase 2b: 256-point transforms of the 16 columns along y
    {
        const int c = tid & 15, jy = tid >> 4;
        float2 v[16];
        static_for<0, 16>([&](auto nc) { v[decltype(nc)::value] = tile[el16(jy + 16 * decltype(nc)::value, c)]; });
        stage_a_fwd<float, -1, 16, 16>(v, jy, twy);
        // element (k1, jy) at row 16 k1 + jy: the positions this thread just read
        static_for<0, 16>([&](auto kc) { tile[el16(16 * decltype(kc)::value + jy, c)] = v[decltype(kc)::value]; });
        __syncthreads();
        static_for<0, 16>([&](auto jc) { v[decltype(jc)::value] = tile[el16(16 * jy + decltype(jc)::value, c)]; });
        reg_dft<float, -1, 16>(v);                     // v[k2] = Y[jy + 16 k2]
        if (r == 0) {                                  // unpack slot 0 = column 0 (block-uniform branch)
            if (c == 0) static_for<0, 16>([&](auto kc) { col0[jy + 16 * decltype(kc)::value] = v[decltype(kc)::value]; });
            __syncthreads();
            if (c == 0) {
                static_for<0, 16>([&](auto kc) {
                    constexpr int k2 = decltype(kc)::value;
                    const int ky = jy + 16 * k2;
                    const float2 P = v[k2], Pm = col0[(kNy - ky) & (kNy - 1)];
                    v[k2] = make_float2(0.5f * (P.x + Pm.x), 0.5f * (P.y - Pm.y));
                    NQ.at(nq, ky) = make_float2(0.5f * (P.y + Pm.y), -0.5f * (P.x - Pm.x));
                });
            }
        }
        float2* out = plane + 16 * r + slot_of_col(c);
        static_for<0, 16>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            st_field(&F.at(out, (long long)(jy + 16 * k2) * kM), v[k2]);
        });
    }
}

// c2r phase 1: inverse y on the block's slots from v (thread (c, jy) holds
// slot 16 r + slot_of_col(c) at rows jy + 16 k2), block 0 repacks slot 0 as
// S0 + i SN first; the column results end in the tile in the row layout.
__device__ __forceinline__ void c2r_columns(float2 (&v)[16], float2* tile, int r, int c, int jy,
                                            const float2* __restrict__ twy, const float2* __restrict__ nq,
                                            const GBuf<const float2>& NQ) {
    const GBuf<const float2> TY{twy, 256};
    if (r == 0 && c == 0) {                            // repack slot 0: S0 + i SN
        static_for<0, 16>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            const float2 sn = NQ.at(nq, jy + 16 * k2);
            v[k2] = make_float2(v[k2].x - sn.y, v[k2].y + sn.x);
        });
    }
    reg_dft<float, +1, 16>(v);                         // over k2, k1 = jy
    static_for<0, 16>([&](auto nc) {
        constexpr int n2 = decltype(nc)::value;
        float2 val = v[n2];
        if (n2 > 0 && jy > 0) val = cmulc(val, TY[n2 * jy]);
        tile[el16(16 * jy + n2, c)] = val;              // element (k1 = jy, n2)
    });
    __syncthreads();
    static_for<0, 16>([&](auto kc) { v[decltype(kc)::value] = tile[el16(16 * decltype(kc)::value + jy, c)]; });
    reg_dft<float, +1, 16>(v);                         // v[n1] = y[jy + 16 n1]
    static_for<0, 16>([&](auto nc) { tile[el16(jy + 16 * decltype(nc)::value, c)] = v[decltype(nc)::value]; });
}

// c2r phase 1b: c2r pairing and inverse stage B of row y = tid, then the
// exchange of the rows to their owners (arrives on and waits for the cluster
// barrier that frees every block's tile).
__device__ __forceinline__ void c2r_rows(float4* tile4, cg::cluster_group& cluster, int r, int tid,
                                         const float2* __restrict__ twx) {
    const GBuf<const float2> TX{twx, 256};
    const int y = tid;
    float2 x[2][8];
    static_for<0, 8>([&](auto kc) {
        constexpr int k2 = decltype(kc)::value;
        const float4 q = tile4[pr8(y, k2)];
        x[0][k2] = make_float2(q.x, q.y);
        x[1][k2] = make_float2(q.z, q.w);
    });
    cluster.barrier_arrive();                          // this block's tile is free for the remote stores
    float2 z[2][8];
    if (r == 0) {
        z[0][0] = make_float2(x[0][0].x + x[0][0].y, x[0][0].x - x[0][0].y);   // X[0] = re, X[128] = im
        static_for<1, 5>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            c2r_pair(x[0][k2], x[0][8 - k2], w256<16 * k2>(), &z[0][k2], &z[0][8 - k2]);
        });
        static_for<0, 4>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            c2r_pair(x[1][k2], x[1][7 - k2], w256<8 + 16 * k2>(), &z[1][k2], &z[1][7 - k2]);
        });
    } else {
        static_for<0, 8>([&](auto kc) {
            constexpr int k2 = decltype(kc)::value;
            c2r_pair(x[0][k2], x[1][7 - k2], TX[r + 16 * k2], &z[0][k2], &z[1][7 - k2]);
        });
    }
    const int k1s[2] = {r == 0 ? 0 : r, r == 0 ? 8 : 16 - r};
    static_for<0, 2>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        reg_dft<float, +1, 8>(z[s]);                   // over k2 -> j
        const int k1 = k1s[s];
        static_for<1, 8>([&](auto jc) {
            constexpr int j = decltype(jc)::value;
            if (k1) z[s][j] = cmulc(z[s][j], TX[2 * j * k1]);
        });
    });
    cluster.barrier_wait();
    // row y goes to block y / 32: the pair (k1(r, 0), k1(r, 1)) of local row yl
    // and stage-A lane j at (j * 8 + r) * 32 + (yl ^ j)
    const int yl = y & 31;
    float4* dst = cluster.map_shared_rank(tile4, y >> 5) + r * 32;
    static_for<0, 8>([&](auto jc) {
        constexpr int j = decltype(jc)::value;
        dst[j * 256 + (yl ^ j)] = pack2(z[0][j], z[1][j]);
    });
}

// c2r phase 3: inverse stage A of the block's rows 32 r .. 32 r + 31, stored.
__device__ __forceinline__ void c2r_stage_a_store(const float4* tile4, int r, int tid, float2* __restrict__ plane,
                                                  const GBuf<float2>& F) {
    const int w = tid >> 5, lane = tid & 31, g = lane >> 3, j = lane & 7;
    const int yl = w + 8 * g;
    const float4* src = tile4 + j * 256 + (yl ^ j);
    float2 v[16];
    static_for<0, 8>([&](auto qc) {                    // the pair sent by block q
        constexpr int q = decltype(qc)::value;
        const float4 t = src[q * 32];
        v[k1_of(q, 0)] = make_float2(t.x, t.y);
        v[k1_of(q, 1)] = make_float2(t.z, t.w);
    });
    reg_dft<float, +1, 16>(v);                         // v[n1] = z[j + 8 n1]
    float2* p = plane + (size_t)(32 * r + yl) * kM;
    static_for<0, 16>([&](auto nc) { st_field(&F.at(p, j + 8 * decltype(nc)::value), v[decltype(nc)::value]); });
}

constexpr size_t kTileBytes = (size_t)kM * kNy / kRcC * sizeof(float2);   // 32 KB

// L2 prefetch distance in planes (0: none).  Block r of the cluster on plane pl
// asks L2 for its 32 KB share of plane pl + kPlanePf, so that the cluster that
// takes that plane about one block lifetime later finds its input in L2.
#ifndef PSATD_PLANE_PF
#define PSATD_PLANE_PF 20
#endif
constexpr int kPlanePf = PSATD_PLANE_PF;

__device__ __forceinline__ void prefetch_plane(const float2* data, int pl, int r) {
    if constexpr (kPlanePf > 0) {
        const int npl = (int)(gridDim.x / kRcC);
        if (threadIdx.x == 0 && pl + kPlanePf < npl)
            prefetch_l2_bulk(data + (size_t)(pl + kPlanePf) * (kM * kNy) + (size_t)r * (kTileBytes / sizeof(float2)),
                             (uint32_t)kTileBytes);
    }
}

// 64 registers: four blocks per SM
#ifndef PSATD_RC_MINB_R2C
#define PSATD_RC_MINB_R2C 4
#endif
#ifndef PSATD_RC_MINB_C2R
#define PSATD_RC_MINB_C2R 5
#endif
__global__ void __launch_bounds__(kRcThreads, PSATD_RC_MINB_R2C)
plane_r2c_kernel(float2* __restrict__ data, const float2* __restrict__ twx, const float2* __restrict__ twy,
                 float2* __restrict__ nyq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* tile4 = reinterpret_cast<float4*>(smem_raw);
    __shared__ float2 col0[kNy];                       // block 0: the packed column after the y transform

    pdl_launch_dependents();
    cg::cluster_group cluster = cg::this_cluster();
    cluster.barrier_arrive();                          // wait for all blocks before the first remote store
    const int r = (int)cluster.block_rank();
    const int pl = blockIdx.x / kRcC;
    float2* plane = data + (size_t)pl * (kM * kNy);
    const int tid = threadIdx.x;
    const long long npl = gridDim.x / kRcC;
    const GBuf<float2> F{data, npl * kM * kNy}, NQ{nyq, npl * kNy};
    pdl_wait();
    prefetch_plane(data, pl, r);

    {
        const int w = tid >> 5, lane = tid & 31, g = lane >> 3, j = lane & 7;
        const int y = 32 * r + 4 * w + g;              // a warp's four rows adjacent: 512 contiguous bytes per remote store
        const float2* p = plane + (size_t)y * kM;
        float2 v[16];
        static_for<0, 16>([&](auto nc) { v[decltype(nc)::value] = ld_field(&F.at(p, j + 8 * decltype(nc)::value)); });
        r2c_stage_a(v, j, twx);
        cluster.barrier_wait();
        r2c_scatter(v, cluster, tile4, y, j);
    }
    cluster.sync();
    r2c_columns(tile4, col0, r, tid, twx, twy, plane, nyq + (size_t)pl * kNy, F, NQ);
}

// capped at 48 registers: five blocks per SM (the packed butterfly adds would
// otherwise take it to 54 registers and four blocks)
__global__ void __launch_bounds__(kRcThreads, PSATD_RC_MINB_C2R)
plane_c2r_kernel(float2* __restrict__ data, const float2* __restrict__ twx, const float2* __restrict__ twy,
                 const float2* __restrict__ nyq) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* tile4 = reinterpret_cast<float4*>(smem_raw);  // this block's columns (row layout), then [8][8][32] rows
    float2* tile = reinterpret_cast<float2*>(smem_raw);

    pdl_launch_dependents();
    cg::cluster_group cluster = cg::this_cluster();
    const int r = (int)cluster.block_rank();
    const int pl = blockIdx.x / kRcC;
    float2* plane = data + (size_t)pl * (kM * kNy);
    const int tid = threadIdx.x;
    const long long npl = gridDim.x / kRcC;
    const GBuf<float2> F{data, npl * kM * kNy};
    const GBuf<const float2> NQ{nyq, npl * kNy};
    pdl_wait();
    prefetch_plane(data, pl, r);

    {
        const int c = tid & 15, jy = tid >> 4;
        const float2* in = plane + 16 * r + slot_of_col(c);
        float2 v[16];
        static_for<0, 16>([&](auto kc) { v[decltype(kc)::value] = ld_field(&F.at(in, (long long)(jy + 16 * decltype(kc)::value) * kM)); });
        c2r_columns(v, tile, r, c, jy, twy, nyq + (size_t)pl * kNy, NQ);
    }
    __syncthreads();
    c2r_rows(tile4, cluster, r, tid, twx);
    cluster.sync();
    c2r_stage_a_store(tile4, r, tid, plane, F);
}

}  // namespace

bool plane_rc_supported(int prec, const GridGeom& g) { return prec == 32 && g.Nx == 256 && g.Ny == 256; }

// Real-field plane transform of ncomp components (dir < 0: r2c + y, dir > 0:
// inverse y + c2r) of real FP32 fields [ncomp][Nz][256][256], in place.
cudaError_t launch_plane_rc(float* data, float2* nyq, int ncomp, const GridGeom& g, const Tables<float>& tb, int dir,
                            cudaStream_t s) {
    if (!plane_rc_supported(32, g)) return cudaErrorNotSupported;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)((long long)ncomp * g.Nz * kRcC), 1, 1);
    cfg.blockDim = dim3(kRcThreads, 1, 1);
    cfg.dynamicSmemBytes = kTileBytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[3];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kRcC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;     // may overlap the previous kernel's tail
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    // load-balancing placement lets the blocks of a cluster share an SM: every SM
    // takes blocks (the spread placement left four SMs idle) and the slots freed
    // at the end of a cluster refill sooner (2 % on the plane kernels)
#ifndef PSATD_RC_SCHED
#define PSATD_RC_SCHED 1
#endif
#if PSATD_RC_SCHED
    attr[2].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    attr[2].val.clusterSchedulingPolicyPreference = PSATD_RC_SCHED == 1 ? cudaClusterSchedulingPolicyLoadBalancing
                                                                        : cudaClusterSchedulingPolicySpread;
    cfg.numAttrs = 3;
#endif
    float2* d = reinterpret_cast<float2*>(data);
    if (dir < 0) return cudaLaunchKernelEx(&cfg, plane_r2c_kernel, d, tb.tw[0], tb.tw[1], nyq);
    return cudaLaunchKernelEx(&cfg, plane_c2r_kernel, d, tb.tw[0], tb.tw[1], (const float2*)nyq);
}

// Slot order of the spectra the plane kernels leave in storage: the x mode
// index 0..127 held by slot p (the x Nyquist mode is kept apart, see above).
int plane_rc_slot_mode(int p) {
    const int r = p / 16, s = (p / 8) & 1, k2 = p & 7;
    const int k1 = r == 0 ? (s ? 8 : 0) : (s ? 16 - r : r);
    return k1 + 16 * k2;
}

}  // namespace psatd
