// Fused k-space pass of one PSATD step (Sec. 2.1, Eq. 3-4), fed by the tensor
// copy engine: at block start one thread issues six tiled bulk-tensor loads
// (one per field component, box = W x-columns x 1 y x Nz z, 64 contiguous bytes
// per row) into the six shared-memory slots, each completing on its own
// mbarrier.  The whole tile (6 * Nz * W complex values) is then in flight at
// once; each thread group starts on its first component as soon as that slot
// has landed.  The block's threads form two groups; each group transforms
// three components.  Per component: forward z transform in registers (the slot
// doubles as the exchange buffer; the exchanges synchronise only the group, on
// a named barrier), spectrum back to the slot; the per-mode update over all six
// slots (modes split between the groups, block-wide barriers around it);
// inverse z transforms stored straight from registers to the field.
//
// The waits on the copies are bounded: past the limit the block sets an error
// bit in the context's device error word and runs on with invalid data.
#include "fft_reg.cuh"
#include "tma.cuh"

namespace psatd {

namespace {

// L2 prefetch distance in tiles (0: none): thread 0 of the block on field tile
// bt asks L2 for the six component boxes of tile bt + kKsPf.
#ifndef PSATD_KS_PF
#define PSATD_KS_PF 152
#endif
constexpr int kKsPf = PSATD_KS_PF;

// Barrier over the NT threads of group h only (named barrier 1 + h; barrier 0
// is __syncthreads): the exchange rounds of a group touch only its own
// components' slots, so the other group need not wait.
template <int NT, int G>
__device__ __forceinline__ void group_sync(int h) {
    if constexpr (G > 1) {
        // immediate barrier ids, so that the block claims three barriers, not all sixteen
        if (h == 0) asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
        else asm volatile("bar.sync 2, %0;" ::"n"(NT) : "memory");
    } else {
        __syncthreads();
    }
}

// Shared-memory layout of one component slot: element (row k1, lane j, column c)
// at k1*RP + j*W + c with RP = N2*W, i.e. the dense [z][c] tile the copy engine
// writes (z = N2 k1 + j).  Every copy destination is a whole slot, so it keeps
// the 128-byte alignment bulk-tensor copies require.
//   - raw element z = j + N2 n1 of column c sits at (n1, j): thread (c, j) reads
//     exactly the positions it later scatters to;
//   - the spectrum a thread holds after the forward transform (register
//     r = q N2 + k2 <-> kz = (t + N2 q) + N1 k2) is stored back at the same
//     positions (r, t), so the per-mode update and the first read of the inverse
//     touch only the thread's own positions and need no barrier.
// HALF: the storage holds the half spectrum of real fields in the slot order of
// the real-field plane kernels (x extent = Nx/2 slots): the slot's wave number
// comes from kxs and the coefficient table is in slot order along x (column =
// slot, so neighbouring threads read neighbouring entries; column Nx/2 = the x
// Nyquist mode), and modes on Nyquist planes take the mean update that keeps the
// field real (project_b / project_e: B / E is first projected the same way, the
// mean of the projections along the two mirrored wave vectors; that mean is not
// idempotent on Nyquist planes, so a projection followed by a step needs both).  The x Nyquist spectrum
// lives in its own array nyq[q][z][k_y]; the blocks after the Ny * Nx/(2W)
// field tiles take its tiles of W k_y values (copied through map_nyq, a 3D map
// {Ny, Nz, 6}).  SPECTRAL_OUT with HALF leaves the updated half spectrum (slots
// and the Nyquist array) in natural k_z order.
// float32: two blocks per SM (128 registers a thread, the 96 KB tile twice)
template <typename T, int N1, int N2, int W, int G, bool SPECTRAL_OUT, bool HALF, bool PROJ = false>
__global__ void __launch_bounds__(W * N2 * G, sizeof(T) == 4 ? 2 : 1)
kspace_tma_kernel(const __grid_constant__ CUtensorMap map, const __grid_constant__ CUtensorMap map_nyq,
                  cplx<T>* __restrict__ data, int Nx, int Ny, const cplx<T>* __restrict__ tw,
                  const T* __restrict__ kxs, const T* __restrict__ kys, const T* __restrict__ kzs,
                  const ModeCoef<T>* __restrict__ coef, int* __restrict__ err, bool project_b, int coef_nx,
                  cplx<T>* __restrict__ nyq, T kx_nyq, bool project_e) {
    constexpr int Nz = N1 * N2;
    constexpr int RP = N2 * W;
    constexpr int SLOT = N1 * RP;
    constexpr int NT = W * N2;                                  // threads of one group
    constexpr int NC = 6 / G;                                   // components transformed by one group
    constexpr int NB = (G == 1 && sizeof(T) == 4) ? 2 : 1;      // components per exchange round
    constexpr int NM = N1 / G;                                  // modes updated per thread
    constexpr uint32_t kBytes = 6u * Nz * W * sizeof(cplx<T>);
    static_assert(kBytes < (1u << 20), "mbarrier transaction count is 20 bits");
    static_assert(NC % NB == 0 && N1 % G == 0, "group split");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cplx<T>* spec = reinterpret_cast<cplx<T>*>(smem_raw);      // [6][N1][RP]
    __shared__ __align__(8) uint64_t bar[6];                    // one mbarrier per component slot

    const int t = threadIdx.x % NT, h = threadIdx.x / NT;       // group h: components NC h .. NC h + NC - 1
    const int c = t % W, j = t / W;
    const int ntile = Nx / W;
    const bool nq = HALF && (int)blockIdx.x >= ntile * Ny;      // a tile of the x Nyquist array
    const int bt = nq ? (int)blockIdx.x - ntile * Ny : (int)blockIdx.x;
    const int xt = nq ? 0 : bt % ntile;
    const int y = nq ? bt * W + c : bt / ntile;                 // this thread's k_y index
    const int ix = nq ? 0 : xt * W + c;
    const size_t plane = nq ? (size_t)Ny : (size_t)Nx * Ny;
    const size_t cstride = plane * Nz;
    pdl_launch_dependents();

    if (threadIdx.x == 0) {
        for (int q = 0; q < 6; ++q) mbar_init(&bar[q], 1);
        fence_mbar_init();
    }
    __syncthreads();

    // before the field is read (this part may overlap the previous kernel):
    // outer twiddles W_N^{j k1} (the inverse uses their conjugates with k1 = j)
    // and the per-mode coefficients of this thread's modes (registers
    // r = h NM .. h NM + NM - 1 of position (c, j)); their loads complete while
    // the tile copies fly
    cplx<T> twr[N1];
    static_for<1, N1>([&](auto kc) { twr[decltype(kc)::value] = tw[PSATD_IX(j * decltype(kc)::value, Nz)]; });
    const int Nxh = coef_nx, Nyh = Ny / 2 + 1;
    const int ax = HALF ? (nq ? coef_nx - 1 : ix) : min(ix, Nx - ix), ay = min(y, Ny - y);
    const T kx = nq ? kx_nyq : kxs[PSATD_IX(ix, Nx)], ky = kys[PSATD_IX(y, Ny)];
    const long long ncoef = (long long)(Nz / 2 + 1) * Nyh * Nxh;
    ModeCoef<T> mc[NM];
    T kzr[NM];
    static_for<0, NM>([&](auto mcix) {
        constexpr int m = decltype(mcix)::value;
        const int r = h * NM + m;
        const int iz = (j + N2 * (r / N2)) + N1 * (r % N2);
        const int az = min(iz, Nz - iz);
        mc[m] = coef[PSATD_IX(((size_t)az * Nyh + ay) * Nxh + ax, ncoef)];
        kzr[m] = kzs[PSATD_IX(iz, Nz)];
    });

    pdl_wait();
    if (threadIdx.x == 0) {
        constexpr int xw = (int)(sizeof(cplx<T>) / 8);        // 8-byte elements per complex
        for (int i = 0; i < 6; ++i) {
            // each group's first component first (0, 3, 1, 4, 2, 5 for two groups)
            const int q = (i % G) * NC + i / G;
            mbar_arrive_expect_tx(&bar[q], kBytes / 6);
            if (nq) tma_load_3d(spec + q * SLOT, &map_nyq, &bar[q], bt * W * xw, 0, q);
            else tma_load_4d(spec + q * SLOT, &map, &bar[q], xt * W * xw, y, 0, q);
        }
        if constexpr (kKsPf > 0) {
            const int bn = bt + kKsPf;
            if (!nq && bn < ntile * Ny)
                for (int q = 0; q < 6; ++q) tma_prefetch_4d(&map, (bn % ntile) * W * xw, bn / ntile, 0, q);
        }
    }

    // every thread waits for a component just before its first read of it, so
    // a group starts on its first component while the others are in flight; an
    // expired wait records the error and the block runs on (its barriers stay
    // matched), and the block's last act is a second bounded wait on every copy
    // so that none is in flight when it exits
    auto wait_slot = [&](int q) {
        if (!mbar_wait_bounded(&bar[q], 0) && (threadIdx.x & 31) == 0) atomicOr(err, DEV_ERR_TMA_TIMEOUT);
    };
    auto drain = [&]() {
        if (threadIdx.x == 0)
            for (int q = 0; q < 6; ++q) mbar_wait_bounded(&bar[q], 0);
    };

    cplx<T>* own = spec + j * W + c;                           // (row r, position (c, j)) at own[r * RP]
    cplx<T> v[NB][N1];

    // Exchange layout: between the two passes of a transform, odd rows hold
    // their column pairs (2m, 2m + 1) swapped, i.e. logical column n of row k
    // sits at column n ^ (k & 1).  A half-warp (quarter-warp in FP64) spans
    // lanes j = 2m, 2m + 1; in the exchange it reads (writes) one row per lane,
    // two rows RP apart on the same banks, and the swap sends its two rows to
    // columns of opposite parity, i.e. to the two halves of the bank array, so
    // no access of the exchange has a bank conflict.  Row parity and column
    // parity are known per access, so every access is a fixed base pointer
    // plus an immediate offset.
    static_assert(N2 % 2 == 0, "row parity of the exchange row = parity of j");
    const int odd = j & 1;
    cplx<T>* own_x = spec + (j ^ 1) * W + c;                   // position (c, j) of an odd row

    // forward z transforms of this group's components, NB per exchange round
#pragma unroll 1
    for (int q0 = NC * h; q0 < NC * h + NC; q0 += NB) {
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            wait_slot(q0 + b);
            cplx<T>* sl = own + (q0 + b) * SLOT;
            static_for<0, N1>([&](auto nc) { v[b][decltype(nc)::value] = sl[decltype(nc)::value * RP]; });
            reg_dft<T, -1, N1>(v[b]);
            static_for<1, N1>([&](auto kc) {
                constexpr int k1 = decltype(kc)::value;
                if (j) v[b][k1] = cmul(v[b][k1], twr[k1]);
            });
            cplx<T>* sx = own_x + (q0 + b) * SLOT;
            static_for<0, N1>([&](auto kc) {
                constexpr int k1 = decltype(kc)::value;
                ((k1 & 1) ? sx : sl)[k1 * RP] = v[b][k1];
            });
        });
        group_sync<NT, G>(h);
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            const cplx<T>* sl = spec + (q0 + b) * SLOT + c;
            static_for<0, N1 / N2>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                cplx<T> w[N2];
                const cplx<T>* row = sl + (j + N2 * q) * RP;
                const cplx<T>* ev = row + odd * W;              // even columns of this row's parity
                const cplx<T>* od = row - odd * W;              // odd columns
                static_for<0, N2>([&](auto jc) {
                    constexpr int n = decltype(jc)::value;
                    w[n] = ((n & 1) ? od : ev)[n * W];
                });
                reg_dft<T, -1, N2>(w);
                static_for<0, N2>([&](auto kc) { v[b][q * N2 + decltype(kc)::value] = w[decltype(kc)::value]; });
            });
        });
        group_sync<NT, G>(h);
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            cplx<T>* sl = own + (q0 + b) * SLOT;
            static_for<0, N1>([&](auto rc) { sl[decltype(rc)::value * RP] = v[b][decltype(rc)::value]; });
        });
    }
    if constexpr (G > 1) __syncthreads();                      // the update reads the other group's components

    // per-mode update on this thread's modes of position (c, j)
    static_for<0, NM>([&](auto mcix) {
        constexpr int m = decltype(mcix)::value;
        const int r = h * NM + m;
        cplx<T>* o = own + r * RP;
        cplx<T> Ex = o[0], Ey = o[SLOT], Ez = o[2 * SLOT];
        cplx<T> Bx = o[3 * SLOT], By = o[4 * SLOT], Bz = o[5 * SLOT];
        const ModeCoef<T> mm = mc[m];
        if constexpr (HALF) {
            const bool fz = ((j + N2 * (r / N2)) + N1 * (r % N2)) == Nz / 2;
            if constexpr (PROJ) {                       // (the step's instance carries no projection)
                if (project_e)
                    project_b_mean<T>(Ex, Ey, Ez, kx * mm.kinv, ky * mm.kinv, kzr[m] * mm.kinv, nq, 2 * y == Ny, fz);
                if (project_b)
                    project_b_mean<T>(Bx, By, Bz, kx * mm.kinv, ky * mm.kinv, kzr[m] * mm.kinv, nq, 2 * y == Ny, fz);
            }
            rotate_mode_mean<T>(Ex, Ey, Ez, Bx, By, Bz, kx * mm.kinv, ky * mm.kinv, kzr[m] * mm.kinv, nq,
                                2 * y == Ny, fz, mm.C, mm.S);
        } else {
            rotate_mode<T>(Ex, Ey, Ez, Bx, By, Bz, kx * mm.kinv, ky * mm.kinv, kzr[m] * mm.kinv, mm.C, mm.S,
                           project_b);
        }
        o[0] = Ex; o[SLOT] = Ey; o[2 * SLOT] = Ez;
        o[3 * SLOT] = Bx; o[4 * SLOT] = By; o[5 * SLOT] = Bz;
    });
    if constexpr (G > 1) __syncthreads();                      // the inverse reads the other group's modes

    cplx<T>* base = nq ? nyq + y : data + (size_t)y * Nx + ix;
    const GBuf<cplx<T>> F = nq ? GBuf<cplx<T>>{nyq, 6LL * Ny * Nz} : GBuf<cplx<T>>{data, 6LL * Nx * Ny * Nz};
    if constexpr (SPECTRAL_OUT) {
        // store the updated spectrum in natural kz order (one-shot focal path)
        for (int q = NC * h; q < NC * h + NC; ++q) {
            const cplx<T>* sl = own + q * SLOT;
            cplx<T>* p = base + q * cstride;
            static_for<0, N1 / N2>([&](auto qc) {
                constexpr int qq = decltype(qc)::value;
                static_for<0, N2>([&](auto kc) {
                    constexpr int k2 = decltype(kc)::value;
                    F.at(p, (long long)((j + N2 * qq) + N1 * k2) * plane) = sl[(qq * N2 + k2) * RP];
                });
            });
        }
        drain();
        return;
    }

    // inverse z transforms of this group's components, NB per exchange round
#pragma unroll 1
    for (int q0 = NC * h; q0 < NC * h + NC; q0 += NB) {
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            const cplx<T>* sl = own + (q0 + b) * SLOT;
            static_for<0, N1>([&](auto rc) { v[b][decltype(rc)::value] = sl[decltype(rc)::value * RP]; });
        });
        group_sync<NT, G>(h);
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            cplx<T>* sl = spec + (q0 + b) * SLOT + c;
            static_for<0, N1 / N2>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                cplx<T> w[N2];
                static_for<0, N2>([&](auto kc) { w[decltype(kc)::value] = v[b][q * N2 + decltype(kc)::value]; });
                reg_dft<T, +1, N2>(w);
                const int k1 = j + N2 * q;
                cplx<T>* row = sl + k1 * RP;
                cplx<T>* ev = row + odd * W;                    // even columns of this row's parity
                cplx<T>* od = row - odd * W;                    // odd columns
                static_for<0, N2>([&](auto nc) {
                    constexpr int n2 = decltype(nc)::value;
                    cplx<T> val = w[n2];
                    if (n2 > 0 && k1 > 0) {
                        // W_N^{-n2 k1}; for q = 0 this is conj(twr[n2]) (k1 = j)
                        const cplx<T> tv = (q == 0) ? twr[n2] : tw[PSATD_IX(n2 * k1, Nz)];
                        val = cmulc(val, tv);
                    }
                    ((n2 & 1) ? od : ev)[n2 * W] = val;
                });
            });
        });
        group_sync<NT, G>(h);
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            const cplx<T>* sl = own + (q0 + b) * SLOT;
            const cplx<T>* sx = own_x + (q0 + b) * SLOT;
            static_for<0, N1>([&](auto kc) {
                constexpr int k1 = decltype(kc)::value;
                v[b][k1] = ((k1 & 1) ? sx : sl)[k1 * RP];
            });
        });
        static_for<0, NB>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            reg_dft<T, +1, N1>(v[b]);
            cplx<T>* p = base + (q0 + b) * cstride;
            static_for<0, N1>([&](auto nc) { F.at(p, (long long)(j + N2 * decltype(nc)::value) * plane) = v[b][decltype(nc)::value]; });
        });
    }
    drain();
}

// Two thread groups per block (each transforms three components; the update
// splits the tile's modes between them): 256 threads at ~128 registers, twice
// the resident warps of one group per block at the same shared memory.
template <typename T, int N1, int N2, int W>
cudaError_t kspace_tma_launch(const CUtensorMap& map, cplx<T>* data, const GridGeom& g, const Tables<T>& tb,
                              int* err, cudaStream_t s, bool spectral_out, bool project_b, const HalfSlots<T>* half) {
    constexpr int G = 2;
    const size_t smem = (size_t)6 * N1 * N2 * W * sizeof(cplx<T>);
    const bool proj = half && (project_b || half->project_e);
    auto k = half ? (spectral_out ? kspace_tma_kernel<T, N1, N2, W, G, true, true, true>
                                  : (proj ? kspace_tma_kernel<T, N1, N2, W, G, false, true, true>
                                          : kspace_tma_kernel<T, N1, N2, W, G, false, true, false>))
                  : (spectral_out ? kspace_tma_kernel<T, N1, N2, W, G, true, false>
                                  : kspace_tma_kernel<T, N1, N2, W, G, false, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int nx = half ? g.Nx / 2 : g.Nx;             // complex elements per stored row
    const unsigned blocks = (unsigned)((long long)g.Ny * (nx / W) + (half ? g.Ny / W : 0));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(W * N2 * G, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // may overlap the previous kernel's tail
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, map, half ? *half->map_nyq : map, data, nx, g.Ny, tb.tw[2],
                              half ? half->k : tb.k[0], tb.k[1], tb.k[2], half ? half->coef : tb.coef, err, project_b,
                              g.Nx / 2 + 1, half ? half->nyq : (cplx<T>*)nullptr,
                              (T)(-3.14159265358979323846 / g.dx), half ? half->project_e : false);
}

// Self-test of the bounded-wait path: waits on an mbarrier whose 16 expected
// bytes no copy will ever deliver, gives up after `limit` polls and reports
// DEV_ERR_TMA_TIMEOUT.  No asynchronous copy is issued, so nothing is in flight
// when the block exits.
__global__ void wait_timeout_selftest_kernel(int* err, uint32_t limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        mbar_arrive_expect_tx(&bar, 16);
        bool ok = false;
        for (uint32_t it = 0; it < limit && !ok; ++it) ok = mbar_try_wait(&bar, 0);
        if (!ok) atomicOr(err, DEV_ERR_TMA_TIMEOUT);
    }
}

}  // namespace

cudaError_t launch_wait_timeout_selftest(int* err, cudaStream_t s) {
    wait_timeout_selftest_kernel<<<1, 32, 0, s>>>(err, 1024);
    return cudaGetLastError();
}

template <typename T> constexpr int kspace_tma_width() { return 64 / (int)sizeof(cplx<T>); }

template <typename T>
cudaError_t launch_kspace_tma(const CUtensorMap& map, cplx<T>* data, const GridGeom& g, const Tables<T>& tb,
                              int* err, cudaStream_t s, bool spectral_out, bool project_b, const HalfSlots<T>* half) {
    constexpr int W = kspace_tma_width<T>();
    if ((half ? g.Nx / 2 : g.Nx) % W != 0 || (half && g.Ny % W != 0)) return cudaErrorNotSupported;
    switch (g.Nz) {
        case 64: return kspace_tma_launch<T, 8, 8, W>(map, data, g, tb, err, s, spectral_out, project_b, half);
        case 128: return kspace_tma_launch<T, 16, 8, W>(map, data, g, tb, err, s, spectral_out, project_b, half);
        case 256: return kspace_tma_launch<T, 16, 16, W>(map, data, g, tb, err, s, spectral_out, project_b, half);
        default: return cudaErrorNotSupported;
    }
}

int kspace_tma_box_x(int prec) { return prec == 64 ? kspace_tma_width<double>() * 2 : kspace_tma_width<float>(); }

// z-extent of one copy box: the whole pencil (0 if Nz has no plan here)
int kspace_tma_box_z(int Nz) { return (Nz == 64 || Nz == 128 || Nz == 256) ? Nz : 0; }

template cudaError_t launch_kspace_tma<float>(const CUtensorMap&, cplx<float>*, const GridGeom&, const Tables<float>&, int*, cudaStream_t, bool, bool, const HalfSlots<float>*);
template cudaError_t launch_kspace_tma<double>(const CUtensorMap&, cplx<double>*, const GridGeom&, const Tables<double>&, int*, cudaStream_t, bool, bool, const HalfSlots<double>*);

}  // namespace psatd
