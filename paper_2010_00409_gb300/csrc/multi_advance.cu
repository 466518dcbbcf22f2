// Persistent batched PSATD advance: many periodic boxes (pulse realisations on
// grids of different sizes) stepped together in ONE cooperative launch.
//
// A step of every box is the same five phases (Sec. 2.1, Eq. 3-4 between the
// forward and inverse 3D DFTs): x forward, y forward, the fused z pass (z
// forward, the per-mode update, z inverse), y inverse, x inverse.  Each phase is
// one list of work items over all boxes (box p owns items [pre[p], pre[p+1])),
// which the resident blocks draw one at a time from a global ticket counter
// (a block that drew small items takes more); a grid-wide barrier separates the
// phases, because a phase reads what every block wrote in the one before.  The
// launch runs n steps, i.e. 5 n - 1 barriers, without returning to the host;
// a box with fewer steps of its own skips its items in the later steps.
//
// Work items (the generic shared-memory Stockham tiles of fft_core.cuh, so any
// axis length with factors 2, 3, 5 works):
//   x: W_x consecutive rows of one box (contiguous in memory);
//   y: W_y consecutive x-columns at one (component, z), read row by row;
//   z: W_z consecutive x-columns at one y, all six components: forward z
//      transforms, the update of every mode of the tile, inverse z transforms.
// The radix schedule of each axis and the three tile widths come from the host
// (the batch autotuner picks them per axis length).
//
// The barrier: every block adds one to a global counter after a fence, and
// thread 0 polls the counter (acquire loads, a short sleep between polls) until
// it reaches the number of arrivals that barrier needs.  The wait is bounded by
// the global nanosecond timer; a block whose wait expires sets
// DEV_ERR_GRID_TIMEOUT in the device error word and leaves the kernel, and so
// does every other block at the next barrier it cannot pass, so no block spins
// forever.  Field loads go around L1 (cache-global) so that no block reads a
// line another block rewrote in the previous phase.
#include "fft_reg.cuh"
#include "tma.cuh"

namespace psatd {

namespace {

constexpr int kMT = 256;

template <typename T> constexpr size_t desc_bytes() { return (sizeof(MultiProblem<T>) + 127) / 128 * 128; }

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier number `target / gridDim.x` (see above); false if this block's
// wait expired.
__device__ bool grid_barrier(unsigned* bar, unsigned target, int* err, unsigned long long limit_ns) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned long long t0 = global_ns();
        int done = 0;
        for (unsigned it = 0; it < (1u << 30); ++it) {
            if (ld_acquire_gpu(bar) >= target) {
                done = 1;
                break;
            }
            if (global_ns() - t0 > limit_ns) break;
            __nanosleep(128);
        }
        if (!done) atomicOr(err, DEV_ERR_GRID_TIMEOUT);
        __threadfence();
        ok = done;
    }
    __syncthreads();
    return ok != 0;
}

// x phase: rows row0 .. row0 + nrow - 1 of the box ([6][Nz][Ny] rows of Nx).
template <typename T, int S>
__device__ void x_tile(const MultiProblem<T>& P, long long item, cplx<T>* sm) {
    const int Nx = P.N[0], W = P.W[0], Pp = pencil_stride(Nx);
    const long long rows = 6LL * P.N[1] * P.N[2];
    const long long row0 = item * W;
    const int nrow = (int)min((long long)W, rows - row0);
    cplx<T>* A = sm;
    cplx<T>* B = sm + (size_t)W * Pp;
    cplx<T>* base = P.f + row0 * Nx;
    const GBuf<cplx<T>> F{P.f, rows * Nx};
    const int n = nrow * Nx;
    const FastDiv dn = fast_div(Nx);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int w = fdiv(e, dn), i = e - w * Nx;
        A[w * Pp + pad32(i)] = __ldcg(&F.at(base, e));
    }
    __syncthreads();
    const cplx<T>* res = fft_tile<T, S>(A, B, P.plan[0], nrow, Pp, P.tw[0]);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int w = fdiv(e, dn), i = e - w * Nx;
        F.at(base, e) = res[w * Pp + pad32(i)];
    }
}

// y phase: x-columns x0 .. x0 + nw - 1 of plane (comp, z).
template <typename T, int S>
__device__ void y_tile(const MultiProblem<T>& P, long long item, cplx<T>* sm) {
    const int Nx = P.N[0], Ny = P.N[1], Nz = P.N[2], W = P.W[1], Pp = pencil_stride(Ny);
    const int ntile = (Nx + W - 1) / W;
    const int t = (int)(item % ntile);
    const long long rest = item / ntile;                      // comp * Nz + z
    const int z = (int)(rest % Nz), comp = (int)(rest / Nz);
    const int x0 = t * W, nw = min(W, Nx - x0);
    const size_t plane = (size_t)Nx * Ny;
    cplx<T>* A = sm;
    cplx<T>* B = sm + (size_t)W * Pp;
    cplx<T>* base = P.f + (size_t)comp * plane * Nz + (size_t)z * plane + x0;
    const GBuf<cplx<T>> F{P.f, 6LL * (long long)plane * Nz};
    const int n = Ny * nw;
    const FastDiv dw = fast_div(nw);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int r = fdiv(e, dw), w = e - r * nw;
        A[w * Pp + pad32(r)] = __ldcg(&F.at(base, (long long)r * Nx + w));
    }
    __syncthreads();
    const cplx<T>* res = fft_tile<T, S>(A, B, P.plan[1], nw, Pp, P.tw[1]);
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int r = fdiv(e, dw), w = e - r * nw;
        F.at(base, (long long)r * Nx + w) = res[w * Pp + pad32(r)];
    }
}

// z pass of one tile, transforming component c of F in place (scratch as the
// Stockham partner buffer).
template <typename T, int S>
__device__ void z_transform(cplx<T>* Fc, cplx<T>* scratch, const MultiProblem<T>& P, int nw, int Pp) {
    cplx<T>* res = fft_tile<T, S>(Fc, scratch, P.plan[2], nw, Pp, P.tw[2]);
    if (res != Fc) {
        for (int e = threadIdx.x; e < nw * Pp; e += blockDim.x) Fc[e] = scratch[e];
        __syncthreads();
    }
}

// z phase: x-columns x0 .. x0 + nw - 1 at one y, all six components.
template <typename T>
__device__ void z_tile(const MultiProblem<T>& P, long long item, cplx<T>* sm) {
    const int Nx = P.N[0], Ny = P.N[1], Nz = P.N[2], W = P.W[2], Pp = pencil_stride(Nz);
    const int ntile = (Nx + W - 1) / W;
    const int t = (int)(item % ntile);
    const int y = (int)(item / ntile);
    const int x0 = t * W, nw = min(W, Nx - x0);
    const size_t plane = (size_t)Nx * Ny, cstride = plane * Nz, ct = (size_t)W * Pp;
    cplx<T>* F = sm;                                          // [6][W][Pp]
    cplx<T>* scratch = sm + 6 * ct;                           // [W][Pp]
    cplx<T>* base = P.f + (size_t)y * Nx + x0;
    const GBuf<cplx<T>> G{P.f, 6LL * (long long)cstride};
    const int n = Nz * nw;
    const FastDiv dw = fast_div(nw), dz = fast_div(Nz);
    for (int c = 0; c < 6; ++c)
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int r = fdiv(e, dw), w = e - r * nw;
            F[c * ct + w * Pp + pad32(r)] = __ldcg(&G.at(base, c * cstride + (size_t)r * plane + w));
        }
    __syncthreads();
    for (int c = 0; c < 6; ++c) z_transform<T, -1>(F + c * ct, scratch, P, nw, Pp);

    const int Nxh = Nx / 2 + 1, Nyh = Ny / 2 + 1;
    const int ay = min(y, Ny - y);
    const T ky = P.k[1][PSATD_IX(y, Ny)];
    const long long ncoef = (long long)(Nz / 2 + 1) * Nyh * Nxh;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int w = fdiv(e, dz), r = e - w * Nz;
        const int ix = x0 + w;
        const int ax = min(ix, Nx - ix), az = min(r, Nz - r);
        const ModeCoef<T> m = P.coef[PSATD_IX(((size_t)az * Nyh + ay) * Nxh + ax, ncoef)];
        cplx<T>* o = F + w * Pp + pad32(r);
        cplx<T> Ex = o[0], Ey = o[ct], Ez = o[2 * ct], Bx = o[3 * ct], By = o[4 * ct], Bz = o[5 * ct];
        rotate_mode<T>(Ex, Ey, Ez, Bx, By, Bz, P.k[0][PSATD_IX(ix, Nx)] * m.kinv, ky * m.kinv,
                       P.k[2][PSATD_IX(r, Nz)] * m.kinv, m.C, m.S);
        o[0] = Ex; o[ct] = Ey; o[2 * ct] = Ez;
        o[3 * ct] = Bx; o[4 * ct] = By; o[5 * ct] = Bz;
    }
    __syncthreads();
    for (int c = 0; c < 6; ++c) z_transform<T, +1>(F + c * ct, scratch, P, nw, Pp);

    for (int c = 0; c < 6; ++c)
        for (int e = threadIdx.x; e < n; e += blockDim.x) {
            const int r = fdiv(e, dw), w = e - r * nw;
            G.at(base, c * cstride + (size_t)r * plane + w) = F[c * ct + w * Pp + pad32(r)];
        }
}

template <typename T>
__global__ void __launch_bounds__(kMT)
multi_advance_kernel(const MultiProblem<T>* __restrict__ probs, const long long* __restrict__ prefix, int nprob,
                     int nsteps, unsigned* bar, unsigned long long* ticket, int* err, unsigned long long limit_ns,
                     unsigned extra) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    MultiProblem<T>* P = reinterpret_cast<MultiProblem<T>*>(smem_raw);
    cplx<T>* tile = reinterpret_cast<cplx<T>*>(smem_raw + desc_bytes<T>());
    __shared__ long long s_item;
    int cur = -1;                                               // box whose descriptor is in P
    unsigned nbar = 0;
    unsigned long long base = 0;                                // first ticket of this phase
    for (int s = 0; s < nsteps; ++s) {
        for (int ph = 0; ph < 5; ++ph) {
            const int a = ph <= 2 ? ph : 4 - ph;               // axis of the phase: x, y, z, y, x
            const long long* pre = prefix + (size_t)a * (nprob + 1);
            const long long total = pre[nprob];
            // items are handed out one at a time from a global ticket counter, so
            // blocks that drew cheap items (small boxes) take more of them; every
            // block stops at its first ticket past the phase, so the phase uses
            // exactly total + gridDim.x tickets
            for (;;) {
                if (threadIdx.x == 0) s_item = (long long)(atomicAdd(ticket, 1ull) - base);
                __syncthreads();
                const long long g = s_item;
                if (g >= total) break;
                int lo = 0, hi = nprob - 1;                     // the box p with pre[p] <= g < pre[p + 1]
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pre[PSATD_IX(mid, nprob + 1)] <= g) lo = mid;
                    else hi = mid - 1;
                }
                if (lo != cur) {
                    const int* src = reinterpret_cast<const int*>(probs + lo);
                    int* dst = reinterpret_cast<int*>(P);
                    for (int i = threadIdx.x; i < (int)(sizeof(MultiProblem<T>) / 4); i += blockDim.x) dst[i] = src[i];
                    cur = lo;
                    __syncthreads();
                }
                const long long item = g - pre[lo];
                if (s < P->nsteps) {                            // a box past its own step count is skipped
                    if (ph == 0) x_tile<T, -1>(*P, item, tile);
                    else if (ph == 1) y_tile<T, -1>(*P, item, tile);
                    else if (ph == 2) z_tile<T>(*P, item, tile);
                    else if (ph == 3) y_tile<T, +1>(*P, item, tile);
                    else x_tile<T, +1>(*P, item, tile);
                }
                __syncthreads();                                // the next item reuses s_item, the descriptor and tile
            }
            base += (unsigned long long)total + gridDim.x;
            if (s == nsteps - 1 && ph == 4) return;
            ++nbar;
            if (!grid_barrier(bar, nbar * gridDim.x + extra, err, limit_ns)) return;
        }
    }
}

}  // namespace

template <typename T>
size_t multi_tile_bytes(int axis, int N_axis, int W) {
    const size_t es = sizeof(cplx<T>);
    return (axis == 2 ? 7 : 2) * (size_t)W * pencil_stride(N_axis) * es;
}

template <typename T>
cudaError_t launch_multi_advance(const MultiProblem<T>* probs, const long long* prefix, int nprob, int nsteps,
                                 size_t tile_bytes, long long max_items, unsigned* bar, int* err,
                                 unsigned long long limit_ns, unsigned extra, cudaStream_t s, int* grid_out) {
    auto k = multi_advance_kernel<T>;
    const size_t smem = desc_bytes<T>() + tile_bytes;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kMT, smem)) != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long grid = (long long)per_sm * sms;
    if (max_items < grid) grid = max_items < 1 ? 1 : max_items;
    // barrier counter at bar[0], ticket counter at bar[2] (8-byte aligned)
    unsigned long long* ticket = reinterpret_cast<unsigned long long*>(bar + 2);
    if ((e = cudaMemsetAsync(bar, 0, 16, s)) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(kMT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;            // all blocks resident at once (the barrier needs it)
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (grid_out) *grid_out = (int)grid;
    return cudaLaunchKernelEx(&cfg, k, probs, prefix, nprob, nsteps, bar, ticket, err, limit_ns, extra);
}

template size_t multi_tile_bytes<float>(int, int, int);
template size_t multi_tile_bytes<double>(int, int, int);
template cudaError_t launch_multi_advance<float>(const MultiProblem<float>*, const long long*, int, int, size_t,
                                                 long long, unsigned*, int*, unsigned long long, unsigned,
                                                 cudaStream_t, int*);
template cudaError_t launch_multi_advance<double>(const MultiProblem<double>*, const long long*, int, int, size_t,
                                                  long long, unsigned*, int*, unsigned long long, unsigned,
                                                  cudaStream_t, int*);

}  // namespace psatd
