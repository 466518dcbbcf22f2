// Shared device/host helpers of the PSATD library: complex arithmetic, the
// per-axis FFT plan, and the launch interfaces of the kernel translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace psatd {

// ---------------------------------------------------------------------------
// Bounds-checked global indices (builds with -DPSATD_DEBUG).  PSATD_IX(i, n) is
// the index i of a global buffer of n elements.  In a debug build an index
// outside [0, n) is counted (the first one is kept with its bound) and replaced
// by 0, so the access stays inside the buffer; psatd_debug_bounds_report reads
// and clears the counts of every translation unit.  In other builds it is i.
#ifdef PSATD_DEBUG
void debug_register_reader(long long (*reader)(long long* first_index, long long* first_bound));
namespace dbg {
static __device__ unsigned long long g_oob;
static __device__ long long g_first[2];
__device__ __forceinline__ long long idx(long long i, long long n) {
    if (i < 0 || i >= n) {
        if (atomicAdd(&g_oob, 1ull) == 0ull) {
            g_first[0] = i;
            g_first[1] = n;
        }
        return 0;
    }
    return i;
}
// this translation unit's counts, read and cleared (host)
static long long read_and_clear(long long* first_index, long long* first_bound) {
    unsigned long long n = 0;
    long long f[2] = {0, 0};
    if (cudaMemcpyFromSymbol(&n, g_oob, sizeof n) != cudaSuccess) return -1;
    cudaMemcpyFromSymbol(f, g_first, sizeof f);
    const unsigned long long zero = 0;
    cudaMemcpyToSymbol(g_oob, &zero, sizeof zero);
    if (first_index) *first_index = f[0];
    if (first_bound) *first_bound = f[1];
    return (long long)n;
}
struct Registrar {
    Registrar() { debug_register_reader(&read_and_clear); }
};
static Registrar g_registrar;
}  // namespace dbg
#define PSATD_IX(i, n) (::psatd::dbg::idx((long long)(i), (long long)(n)))
#else
#define PSATD_IX(i, n) (i)
#endif

// A global buffer of n elements: at(p, k) is p[k] for a pointer p into it,
// bounds-checked against the whole buffer in debug builds.
template <typename V> struct GBuf {
    V* base;
    long long n;
    __device__ __forceinline__ V& at(const V* p, long long k) const {
#ifdef PSATD_DEBUG
        return base[PSATD_IX((long long)(p - base) + k, n)];
#else
        return const_cast<V&>(p[k]);                 // release: exactly p[k]
#endif
    }
    __device__ __forceinline__ V& operator[](long long i) const { return base[PSATD_IX(i, n)]; }
};

// ---------------------------------------------------------------------------
// complex helpers over float2 / double2
// ---------------------------------------------------------------------------
template <typename T> struct vec2;
template <> struct vec2<float>  { using type = float2; };
template <> struct vec2<double> { using type = double2; };
template <typename T> using cplx = typename vec2<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
    cplx<T> r; r.x = re; r.y = im; return r;
}
template <typename V> __host__ __device__ __forceinline__ V cadd(V a, V b) { a.x += b.x; a.y += b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V csub(V a, V b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <typename V> __host__ __device__ __forceinline__ V cmulc(V a, V b) {
    V r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <typename V, typename S> __host__ __device__ __forceinline__ V cscale(V a, S s) { a.x *= s; a.y *= s; return a; }

// ---------------------------------------------------------------------------
// float32 twiddles.  A forward transform multiplies by w and the inverse by
// conj w, so per step the field's energy is scaled by |w|^2 along every path a
// twiddle sits on: the rounding of cos and sin to float32 leaves |w|^2 - 1 at
// ~1e-8 per twiddle, a drift that repeats every step.  Among the float32 pairs
// within one ulp of (cos, sin) this picks the one minimising
// |c^2 + s^2 - 1| + |angle error|; values exactly representable stay as they are.
struct UnitF { float c, s; };

__host__ __device__ constexpr double ulp_f32(double x) {
    double a = x < 0 ? -x : x, p = 1.0;
    if (a < 1e-30) return 0.0;
    if (a >= 1.0) {
        while (a >= 2.0 * p) p *= 2.0;
    } else {
        while (p > a) p *= 0.5;
    }
    return p * 1.1920928955078125e-07;            // 2^-23 of the binade
}

__host__ __device__ constexpr UnitF unit_f32(double c, double s) {
    const float c0 = (float)c, s0 = (float)s;
    const bool ce = (double)c0 == c, se = (double)s0 == s;
    UnitF best{c0, s0};
    double best_cost = 1e300;
    for (int i = -1; i <= 1; ++i) {
        for (int j = -1; j <= 1; ++j) {
            if ((ce && i != 0) || (se && j != 0)) continue;
            const float cf = (float)((double)c0 + i * ulp_f32(c0));
            const float sf = (float)((double)s0 + j * ulp_f32(s0));
            const double m = (double)cf * cf + (double)sf * sf - 1.0;
            const double a = c * ((double)sf - s) - s * ((double)cf - c);     // angle error (small)
            const double cost = (m < 0 ? -m : m) + (a < 0 ? -a : a);
            if (cost < best_cost) {
                best_cost = cost;
                best = UnitF{cf, sf};
            }
        }
    }
    return best;
}
// multiply by s*i, s = +-1
template <typename V> __host__ __device__ __forceinline__ V cmul_si(V a, int s) {
    V r; if (s > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; } return r;
}

// |a|^2 + |b|^2 + |c|^2 of one cell's three components, formed in the storage
// precision (float32 storage: float32 products and sums, relative error ~1e-7)
// and returned as float64 for the accumulation over cells.  The diagnostics and
// the allocation-free energy kernel share it, so their results differ only in
// the order of the float64 sums.
template <typename T>
__device__ __forceinline__ double cell_energy3(cplx<T> a, cplx<T> b, cplx<T> c) {
    T s = a.x * a.x;
    s = fma(a.y, a.y, s);
    s = fma(b.x, b.x, s);
    s = fma(b.y, b.y, s);
    s = fma(c.x, c.x, s);
    s = fma(c.y, c.y, s);
    return (double)s;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialization may start while the previous kernel's last blocks still run;
// it must call pdl_wait() before touching that kernel's output.  Both are no-ops
// for a normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ---------------------------------------------------------------------------
// 1D plan of one axis: N = prod(radix[0..npass)), radices in {2,3,4,5,8}
// ---------------------------------------------------------------------------
constexpr int kMaxPass = 16;
struct AxisPlan {
    int N;
    int npass;
    int radix[kMaxPass];
};

// Host: factor N into 8, 4, 5, 3, 2 (largest radices first).  Returns false if
// N has another prime factor.
bool make_plan(int N, AxisPlan* p);

// ---------------------------------------------------------------------------
// Per-mode table entry: C/Ntot, S/Ntot, 1/|k| (0 at k = 0).
// Indexed by (|m_z|, |m_y|, |m_x|), each 0..N/2.
// ---------------------------------------------------------------------------
template <typename T> struct alignas(4 * sizeof(T)) ModeCoef { T C, S, kinv, pad; };

// Geometry handed to the kernels (all float64).
struct GridGeom {
    int Nx, Ny, Nz;
    double dx, dy, dz;
    double x_min, y_min, z_min;
    double c;
};

struct ShellGeom { double R0, L; };

struct PulseParams {
    int kind, div_project;
    double lambda, theta, eps, P0, n_cycles, cep, ellipticity, pol_angle;
    double amp;          // A (flat-top, profile) or E0 (Gaussian), computed on the host
    const double2* prof; // profile kind: complex samples a_k = a(prof_z0 + k prof_dz), k < prof_n
    int prof_n;
    double prof_z0, prof_dz;
};

// Device tables of one context.
template <typename T> struct Tables {
    const cplx<T>* tw[3];       // tw[a][t] = exp(-2 pi i t / N_a), t < N_a
    // [32][32] tw[a][(i j) mod N_a] for N_a = 512, 1024 (else null): twiddles of
    // the register kernels read along a thread-indexed j, 32 consecutive entries
    const cplx<T>* tw2[3] = {nullptr, nullptr, nullptr};
    const T* k[3];              // k_a[i] = 2 pi m(i) / (N_a d_a)
    const ModeCoef<T>* coef;    // (Nz/2+1) x (Ny/2+1) x (Nx/2+1)
    AxisPlan plan[3];
    int tile_shift = 0;         // generic kernels: tile width scaled by 2^tile_shift (autotuner)
};

// One periodic box of a persistent batched advance (multi_advance.cu): its
// complex fields [6][Nz][Ny][Nx], tables, the radix schedule of each axis and
// the tile widths of the x (rows per tile), y and z (x-columns per tile) phases.
template <typename T> struct MultiProblem {
    cplx<T>* f;
    const cplx<T>* tw[3];
    const T* k[3];
    const ModeCoef<T>* coef;
    int N[3];
    int W[3];
    int nsteps;                 // this box's steps (the launch runs the largest count)
    AxisPlan plan[3];
};

// Shared-memory bytes of one tile of the phase along `axis` (N_axis points,
// W pencils): two Stockham buffers for x and y, six components and a partner
// buffer for the fused z pass.
template <typename T> size_t multi_tile_bytes(int axis, int N_axis, int W);

// Persistent cooperative launch advancing nprob boxes by up to nsteps PSATD
// steps (box p by its own probs[p].nsteps <= nsteps).
// prefix[a][p] (a = 0, 1, 2; p = 0..nprob) are the first work items of box p in
// the x, y and z phases; tile_bytes the largest tile; bar 16 bytes of device
// memory (8-byte aligned: the barrier and work-ticket counters) the launch
// resets first; err the device error word; limit_ns the bound of each
// barrier wait; extra > 0 makes every barrier unreachable (self-test of the
// bounded wait).  The grid is the co-resident block count (at most max_items).
template <typename T>
cudaError_t launch_multi_advance(const MultiProblem<T>* probs, const long long* prefix, int nprob, int nsteps,
                                 size_t tile_bytes, long long max_items, unsigned* bar, int* err,
                                 unsigned long long limit_ns, unsigned extra, cudaStream_t s, int* grid_out);

// K2 modes: ROTATE = full step (forward z, update, inverse z); PROJECT = the
// one-time transverse projection; ROTATE_SPECTRAL = forward z and update only,
// leaving the spectrum (natural kx, ky, kz order) in storage.
// KS_ROTATE_SPECTRAL_PROJ also removes the longitudinal part of B before the
// update (E's is removed by Eq. 3 itself, and k^ x B does not see it), which
// equals the one-time projection followed by the update.
enum KspaceMode { KS_ROTATE = 0, KS_PROJECT = 1, KS_ROTATE_SPECTRAL = 2, KS_ROTATE_SPECTRAL_PROJ = 3 };

// ---------------------------------------------------------------------------
// Kernel launchers (one translation unit each); all return cudaGetLastError().
// ---------------------------------------------------------------------------
// In-place FFT along one axis (0 = x, 1 = y, 2 = z) of ncomp consecutive
// components of an [ncomp][Nz][Ny][Nx] array.  dir = -1 forward, +1 inverse.
template <typename T>
cudaError_t launch_fft_axis(cplx<T>* data, int ncomp, const GridGeom& g, const Tables<T>& tb,
                            int axis, int dir, cudaStream_t s, long long* nlaunch);

// Register-resident variants; cudaErrorNotSupported (nothing launched) when the
// axis length or layout has no fast kernel.
template <typename T>
cudaError_t launch_fft_axis_fast(cplx<T>* data, int ncomp, const GridGeom& g, const Tables<T>& tb,
                                 int axis, int dir, cudaStream_t s);
template <typename T>
cudaError_t launch_kspace_fast(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, cudaStream_t s);

// Fused x pass of a step in z, y, x order (N_x = 512 or 1024 in float32,
// complex storage): forward x, the Eq. 3-4 update of every mode, inverse x, one
// block per (k_y, k_z) row with all six components; y and z already in k-space.
// cudaErrorNotSupported (nothing launched) for other shapes.
template <typename T>
cudaError_t launch_kspace_rows(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, cudaStream_t s);
bool kspace_rows_supported(int prec, const GridGeom& g);

// Half spectrum of real fields in the slot order of the real-field plane
// kernels: per slot p < Nx/2 the wave number k_x, and the coefficient table
// with its x index in slot order (column p = slot p, column Nx/2 = the x
// Nyquist mode), (Nz/2+1) x (Ny/2+1) x (Nx/2+1) entries.
// nyq: [6][Nz][Ny] complex, the x Nyquist spectrum of the real fields, and
// map_nyq its 3D tensor map {Ny * sizeof(complex)/8, Nz, 6} (box {W, Nz, 1}).
template <typename T> struct HalfSlots {
    const T* k;
    const ModeCoef<T>* coef;
    cplx<T>* nyq;
    const CUtensorMap* map_nyq;
    bool project_e = false;     // project E (mean on Nyquist planes) before the update
};

// Tensor-copy-fed k-space pass; `map` describes the field as a 4D tensor of
// 8-byte elements {nx * sizeof(complex)/8, Ny, Nz, 6} (nx = Nx, or Nx/2 slots
// for the half spectrum) with box {kspace_tma_box_x(prec), 1,
// kspace_tma_box_z(Nz), 1}.  Device errors are OR-ed into *err.  With `half`
// the storage is a real-field half spectrum (rotation only; slot 0 untouched).
template <typename T>
cudaError_t launch_kspace_tma(const CUtensorMap& map, cplx<T>* data, const GridGeom& g, const Tables<T>& tb,
                              int* err, cudaStream_t s, bool spectral_out = false, bool project_b = false,
                              const HalfSlots<T>* half = nullptr);

// Real-field plane transforms (FP32, 256 x 256 planes, in place): dir < 0 =
// r2c along x + y, dir > 0 = inverse y + c2r.  Spectra are in slot order
// (plane_rc_slot_mode(p) = x mode index of slot p); the x Nyquist spectrum goes
// to / comes from nyq [ncomp * Nz][Ny].
cudaError_t launch_plane_rc(float* data, float2* nyq, int ncomp, const GridGeom& g, const Tables<float>& tb,
                            int dir, cudaStream_t s);
bool plane_rc_supported(int prec, const GridGeom& g);
int plane_rc_slot_mode(int p);

int kspace_tma_box_x(int prec);
int kspace_tma_box_z(int Nz);
cudaError_t launch_wait_timeout_selftest(int* err, cudaStream_t s);

// Fused x+y FFT of x-y planes through a thread-block cluster (distributed
// shared memory); cudaErrorNotSupported (nothing launched) for other shapes.
template <typename T>
cudaError_t launch_plane_xy(cplx<T>* data, int ncomp, const GridGeom& g, const Tables<T>& tb, int dir,
                            cudaStream_t s);
bool plane_xy_supported(int prec, const GridGeom& g);

// Fused z-forward FFT, per-mode update, z-inverse FFT over all six components.
template <typename T>
cudaError_t launch_kspace_z(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, int mode,
                            double scale, cudaStream_t s, long long* nlaunch);

// Per-mode update (any KspaceMode's update, no transform) of a spectrum
// transformed along all three axes.
template <typename T>
cudaError_t launch_modes(cplx<T>* data, const GridGeom& g, const Tables<T>& tb, int mode, double scale,
                         cudaStream_t s);

// Pulse initialisation on the mapped grid.
template <typename T>
cudaError_t launch_init_pulse(cplx<T>* data, const GridGeom& g, const ShellGeom& sh,
                              const PulseParams& p, int m_lo, int m_hi, cudaStream_t s,
                              long long* nlaunch);

// Focal-plane sampling scratch and launch.
// The same pulse written as real float32 values (real field storage).
cudaError_t launch_init_pulse_real(float* data, const GridGeom& g, const ShellGeom& sh, const PulseParams& p,
                                   int m_lo, int m_hi, cudaStream_t s, long long* nlaunch);

struct SampleScratch {
    double2* wx;     // [Nx]
    double2* wy;     // [ny][Ny]
    double2* wz;     // [nz][Nz]
    double2* g;      // [ncomp][Nz][Ny]
    double2* h;      // [ncomp][Nz][ny]
};
template <typename T>
cudaError_t launch_sample_plane(const cplx<T>* data, const GridGeom& g, const ShellGeom& sh,
                                double x_phys, int ny, int nz, double y0, double y1, double z0,
                                double z1, double t, const int* comps, int ncomp,
                                const SampleScratch& sc, cplx<T>* out, cudaStream_t s,
                                long long* nlaunch, bool from_spectrum = false);

// Diagnostics: energy partials and spectral divergence partials.
// Sampling of real float32 storage: from the real field (from_spectrum false),
// or from the half spectrum the one-shot leaves (slots [6][Nz][Ny][Nx/2] with
// x mode slot_mode[p], the x Nyquist spectrum in nyq [6][Nz][Ny]).
cudaError_t launch_sample_plane_real(const float* data, const float2* nyq, const int* slot_mode, const GridGeom& g,
                                     const ShellGeom& sh, double x_phys, int ny, int nz, double y0, double y1,
                                     double z0, double z1, double t, const int* comps, int ncomp,
                                     const SampleScratch& sc, float2* out, cudaStream_t s, long long* nlaunch,
                                     bool from_spectrum);

template <typename T>
cudaError_t launch_energy(const cplx<T>* data, size_t n_per_comp, double* partial, int nblocks,
                          cudaStream_t s, long long* nlaunch);
template <typename T>
cudaError_t launch_divergence(const cplx<T>* spec3, const GridGeom& g, const Tables<T>& tb,
                              double* partial, int nblocks, cudaStream_t s, long long* nlaunch);
// Real float32 storage: the energy from the real fields [6][n], and the
// divergence maxima of three real components from their half spectrum in slot
// order (spec [3][Nz][Ny][Nx/2], slot p at wave number slot_k[p]) and x-Nyquist
// array (nyq [3][Nz][Ny], wave number kx_nyq).
cudaError_t launch_energy_real(const float* data, size_t n_per_comp, double* partial, int nblocks, cudaStream_t s,
                               long long* nlaunch);
cudaError_t launch_divergence_half(const float2* spec, const float2* nyq, const GridGeom& g, const float* slot_k,
                                   float kx_nyq, const Tables<float>& tb, double* partial, int nblocks,
                                   cudaStream_t s, long long* nlaunch);
// Final reduction of `nblocks` rows of `width` doubles: columns [0, nsum) are
// summed, columns [nsum, width) are max-reduced.  Result in out[width].
cudaError_t launch_reduce_final(const double* partial, int nblocks, int width, int nsum,
                                double* out, cudaStream_t s, long long* nlaunch);

// Strided batched GEMM on the tensor cores (gemm.cu): C[b] = alpha A[b] B[b] +
// beta C[b], A[b](m,k) = A[b0 sAb0 + b1 sAb1 + m sAm + k sAk], b = (b0, b1), float32
// in memory, bfloat16 tiles, float32 accumulation; ksplit > 1 splits K over
// blocks with float atomics.
struct GemmArgs {
    int M, N, K;
    int nb0, nb1;                 // batch = nb0 x nb1
    const float* A;
    long long sAb0, sAb1, sAm, sAk;
    const float* B;
    long long sBb0, sBb1, sBk, sBn;
    float* C;
    long long sCb0, sCb1, sCm, sCn;
    float alpha, beta;
    int ksplit;
};
cudaError_t launch_gemm(const GemmArgs& a, cudaStream_t s);

// C (M x N, row-major float32) = A B^T with A (M x K) and B (N x K) K-major
// bfloat16 in device memory, fed to the tensor cores by tensor copies; M a
// multiple of 128, N of 256, K of 64, 16-byte aligned pointers
// (cudaErrorInvalidValue otherwise).
cudaError_t launch_gemm_tma(const void* A, const void* B, float* C, int M, int N, int K, cudaStream_t s);
bool gemm_take_error();

}  // namespace psatd
