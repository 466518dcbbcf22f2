/*
 * psatd.h -- C ABI of the GB300 PSATD tight-focusing library.
 *
 * The library advances an electromagnetic pulse in vacuum with the analytic-in-
 * time spectral (PSATD) Maxwell solver of arXiv:2010.00409, Sec. 2.1 (Eq. 3-4),
 * on the periodic layer produced by the mapping of Sec. 2.3 (Eq. 13), and maps
 * the result back to physical space with the cut-out of Eq. 14-16.
 *
 * Conventions shared by every entry point:
 *  - Units are those of the caller; the paper uses CGS (Sec. 2.1).  c is passed.
 *  - Field storage is six complex components in the order Ex, Ey, Ez, Bx, By, Bz,
 *    component-major, each [Nz][Ny][Nx] with x fastest ("SoA").  Precision 32
 *    stores float2 (8 B per value, 48 B per cell); precision 64 stores double2
 *    (16 B per value, 96 B per cell).  Node (i, j, l) sits at
 *    (x_min + i*dx, y_min + j*dy, z_min + l*dz).
 *  - The forward DFT is unnormalised with kernel exp(-i k.x); wave numbers are
 *    k_m = 2*pi*m/(N*d), m in {-floor(N/2), ..., ceil(N/2)-1} (numpy order), so the
 *    Nyquist index of even N is -N/2.  At k = 0 the unit vector k^ is 0.
 *  - Every call returns a psatd_status; nothing throws or aborts across the ABI.
 *    On error the context keeps its previous state and psatd_last_error() holds
 *    a one-line message.
 *  - Work is enqueued on the CUDA stream given to psatd_init_grid and is
 *    asynchronous, except where a call says it synchronises.
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Host pointers are plain pageable or pinned memory owned by the caller;
 *    device pointers are owned by the caller unless stated otherwise.
 *  - Sizes: every N must be 1..2048 and factor into 2, 3 and 5 (else
 *    PSATD_ERR_SIZE).
 */
#ifndef PSATD_H
#define PSATD_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psatd_ctx psatd_ctx;

typedef enum psatd_status {
    PSATD_OK = 0,
    PSATD_ERR_ARG = -1,      /* NULL pointer, bad enum, non-finite or inconsistent value */
    PSATD_ERR_SIZE = -2,     /* N outside 1..2048 or with a prime factor other than 2, 3, 5 */
    PSATD_ERR_OOM = -3,      /* a device allocation failed */
    PSATD_ERR_CUDA = -4,     /* a CUDA runtime call or kernel launch failed */
    PSATD_ERR_TIMEOUT = -5,  /* a bounded device wait expired */
    PSATD_ERR_STATE = -6     /* call not valid in the current state (e.g. no fields) */
} psatd_status;

enum { PSATD_PULSE_FLAT_TOP = 0, PSATD_PULSE_GAUSSIAN = 1, PSATD_PULSE_PROFILE = 2 };
enum { PSATD_FORWARD = -1, PSATD_INVERSE = +1 };
enum { PSATD_FLAG_NO_FIELD_ALLOC = 1,     /* init_grid: caller binds field storage */
       PSATD_FLAG_REAL_FIELDS = 2 };     /* init_grid: real field storage (see below) */

/* The periodic box (Sec. 2.3): D = Nx*dx is the period of the mapped layer. */
typedef struct psatd_grid {
    int Nx, Ny, Nz;
    double dx, dy, dz;
    double x_min, y_min, z_min;   /* node (0,0,0); Eq. 13 layer uses x_min = -R_min - D */
    double c;                     /* speed of light (CGS: 2.99792458e10 cm/s) */
} psatd_grid;

/* Geometry of the initial spherical shell R0 - L/2 <= R <= R0 + L/2 (Sec. 2.2);
 * used by the pulse models and by the cut-out I_S of Eq. 15-16. */
typedef struct psatd_mapping {
    double R0;
    double L;
} psatd_mapping;

/* Pulse models.  FLAT_TOP is Eq. 5-11 (u = A/R u_l(R-R0) u_ts(alpha), A of Eq. 9,
 * E = u s0, B = u s1).  GAUSSIAN is Sec. 3.2.1: u = E0 R0 sin(k(R-R0)+phi) u_l u_ts / R
 * with u_l = exp(-zeta^2 ln4/(n lambda)^2) on |zeta| <= L/2 and
 * u_ts = exp(-alpha^2/theta0^2) times the Eq. 5 edge at 2*theta0 with width eps;
 * E0 = sqrt(4 P0 / (c R0^2 F(theta0))) with the series F of Sec. 3.2.1 (CGS form).
 * alpha is the angle from the -x axis; s0 = |R x (d x R)|^-1 R x (d x R) and
 * s1 = |d x R|^-1 d x R; d1 = (0, cos psi, sin psi), d2 = (0, -sin psi, cos psi);
 * E = u_phi s0(d1) + e u_{phi+pi/2} s0(d2) and likewise B with s1.  Replicas of the
 * pulse spaced D along x are summed at every node (Sec. 2.3). */
typedef struct psatd_pulse {
    int kind;            /* PSATD_PULSE_FLAT_TOP, PSATD_PULSE_GAUSSIAN or PSATD_PULSE_PROFILE */
    int div_project;     /* nonzero: remove k^(k^.E) and k^(k^.B) once after init (Sec. 2.1) */
    double lambda;       /* carrier wavelength */
    double theta;        /* flat-top half angle theta; Gaussian theta0 */
    double eps;          /* edge smoothing angle of Eq. 5 */
    double P0;           /* power (cycle-averaged, as Eq. 9 and Sec. 3.2.1) */
    double n_cycles;     /* Gaussian FWHM duration in wavelengths (n of Sec. 3.2.1) */
    double cep;          /* carrier phase phi */
    double ellipticity;  /* e in [0, 1] */
    double pol_angle;    /* psi */
} psatd_pulse;

/* Energy and spectral divergence of the current fields. */
typedef struct psatd_diag {
    double energy;       /* sum over cells of |E|^2 + |B|^2 */
    double energy_E;
    double energy_B;
    double max_div_E;    /* max over k of |k^ . FFT(E)(k)| (unnormalised DFT) */
    double max_div_B;
    double max_E_hat;    /* max over k of |FFT(E)(k)| (vector norm) */
    double max_B_hat;
} psatd_diag;

/* Create a context for one periodic box and allocate its tables (and, unless
 * flags has PSATD_FLAG_NO_FIELD_ALLOC, the six-component field storage, zeroed).
 * dt is the step of psatd_advance; precision is 32 or 64; cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  The mapping geometry is only
 * needed by psatd_init_pulse and psatd_sample_focal_plane.
 *
 * Field storage is complex [6][Nz][Ny][Nx] (8 or 16 bytes per value) by
 * default.  With PSATD_FLAG_REAL_FIELDS it is real float32 [6][Nz][Ny][Nx]
 * (4 bytes per value; the physical E and B are real): precision must be 32,
 * Nx = Ny = 256 and Nz one of 64, 128, 256 (else PSATD_ERR_ARG).  A real-field
 * step is the real part of the complex step (Sec. 2.1, Eq. 3-4; on Nyquist
 * planes this is the mean of the update at the two mirrored wave vectors) and
 * moves half the bytes.  In that mode psatd_fft returns PSATD_ERR_STATE
 * (psatd_energy_noalloc reads complex storage only) and psatd_autotune keeps
 * the one real-field kernel set.  psatd_init_pulse writes the (real) pulse
 * straight into the real storage and projects it with one real-field pass;
 * psatd_sample_focal_plane reads the real field, and psatd_focal_one_shot
 * leaves and samples the half spectrum (k_x >= 0, in the slot order of the
 * real-field plane pass, the x Nyquist modes in a context-owned array; the
 * negative k_x are their conjugates); psatd_diagnostics takes the energy from
 * the real fields and the divergence from the half spectrum of a real copy of
 * three components (12 bytes per cell, allocated on its first use).
 * Cites: Sec. 2.1 (solver), Sec. 2.3 (periodic layer). */
psatd_status psatd_init_grid(const psatd_grid* grid, const psatd_mapping* mapping,
                             double dt, int precision, void* cuda_stream, int flags,
                             psatd_ctx** out);

/* Release everything the context owns (not caller-bound field storage). */
void psatd_destroy(psatd_ctx* ctx);

/* Change the step; rebuilds the cos/sin table on the host in float64.  Any finite
 * dt is valid, including negative (time reversal) and large (Sec. 2.1: the
 * vacuum solver is exact in time for any step). */
psatd_status psatd_set_dt(psatd_ctx* ctx, double dt);

/* Replace the shell geometry used by later psatd_init_pulse,
 * psatd_focal_one_shot and psatd_sample_focal_plane calls. */
psatd_status psatd_set_mapping(psatd_ctx* ctx, const psatd_mapping* mapping);

/* Use caller-owned device memory (e.g. a torch tensor) as the field storage.
 * bytes must be at least 6*Nx*Ny*Nz*(8 or 16; 4 with real fields) and dev_ptr
 * 256-byte aligned.
 * Library-owned storage, if any, is freed.  The memory must outlive the context
 * or the next bind. */
psatd_status psatd_bind_fields(psatd_ctx* ctx, void* dev_ptr, size_t bytes);

/* Device pointer and size of the current field storage. */
psatd_status psatd_fields(psatd_ctx* ctx, void** dev_ptr, size_t* bytes);

/* Copy component comp (0..5, or -1 for all six) from src, laid out as the field
 * storage of that component(s).  src_on_device selects device or host memory.
 * Host copies synchronise the stream. */
psatd_status psatd_set_field(psatd_ctx* ctx, int comp, const void* src, int src_on_device);
psatd_status psatd_get_field(psatd_ctx* ctx, int comp, void* dst, int dst_on_device);

/* Initialise all six components from a pulse model on the mapped grid (Eq. 5-13,
 * Sec. 3.2.1).  Coordinates and the pulse are evaluated in float64 and rounded
 * once.  Resets the time to 0. */
psatd_status psatd_init_pulse(psatd_ctx* ctx, const psatd_pulse* pulse);

/* Longitudinal profile of PSATD_PULSE_PROFILE pulses.  Sec. 2.2 lets the pulse
 * have an arbitrary profile along the radial direction; this kind keeps the
 * flat-top transverse shape of Eq. 5 and the amplitude A/R of Eq. 8-9, and takes
 * the longitudinal factor from a table: u_l(zeta) = Re(a(zeta) e^{i phi}) with
 * zeta = R - R0, phi the pulse's cep (cep + pi/2 for the second polarisation)
 * and a(zeta) the complex (analytic) waveform linearly interpolated between the
 * samples a_k = a(zeta0 + k dzeta), k < n; u_l = 0 outside [zeta0, zeta0 +
 * (n-1) dzeta] and outside |zeta| <= L/2.  With a the analytic signal g + i H[g]
 * of a real waveform g (H the Hilbert transform along zeta), phi acts as a
 * carrier-envelope phase: a = -i e^{i k zeta} cos^2(pi zeta/L) gives Eq. 7's
 * sin(k zeta + phi) cos^2(pi zeta/L).
 * samples: 2n float64 (re, im interleaved), host memory, copied; n in
 * 2..1048576, dzeta > 0, all finite.  The table stays with the context until
 * replaced.  Synchronises. */
psatd_status psatd_set_pulse_profile(psatd_ctx* ctx, const double* samples, int n, double zeta0, double dzeta);

/* Advance n_steps >= 0 PSATD steps of size dt (Eq. 3-4): per step a forward 3D
 * FFT of the six components, the per-mode update, and an inverse 3D FFT; the
 * physical field is in storage after every step.  Asynchronous. */
psatd_status psatd_advance(psatd_ctx* ctx, int n_steps);

/* In-place 3D DFT of all six components with the library's FFT kernels:
 * direction PSATD_FORWARD (exp(-ikx)) or PSATD_INVERSE (exp(+ikx)); both
 * unnormalised.  Asynchronous. */
psatd_status psatd_fft(psatd_ctx* ctx, int direction);

/* After psatd_focal_one_shot (storage holds the updated spectrum) this samples
 * the same interpolant from the spectrum, so further planes of the focal region
 * cost no transform.
 * Sample the physical field on the plane x = x_phys at y_p = y0 + p (y1-y0)/ny,
 * z_q = z0 + q (z1-z0)/nz (p < ny, q < nz) at the current time t, as
 * u(R, t) = u~(T(R)) I_S(t)(R) (Eq. 13-16) with u~ the exact trigonometric
 * interpolant of the grid field.  comp_mask selects components (bit c = component
 * c); dst receives popcount(comp_mask) planes [nz][ny] of complex values in the
 * context precision, in increasing component order.  Synchronises when dst is
 * on the host.  ny, nz in 1..4096. */
psatd_status psatd_sample_focal_plane(psatd_ctx* ctx, double x_phys, int ny, int nz,
                                      double y0, double y1, double z0, double z1,
                                      int comp_mask, void* dst, int dst_on_device);

/* One-shot focal field (the solver is exact in time in vacuum, Sec. 2.1 and the
 * single step of Delta t = R0/c of Sec. 3.1): initialise the pulse (as
 * psatd_init_pulse, including its div_project), advance by ONE step of size T,
 * and sample the plane x = x_phys at time T exactly as psatd_sample_focal_plane,
 * evaluating the interpolant straight from the updated spectrum (no inverse 3D
 * transform).  Afterwards the field storage holds that spectrum, so advance,
 * fft and diagnostics return PSATD_ERR_STATE until a pulse
 * or all six components are set again (psatd_sample_focal_plane keeps working,
 * from the spectrum); psatd_time() is T.  The coefficient
 * table for T is built on the host (float64) and cached for the next call with
 * the same T.  With real field storage the spectrum is the half spectrum of
 * real fields (the update is the real-field one, with the projection of B
 * folded in) and the sample is the same interpolant of the real field. */
psatd_status psatd_focal_one_shot(psatd_ctx* ctx, const psatd_pulse* pulse, double T, double x_phys,
                                  int ny, int nz, double y0, double y1, double z0, double z1,
                                  int comp_mask, void* dst, int dst_on_device);

/* Energy and spectral divergence of the current fields (float64 accumulation).
 * Synchronises. */
psatd_status psatd_diagnostics(psatd_ctx* ctx, psatd_diag* out);

/* Current time t = (steps taken since init_pulse or set_time) * dt, summed. */
double psatd_time(const psatd_ctx* ctx);
psatd_status psatd_set_time(psatd_ctx* ctx, double t);

/* Wait for all work of the context's stream.  Returns PSATD_ERR_TIMEOUT if a
 * kernel reported an expired bounded wait since the last check (the affected
 * step left the field unchanged); the error word is then cleared.  get_field
 * to host, sample_focal_plane to host and diagnostics check it too. */
psatd_status psatd_synchronize(psatd_ctx* ctx);

/* Eq. 12: D_min = -R_min cos(theta) + sqrt(R_max^2 - R_min^2 sin^2(theta)). */
double psatd_d_min(double R0, double L, double theta);

/* Message of the last failed call on ctx (or of the last failed psatd_init_grid
 * when ctx is NULL).  Never NULL. */
const char* psatd_last_error(const psatd_ctx* ctx);

/* Static name of a status code. */
const char* psatd_status_string(psatd_status s);

/* Number of kernel launches the context has issued since creation. */
long long psatd_launch_count(const psatd_ctx* ctx);

/* Kernel selection: AUTO uses the register-resident kernels where the axis
 * length has one (64, 128, 256, 512; the k-space pass for Nz in 64, 128, 256,
 * fed by tensor copies), and the generic shared-memory Stockham kernels
 * elsewhere; REGISTER is AUTO without the tensor-copy feed; GENERIC forces the
 * generic kernels everywhere.  All compute the same transform; default AUTO. */
enum { PSATD_PATH_AUTO = 0, PSATD_PATH_GENERIC = 1, PSATD_PATH_REGISTER = 2 };
psatd_status psatd_set_kernel_path(psatd_ctx* ctx, int path);

/* Self-test of device wait reporting: launches one block that waits, with a
 * short bound, on a barrier nothing completes, and returns what
 * psatd_synchronize reports (PSATD_ERR_TIMEOUT when the bound works).  The
 * context stays usable afterwards.  The paper has no counterpart. */
psatd_status psatd_selftest_wait_timeout(psatd_ctx* ctx);

/* Energy sums (|E|^2 and |B|^2 over all cells, float64) of a six-component field
 * in the storage layout above, for callers that cannot allocate device memory
 * when they need it: during CUDA graph capture, under a framework allocator
 * that has reserved the whole device, or in loops where cudaMalloc/cudaFree
 * (which may synchronise the device) are not acceptable.  It allocates nothing:
 * its partial sums live in a 1 MB array compiled into the library, so n_cells
 * must be 1..2^30 (else PSATD_ERR_SIZE).  fields is a device pointer to
 * 6 * n_cells complex values of the given precision (32 or 64); out receives
 * {energy_E, energy_B}, on the device (out_on_device != 0, asynchronous on
 * cuda_stream) or on the host (the call then synchronises the stream).  The
 * first call on each device looks up the array's device address and loads the
 * entry point's kernels for both precisions (the runtime would otherwise load
 * each kernel on its first launch, which can allocate); make that first call
 * before any stream capture.  After it, no call on that device allocates.  All
 * calls share the array, so calls that overlap on the GPU race and must be
 * serialised by the caller.  Needs no context; errors are returned only as the
 * status, and a launch failure is reported from the launch itself: an error the
 * caller left pending is not consumed.  The paper has no counterpart. */
psatd_status psatd_energy_noalloc(const void* fields, int precision, long long n_cells, double* out,
                                  int out_on_device, void* cuda_stream);

/* Failure injection for host-side tests (the paper has no counterpart).
 * psatd_debug_set_alloc_limit caps the bytes of device memory the library's
 * contexts hold (fields it allocates, tables, scratch): an allocation that
 * would pass the cap fails as cudaMalloc would (the call returns
 * PSATD_ERR_OOM) without reaching the driver; bytes < 0 removes the cap.
 * psatd_debug_alloc_live returns the bytes held now.
 * psatd_debug_inject_cuda_error makes the after_calls-th checked CUDA call of
 * the C ABI from now (counted over all contexts; a step launch of
 * psatd_advance counts as one) return cuda_error (a cudaError_t value) without
 * being made, so the entry point returns PSATD_ERR_CUDA (PSATD_ERR_OOM for
 * cudaErrorMemoryAllocation); after_calls <= 0 disarms.  Both are
 * process-wide and not synchronised with calls in flight on other threads. */
void psatd_debug_set_alloc_limit(long long bytes);
/* In a library built with -DPSATD_DEBUG (libpsatd_debug.so) every global index
 * of the field, table and scratch buffers the kernels touch is checked against
 * its buffer: an index outside the buffer is counted and replaced by 0 (the
 * access stays inside), the first one kept with its bound.  This call
 * synchronises the device, returns the number of such indices since the last
 * call (and clears it) and writes the first index and bound when it is > 0;
 * -1 on a CUDA error, -2 in a library built without the checks. */
long long psatd_debug_bounds_report(long long* first_index, long long* first_bound);
long long psatd_debug_alloc_live(void);
void psatd_debug_inject_cuda_error(int after_calls, int cuda_error);

/* Batches: record a sequence of calls on contexts that share one (non-default)
 * CUDA stream into a CUDA graph and replay it with a single launch, e.g. one
 * exact step per pulse realisation for parameter sweeps.  Between
 * psatd_batch_begin and psatd_batch_end (same host thread) only psatd_advance
 * and psatd_focal_one_shot with a device dst are recorded; calls that need the
 * host to wait (host copies, diagnostics, set_dt, synchronize,
 * sample_focal_plane) return PSATD_ERR_STATE, and a one-shot must have run once
 * outside the capture with the same T and plane size (tables and buffers are
 * prepared then).  psatd_batch_launch enqueues the graph on the stream and
 * moves each context's time as the recorded calls would have. */
typedef struct psatd_batch psatd_batch;
psatd_status psatd_batch_begin(void* cuda_stream, psatd_batch** out);
psatd_status psatd_batch_end(psatd_batch* batch);
psatd_status psatd_batch_launch(psatd_batch* batch);
long long psatd_batch_nodes(const psatd_batch* batch);      /* graph nodes, 0 if none */
void psatd_batch_destroy(psatd_batch* batch);

/* Persistent batched advance (the parameter sweeps of Sec. 3.2.3: statistics
 * over many perturbed pulse realisations, each on its own periodic layer of
 * Sec. 2.3).  Advances context ctxs[p] by n_steps[p] >= 0 PSATD steps of its
 * own dt (Sec. 2.1, Eq. 3-4), for all p < n_ctx, in ONE cooperative kernel
 * launch on the stream of ctxs[0] that runs the largest count (a box past its
 * own count skips its work): each step is five phases (x, y, the fused z pass with the
 * update, y inverse, x inverse), each a list of work items over all boxes, with
 * a grid-wide barrier between phases.  The contexts need complex field storage
 * (not PSATD_FLAG_REAL_FIELDS), one precision, one device and one stream,
 * distinct field storage and axis lengths up to 1024; grids may all differ.
 * Each barrier wait is bounded (2 s): if one expires the blocks leave the
 * kernel, the boxes' fields are invalid, and the next psatd_synchronize of
 * ctxs[0] returns PSATD_ERR_TIMEOUT.  Radix schedules and tile widths come from
 * psatd_multi_autotune when it has run for the axis lengths, else defaults.
 * Asynchronous; recorded into a batch capture when ctxs[0]'s stream is being
 * captured (the same boxes with the same step counts must have been advanced
 * once before the capture: that call uploads their descriptors).  Errors are reported through ctxs[0] (psatd_last_error). */
psatd_status psatd_multi_advance(psatd_ctx* const* ctxs, int n_ctx, const int* n_steps);

/* Autotuner of the batched advance: on copies of the fields (the contexts'
 * fields are left unchanged), times trial_steps steps of the whole batch for
 * every distinct radix schedule (radices 8/4/5/3/2 or 4/5/3/2, largest or
 * smallest first) and tile-width scale (1/2, 1, 2) of each axis length in turn
 * (coordinate descent), keeps the fastest and caches it per (precision, axis
 * length) for later psatd_multi_advance calls in this process.  Writes the best
 * time per step.  Synchronises the stream; needs memory for one copy of all
 * the fields (PSATD_ERR_OOM otherwise, nothing changed). */
psatd_status psatd_multi_autotune(psatd_ctx* const* ctxs, int n_ctx, int trial_steps, double* ms_per_step);

/* Self-test of the batched advance's bounded grid barrier: launches it on this
 * context with one arrival more than the grid can give, so every block's first
 * barrier wait expires after 2 ms; returns what psatd_synchronize reports
 * (PSATD_ERR_TIMEOUT when the bound works).  The field content is undefined
 * afterwards; the context stays usable.  The paper has no counterpart. */
psatd_status psatd_selftest_grid_barrier_timeout(psatd_ctx* ctx);

/* Autotuner: times trial_steps PSATD steps of each kernel path (AUTO, REGISTER,
 * GENERIC) and generic tile width scale (1/2, 1, 2) on a scratch copy of the
 * field, keeps the fastest for this context and caches it per grid shape and
 * precision for the process (later calls for the same shape apply the cached
 * choice without timing and report ms_per_step = -1).  Outputs may be NULL. */
psatd_status psatd_autotune(psatd_ctx* ctx, int trial_steps, int* path, int* tile_shift, double* ms_per_step);

/* ---------------------------------------------------------------------------
 * Surrogate: a Fourier neural operator from pulse parameters to the field on a
 * focal patch, trained and evaluated with the library's own kernels (tensor-core
 * GEMMs in bfloat16 with float32 accumulation, float32 elsewhere).  The paper
 * has no counterpart; it motivates statistical sweeps (Sec. 3.2.3) whose focal
 * fields the solver produces and judges.
 *   v0 = W_lift [p_1..p_n, x, y, z] + b,  v_l = act(S_l v_{l-1} + W_l v_{l-1} + b_l)
 *   out = W_q2 GELU(W_q1 v_L + b_q1) + b_q2
 * S_l: truncated DFT (kx in [0, modes), ky, kz in {0..modes-1, P-modes..P-1}),
 * a complex width x width matrix per kept mode, inverse DFT; act = GELU except
 * on the last layer.  Coordinates are -1 + 2 i / patch.  Tensors are float32,
 * sample-major: params [batch][in_params], output and targets
 * [batch][out_channels][patch^3] with x fastest. */
typedef struct psatd_fno psatd_fno;
typedef struct psatd_fno_config {
    int in_params;      /* scalar inputs per sample (coordinates are added) */
    int width;          /* channels */
    int layers;         /* spectral layers */
    int patch;          /* P: output patch P^3, even, 4..128 */
    int modes;          /* kept modes per sign and axis, 2*modes <= P */
    int hidden;         /* projection hidden channels */
    int out_channels;
    int max_batch;
} psatd_fno_config;
/* Allocate parameters (seeded uniform initialisation), Adam state and the
 * activation buffers for max_batch samples on the current device. */
psatd_status psatd_fno_create(const psatd_fno_config* cfg, unsigned long long seed, void* cuda_stream,
                              psatd_fno** out);
void psatd_fno_destroy(psatd_fno* fno);
long long psatd_fno_num_params(const psatd_fno* fno);
/* Device pointers of the flat parameter vector, its gradient and the last
 * forward output (owned by the model). */
psatd_status psatd_fno_buffers(psatd_fno* fno, float** params, float** grads, float** output);
/* Forward pass; out may be NULL (the result stays in the model's output buffer). */
psatd_status psatd_fno_forward(psatd_fno* fno, const float* params_dev, int batch, float* out_dev);
/* Forward, mean squared error against target, backward: gradients overwrite the
 * gradient vector; *loss (may be NULL) is set after a synchronisation. */
psatd_status psatd_fno_loss_backward(psatd_fno* fno, const float* params_dev, int batch, const float* target_dev,
                                     double* loss);
psatd_status psatd_fno_adam_step(psatd_fno* fno, float lr, float beta1, float beta2, float eps, float weight_decay);
psatd_status psatd_fno_synchronize(psatd_fno* fno);
const char* psatd_fno_last_error(const psatd_fno* fno);

/* The tensor-core GEMM used by the surrogate (the surrogate is not in the
 * paper; its dense contractions), on device float32 matrices with arbitrary
 * strides: C = alpha A B + beta C (A: M x K, B: K x N), operands rounded to
 * bfloat16, tcgen05.mma with float32 accumulation in tensor memory.  ksplit > 1
 * splits K over tiles (partial sums added atomically).  Asynchronous on
 * cuda_stream; returns PSATD_ERR_ARG for NULL pointers or negative sizes.  An
 * expired bounded wait inside the kernel is reported by the next
 * psatd_fno_synchronize. */
psatd_status psatd_gemm_bf16(int M, int N, int K, const float* A, long long sAm, long long sAk, const float* B,
                             long long sBk, long long sBn, float* C, long long sCm, long long sCn, float alpha,
                             float beta, int ksplit, void* cuda_stream);

/* Tensor-core GEMM with bfloat16 operands in memory (the surrogate's dense
 * contractions at scale; the paper has none): C = A B^T, A (M x K) and B (N x K)
 * row-major bfloat16 (K contiguous), C (M x N) row-major float32, float32
 * accumulation in tensor memory.  Operands reach shared memory through tensor
 * copies with 128-byte swizzle, four stages deep; tiles 128 x 256.  M must be a
 * multiple of 128, N of 256, K of 64, and the three device pointers 16-byte
 * aligned (PSATD_ERR_ARG otherwise).  Asynchronous on cuda_stream. */
psatd_status psatd_gemm_bf16_tma(int M, int N, int K, const void* A, const void* B, float* C, void* cuda_stream);

/* Synchronise cuda_stream; PSATD_ERR_TIMEOUT if a bounded wait inside a GEMM
 * kernel expired since the last check (the results of that GEMM are invalid). */
psatd_status psatd_gemm_synchronize(void* cuda_stream);

/* Float64 arithmetic rate probe, the denominator of the float64 solver's
 * roofline (that path is bound by float64 arithmetic, not by memory): launches
 * blocks x threads threads on cuda_stream; each runs eight independent chains
 * of iters float64 fused multiply-adds, i.e. 16 * iters floating-point
 * operations per thread, and writes one double to out[thread] (device memory
 * of blocks * threads doubles, owned by the caller).  The caller times the
 * launch (CUDA events on the same stream).  PSATD_ERR_ARG for a NULL out,
 * blocks outside 1..2^20, threads not a multiple of 32 in 32..1024 or
 * iters < 1; PSATD_ERR_CUDA if the launch fails.  Asynchronous.  The paper has
 * no counterpart. */
psatd_status psatd_fp64_fma_probe(double* out, int blocks, int threads, int iters, void* cuda_stream);

/* Kernel kinds for per-kernel timing. */
enum {
    PSATD_KERNEL_FFT_X = 0,      /* generic FFT along x */
    PSATD_KERNEL_FFT_Y = 1,      /* generic FFT along y */
    PSATD_KERNEL_FFT_Z = 2,      /* generic FFT along z */
    PSATD_KERNEL_KSPACE = 3,     /* fused z-FFT / per-mode update / inverse z-FFT */
    PSATD_KERNEL_INIT = 4,       /* pulse initialisation */
    PSATD_KERNEL_SAMPLE = 5,     /* focal-plane sampling (all of its launches) */
    PSATD_KERNEL_DIAG = 6,       /* energy / divergence reductions */
    PSATD_KERNEL_PLANE_XY = 7,   /* fused x+y plane FFT (real fields: r2c / c2r plane kernels) */
    PSATD_KERNEL_KINDS = 8
};

/* Start (enable != 0) or stop per-kernel timing: while enabled every launch of
 * the context is bracketed by a pair of CUDA events on its stream.  Enabling
 * clears the accumulated totals. */
psatd_status psatd_profile_enable(psatd_ctx* ctx, int enable);

/* Accumulated device time (ms) and number of timed launches of one kernel kind
 * since profiling was enabled.  Synchronises the stream. */
psatd_status psatd_profile_read(psatd_ctx* ctx, int kind, double* total_ms, long long* launches);

/* Static name of a kernel kind ("fft_x", ...). */
const char* psatd_kernel_name(int kind);

#ifdef __cplusplus
}
#endif

#endif /* PSATD_H */
