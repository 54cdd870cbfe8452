/*
 * fsp.h -- C ABI of the GB300 (sm_103a) free-space spectral Poisson solver.
 *
 * The solver computes the free-space potential of a source sampled on an N^3
 * cell-centred grid of spacing h (cube side L = N h), the convolution
 * phi = G * rho with G(x) = 1/(4 pi |x|) (Sec. 1, Eq. convolution_eq of
 * Mayani et al., arXiv 2405.02603, with eps0 = 1), by the Hockney-Eastwood
 * doubled-grid FFT convolution (Sec. 2.2, steps 1-5):
 *
 *   phi_i = h^3 sum_{j in [0,N)^3} T[|i - j|] rho_j ,   i in [0,N)^3,
 *
 * where T is the real-space kernel of the chosen method (fsp_algo):
 *   FSP_HE     Hockney-Eastwood: T[m] = 1/(4 pi h |m|), T[0] = 1/(4 pi)
 *              (Sec. 2.2 step 3; origin value in this sign convention).
 *   FSP_VG     Vico-Greengard: inverse DFT on the (4N)^3 grid of the truncated
 *              spectral kernel G_L(k) = 2 (sin(L_t|k|/2)/|k|)^2 (Sec. 2.3, Eq.
 *              green_vico), L_t = 1.1 sqrt(3) L, restricted to the doubled grid.
 *   FSP_VG_DCT the paper's memory-reduced variant: the same kernel from a DCT-I
 *              on (2N+1)^3 samples (Sec. 2.4).
 *
 * Arrays: rho and phi are dense C-order arrays of N^3 reals, index
 * (z*N + y)*N + x, x fastest; `double` for FSP_F64, `float` for
 * FSP_F32_MIXED.  They belong to the caller.  phi == rho (in place) is allowed.
 *
 * Streams: `fsp_stream` is a cudaStream_t (NULL = the legacy default stream).
 * Device work is enqueued asynchronously on the given stream; an asynchronous
 * CUDA fault surfaces as FSP_ECUDA from a later call or from fsp_plan_sync.
 *
 * Errors: every entry point returns an fsp_status and never aborts the
 * process.  Arguments are validated synchronously before any device work is
 * enqueued; on an error return nothing has been enqueued and no output or
 * plan state has changed unless stated otherwise.
 */
#ifndef FSP_H
#define FSP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fsp_stream; /* identical to cudaStream_t */

typedef enum {
    FSP_OK = 0,
    FSP_EINVAL = 1,       /* bad argument, NULL or misaligned pointer, unknown or destroyed plan */
    FSP_EUNSUPPORTED = 2, /* size outside what the kernels support (e.g. 2N not 2/3/5-smooth) */
    FSP_ENOMEM = 3,       /* device allocation failed or exceeded a memory budget */
    FSP_ECUDA = 4,        /* a CUDA runtime call or a kernel launch failed */
    FSP_EBUSY = 5,        /* a queue or slot limit is reached; retry later */
    FSP_ETIMEOUT = 6      /* a bounded device-side wait ran out */
} fsp_status;

/* The paper's solver names HOCKNEY, VICO and VICO_2 (Sec. 4, availability). */
typedef enum { FSP_HE = 0, FSP_VG = 1, FSP_VG_DCT = 2 } fsp_algo;

/* FSP_F64: every step in double precision.
 * FSP_F32_MIXED: the solve (all transforms and the spectral multiply) in
 * single precision; the Green's spectrum is precomputed in double precision
 * and rounded once to single precision.
 * FSP_F64_DF: double arrays in and out, FP64-class accuracy (about 1e-14
 * relative), but the transforms run in double-float arithmetic (each value a
 * pair of floats, hi + lo) on the FP32 pipes, which on this GPU are far faster
 * than its FP64 pipes; the spectrum is the FP64 one split into float pairs.
 * Only where the specialised kernels run: N = 32, 64, 128, 256, 512, or a
 * non-cubic box whose sizes are powers of two in that range
 * (FSP_EUNSUPPORTED otherwise); not in batches.  Double-float keeps FP32's
 * exponent range: plan creation returns FSP_EUNSUPPORTED when the largest
 * spectrum value lies outside [2^-80, 2^80] (that value is about
 * 3e-6 L^2 (32/N)^3, so the box side L may range over about 1e-8 .. 1e14 at
 * N = 32 .. 512), and the caller keeps 8 N^3 max|rho| below about 2^80. */
typedef enum { FSP_F64 = 0, FSP_F32_MIXED = 1, FSP_F64_DF = 2 } fsp_dtype;

typedef struct fsp_plan fsp_plan;

/* Human-readable name of a status code (static string, never NULL). */
const char *fsp_status_str(fsp_status s);

/*
 * fsp_plan_create -- build a solver for one (N, L, h, algo, dtype) on the
 * current CUDA device.
 *
 * N      grid points per axis, N >= 2; 2N must be 2/3/5-smooth, and 4N too for
 *        FSP_VG (otherwise FSP_EUNSUPPORTED); N <= 1024.
 * L      cube side, L > 0 and finite.
 * h      grid spacing; must equal L/N to 1e-12 relative (else FSP_EINVAL).
 * algo   FSP_HE, FSP_VG or FSP_VG_DCT.
 * dtype  FSP_F64, FSP_F32_MIXED or FSP_F64_DF.
 * stream the precompute (plan-time Green's spectrum, Sec. 2.2 step 3, Sec. 2.3
 *        and Sec. 2.4) runs on this stream; the call returns after it has
 *        completed (it synchronises the stream) and temporaries are freed.
 *
 * The plan owns the spectrum S ((N+1)^3 reals) and the solve workspace
 * (3 N^2 P complex values, P = N+1 rounded up to 16).  FSP_VG needs a
 * (4N)^3 complex FP64 temporary, FSP_VG_DCT a (2N+1)^3 FP64 one, during the
 * call only.  On failure *out is set to NULL and nothing is leaked.
 */
fsp_status fsp_plan_create(fsp_plan **out, int N, double L, double h, fsp_algo algo, fsp_dtype dtype,
                           fsp_stream stream);

/*
 * fsp_plan_create_aniso -- a plan for a non-cubic box of nx x ny x nz cells
 * with spacings hx, hy, hz (sides L_a = n_a h_a), such as the 512^2 x 1024
 * grids of the paper's weak-scaling runs (Sec. 3.2).  The methods of
 * Sec. 2.2-2.4 per axis: HE samples 1/(4 pi |(m_x hx, m_y hy, m_z hz)|) with
 * T[0] = 1/(4 pi); VG and VG-DCT sample G_L on the (4 n_a) frequency grid
 * k_a = 2 pi j_a / (4 n_a h_a) (resp. its octant) with the window
 * L_t = 1.1 |(L_x, L_y, L_z)| (1.1 sqrt(3) L for a cube).  Layout of rho and
 * phi: nz x ny x nx reals, x fastest.
 *
 * A cube (nx = ny = nz, hx = hy = hz) returns the cubic plan of
 * fsp_plan_create, with its specialised kernels.  Otherwise, when every n_a
 * is a power of two in [32, 512] (FSP_F32_MIXED: n_y and n_z up to 1024), the
 * solve runs on the specialised kernels
 * (rows of n_x; column passes with runtime strides), in any dtype; else on
 * the generic engine (any 2/3/5-smooth 2 n_a, and 4 n_a for FSP_VG), dtype
 * FSP_F64 or FSP_F32_MIXED (FSP_F64_DF: FSP_EUNSUPPORTED).  FSP_VG and
 * FSP_VG_DCT need 3 min_a L_a >= L_t (the (4 n_a h_a)-periodic images of the
 * truncated kernel must stay outside the box): FSP_EUNSUPPORTED otherwise,
 * e.g. for a 1 x 1 x a box with a > 2.33.  The workspace is
 * 3 nz ny P complex values (P = nx+1 rounded up to 16), the spectrum
 * (nz+1)(ny+1)P reals.  fsp_solve, fsp_solve_host(_many), fsp_plan_sync,
 * fsp_plan_set_timing, fsp_plan_spectrum ((nz+1)(ny+1)(nx+1) doubles) and
 * fsp_plan_destroy accept the plan, and so do fsp_plan_field_init and
 * fsp_solve_field (the field kernels per axis, F_a = m_a h_a / (4 pi |r|^3)
 * for HE and the octant route with the box's window for VG); batches
 * (fsp_batch_create) return FSP_EUNSUPPORTED for it.
 */
fsp_status fsp_plan_create_aniso(fsp_plan **out, int nx, int ny, int nz, double hx, double hy, double hz,
                                 fsp_algo algo, fsp_dtype dtype, fsp_stream stream);

/*
 * fsp_solve -- one free-space solve, phi = G * rho (Sec. 2.2 steps 1-5):
 * zero-pad to (2N)^3 (never materialised), 3D real-to-complex FFT, multiply
 * by the plan's spectrum, inverse FFT, restrict to N^3.  Five kernel launches
 * on `stream`, asynchronous.
 *
 * rho, phi: DEVICE pointers on the plan's device, 16-byte aligned, N^3 reals
 * of the plan's dtype; phi == rho allowed, other overlaps are not.  One solve
 * per plan may be in flight at a time (the workspace is per plan): solves on
 * one stream serialise naturally; concurrent streams need separate plans.
 */
fsp_status fsp_solve(fsp_plan *plan, const void *rho, void *phi, fsp_stream stream);

/*
 * fsp_plan_field_init -- plan-time set-up of field solves (fsp_solve_field):
 * the field kernels F_a = -dG/dx_a (a = x, y, z) of the plan's method and
 * their spectra, FP64, rounded to the plan's type, plus a third workspace of
 * 2 N^2 P complex values.  E = -grad phi is the field of Appendix B (Eq.
 * efield), the step after the solve in the paper's particle-in-cell loop.
 *   FSP_HE:            F_a[m] = m_a / (4 pi h^2 |m|^3), F_a[0] = 0 (the
 *                      sampled gradient of the kernel of Sec. 2.2).
 *   FSP_VG, FSP_VG_DCT: the inverse transform of -i k_a G_L(k) (Sec. 2.3,
 *                      Eq. green_vico), evaluated through the (2N+1)^3
 *                      octant as a DST-I along a and DCT-I along the other
 *                      axes (Sec. 2.4), with the Nyquist plane j_a = -2N at
 *                      zero.  Both forms use this octant route: it equals the
 *                      (4N)^3 transform to rounding and needs 1/64 of its
 *                      memory.
 * The spectrum of F_a is odd in k_a: S_a = h^3 / (2N)^3 DST_a DCT DCT (F_a);
 * the solve multiplies by -i S_a.  Runs on `stream` and returns after it has
 * completed; temporaries ((2N+1)^3 FP64 for the Vico-Greengard forms) are
 * freed.  Calling it again is a no-op.  FSP_EINVAL for a spectrum-only plan
 * (no workspace); FSP_ENOMEM when the buffers do not fit, leaving the plan
 * usable for potential solves.
 */
fsp_status fsp_plan_field_init(fsp_plan *plan, fsp_stream stream);

/*
 * fsp_solve_field -- the field E = -grad phi of rho (Appendix B, Eq. efield)
 * and optionally phi itself: E_a[i] = h^3 sum_j F_a[i - j] rho_j for
 * a = x, y, z, each through the doubled grid like fsp_solve with the odd
 * spectrum -i S_a in place of S.  The forward transforms of rho (P1, P2)
 * run once; each output then takes its own P3 (z-FFT, multiply, z-IFFT, into
 * the third workspace), P4 and P5, so one call is 2 + 3 x 3 launches (+3
 * with phi) on `stream`, asynchronous.
 *
 * rho: DEVICE pointer, N^3 reals of the plan's dtype.  ex, ey, ez: DEVICE
 * pointers, N^3 reals each, the components along x (the fastest index), y
 * and z; phi: the same for the potential, or NULL.  All 16-byte aligned.
 * The outputs must not overlap one another; any of them may be rho (rho is
 * read completely before the first output is written).  Runs
 * fsp_plan_field_init first if it has not been called (synchronously, on
 * `stream`).  One solve per plan in flight, as for fsp_solve.
 */
fsp_status fsp_solve_field(fsp_plan *plan, const void *rho, void *phi, void *ex, void *ey, void *ez,
                           fsp_stream stream);

/*
 * fsp_solve_host -- the same solve on HOST arrays: copies rho host->device,
 * solves, copies phi device->host, all on `stream`, and returns after the
 * stream has completed the copy back.  rho/phi: host pointers (pinned memory
 * gives asynchronous, full-bandwidth copies), N^3 reals of the plan's dtype.
 * The first call allocates two N^3 device staging buffers kept by the plan.
 */
fsp_status fsp_solve_host(fsp_plan *plan, const void *rho_host, void *phi_host, fsp_stream stream);

/*
 * fsp_solve_host_many -- `count` solves of HOST arrays, pipelined: the copy of
 * source i+1 to the device and the copy of result i-1 back to the host run on
 * their own streams while solve i runs on `stream`, through three device
 * staging slots (each copy may take as long as two solves before it holds up
 * the next solve).  rho_host[i], phi_host[i]: host pointers (pinned for
 * asynchronous, full-bandwidth copies), N^3 reals of the plan's dtype.  The
 * first call allocates six N^3 staging buffers, two streams and nine events,
 * kept by the plan.  Returns after every result is on the host.
 */
fsp_status fsp_solve_host_many(fsp_plan *plan, const void *const *rho_host, void *const *phi_host, int count,
                               fsp_stream stream);

/* Wait for all work enqueued for this plan's solves and report any
 * asynchronous CUDA error as FSP_ECUDA.  FSP_ETIMEOUT: a bounded device-side
 * wait of a solve since the last check ran out (the results of that solve are
 * not valid; the plan and the context stay usable; the flag is cleared). */
fsp_status fsp_plan_sync(fsp_plan *plan, fsp_stream stream);

/* Time limit (milliseconds, > 0; default 1000) of each device-side wait in
 * this plan's solves.  Only the TMA-staged P3 waits (FP32-mixed, N = 64, 128,
 * 256, selected by FSP_P3_TMA=1 in the environment at plan creation; the
 * default register-direct P3 measured faster): on an mbarrier, for each input
 * tile of Sec. 2.2 step 4's z-transforms. */
fsp_status fsp_plan_set_wait_timeout(fsp_plan *plan, double ms);
/* Fault injection for tests, made on the host: the next solve's TMA-staged P3
 * expects 16 bytes more per input tile than the copy delivers, so each of its
 * CTAs' first wait can only end by the time limit; fsp_plan_sync then returns
 * FSP_ETIMEOUT.  FSP_EUNSUPPORTED when the plan's P3 has no such wait. */
fsp_status fsp_plan_inject_stall(fsp_plan *plan);

/* Release the plan and all its device memory.  Waits for the device first.
 * A destroyed or unknown pointer returns FSP_EINVAL (plans are tracked in a
 * registry, so a stale pointer is detected instead of dereferenced). */
fsp_status fsp_plan_destroy(fsp_plan *plan);

/*
 * fsp_plan_set_timing -- per-pass timing hook.  With nevents == 6, every later
 * fsp_solve on this plan records events[i] on the solve's stream just before
 * pass i (i = 0..4: pad+x-R2C, y-FFT, z-FFT*S*z-IFFT, y-IFFT, x-C2R) and
 * events[5] after the last pass, so that each kernel can be timed on the
 * stream it runs on.  events are cudaEvent_t handles owned by the caller
 * (created and destroyed by it, on the plan's device); nevents == 0 (events
 * may be NULL) turns the hook off.  Any other count returns FSP_EINVAL.
 */
fsp_status fsp_plan_set_timing(fsp_plan *plan, void *const *events, int nevents);

/* 1 when this plan's solves run the specialised kernels (N = 32, 64, 128,
 * 256, 512, or a non-cubic box of such sizes; FSP_F64 and FSP_F32_MIXED also
 * N = 48, 96, 192; compile-time radix schedules, register-resident), 0 when
 * they run the generic mixed-radix
 * engine, -1 for an invalid plan.  Setting
 * the environment variable FSP_GENERIC_ONLY=1 before fsp_plan_create forces
 * the generic engine (used to test both paths on the same sizes). */
int fsp_plan_uses_fast_path(const fsp_plan *plan);
/* Bounds evidence without a sanitizer.  With FSP_CHECK_BOUNDS=1 in the
 * environment at plan creation, every device buffer the plan allocates (the
 * spectrum, workspaces, roots tables, staging buffers, the field's spectra and
 * workspace, and the plan-time temporaries) is surrounded by 1 MB guard bands
 * of one byte pattern.  fsp_plan_check_bounds synchronises the device and
 * counts the guard bytes around the plan's live buffers that no longer hold
 * the pattern (0 when every kernel stayed inside its buffers);
 * FSP_EUNSUPPORTED for a plan created without the variable.
 * fsp_bounds_freed_bad: such bytes found, process-wide, in guarded buffers
 * when they were freed (temporaries at the end of plan creation, buffers of
 * destroyed plans).  Nothing traps: the counts are read on the host. */
fsp_status fsp_plan_check_bounds(const fsp_plan *plan, unsigned long long *bad_bytes);
unsigned long long fsp_bounds_freed_bad(void);

/* Kernel launches per fsp_solve: 3 when the fused plane passes serve the
 * plan (PA = pad + x-R2C + y-FFT of each z-plane in one thread-block
 * cluster, P3, PC = y-IFFT + x-C2R + crops; the plane's intermediate W1 goes
 * through L2 only), else 5 (Sec. 2.2 steps 1-5, one axis per launch).  The
 * plane passes exist for FSP_F32_MIXED at N = 64, 128, 256 and are used by
 * default at N = 64, where they measured faster; FSP_PLANE=1 (or 0) in the
 * environment at plan creation forces them on (or off).  -1 for an invalid
 * plan. */
int fsp_plan_launches(const fsp_plan *plan);

/* Device bytes the plan holds (spectrum + workspace + tables), 0 if invalid. */
size_t fsp_plan_bytes(const fsp_plan *plan);

/* Wall time of the plan-time precompute in milliseconds, < 0 if invalid. */
double fsp_plan_precompute_ms(const fsp_plan *plan);

/*
 * fsp_plan_spectrum -- copy the plan's multiplier to host memory as doubles:
 * S[q] = h^3 DFT_{2N}{G_2}[q] / (2N)^3 for q in [0,N]^3, shape (N+1)^3,
 * index (qz*(N+1) + qy)*(N+1) + qx (the spectrum of the mirrored kernel is
 * real and even per axis, so this octant holds all of it).  For
 * FSP_F32_MIXED the values are the single-precision ones the solve uses.
 * Synchronous.  s_host must hold (N+1)^3 doubles.
 */
fsp_status fsp_plan_spectrum(const fsp_plan *plan, double *s_host);

/*
 * fsp_plan_create_from_spectrum -- a cubic plan whose multiplier is a stored
 * one: s_host holds the (N+1)^3 doubles fsp_plan_spectrum wrote for a plan of
 * the same N and L (same layout, already scaled by h^3 / (2N)^3), so the
 * plan-time precompute of Sec. 2.2-2.4 (for FSP_VG a DFT of the (4N)^3
 * grid) is replaced by one host-to-device copy.  Checkpoint and warm start:
 * a restarted job or server restores its plans without recomputing them.
 * The values are stored as given, rounded to the plan's dtype (a fresh plan
 * rounds its FP64 spectrum the same way), so the spectrum of an FSP_F64 plan
 * restores a plan of any dtype to exactly the multiplier a fresh plan of that
 * dtype holds, and one of an FSP_F32_MIXED plan restores an FSP_F32_MIXED
 * plan bit for bit (FP32 values are exact doubles).
 * N, L and algo are checked as in fsp_plan_create; nothing checks that
 * s_host belongs to that (N, L, algo).
 * s_host is read during the call only (the caller keeps it).  FSP_EINVAL for
 * a null pointer or a non-finite value, otherwise the statuses of
 * fsp_plan_create (for FSP_F64_DF also the range check of its spectrum).
 * Synchronous on stream.
 */
fsp_status fsp_plan_create_from_spectrum(fsp_plan **out, int N, double L, fsp_algo algo, fsp_dtype dtype,
                                         const double *s_host, fsp_stream stream);

/*
 * fsp_kernel_T -- the real-space kernel T[m], m in [0,N]^3, of `algo`
 * (Sec. 2.2 step 3, Sec. 2.3, Sec. 2.4), computed on the current device in
 * FP64 exactly as fsp_plan_create computes it, written to the DEVICE array
 * t_dev ((N+1)^3 doubles, index (mz*(N+1)+my)*(N+1)+mx).  Same size rules as
 * fsp_plan_create.  Synchronises `stream`; temporaries are freed.
 */
fsp_status fsp_kernel_T(int N, double L, fsp_algo algo, double *t_dev, fsp_stream stream);

/*
 * fsp_fft_c2c -- `count` independent unnormalised 1D FFTs of length n
 * (2/3/5-smooth, 1 <= n <= 4096) with the solver's line kernels:
 * X[k] = sum_j x[j] exp(sign 2 pi i jk / n), sign = -1 (forward) or +1.
 * in/out: DEVICE arrays of count*n interleaved complex values (re, im),
 * contiguous lines, `double` (dtype FSP_F64) or `float` (FSP_F32_MIXED);
 * in == out allowed.  Asynchronous on `stream`.
 */
fsp_status fsp_fft_c2c(int n, int count, fsp_dtype dtype, int sign, const void *in, void *out, fsp_stream stream);

/* ------------------------------------------------------------- batches --
 * Many independent solves of mixed sizes in ONE persistent kernel launch,
 * replayed as a CUDA graph (a systems form; the paper solves one grid at a
 * time).  The launch walks a work list of tiles ordered pass by pass; a tile
 * of pass p waits, on the device, for pass p-1 of its own solve.  Every such
 * wait is bounded in time (default 1000 ms): when a limit runs out the kernel
 * records FSP_ETIMEOUT, all blocks stop taking work and the launch ends, and
 * fsp_batch_wait returns FSP_ETIMEOUT with the context still usable.
 */
typedef struct fsp_batch fsp_batch;

/* Build a batch over `count` solves: plans[i] with device arrays rho[i] ->
 * phi[i] (16-byte aligned, N_i^3 reals).  The plans must be distinct (each
 * owns its workspace), live, of one dtype and on the current device; they
 * must outlive the batch.  The work list and the graph are built once; each
 * launch re-reads rho[i] and rewrites phi[i].  Every tile uses the generic
 * mixed-radix engine with the plan's tile shapes, so a batched result is
 * bitwise equal to a single solve through that engine (FSP_GENERIC_ONLY=1).
 * Synchronises `stream`. */
fsp_status fsp_batch_create(fsp_batch **out, fsp_plan *const *plans, const void *const *rho, void *const *phi,
                            int count, fsp_stream stream);
/* Launch the batch's graph on `stream` (asynchronous).  One launch of a batch
 * may be in flight at a time. */
fsp_status fsp_batch_launch(fsp_batch *batch, fsp_stream stream);
/* Synchronise `stream` and return the last launch's device status: FSP_OK or
 * FSP_ETIMEOUT. */
fsp_status fsp_batch_wait(fsp_batch *batch, fsp_stream stream);
/* Change the per-wait time limit (milliseconds, > 0); rebuilds the graph. */
fsp_status fsp_batch_set_timeout(fsp_batch *batch, double ms);
/* The form a batch's graph takes (rebuilds the graph): 0 (default) the
 * persistent kernel above; 1 the solves' own launches (each plan's
 * fsp_solve kernels: the specialised ones for power-of-two N, else the
 * generic engine) on 8 captured streams, a plan's solves on one stream, plans
 * dealt round-robin.  Results are those of fsp_solve with each plan. */
fsp_status fsp_batch_set_form(fsp_batch *batch, int form);
/* Fault injection for tests, made on the host: one dependency of the work
 * list is raised by one tile that never exists, so that wait can only end by
 * its time limit.  Later launches then end with FSP_ETIMEOUT. */
fsp_status fsp_batch_inject_stall(fsp_batch *batch);
fsp_status fsp_batch_destroy(fsp_batch *batch);
/* Tune this batch's tile shapes in place: coordinate descent over the
 * generic engine's row and column shapes of each distinct N (largest first),
 * timing graph replays of the batch itself; the winners are kept by the batch
 * and recorded in the tuning table (fsp_tuning_get).  Launches the batch many
 * times (it reads rho, overwrites phi); synchronises `stream`. */
fsp_status fsp_batch_autotune(fsp_batch *batch, fsp_stream stream);
/* create + launch + wait + destroy in one call. */
fsp_status fsp_solve_batched(fsp_plan *const *plans, const void *const *rho, void *const *phi, int count,
                             fsp_stream stream);

/* -------------------------------------------------------------- server --
 * Continuous-batching solve server (a systems form; no counterpart in the
 * paper).  A worker thread owned by the server admits queued requests into
 * free slots (one CUDA stream each) as soon as a slot and device memory are
 * free, so solves of different sizes overlap on the device.  Spectra are
 * cached per (N, L, algo, dtype) and evicted least-recently-used.  A cache
 * miss is built by a second server thread on its own stream, outside the
 * worker's lock: meanwhile the worker keeps admitting (FIFO among requests
 * whose spectrum is ready; requests waiting for a build keep their place
 * without holding back the ones behind them) and retiring solves.  Spectra,
 * workspaces and the temporaries of builds in progress (the kernel on the
 * (4N)^3 grid for FSP_VG, the (2N+1)^3 octant for FSP_VG_DCT, reserved before
 * a build starts) together never exceed the budget; a request that cannot fit
 * with nothing else running fails with FSP_ENOMEM.  Every solve uses the same
 * kernels as fsp_solve, so a result is bitwise the same alone or in a mix.
 */
typedef struct fsp_server fsp_server;

typedef struct {
    uint64_t submitted, admitted, completed;
    uint64_t spec_hits, spec_misses, evictions;
    uint64_t queued, running;
    uint64_t cached_spectra;
    size_t bytes_in_use, budget;
    uint64_t builds_in_flight;  /* spectra being built now */
    size_t peak_bytes_in_use;   /* the most bytes_in_use has been */
} fsp_server_stats;

/* hbm_budget_bytes > 0; 1 <= max_slots <= 64 (concurrent solves). */
fsp_status fsp_server_create(fsp_server **out, size_t hbm_budget_bytes, int max_slots);
/* Queue one solve phi = G * rho (DEVICE arrays, 16-byte aligned, N^3 reals of
 * dtype) on the server's device; h = L/N.  Sizes are validated now
 * (FSP_EINVAL / FSP_EUNSUPPORTED); FSP_EBUSY when 65536 requests are queued.
 * rho and phi must stay valid and untouched until the request is done. */
fsp_status fsp_server_submit(fsp_server *server, int N, double L, fsp_algo algo, fsp_dtype dtype, const void *rho,
                             void *phi, uint64_t *ticket);
/* *state: 0 queued, 1 running, 2 done, 3 failed.  When done or failed,
 * *latency_ms (may be NULL) is submit-to-completion wall time, the request is
 * forgotten (a later poll of it returns FSP_EINVAL) and the return value is
 * its status; otherwise FSP_OK. */
fsp_status fsp_server_poll(fsp_server *server, uint64_t ticket, int *state, double *latency_ms);
fsp_status fsp_server_get_stats(fsp_server *server, fsp_server_stats *out);
/* Stops the worker, waits for the device, frees everything. */
fsp_status fsp_server_destroy(fsp_server *server);

/* ------------------------------------------------------------ autotune --
 * Tile shapes of the generic mixed-radix engine (the lines per CTA of its row
 * and column passes; used by every solve of a non-power-of-two N and by all
 * batched solves).  The shape changes no result bit (each line's arithmetic is
 * the same), only speed.
 *
 * fsp_autotune times every feasible shape for (N, dtype) on the current device
 * (builds a temporary plan, a few ms of solves per shape; synchronises
 * `stream`), records the fastest in a process-wide table and returns it.
 * dtype: FSP_F64 or FSP_F32_MIXED.  Plans created later for (N, dtype) use the
 * table's shape.
 * fsp_tuning_get writes the table as text, one "N dtype lgL_row lgL_col" line
 * per entry (NUL-terminated); *len receives the size needed (buf may be NULL).
 * fsp_tuning_set merges such text into the table (pins a tuned table). */
fsp_status fsp_autotune(int N, fsp_dtype dtype, fsp_stream stream, int *lgL_row, int *lgL_col);
fsp_status fsp_tuning_get(char *buf, size_t cap, size_t *len);
fsp_status fsp_tuning_set(const char *text);

/* ---------------------------------------------- slab-decomposed solve --
 * One rank's share of a solve distributed over R ranks (the paper's
 * distributed solver transposes pencils with all-to-all exchanges, Sec. 3.2;
 * the physical grid maps onto the doubled one as in Appendix A, Algorithm 1).
 * Rank r owns the z-planes [z0, z1) of rho and phi (dense slabs of
 * (z1-z0) N^2 reals, C order as for fsp_solve) and the half-spectrum columns
 * k_x in [kx0, kx1), with z0 = floor(r N / R), kx0 = floor(r (N+1) / R).
 * A solve is
 *   fsp_dist_forward   P1 and P2 on the z-slab; writes send block q for every
 *                      rank q (phase 0);
 *   (caller)           block r -> q of every pair is copied into q's receive
 *                      block from r (an all-to-all: NCCL, peer copies, or
 *                      device copies when the ranks share a process);
 *   fsp_dist_middle    assembles the k_x slab from the phase-0 receive blocks,
 *                      P3 and P4 on it; writes the phase-1 send blocks;
 *   (caller)           the phase-1 all-to-all;
 *   fsp_dist_backward  assembles the z-slab's rows, P5 into phi.
 * Blocks are the caller's device arrays of fsp_dist_block_elems complex
 * values (double2 for FSP_F64, float2 for FSP_F32_MIXED), 16-byte aligned,
 * one per peer (including the rank itself), indexed by peer rank.  Phase-0
 * block s -> q: [zl][k_y][j], zl < nz_s, k_y < 2N, j < kx-width of q.
 * Phase-1 block s -> q: [zl][y][j], zl < nz_q, y < N, j < kx-width of s.
 * Generic engine (2N 2/3/5-smooth, 4N for FSP_VG), FSP_F64 or
 * FSP_F32_MIXED (else FSP_EUNSUPPORTED); 1 <= R <= N.  Asynchronous on
 * `stream`.  fsp_dist_partition and fsp_dist_block_elems are host arithmetic
 * only (no device); fsp_dist_block_elems returns -1 for invalid arguments. */
typedef struct fsp_dist fsp_dist;
fsp_status fsp_dist_partition(int N, int nranks, int rank, int *z0, int *z1, int *kx0, int *kx1);
long long fsp_dist_block_elems(int N, int nranks, int rank, int phase, int peer, int sending);
fsp_status fsp_dist_create(fsp_dist **out, int N, double L, fsp_algo algo, fsp_dtype dtype, int nranks, int rank,
                           fsp_stream stream);
fsp_status fsp_dist_forward(fsp_dist *d, const void *rho_slab, void *const *send, fsp_stream stream);
fsp_status fsp_dist_middle(fsp_dist *d, const void *const *recv, void *const *send, fsp_stream stream);
fsp_status fsp_dist_backward(fsp_dist *d, const void *const *recv, void *phi_slab, fsp_stream stream);
fsp_status fsp_dist_destroy(fsp_dist *d);

/* ------------------------------------------------------- host buffers --
 * Pinned host memory for the host-buffer solves (fsp_solve_host,
 * fsp_solve_host_many), placed on one host NUMA node.  The paper has no
 * counterpart; its solver keeps its fields in device memory.
 *
 * fsp_device_host_numa: the host NUMA node closest to `device`
 * (cudaDevAttrHostNumaId), -1 when unknown or the system has no NUMA.
 * fsp_host_alloc: `bytes` of anonymous memory bound to `numa_node` (none when
 * numa_node < 0), every page touched, then page-locked for the device.  The
 * caller owns it and releases it with fsp_host_free(p, bytes).  FSP_ENOMEM
 * when the mapping fails, FSP_EUNSUPPORTED when the node cannot be bound,
 * FSP_ECUDA when page-locking fails. */
int fsp_device_host_numa(int device);
fsp_status fsp_host_alloc(void **out, size_t bytes, int numa_node);
fsp_status fsp_host_free(void *p, size_t bytes);

/*
 * fsp_solve_noalloc -- an FP64 solve that allocates no device memory.  The
 * paper has no counterpart: it is an interface for callers that do not call
 * cudaMalloc (real-time loops that forbid allocator calls; applications whose
 * device memory is entirely held by their own allocator).  The caller passes
 * everything that has a size: the spectrum, the source and the result.
 *
 * N    2 <= N <= 32 and 2N 2/3/5-smooth; larger or unsupported sizes return
 *      FSP_EUNSUPPORTED (N < 2: FSP_EINVAL) before any device work.
 * S    DEVICE array of (N+1)^3 doubles, index (qz*(N+1)+qy)*(N+1)+qx: the
 *      multiplier of the method, h^3 DFT_{2N}{G_2}[q] / (2N)^3, e.g. what
 *      fsp_plan_spectrum returns for an FSP_F64 plan, copied to the device.
 * rho, phi  DEVICE arrays of N^3 doubles, 16-byte aligned (as fsp_solve).
 *
 * Scratch: the two transform buffers and the roots tables live in one
 * file-scope device array of 2.36 MB (N = 32 at row pitch 48), which every
 * GPU that loads the library holds until the process exits.  Every call looks
 * up that array's device address in the current context
 * (cudaGetSymbolAddress, which allocates nothing), so the address stays right
 * after a device reset or a new primary context.  The first lookup in a
 * context may load the library's device code.  All calls on a
 * device share the one array and leave their intermediate values in it; no
 * part of it needs to start at zero (each call writes every element before
 * reading it).  Calls whose device work overlaps in time (different streams,
 * or host threads racing on one device) corrupt each other's results:
 * serialise them, e.g. on one stream.  Asynchronous on `stream`.
 */
fsp_status fsp_solve_noalloc(int N, const double *S, const double *rho, double *phi, fsp_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* FSP_H */
