/*
 * dgpe.h -- C ABI of the GB300 split-step Crank-Nicolson (SSCN) solver for the 3D dipolar
 * Gross-Pitaevskii equation (arXiv 1610.05329).
 *
 * What is computed.  The paper ("Nature of problem", "Solution method") solves the
 * time-dependent GP equation with contact and dipolar interaction in an anisotropic
 * harmonic trap by the split-step Crank-Nicolson method, in imaginary or real time, with
 * the dipolar term evaluated in momentum space through the convolution theorem, using a
 * real-to-complex FFT ("Summary of revisions", DBEC-GP-OMP).  The dimensionless model this
 * library implements is
 *
 *     i dpsi/dt = [ -1/2 lap + V + g |psi|^2 + gdd Phi ] psi
 *     V   = 1/2 (nu_x^2 x^2 + nu_y^2 y^2 + nu_z^2 z^2)
 *     Phi = IDFT[ Ut(k) DFT(|psi|^2) ],  Ut(k) = 3 k_z^2 / |k|^2 - 1,  Ut(0) = 0
 *
 * on the grid x_i = (i - nx/2) hx (same for y, z), k_m = 2 pi m / (n h) with m signed.
 * One step is: the potential step psi <- psi exp(-i theta) (real time) or
 * psi exp(-theta) (imaginary time), theta = dt (V + g n + gdd Phi) with n, Phi of the
 * incoming state; then Crank-Nicolson along x, y and z,
 * (1 - c D) psi' = (1 + c D) psi on the interior of every grid line, D the 3-point second
 * difference, psi = 0 on the two wall points of the line, c = i dt/(4 h^2) (real time) or
 * dt/(4 h^2) (imaginary time); in imaginary time psi is then divided by sqrt(norm),
 * norm = hx hy hz sum |psi|^2.  The three sweeps commute exactly, so the library may run
 * them in any order.
 *
 * Memory and layout.  psi is row-major [nx][ny][nz] (z fastest), complex values stored as
 * interleaved (re, im) pairs: complex128 for DGPE_FP64 and DGPE_DF64, complex64 for
 * DGPE_MIXED.  All
 * device memory the solver uses is one workspace of dgpe_workspace_bytes() bytes: the
 * caller may own it (params.workspace, e.g. a PyTorch tensor) or let dgpe_create allocate
 * it with cudaMalloc.  The one exception is dgpe_step_host, which allocates its second psi
 * buffer at its first call.  Nothing is kept in global variables: one context per stream.
 *
 * Errors.  Every int-returning call returns DGPE_OK (0) or a negative DGPE_E* code; no C++
 * exception crosses the ABI.  Parameter checks happen before any CUDA call, so invalid
 * parameters are reported even on a machine without a GPU.  Errors found on the device
 * (a non-finite norm, or a zero norm in imaginary time, which cannot be renormalised) are
 * latched and returned by the next synchronising call
 * (dgpe_sync, dgpe_observables, dgpe_get_psi with a host buffer, dgpe_get_phi).
 * A context is not thread-safe: calls on one context must not overlap.
 */
#ifndef DGPE_H
#define DGPE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGPE_OK 0
#define DGPE_EINVAL (-1)        /* bad argument or parameter */
#define DGPE_ENOMEM (-2)        /* device allocation failed or workspace too small */
#define DGPE_ECUDA (-3)         /* a CUDA runtime call or kernel launch failed */
#define DGPE_ENONFINITE (-4)    /* NaN/Inf in a reduction (norm, observables), or a zero norm to renormalise */
#define DGPE_ETIMEOUT (-5)      /* reserved: a bounded device-side wait gave up.  No kernel of this
                                   build waits on a flag or on another block, so no call returns it */
#define DGPE_EUNSUPPORTED (-6)  /* valid request this build does not support */

#define DGPE_REAL_TIME 0
#define DGPE_IMAG_TIME 1

#define DGPE_FP64 0   /* complex128 psi; FFT, phase and CN in FP64 */
/* complex64 psi; FFT, phase and CN in FP32; the norm and the observables' sums FP64-class
 * (FP32 terms, exact weights, double-float sums per point, FP64 across blocks).  In real time every
 * step restores the norm the real-time run began with (the norm of the state its first step
 * started from), undoing the drift of the FP32-rounded Crank-Nicolson factors (about 3e-7
 * of the norm per step, systematic); the exact scheme conserves the norm, so this corrects
 * rounding only.  dgpe_grad_z2 runs its trajectory without it. */
#define DGPE_MIXED 1
/* Double-float: every value is a pair of FP32 numbers hi + lo (about 48 significant bits)
 * and every operation runs on the FP32 pipe, which GB300 issues 64 times as fast as FP64.
 * The caller sees complex128 (dgpe_set_psi/dgpe_get_psi convert at the boundary) and FP64
 * observables; the differentiation calls return DGPE_EUNSUPPORTED.  The paper has no
 * counterpart: this is an implementation choice for FP64-starved hardware. */
#define DGPE_DF64 2

#define DGPE_HOST 0
#define DGPE_DEVICE 1

/* Quadrature of the norm (hence the imaginary-time renormalisation) and of the observables. */
#define DGPE_RECTANGLE 0  /* h^3 sum over all points */
#define DGPE_SIMPSON 1    /* composite Simpson (1,4,2,...,4,1)/3 per axis on indices 0..n-2 (the last point is a wall) */
/* Kinetic-energy form of the observables. */
#define DGPE_KINETIC_LAPLACIAN3 0  /* 1/2 Re conj(psi)(-lap psi), the step's own 3-point Laplacian */
#define DGPE_KINETIC_GRADIENT5 1   /* 1/2 |grad psi|^2 with 4th-order 5-point first derivatives */

/* Sub-steps for dgpe_substep (each is one factor of the split step). */
#define DGPE_SUB_POTENTIAL 0  /* psi <- psi e^{-i theta} (or e^{-theta}); no renormalisation */
#define DGPE_SUB_CN_X 1
#define DGPE_SUB_CN_Y 2
#define DGPE_SUB_CN_Z 3

/*
 * Problem description.  Sizes: 4 <= n <= 512, n even, n = 2^a 3^b 5^c 7^d (the sizes the
 * paper recommends for its transforms, except factors 11 and 13; radix-2/3/4/5/7/8
 * transforms), e.g.
 * the paper's own 480 x 480 x 500 and 480 x 480 x 250 grids.
 * h, dt > 0 and finite; nu, g, gdd finite.  workspace: NULL, or device memory of at least
 * workspace_bytes >= dgpe_workspace_bytes(p) bytes, 256-byte aligned, owned by the caller
 * and kept alive until dgpe_destroy.
 */
typedef struct dgpe_params {
  int nx, ny, nz;
  double hx, hy, hz;
  double dt;
  int mode;           /* DGPE_REAL_TIME or DGPE_IMAG_TIME */
  int precision;      /* DGPE_FP64, DGPE_MIXED or DGPE_DF64 */
  double nu[3];       /* trap frequencies nu_x, nu_y, nu_z */
  double g;           /* contact strength */
  double gdd;         /* dipolar strength (dipoles along z) */
  double cutoff;      /* spherical cutoff radius R of the dipolar interaction (interaction
                         restricted to r < R: Ut(k) times 1 + 3cos(kR)/(kR)^2 - 3sin(kR)/(kR)^3);
                         <= 0: no cutoff */
  int integration;    /* DGPE_RECTANGLE (default 0) or DGPE_SIMPSON */
  int kinetic;        /* DGPE_KINETIC_LAPLACIAN3 (default 0) or DGPE_KINETIC_GRADIENT5 */
  void *workspace;    /* optional caller-owned device memory */
  size_t workspace_bytes;
} dgpe_params;

/* Observables of the current state, FP64.  norm = h^3 sum |psi|^2 (sums weighted by the
 * chosen quadrature); the energy terms use the 3-point Laplacian with zero values outside
 * the grid (or the 5-point gradient, see dgpe_params.kinetic):
 *   e_kin = h^3 sum 1/2 Re conj(psi) (-lap psi),  e_trap = h^3 sum V n,
 *   e_contact = h^3 sum g n^2 / 2,  e_dipolar = h^3 sum gdd Phi n / 2,
 *   energy = e_kin + e_trap + e_contact + e_dipolar,
 *   mu = (e_kin + e_trap + 2 e_contact + 2 e_dipolar) / norm,
 *   rms[d] = sqrt(sum d^2 n / sum n). */
typedef struct dgpe_obs {
  double norm, mu, energy;
  double rms[3];
  double e_kin, e_trap, e_contact, e_dipolar;
} dgpe_obs;

/* Per-kernel timing record (see dgpe_set_timing). bytes_per_launch is the kernel's
 * algorithmic HBM traffic (each input read once, each output written once). */
typedef struct dgpe_kernel_time {
  char name[32];
  double total_ms;
  long long launches;
  double bytes_per_launch;
} dgpe_kernel_time;

typedef struct dgpe_ctx dgpe_ctx;

/* Device bytes the solver needs for p (only shape and precision matter).  Host-only.
 * Paper: Summary of revisions, DBEC-GP-OMP (the memory of the dipolar transform is set by
 * the half spectrum of the real-to-complex FFT). */
int dgpe_workspace_bytes(const dgpe_params *p, size_t *bytes);

/* Validate p, set up the workspace, FFT twiddles and Crank-Nicolson factor tables on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).  psi starts at zero.
 * On success *out owns the context; free it with dgpe_destroy.
 * Paper: Nature of problem (the GP equation with contact and dipolar interaction in a
 * harmonic anisotropic trap: nu, g, gdd); Solution method (discretised in space and time:
 * the grid and dt); Additional comments (grid sizes are checked and an error is reported). */
int dgpe_create(const dgpe_params *p, void *cuda_stream, dgpe_ctx **out);

/* Change dt, mode, nu, g, gdd or h (e.g. the quench or a trap schedule) without
 * reallocation; shape and precision must stay the same (else DGPE_EINVAL).
 * Stream-ordered: takes effect for work enqueued afterwards.
 * Paper: Nature of problem (the trap and interaction strengths); Solution method (imaginary
 * or real time: stationary then non-stationary problems on one state). */
int dgpe_set_params(dgpe_ctx *ctx, const dgpe_params *p);

/* Copy psi in from `where` = DGPE_HOST or DGPE_DEVICE memory (layout above; complex128 for
 * FP64 and DF64, complex64 for MIXED).  The caller keeps ownership.  Clears latched device
 * errors.  Paper: Solution method (the state the propagation starts from). */
int dgpe_set_psi(dgpe_ctx *ctx, const void *psi, int where);

/* Copy the current psi (pending renormalisation applied) to `out` in host or device memory.
 * Host copies synchronise the stream; device copies are stream-ordered.
 * Paper: Solution method (the stationary or non-stationary solution the propagation yields). */
int dgpe_get_psi(dgpe_ctx *ctx, void *out, int where);

/* Enqueue nsteps >= 0 SSCN steps (stream-ordered, asynchronous; replayed from a CUDA graph).
 * In imaginary time every step renormalises (applied lazily: see dgpe_get_psi).
 * Paper: Solution method (split-step Crank-Nicolson, propagation in imaginary or real time
 * over small time steps, the dipolar term in momentum space by the convolution theorem);
 * Summary of revisions, DBEC-GP-OMP (the transform of the density is real-to-complex). */
int dgpe_step(dgpe_ctx *ctx, int nsteps);

/* Host-resident states through the solver: copy psi in from host memory `in` (as
 * dgpe_set_psi), run nsteps steps, copy the result (as dgpe_get_psi) to host memory `out`.
 * Asynchronous: the copies run on two internal streams, and successive calls alternate the
 * state between the workspace's psi buffer and a second one of the same size (allocated at
 * the first call with cudaMalloc, outside the workspace, freed by dgpe_destroy; double-float
 * also stages its converted output), so the input copy of one call overlaps the previous
 * call's steps and its output copy the next call's, with no device-side copy.  `in` must stay
 * unchanged and `out` unread until dgpe_sync (which waits for the copies too); later calls
 * that change psi on this context wait for the output copy by themselves.  Pinned host
 * memory lets the copies run asynchronously.  Device errors surface at dgpe_sync, as for
 * dgpe_step.  NULL in/out or nsteps < 0: DGPE_EINVAL.
 * Paper: Solution method (propagation); states that live in host memory between steps. */
int dgpe_step_host(dgpe_ctx *ctx, const void *in, void *out, int nsteps);

/* Apply one factor of the split step (DGPE_SUB_*) once, without renormalisation.
 * Paper: Solution method (the factors of the split step). */
int dgpe_substep(dgpe_ctx *ctx, int which);

/* Compute the observables of the current state; synchronises the stream.
 * Returns DGPE_ENONFINITE if a sum is NaN/Inf.
 * Paper: Nature of problem (the properties of the condensate the GP equation describes);
 * the paper prints no formula for them, so the forms are the readings stated at dgpe_obs
 * (the step's own discrete Hamiltonian; the rectangle or Simpson quadrature). */
int dgpe_observables(dgpe_ctx *ctx, dgpe_obs *o);

/* Dipolar potential Phi = IDFT[Ut DFT(|psi|^2)] of the current state (real, [nx][ny][nz],
 * double for FP64 and DF64, float for MIXED) into host or device memory.  Synchronises for
 * host.  Paper: Solution method (the dipolar contribution evaluated in momentum space by
 * the convolution theorem). */
int dgpe_get_phi(dgpe_ctx *ctx, void *out, int where);

/* ---- Differentiation (real time only) ----------------------------------------------
 * Discrete adjoint of the real-time step, written by hand (the paper has no adjoint; this
 * differentiates the step it describes).  Cotangent convention: for a real loss L,
 * gbar = 2 dL/d conj(psi), so that dL = Re sum conj(gbar) dpsi.  Of one step
 * psi' = X Y Z P(psi): each Crank-Nicolson sweep's adjoint is the same sweep with
 * dt -> -dt, and the potential step's adjoint is
 *   gbar = e^{+i theta} gbar1 + 2 dt (g s + gdd Phi[s]) psi,  s = Im(conj(gbar1) P(psi)),
 * with dL/dg = dt sum s |psi|^2, dL/dgdd = dt sum s Phi[|psi|^2], dL/dnu_z = dt nu_z sum s z^2.
 */

/* One adjoint step.  psi_k: device, the step's input state ([nx][ny][nz], the context's
 * complex type), not modified.  gbar: device, in = cotangent of the step's output,
 * out = cotangent of psi_k.  Adds the step's dL/dg, dL/dgdd, dL/dnu_z to the context's
 * accumulators (dgpe_adjoint_grads).  Uses the context's parameters (nu_z, g, gdd, dt),
 * which must be those of the forward step.  DGPE_EUNSUPPORTED in imaginary time. */
int dgpe_adjoint_step(dgpe_ctx *ctx, const void *psi_k, void *gbar);

/* Synchronises and copies the accumulated {dL/dg, dL/dgdd, dL/dnu_z} into out[3]; reset != 0
 * zeroes the accumulators afterwards.  (No paper counterpart: the paper has no adjoint.) */
int dgpe_adjoint_grads(dgpe_ctx *ctx, double *out, int reset);

/* Device bytes of the work buffer of dgpe_grad_z2 for nseg segments of steps_per_seg
 * steps: sqrt(N) checkpointing keeps ceil(N/k) checkpoints plus the k states of one
 * segment (k = ceil(sqrt(N)), N = nseg * steps_per_seg), the cotangent and nseg sums.
 * (No paper counterpart: the paper has no adjoint.) */
int dgpe_grad_z2_workspace_bytes(const dgpe_ctx *ctx, int nseg, int steps_per_seg, size_t *bytes);

/* Gradient of L = hx hy hz sum z^2 |psi_N|^2 (= <z^2> of a unit-norm state) after
 * N = nseg * steps_per_seg real-time steps from the current psi, with the trap frequency
 * nu_z = nu_z[s] (host array) during steps [s*steps_per_seg, (s+1)*steps_per_seg), the other
 * parameters fixed.  Outputs (host): *loss, dnu[s] = dL/dnu_z[s] (nseg values), *dg, *dgdd.
 * work: device memory of dgpe_grad_z2_workspace_bytes(), 256-byte aligned, caller-owned.
 * Cost: one forward pass storing a checkpoint every k steps, then per segment (backwards)
 * a recomputation from its checkpoint and the adjoint steps through it.  On return the
 * context holds the initial psi and the initial nu_z again.  Synchronises.  (No paper
 * counterpart: the paper has no adjoint; the forward steps are its Solution method.) */
int dgpe_grad_z2(dgpe_ctx *ctx, int nseg, int steps_per_seg, const double *nu_z, void *work, size_t work_bytes,
                 double *loss, double *dnu, double *dg, double *dgdd);

/* ---- Batching and launch-shape tuning -----------------------------------------------
 * Many independent condensates (different shapes and parameters) advanced together: one
 * CUDA graph holds every context's steps as parallel branches, so small grids that cannot
 * fill the GPU alone run concurrently.  The paper runs one condensate per program; this
 * serves many small independent ones (parameter scans). */
typedef struct dgpe_batch dgpe_batch;

/* n >= 1 distinct contexts on the current device; they must outlive the batch.  The batch
 * launches on cuda_stream; do not enqueue work on a context's own stream while a batch step
 * may still run (synchronise first).  FP32-mixed contexts of the same shape, mode and
 * launch shape are stepped as a group: each kernel of the step is one launch for all of
 * them (their arguments in a device array of n entries that dgpe_batch_create allocates with
 * cudaMalloc); other contexts run their own kernels.  Results are bitwise those of each
 * context's own steps.  (No paper counterpart: see above.) */
int dgpe_batch_create(dgpe_ctx *const *ctxs, int n, void *cuda_stream, dgpe_batch **out);
/* nsteps SSCN steps of every context, as one graph launch: each context's nsteps steps form
 * one chain of kernels (a branch of the graph), and the branches are joined once, at the
 * end, so no context waits for another between steps; branches with less work (fewer points)
 * run at a higher stream priority, so that short chains of small grids interleave with long
 * ones instead of waiting behind them.  A graph holds at most 2^18 kernel
 * nodes; a longer run launches several graphs of equal length (and one shorter).  Graphs
 * are built at the first call with a given nsteps (capture and instantiation, host time
 * that grows with nsteps x contexts), cached for up to four step counts, and rebuilt when a
 * context's step changed through dgpe_set_params or tuning.  Asynchronous.
 * (No paper counterpart: the paper runs one condensate per program.) */
int dgpe_batch_step(dgpe_batch *b, int nsteps);
/* Wait for the batch stream; the first latched device error of any context.  (No paper
 * counterpart.) */
int dgpe_batch_sync(dgpe_batch *b);
/* Free the batch (its graph, capture streams and events) after waiting for its stream.  The
 * contexts stay owned by the caller and usable.  NULL is safe.  (No paper counterpart.) */
void dgpe_batch_destroy(dgpe_batch *b);

/* Launch shape of a context's step.  Paper: Summary of revisions, DBEC-GP-MPI (performance
 * depends on the grid sizes and the machine, and configurations should be tried). */
typedef struct dgpe_tuning {
  int plan_style[3];     /* FFT radix order per axis: 0 radix-8 first, 1 radix-4, 2 radix-3 first */
  int ylines;            /* lines per CTA of the y transforms: 2, 4, 8, 16 or 32 */
  int fft_threads;       /* threads per CTA of the y/x transforms: 128 or 256 */
  int cn_per_sm;         /* CTAs per SM of the persistent Crank-Nicolson sweeps: 1 or 2 (an upper
                            bound: the FP32 sweeps of 512-thread CTAs fit one per SM by registers;
                            those of short lines run four per SM regardless) */
  double step_ms_default, step_ms_tuned;  /* measured by dgpe_autotune (0 otherwise) */
} dgpe_tuning;

/* Time candidate launch shapes on this context's own shape (a few steps each, with CUDA
 * events per kernel), choose the fastest per kernel class (a radix order other than the
 * default only when it is more than 3 % faster), apply it and report it in *out.
 * psi and the device state are restored afterwards.  Synchronises; allocates one
 * psi-sized temporary with cudaMallocAsync.  Paper: as dgpe_tuning. */
int dgpe_autotune(dgpe_ctx *ctx, dgpe_tuning *out);
/* Apply a tuning (e.g. one found earlier for the same shape). DGPE_EINVAL if invalid.
 * Paper: as dgpe_tuning. */
int dgpe_set_tuning(dgpe_ctx *ctx, const dgpe_tuning *t);
/* The launch shape in use (the defaults of dgpe_create until dgpe_autotune or
 * dgpe_set_tuning changes it); step_ms_default and step_ms_tuned are 0.  No CUDA call.
 * Paper: as dgpe_tuning. */
int dgpe_get_tuning(const dgpe_ctx *ctx, dgpe_tuning *out);
/* Kernel launches of one dgpe_step step (7, or 8 where the z sweep is a pass of its own:
 * FP64 and double-float).  No CUDA call.  (No paper counterpart; the paper times whole
 * runs of the step loop, Tables 1-3.) */
int dgpe_step_launches(const dgpe_ctx *ctx, int *n);

/* Wait for the stream; returns a latched device error if any.  (No paper counterpart.) */
int dgpe_sync(dgpe_ctx *ctx);

/* Per-kernel timing: when enabled, dgpe_step launches kernels one by one with CUDA events
 * around each (instead of replaying the graph) and accumulates their durations.  A record
 * covers one stage of the step: in FP64 the "k5" record times its two launches (the
 * phase-only pass and the per-line z sweep) together.  (No paper counterpart; the paper
 * times whole runs of the step loop, Tables 1-3.) */
int dgpe_set_timing(dgpe_ctx *ctx, int enable);
/* Synchronises, then copies up to `max` records into out and sets *n to the number of
 * kernels timed.  (No paper counterpart.) */
int dgpe_kernel_times(dgpe_ctx *ctx, dgpe_kernel_time *out, int max, int *n);

/* Norm and rms sizes of a caller's psi without allocating any device memory.
 *
 * The paper has no counterpart of this call; it exists for callers that cannot allocate:
 * a framework that owns all device memory through its own pool and treats any outside
 * cudaMalloc as a bug, a monitoring hook run every step of a time-critical loop where
 * cudaMalloc/cudaFree would synchronise the device and stall other streams, or a process
 * running so close to its memory limit that a new allocation may fail.  It needs no
 * context and no workspace: the scratch of its reduction (per-block partial sums and a
 * counter, 256 KiB) is one fixed array inside the library, of which every GPU that loads
 * the library keeps one copy until the process exits.
 *
 * psi: device memory, [nx][ny][nz], owned by the caller: complex128 for p->precision =
 * DGPE_FP64 or DGPE_DF64 (the double-float mode's caller format, as at dgpe_set_psi), complex64
 * for DGPE_MIXED.  Only p->nx, ny, nz, hx, hy, hz, precision and integration are read; the
 * grid is x_i = (i - nx/2) hx as everywhere in this library, and with DGPE_SIMPSON every sum
 * carries the composite Simpson weights, as in dgpe_observables.
 * out: device memory for 4 doubles, owned by the caller: norm = hx hy hz sum w |psi|^2,
 * rms_x, rms_y, rms_z (sqrt(sum w d^2 |psi|^2 / sum w |psi|^2)), written in stream order.
 * Sizes: each axis at most 512 (the library's grid limit; the kernel keeps the z weights
 * in a fixed table of 512 entries and its partial sums in the fixed scratch, whatever the
 * size); larger axes return DGPE_EUNSUPPORTED.  Bad pointers, sizes, spacings, precision
 * or integration: DGPE_EINVAL.
 * The first call on each GPU looks up that GPU's copy of the scratch array; make that
 * first call before any stream capture.  Every call on a GPU shares the same scratch, so
 * calls whose GPU work may overlap (e.g. on unordered streams) race and give wrong
 * results: order them on one stream or with events.  Asynchronous: returns after
 * enqueueing a memset and one kernel on cuda_stream (NULL = legacy default stream). */
int dgpe_moments_noalloc(const void *psi, const dgpe_params *p, double *out, void *cuda_stream);

/* Static text for an error code.  Paper: Additional comments (invalid grid sizes are
 * reported to the user as an error). */
const char *dgpe_strerror(int code);

/* Name and text of the last CUDA runtime error this thread's calls met (empty if none);
 * valid until the next call on the same thread.  (No paper counterpart.) */
const char *dgpe_last_cuda_error(void);

/* Free the context and whatever it allocated (not a caller-owned workspace). NULL is ok.
 * (No paper counterpart.) */
void dgpe_destroy(dgpe_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* DGPE_H */
