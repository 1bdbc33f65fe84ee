/*
 * gpe.h -- C ABI of the GB300 spin-1 Gross-Pitaevskii split-step library (libgpe.so).
 *
 * Method: "Universal Dynamics at the Lowest Temperatures", Sec. 2.2.  The library
 * propagates many truncated-Wigner trajectories of the three-component equation
 * Eq. (GPE) on periodic 1D/2D/3D grids with the paper's split-step Fourier scheme
 * (kinetic step in momentum space, diagonal phase step, off-diagonal 3x3 spin-mixing
 * step with predictor), symmetrised as K(dt/2) D(dt/2) O(dt) D(dt/2) K(dt/2), and
 * accumulates the ensemble spectra of Sec. 2.1 (occupations n_m(k), transverse spin
 * structure factor S_perp(k)) plus norm / energy diagnostics in FP64.
 *
 * Conventions shared by every entry point:
 *  - hbar = m = 1; external potential V_m(x) = 0 unless set with
 *    gpe_batch_set_potential.  Field components are ordered (psi_1, psi_0, psi_-1).
 *  - Field layout of one trajectory: [3][n2][n1][n0] complex numbers, contiguous,
 *    x (n[0]) fastest; complex = interleaved (re, im) float (GPE_C64) or double
 *    (GPE_C128).  The buffer must be 16-byte aligned.
 *  - Memory: every buffer passed in is caller-owned device memory unless stated; the
 *    library never frees caller memory.  The handle owns its tables and workspace.
 *  - Streams: ``stream`` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously; results are valid once the stream
 *    has reached the point after the call.
 *  - Errors: argument and CUDA launch errors are returned synchronously as a
 *    gpe_status; gpe_last_error() gives a thread-local message.  Device-side
 *    conditions (non-finite values, bounded waits that expired) latch in a status word
 *    that gpe_sync_status() reads.  No C++ exception crosses the ABI.
 */
#ifndef GPE_H
#define GPE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPE_OK = 0,
    GPE_EINVAL = 1,        /* invalid argument (sizes, pointers, alignment, flags)      */
    GPE_ENOMEM = 2,        /* device allocation for the handle's workspace failed       */
    GPE_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed               */
    GPE_ETIMEOUT = 4,      /* a bounded device-side wait expired                        */
    GPE_ENONFINITE = 5,    /* a reduction met a non-finite value                        */
    GPE_EUNSUPPORTED = 6   /* valid request that this build does not implement          */
} gpe_status;

typedef enum { GPE_C64 = 0, GPE_C128 = 1 } gpe_dtype;

/* One trajectory.  ndim in {1,2,3}; n[a] = points along axis a (x = 0), each a power
 * of two in [64, 1024] for ndim >= 2 and in [64, 32768] (C64) / [64, 16384] (C128) for
 * ndim = 1 (beyond 4096 / 2048 points a 1D trajectory runs on a thread-block cluster,
 * and its spectra take a four-step transform); unused axes must be 1.  dx = lattice
 * spacing (all axes).  psi = device pointer to the [3][n2][n1][n0] field (caller-owned,
 * 16-byte aligned). */
typedef struct {
    int32_t ndim;
    int32_t n[3];
    double dx;
    void* psi;
} gpe_traj;

/* Couplings of Eq. (GPE) and the time step.  q is constant when n_knots == 0;
 * otherwise q(t) is piecewise linear through q_knots[j] at t_j = j t_end / (n_knots-1),
 * clamped outside [0, t_end], and step n (time t_n = n dt) uses q(t_n + dt/2).
 * q_knots is a host array copied at gpe_batch_create. */
typedef struct {
    double c0, c1, q, dt;
    const double* q_knots;
    int32_t n_knots;
    double t_end;
} gpe_params;

typedef struct gpe_batch gpe_batch;

/* Creates a batch over ntraj trajectories (copied; psi buffers stay caller-owned and
 * must outlive the handle).  Trajectories of equal shape are advanced together.
 * Allocates the handle's tables and workspace on the current device.  Errors:
 * GPE_EINVAL (sizes, NULL or misaligned psi, dt <= 0), GPE_EUNSUPPORTED (sizes outside
 * the ranges above), GPE_ENOMEM. */
gpe_status gpe_batch_create(const gpe_traj* trajs, int32_t ntraj, gpe_dtype dtype,
                            const gpe_params* params, gpe_batch** out);

/* Frees the handle and its workspace (synchronises the device first). */
gpe_status gpe_batch_destroy(gpe_batch* batch);

/* Initial truncated-Wigner state (Sec. 2.2: runs start from slightly fluctuating
 * initial conditions): psi_m(x) = mean_m [+ mean_field_m(x)] + eta_m(x) for every
 * trajectory, with mean_spinor = (re, im) of (psi_1, psi_0, psi_-1), the optional
 * mean field of gpe_batch_set_mean_field, and eta complex Gaussian,
 * <|eta|^2> = noise_per_mode / dx^d (noise_per_mode particles per plane-wave mode).
 * eta comes from Philox4x32-10 (Salmon et al., SC'11) keyed by the seed, counter
 * (site mod 2^32, m, trajectory base + index in the batch, site >> 32), and Box-Muller
 * in FP64.  Resets the batch time to t = 0.  Errors: GPE_EINVAL (NULL mean_spinor,
 * noise_per_mode < 0). */
gpe_status tw_init_noise(gpe_batch* batch, uint64_t seed, const double mean_spinor[6],
                         double noise_per_mode, void* stream);

/* Advances every trajectory by nsteps Strang steps of dt (Sec. 2.2 split-step scheme)
 * starting from the batch time, which then increases by nsteps dt.  The fields hold
 * psi(t) (not a half-kicked state) before and after the call.  The first call on an FP32
 * batch also runs the tile autotuner (gpe_batch_set_autotune), which allocates a
 * temporary scratch batch and synchronises the stream: make it before any stream capture
 * of your own.  Errors: GPE_EINVAL (nsteps < 0). */
gpe_status gpe_step_batch(gpe_batch* batch, int64_t nsteps, void* stream);

/* Observable flags. */
#define GPE_OBS_SPECTRA 1u   /* n_1, n_0, n_-1 and S_perp, radially binned, summed over trajectories */
#define GPE_OBS_DIAG    2u   /* per-trajectory N_1, N_0, N_-1, E_kin, E_q, E_c0, E_c1, E_V         */
#define GPE_OBS_WINDING 4u   /* per-trajectory winding number of the Larmor angle (1D batches)     */

/* Accumulates observables of the current fields into acc (caller-owned device FP64):
 * acc += contributions, at offset sample_slot * slot_doubles (see gpe_obs_layout).
 * Within one slot: [4][nbins] spectra sums (quantity order n_1, n_0, n_-1, S_perp) --
 * a batch of several shapes has one such block per shape group with equal side lengths,
 * one after the other in group order (gpe_obs_group_layout), a single shape just one --
 * each the sum over the group's trajectories and over the grid modes of a bin of
 *   n_m(k) = |A_m(k)|^2 - 1/2,  A_m(k) = dx^d / sqrt(L^d) sum_x psi_m(x) e^{-ik.x},
 *   S_perp(k) = |F_perp(k)|^2 / L^d,  F_perp(k) = dx^d sum_x F_perp(x) e^{-ik.x},
 *   F_perp = sqrt(2) (psi_1^* psi_0 + psi_0^* psi_-1)   (Sec. 2.1),
 * with bin b = round(|k| / (2 pi / L)); then [ntraj][8] diagnostics (N_1, N_0, N_-1,
 * E_kin, E_q, E_c0, E_c1, E_V), E = dx^d sum_x [psi^*(-Laplacian/2)psi + q (n_1 + n_-1)
 * + c0 rho^2 / 2 + c1 (F_z^2 + |F_perp|^2) / 2 + sum_m V_m n_m] at the current q
 * (E_V = 0 without a potential); then [ntraj] winding numbers Q_w / (2 pi) of the Larmor
 * angle phi_L = arg(F_perp) (Sec. 1: Q_w = int dx d_x phi_L), each the sum over x of
 * arg(F_perp(x)^* F_perp(x+1)) in (-pi, pi] around the periodic grid, an integer up to
 * rounding (1D trajectories only).  Sums are
 * deterministic (fixed reduction order).  The fields are not modified.  The first call
 * on a batch allocates the handle's spectra workspace (four fields per trajectory, in
 * chunks of at most 1 GiB); make it before capturing a stream.
 * Errors: GPE_EINVAL (NULL acc, sample_slot < 0, unknown flags), GPE_EUNSUPPORTED
 * (spectra requested for a batch in which no shape group has equal side lengths; the
 * winding number for a batch with 2D or 3D trajectories).  Groups with unequal sides add
 * diagnostics but no spectra.  The winding number alone allocates no workspace. */
gpe_status observables_accumulate(gpe_batch* batch, double* acc, uint32_t flags,
                                  int32_t sample_slot, void* stream);

/* Accumulator geometry: number of radial bins of all shape groups together (0 if spectra
 * are unavailable) and the number of doubles per sample slot (4 * nbins + 9 * ntraj). */
gpe_status gpe_obs_layout(const gpe_batch* batch, int32_t* nbins, int64_t* slot_doubles);

/* Spectra block of trajectory traj's shape group: its number of radial bins (0 if the
 * group has unequal sides) and the offset, in doubles from the start of a slot, of its
 * [4][nbins] block.  Errors: GPE_EINVAL. */
gpe_status gpe_obs_group_layout(const gpe_batch* batch, int32_t traj, int32_t* nbins, int64_t* spectra_offset);

/* Number of grid modes in each radial bin (host array of nbins int64; the groups' bins one
 * after the other, as in the slot). */
gpe_status gpe_bin_counts(const gpe_batch* batch, int64_t* counts);

/* Offset added to the batch's trajectory indices in the noise counter (default 0), so
 * that batches on several devices draw disjoint members of one ensemble: a batch with
 * base b and n trajectories draws exactly trajectories b .. b+n-1 of a single large
 * batch with the same seed. */
gpe_status gpe_batch_set_traj_base(gpe_batch* batch, int64_t base);

/* External potential V_m(x) (Sec. 2.2: the diagonal part of the split step applies
 * exp(-i [V_m(x_j) + f_m] dt)).  V: caller-owned device array [3][n2][n1][n0] of reals in
 * the batch's precision (float for GPE_C64, double for GPE_C128), components V_1, V_0,
 * V_-1; it applies to every trajectory whose grid is n (unused axes 1) and must stay
 * valid while steps, observables or adjoint steps of the batch run.  V = NULL removes
 * it.  Both local-step integrators and the adjoint include it, and the diagnostics
 * record carries E_V = dx^d sum_x sum_m V_m n_m.  Drops cached step graphs.  Errors:
 * GPE_EINVAL (NULL n, V not aligned to its element size, no trajectory on grid n). */
gpe_status gpe_batch_set_potential(gpe_batch* batch, const int32_t n[3], const void* V);

/* Non-uniform initial states: mean_field (caller-owned device array [3][n2][n1][n0] of
 * complex FP64 as (re, im) pairs, 16-byte aligned) is added to the mean spinor by
 * tw_init_noise for every trajectory whose grid is n; NULL removes it.  It is read
 * during tw_init_noise only.  Errors: GPE_EINVAL (as gpe_batch_set_potential). */
gpe_status gpe_batch_set_mean_field(gpe_batch* batch, const int32_t n[3], const double* mean_field);

/* Local step of the split step.  GPE_INTEGRATOR_PAPER (default): the paper's diagonal
 * and predictor-averaged spin-mixing steps, D(dt/2) O(dt) D(dt/2) (Sec. 2.2).
 * GPE_INTEGRATOR_ROTATION: the same interaction of Eq. (GPE) written as
 * c0 rho + c1 F.f + q f_z^2 and split as Q(dt/2) R(dt) Q(dt/2), where R is the exact
 * flow exp(-i c0 rho dt) exp(-i c1 dt F.f) (rho and F are invariant under it) and Q the
 * quadratic Zeeman phase; it conserves F_z exactly.  The adjoint supports only the
 * paper's step. */
#define GPE_INTEGRATOR_PAPER 0
#define GPE_INTEGRATOR_ROTATION 1
gpe_status gpe_batch_set_integrator(gpe_batch* batch, int32_t kind);

/* Graph replay.  When enabled and q is constant (n_knots == 0), the first
 * gpe_step_batch call with a given nsteps captures its whole kernel sequence (all shape
 * groups, which run concurrently on internal streams forked from and joined back into
 * the caller's stream) into a CUDA graph, and later calls with the same nsteps replay it
 * with one launch.  The capture creates graph resources: make the first call for each
 * nsteps before any stream capture of your own.  Disabled by default; ignored while
 * profiling is enabled. */
gpe_status gpe_batch_set_graph(gpe_batch* batch, int32_t enable);

/* Trajectory lanes (scheduling only; the paper runs many independent trajectories per
 * GPU, Sec. 2.2, and prescribes no order).  gpe_step_batch splits the trajectories of
 * each 2D/3D shape group into ``lanes`` consecutive ranges of nearly equal size and
 * advances each range on its own internal stream (forked from and joined back into the
 * caller's stream; captured together in graph mode), so that one range's kernels fill
 * the tail and launch gap of the other's.  lanes = -1 restores the default (2 for a batch
 * of one 2D shape, else 1: the groups of a batch of several shapes already overlap on
 * their own streams); 1 turns lanes off; at most 64, and never more than a group's
 * trajectories.  1D groups and profiled steps always run as one lane.  The split changes
 * no result bit.  Errors: GPE_EINVAL (lanes not -1 or 1..64). */
gpe_status gpe_batch_set_lanes(gpe_batch* batch, int32_t lanes);
/* Lanes the group of trajectory ``traj`` is stepped in now.  Errors: GPE_EINVAL. */
gpe_status gpe_batch_get_lanes(const gpe_batch* batch, int32_t traj, int32_t* lanes);

/* Test hook for the bounded waits (failure handling; the paper has no counterpart).  Sets
 * how many times the first wait of each block of the x pass and of the tensor-map
 * strided pass may poll its copy barrier before the wait counts as expired: -1 restores
 * the default (2^22 polls), 0 makes that wait expire at once.  An expired wait records
 * GPE_ETIMEOUT in the status word (read by gpe_sync_status); the block then waits, with
 * the default limit, for its copies in flight and returns without writing, so that step's
 * fields are not a valid result.  Drops the batch's captured graphs.  Errors: GPE_EINVAL
 * (NULL batch, value below -1 or not below 2^32 - 1). */
gpe_status gpe_batch_set_wait_limit(gpe_batch* batch, int64_t first_wait_polls);

/* Test hook for the allocation-failure paths (the paper has no counterpart): after
 * ``after`` more successful device allocations by this library (any batch, any thread),
 * the next one fails as if the device were out of memory -- the call that needed it
 * returns GPE_ENOMEM -- and the hook switches itself off; after < 0 switches it off.
 * Always returns GPE_OK. */
gpe_status gpe_debug_fail_alloc(int64_t after);

/* Test hook for the table placement (the paper has no counterpart): mode 1 (the default)
 * lets the kernels built for it keep each thread's stage twiddles and kinetic phases in
 * its own row of tensor memory (the resident 1D kernel at 2048 and 4096 points and the
 * cluster kernel's 4096-point slices, FP32); mode 0 makes them read those tables through L1.  Both give the same result bits.  Process-wide, read at
 * each launch (graphs captured earlier keep the kernels they captured).  Errors:
 * GPE_EINVAL (mode not 0 or 1). */
gpe_status gpe_debug_table_memory(int32_t mode);

/* Tile autotuner of the kinetic passes (the paper prescribes none; the choices change no
 * result bit).  Enabled by default: the first gpe_step_batch call of an FP32 batch times,
 * per 2D/3D shape group, on a zero-filled scratch batch of the group's shape (at most
 * 256 MiB, freed again; if it cannot be allocated the defaults stay), every block size the
 * x pass is built for and, for groups with back-to-back fields, every tile width (complex
 * columns per block) the strided passes are built for, and keeps the fastest of each.
 * Skipped while the stream is being captured.  Disabled, or for FP64 and non-contiguous
 * groups, fixed per-size defaults are used. */
gpe_status gpe_batch_set_autotune(gpe_batch* batch, int32_t enable);

/* Fixes the tile widths of the strided passes for trajectory traj's group (and so for
 * every trajectory of its shape group): cols_y for y, cols_z for z, 0 keeps the current
 * width.  Each must be a width the pass is built for at that size (2, 4, 8 from n = 256,
 * 4, 8, 16 below) and divide nx; the autotuner then leaves the group alone.  The width
 * changes no result bit.  Errors: GPE_EINVAL (bad batch, trajectory or width),
 * GPE_EUNSUPPORTED (FP64 batches, 1D groups, groups whose fields are not back to back),
 * GPE_ECUDA. */
gpe_status gpe_batch_set_tiles(gpe_batch* batch, int32_t traj, int32_t cols_y, int32_t cols_z);

/* Tile widths in use for trajectory traj's group: cols[0] for y, cols[1] for z (0 where the
 * group has no such pass or uses the non-tensor-map pass), *tuned = 1 once the autotuner
 * has run for the group (tuned may be NULL).  Errors: GPE_EINVAL. */
gpe_status gpe_batch_get_tiles(const gpe_batch* batch, int32_t traj, int32_t cols[2], int32_t* tuned);

/* Block size of the x pass (local step fused with the x kinetic pass) for trajectory
 * traj's group.  FP32 2D/3D groups run it with 128 or 256 threads, or 192 at an x extent of
 * 512 (the autotuner times each on the first step and keeps the fastest; every row goes
 * through the same arithmetic, so the choice changes no result bit).  set: one of those
 * sizes fixes it (the autotuner then
 * leaves it), 0 restores the default; drops the batch's captured graphs.  Errors:
 * GPE_EINVAL (bad batch, trajectory or size), GPE_EUNSUPPORTED (FP64 batches, 1D groups). */
gpe_status gpe_batch_set_xpass_threads(gpe_batch* batch, int32_t traj, int32_t threads);
/* get: the block size in use (0 for 1D groups, which have no x pass).  Errors: GPE_EINVAL. */
gpe_status gpe_batch_get_xpass_threads(const gpe_batch* batch, int32_t traj, int32_t* threads);

/* Batch time as a step count (t = step * dt); settable for replaying segments. */
int64_t gpe_batch_get_step(const gpe_batch* batch);
gpe_status gpe_batch_set_step(gpe_batch* batch, int64_t step);

/* Checkpoint and resume (the paper has no counterpart; long runs and preemptible jobs need
 * it).  save: synchronises ``stream`` and writes to ``path`` (host file) the batch's step
 * counter (which also fixes the position in a q(t) schedule), trajectory base, dtype,
 * integrator, couplings, q knots, every trajectory's shape and spacing, and the fields of
 * every trajectory, with a hash of the whole.  load: reads such a file into a batch of the
 * same configuration -- the fields are copied into the batch's (caller-owned) field
 * buffers and the step counter and trajectory base are restored; the noise is drawn only
 * by tw_init_noise, so there is no generator state.  FP64 accumulators are the caller's
 * and are not included.  Errors: GPE_EINVAL (NULL arguments, unreadable or unwritable
 * file, not a checkpoint, hash mismatch, another configuration or size), GPE_ENOMEM
 * (host buffer), GPE_ECUDA. */
gpe_status gpe_batch_save(const gpe_batch* batch, const char* path, void* stream);
gpe_status gpe_batch_load(gpe_batch* batch, const char* path, void* stream);

/* Host transfers (no counterpart in the paper; for callers whose data live in host
 * memory).  gpe_batch_upload copies host_psi -- every trajectory of the batch in batch order,
 * each its [3][n2][n1][n0] field in the batch's precision, back to back -- into the
 * trajectories' device fields; gpe_batch_download copies the fields out in the same layout.
 * Trajectories whose fields are adjacent on the device go as one copy.  Asynchronous on
 * ``stream`` (page-locked host memory lets the copy overlap other work).
 * gpe_obs_download copies accumulator slot ``sample_slot`` of acc (device, slot_doubles of
 * gpe_obs_layout per slot) to host.  Errors: GPE_EINVAL (NULL pointer, sample_slot < 0),
 * GPE_ECUDA. */
gpe_status gpe_batch_upload(gpe_batch* batch, const void* host_psi, void* stream);
gpe_status gpe_batch_download(const gpe_batch* batch, void* host_psi, void* stream);
gpe_status gpe_obs_download(const gpe_batch* batch, const double* acc, int32_t sample_slot, double* host,
                            void* stream);

/* Reverse-mode step (vector-Jacobian product of one Strang step, Sec. 2.2 scheme; the
 * paper itself has no adjoint).  With psi_step_in = psi_n, the fields at the start of
 * step n = step_index (contiguous [ntraj][3][sites] complex, caller-owned device memory,
 * the batch's layout), and lam = dL/dpsi_{n+1} on entry, lam holds dL/dpsi_n on return
 * (same layout; gradients in the convention dL/dRe + i dL/dIm).  dL/dq_n, reduced in
 * FP64 in a fixed order, is added to dLdq (device, max(1, n_knots) doubles) with the
 * linear interpolation weights of q at t_n + dt/2 (dLdq[0] for constant q).  The first
 * call allocates the handle's adjoint workspace.  Errors: GPE_EINVAL, GPE_EUNSUPPORTED
 * (more than one shape, or x extent > 1024). */
gpe_status gpe_adjoint_step(gpe_batch* batch, const void* psi_step_in, void* lam, int64_t step_index,
                            double* dLdq, void* stream);

/* One checkpoint segment of the reverse sweep (Sec. 2.2 scheme; no counterpart in the
 * paper): from psi_ckpt = psi_{n0} (contiguous [ntraj][3][sites], not modified) it
 * recomputes the states the reverse steps need into ``states`` (caller-owned device
 * workspace of nseg such fields, back to back, 16-byte aligned), using the batch's own
 * fields as scratch (their contents on return are unspecified; the step counter is
 * n0 + nseg - 1), then pulls lam back over steps n0 + nseg - 1 down to n0: lam =
 * dL/dpsi_{n0+nseg} on entry, dL/dpsi_{n0} on return, dL/dq added to dLdq, as
 * gpe_adjoint_step would.  2D/3D batches recompute with merged kinetic half steps and keep
 * K(dt/2) psi_n, the state each reverse step starts from, so the segment needs two field
 * passes fewer per step than those calls (the results agree to rounding); 1D batches make
 * exactly those calls.  Errors: GPE_EINVAL (NULL or misaligned pointer, n0 < 0, nseg < 1),
 * GPE_EUNSUPPORTED (as gpe_adjoint_step). */
gpe_status gpe_adjoint_segment(gpe_batch* batch, const void* psi_ckpt, void* states, int64_t n0, int64_t nseg,
                               void* lam, double* dLdq, void* stream);

/* Late-time spin structure factor loss over a band of wave numbers:
 * loss[0] = (1/ntraj) sum_traj sum_{grid modes with kmin <= |k| <= kmax} S_perp(k) of
 * the fields psi (contiguous [ntraj][3][sites]; S_perp as in observables_accumulate),
 * FP64, deterministic.  If lam_out is not NULL it receives dloss/dpsi (same layout).
 * Errors: GPE_EINVAL, GPE_EUNSUPPORTED (as gpe_adjoint_step). */
gpe_status gpe_sf_band_loss(gpe_batch* batch, const void* psi, double kmin, double kmax, double* loss,
                            void* lam_out, void* stream);

/* Measurement: when enabled, every launch the batch makes is bracketed by CUDA events on
 * its stream, summed per kernel class: 0 = x pass (local step fused with the x kinetic
 * pass), 1 = strided kinetic pass (y or z), 2 = resident 1D kernel, 3 = noise,
 * 4 = observables (whole pipeline of one call), 5 = adjoint (one gpe_adjoint_step call, or
 * one gpe_adjoint_segment call: its recompute and strided passes are also counted in classes
 * 0 and 1, so the classes then overlap).  gpe_profile_read synchronises the
 * device, writes the summed milliseconds and launch counts of each class (arrays of 6,
 * host) since the last read, and resets them. */
gpe_status gpe_profile_enable(gpe_batch* batch, int32_t enable);
gpe_status gpe_profile_read(gpe_batch* batch, double* ms, int64_t* launches);

/* Real-space diagnostics that allocate no device memory (the paper has no counterpart;
 * this is a service entry point).  For callers that cannot let the library allocate:
 * code that must not synchronise the device (cudaMalloc and cudaFree can), a process
 * whose device memory is all handed out by another allocator, or a health check run
 * while the device is out of memory.  psi: ntraj caller-owned fields laid out back to
 * back, each [3][n2][n1][n0] complex (dtype), 16-byte aligned.  out: caller-owned device
 * array of ntraj * 8 doubles, overwritten (not accumulated) with
 * (N_1, N_0, N_-1, 0, E_q, E_c0, E_c1, 0) per trajectory -- the diagnostics record of
 * observables_accumulate with the kinetic energy (slot 3) and the potential energy
 * (slot 7) always zero: no potential is taken, even for fields of a batch that has one.
 * Any extents are accepted (not only powers of two).  Partial sums live in a fixed
 * 192 KiB array compiled into the library (held on every device that loads it until the
 * process exits); capacity: ntraj * ceil(sites / 4096) <= 4096 site blocks, larger
 * requests return GPE_EINVAL with a message.  The first call on a device looks up the
 * array's device address, so make it before any stream capture; the address is kept for
 * the process's life, so after a cudaDeviceReset the entry point must not be called
 * again.  Calls share the array: calls that overlap on the same GPU race; serialise them.
 * Errors: GPE_EINVAL (NULL or misaligned pointers, bad sizes, capacity), GPE_ECUDA (also
 * when an error from earlier work is already pending; it is left for its owner). */
gpe_status gpe_diagnostics_noalloc(const void* psi, int32_t ntraj, int32_t ndim, const int32_t n[3],
                                   double dx, gpe_dtype dtype, double c0, double c1, double q,
                                   double* out, void* stream);

/* Verification of the FP32 sine/cosine the local step uses (Cody-Waite reduction plus
 * Taylor polynomials): for each of n device floats x, writes 4 floats to out (device):
 * its sin and cos, then CUDA's sincosf of the same x.  Errors: GPE_EINVAL (NULL, n < 0). */
gpe_status gpe_check_sincos(const float* x, float* out, int64_t n, void* stream);

/* Arithmetic-rate probe (measurement support for the roofline of the compute-bound
 * passes; not part of the method): times one launch that fills every SM with independent
 * FMA chains and writes the rate to *flops_per_s (host), counting an FMA as 2 flops.
 * kind 0: FP32 fma, 1: FP32 through the packed two-lane fma, 2: FP64 fma.  iters sets
 * the work per thread (256 flops per trip; about 2^16 for FP32, 2^10 for FP64 gives a
 * launch of tens of ms).  Synchronises the stream.  Errors: GPE_EINVAL (NULL, iters <= 0,
 * unknown kind), GPE_ECUDA. */
gpe_status gpe_fma_rate(int32_t kind, int64_t iters, double* flops_per_s, void* stream);

/* Number of kernels this library has launched since it was loaded (all batches). */
int64_t gpe_launch_count(void);

/* Synchronises ``stream`` and returns the device status word (GPE_OK if clean) and
 * clears it. */
gpe_status gpe_sync_status(gpe_batch* batch, void* stream);

/* Message of the last failing call on this thread ("" if none). */
const char* gpe_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GPE_H */
