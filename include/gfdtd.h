/*
 * gfdtd.h -- C ABI of the GB300 (sm_103a) generalized-FDTD engine.
 *
 * The engine time-steps batches of independent 1D problems with the
 * generalized Yee cell and stencil of Deck-Leger, Bahrami, Li and Caloz,
 * "Generalized FDTD Scheme for the Simulation of Electromagnetic Scattering in
 * Moving Structures" (arXiv 2304.06586):
 *
 *   Sec. 3 (Fig. 2):   the Yee cell carries the auxiliary fields
 *                      E* = E + v x B and H* = H - v x D (Eq. star) in place of
 *                      the tangential E and H; D sits on integer nodes k and B
 *                      on half nodes k+1/2, as in the standard Yee cell.
 *   Sec. 4:            the leapfrog updates Eqs. Farad_discr and Ampere_discr
 *                      (B and D) and the constitutive updates Eqs.
 *                      Dconst_discr and Bconst_discr (E* and H*), with the
 *                      velocity terms of Table 1 (upwind differences dBa/dBb,
 *                      dDa/dDb and the averages Ba/Bb, Da/Db; column chosen by
 *                      the sign of v).
 *   Eq. const_3d_regular: the medium is a profile eps(z - v t), mu(z - v t)
 *                      that moves rigidly at velocity v (moving perturbation),
 *                      or moving matter whose rest-frame profile eps', mu' is
 *                      made bianisotropic by the motion (footnote tensors of
 *                      Eq. const_3d_regular).
 *   Eq. spectrum_incident: sources are Gaussian-modulated carriers.
 *   Eqs. spectrum_scat_interface, comp_exp: probes accumulate running DFTs of
 *                      the physical E field.
 *
 * Units are normalised: c = eps0 = mu0 = 1, v = beta, the cell size is 1 and
 * the time step is S = dt/dz (the Courant number).  Time level n (B, H*) is
 * t = n S; level n+1/2 (D, E*) is t = (n + 1/2) S.  After n steps the state of
 * an instance is (B^n, D^{n+1/2}); a fresh context starts at n = 0 with all
 * fields zero.  Fields outside [0, nz) are zero (perfectly conducting /
 * magnetic walls one half cell outside the grid).
 *
 * Moving medium.  Positions are given in cells of the moving frame at t = 0.
 * A node at lab position p (k for D, k + 1/2 for B) at time t samples the
 * profile at xi = p - beta t.  xi is evaluated exactly in 32.32 fixed point:
 * profile positions are rounded to multiples of 2^-32 cell and the
 * displacement per half step is round(beta * S * 2^31) units of 2^-32 cell
 * (beta * S taken as the IEEE double product, rounding half away from zero).
 * Layers are half-open intervals [z_{i-1}, z_i).
 *
 * Moving matter.  With rest values eps', mu' (n'^2 = eps' mu') the 1D star
 * relations of Eq. const_3d, solved for E* and H*, read
 *     E* = D / eps_m - beta_c B,   H* = B / mu_m - beta_c D,
 *     1/eps_m = (1 - beta^2) mu' / (n'^2 - beta^2),
 *     1/mu_m  = (1 - beta^2) eps' / (n'^2 - beta^2),
 *     beta_c  = beta (1 - beta^2) / (n'^2 - beta^2);
 * they are discretized like Eqs. Dconst_discr / Bconst_discr with the Table 1
 * averages (beta_c in the averaged terms, beta in the upwind terms).
 *
 * Conventions.  Every call returns a gfdtd_status; nothing aborts or throws
 * across the ABI.  Host input arrays are copied before the call returns.
 * Host output buffers are owned by the caller.  The library owns its device
 * memory, obtained from the allocator installed with gfdtd_set_allocator (by
 * default cudaMalloc).  Work runs asynchronously on the stream given to
 * gfdtd_create; calls that return data to the host synchronise that stream.
 * A context must not be used from two threads at once.
 */
#ifndef GFDTD_H
#define GFDTD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gfdtd_ctx gfdtd_ctx;

typedef enum {
    GFDTD_OK = 0,
    GFDTD_E_ARG = -1,          /* invalid argument (index, size, NULL pointer, range) */
    GFDTD_E_OOM = -2,          /* device or host allocation failed */
    GFDTD_E_CUDA = -3,         /* a CUDA runtime call failed; see gfdtd_last_error */
    GFDTD_E_UNSTABLE = -4,     /* medium outside the scheme's stability region (n|beta| > 1) */
    GFDTD_E_TIMEOUT = -5,      /* a kernel's bounded wait (for its own tile copy) gave up; the
                                  context stays usable, the affected steps are not valid */
    GFDTD_E_STATE = -6,        /* call not valid in the context's current state */
    GFDTD_E_UNSUPPORTED = -7   /* option not built into this library */
} gfdtd_status;

typedef enum { GFDTD_PERTURBATION = 0, GFDTD_MATTER = 1 } gfdtd_kind;

/* Field storage and update precision.  F32: FP32 storage and arithmetic.
 * F32_KAHAN: FP32 with compensated (Kahan) B and D updates.  BF16 / F16:
 * 16-bit storage between time blocks, FP32 arithmetic.  F64: FP64 storage and
 * arithmetic (reference tier; GB300's FP64 rate is low). */
typedef enum {
    GFDTD_F32 = 0, GFDTD_F32_KAHAN = 1, GFDTD_BF16 = 2, GFDTD_F16 = 3, GFDTD_F64 = 4
} gfdtd_prec;

/* Profile interpolation.  LAYERS: n values, n-1 boundaries, value i on
 * [z_{i-1}, z_i).  LINEAR: n knots, linear between knots, constant beyond the
 * first and last knot. */
typedef enum { GFDTD_LAYERS = 0, GFDTD_LINEAR = 1 } gfdtd_interp;

/* Fields readable with gfdtd_read_fields.  D (level n+1/2) and B (level n) are
 * the state; E = physical E at level n+1/2 (moving perturbation: D/eps,
 * Eq. const_1d; moving matter: E* + beta Bbar); ESTAR = E* at level n+1/2
 * (Eq. Dconst_discr with B^n); H = physical H at level n (moving perturbation
 * only: B/mu, Eq. const_1d). */
typedef enum {
    GFDTD_FIELD_D = 0, GFDTD_FIELD_B = 1, GFDTD_FIELD_E = 2, GFDTD_FIELD_H = 3, GFDTD_FIELD_ESTAR = 4
} gfdtd_field;

/* Device allocator hooks: alloc returns a device pointer (NULL on failure),
 * free releases it.  `stream` is the context's CUDA stream. */
typedef void* (*gfdtd_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*gfdtd_free_fn)(void* ptr, size_t bytes, void* stream, void* user);

/* Install process-wide allocator hooks used by contexts created afterwards.
 * Both NULL restores cudaMalloc/cudaFree.  Returns E_ARG if exactly one is NULL. */
gfdtd_status gfdtd_set_allocator(gfdtd_alloc_fn alloc, gfdtd_free_fn free_fn, void* user);

/* Create a context for n_inst independent instances of nz[i] cells each
 * (1 <= nz[i] <= 2^28, n_inst >= 1), Courant number S in (0, 1], field
 * precision prec, on the CUDA stream cuda_stream (a cudaStream_t; NULL = the
 * legacy default stream) of the current device.  Every instance starts as
 * vacuum at rest with no sources or probes.  Allocates all field storage. */
gfdtd_status gfdtd_create(gfdtd_ctx** out, int n_inst, const int64_t* nz, double S,
                          gfdtd_prec prec, void* cuda_stream);

/* Set the moving medium of instance `inst` (Eq. const_3d_regular): kind,
 * velocity beta in (-1, 1), interpolation, n values (n >= 1; n >= 2 for
 * LINEAR) of eps_r[] and mu_r[] (> 0), and positions z[] (LAYERS: n-1
 * strictly increasing boundaries; LINEAR: n strictly increasing knots; may be
 * NULL when n == 1 for LAYERS).  Fails with E_UNSTABLE when some value pair
 * has n|beta| > 1 (the von Neumann limit of the scheme, Sec. 5) unless
 * `allow_unstable` is nonzero, and with E_ARG when |beta| S >= 1. */
gfdtd_status gfdtd_set_medium(gfdtd_ctx* ctx, int inst, gfdtd_kind kind, double beta,
                              gfdtd_interp interp, int n, const double* z,
                              const double* eps_r, const double* mu_r, int allow_unstable);

/* Graded absorbing layers at both ends of instance inst (an option of this
 * library: the paper is silent on the domain ends, and without layers every
 * field is zero beyond them, so waves reflect there).  A field sample at
 * position x (D_k: x = k, B_k: x = k + 1/2) is multiplied right after its
 * update by exp(-sigma d^2), d = (width - x) / width for x < width,
 * (x - (nz - 1 - width)) / width for x > nz - 1 - width, else 0; sources are
 * added after the damping.  width = 0 removes the layers.  With width 64 and
 * sigma 0.2 a pulse of 40-cell carrier wavelength returns below 3e-4 of its
 * amplitude for |beta| <= 0.3 (S = 0.5, vacuum; below 1e-6 at beta = 0).
 * Tiles that reach a layer take the general kernel.  gfdtd_adjoint rejects
 * instances with layers (E_UNSUPPORTED).  E_ARG unless 0 <= width,
 * 2 width < nz and sigma is a finite number >= 0.  Takes effect at the next
 * step. */
gfdtd_status gfdtd_set_absorber(gfdtd_ctx* ctx, int inst, int64_t width, double sigma);

/* Add a soft source to instance `inst` at integer node `node` in [0, nz):
 * after the D update of every step n, D_node += amp sin(omega0 (t - t0))
 * exp(-((t - t0)/tau)^2) with t = (n + 1/2) S (Eq. spectrum_incident, real
 * carrier).  tau > 0. */
gfdtd_status gfdtd_add_source(gfdtd_ctx* ctx, int inst, int64_t node, double omega0,
                              double tau, double t0, double amp);

/* Add a one-way (total-field / scattered-field) source to instance `inst`
 * (an option of this library; the paper's source is the soft one above).
 * Nodes >= node hold the total field, nodes < node the scattered field, and
 * the incident wave enters the total-field region only: it is the right-going
 * wave that a soft source with this waveform emits in an auxiliary grid of
 * the same scheme (FP64 for FP64 fields, FP32 otherwise) filled with the
 * uniform background, taken as the
 * material at `node` at t = 0 (1064 cells: graded layers of 512 cells and
 * strength 0.05 at both ends of a 40-cell interior, the auxiliary soft source
 * 12 cells left of the boundary; 512 is the smallest power-of-two width whose
 * layers reflect below 1e-6 of the incident wave in moving vacuum for
 * |beta| <= 0.6).  Each step, the updates of B at node-2 .. node+1 and of D at
 * node-1 .. node that read a neighbour across the boundary get that
 * neighbour's incident value added (total-field update) or subtracted
 * (scattered-field update).  The background must stay uniform around the
 * boundary for the whole run; what the auxiliary layers reflect (about 1e-6
 * of the incident amplitude for |beta| <= 0.6) reaches the scattered-field
 * region.  Tiles holding those cells take the general kernel; the auxiliary
 * grids advance in their own launch per chunk of steps.  Adding a source
 * restarts every auxiliary grid of the context from rest; write_fields and
 * write_state leave them alone.  gfdtd_step_plain and gfdtd_adjoint reject
 * contexts with one-way sources (E_UNSUPPORTED).  E_ARG unless node is in
 * [0, nz), tau > 0, the other values finite, at most 4 per instance.  Takes
 * effect at the next step. */
gfdtd_status gfdtd_add_tfsf(gfdtd_ctx* ctx, int inst, int64_t node, double omega0, double tau,
                            double t0, double amp);

/* Add a DFT probe at integer node `node` of instance `inst` with n_bins >= 1
 * angular frequencies omega[] (copied).  From the next step on, every step
 * adds E(node, t) exp(+i omega t) S to each bin, t = (n + 1/2) S, in FP64.
 * *probe_id receives the probe's index within the instance. */
gfdtd_status gfdtd_add_probe(gfdtd_ctx* ctx, int inst, int64_t node, int n_bins,
                             const double* omega, int* probe_id);

/* Advance every instance by n_steps >= 0 steps with the batched kernel
 * (register-resident tiles, several steps per HBM round trip, one launch per
 * time block for the whole batch, replayed from a CUDA graph).  The first call
 * may autotune the tile shape; make it before capturing the stream into a
 * graph of your own.  Asynchronous. */
gfdtd_status gfdtd_step(gfdtd_ctx* ctx, int64_t n_steps);

/* Same result as gfdtd_step with the plain kernel: one step and one instance
 * per launch, fields in HBM.  The throughput baseline; also asynchronous. */
gfdtd_status gfdtd_step_plain(gfdtd_ctx* ctx, int64_t n_steps);

/* Copy field `which` of instance `inst` to host_dst[0..n) as doubles, n == nz.
 * Synchronises the context's stream. */
gfdtd_status gfdtd_read_fields(gfdtd_ctx* ctx, int inst, gfdtd_field which,
                               double* host_dst, int64_t n);

/* Overwrite the state field D or B of instance `inst` from host_src[0..n),
 * n == nz (rounded to the storage precision).  Synchronises the stream. */
gfdtd_status gfdtd_write_fields(gfdtd_ctx* ctx, int inst, gfdtd_field which,
                                const double* host_src, int64_t n);

/* Bulk copies of a whole state field (D or B) in device storage format and
 * layout: instance i occupies elements [offsets[i], offsets[i] + nz[i]) of an
 * array of gfdtd_state_elems() elements of gfdtd_state_elem_bytes() bytes
 * (padding elements are zero).  `bytes` must equal the array size.  host
 * buffers should be pinned for full copy bandwidth.  Asynchronous with respect
 * to the host when host memory is pinned; synchronise with gfdtd_synchronize. */
gfdtd_status gfdtd_read_state(gfdtd_ctx* ctx, gfdtd_field which, void* host_dst, int64_t bytes);
gfdtd_status gfdtd_write_state(gfdtd_ctx* ctx, gfdtd_field which, const void* host_src,
                               int64_t bytes);
gfdtd_status gfdtd_state_layout(const gfdtd_ctx* ctx, int64_t* n_elems, int* elem_bytes,
                                int64_t* offsets /* n_inst entries, or NULL */);

/* Read the FP64 DFT accumulators of probe `probe_id` of instance `inst` into
 * re[0..n_bins) and im[0..n_bins).  Synchronises the stream. */
gfdtd_status gfdtd_read_spectrum(gfdtd_ctx* ctx, int inst, int probe_id, double* re, double* im);

/* Steps completed so far (the n of the state (B^n, D^{n+1/2})). */
gfdtd_status gfdtd_steps_done(const gfdtd_ctx* ctx, int64_t* n);

/* Gradient of probe power with respect to the permittivity profile, by the
 * discrete adjoint (the transpose of every step of Sec. 4 / Table 1, applied
 * in reverse time) with sqrt(n_steps) checkpointing.  From the current state,
 * advances every instance by n_steps >= 1 steps exactly as gfdtd_step does
 * (state, step count and DFT accumulators included), and returns, per instance
 * i, loss[i] = L_i = sum_{f = bin_lo}^{bin_hi - 1} |X_f|^2 with X_f the DFT of
 * its probe `probe_id` accumulated over these n_steps only, and in grad the
 * derivatives dL_i / d eps_r[j] of every profile value j of instance i (LAYERS:
 * layer values; LINEAR: knot values), instances concatenated in order.
 * Moving-perturbation instances and FP32 / F32_KAHAN contexts only
 * (E_UNSUPPORTED otherwise).  Every instance needs probe `probe_id` with at
 * least bin_hi bins.  loss: n_inst doubles; grad: sum of n values doubles. */
gfdtd_status gfdtd_adjoint(gfdtd_ctx* ctx, int64_t n_steps, int probe_id, int bin_lo, int bin_hi,
                           double* loss, double* grad);

/* Host-only von Neumann analysis (Sec. 5, App. A): max over kz dz in (0, pi]
 * of the modulus of the eigenvalues of the one-step amplification matrix of a
 * uniform medium (eps_r, mu_r) moving at beta with Courant number S. */
gfdtd_status gfdtd_stability(double S, double beta, double eps_r, double mu_r,
                             gfdtd_kind kind, double* max_abs_zeta);

/* Tile shape of the batched kernel: cells per lane (4 to 24), steps per time
 * block (8 to 32) and the number of 128-thread blocks per SM the fast
 * kernel's registers are limited to (4 to 8; 0 = first built match).  The
 * shapes built depend on the precision (FP32: 8x16x4, 16x16x4, 16x24x8,
 * 20x16x7, 20x24x7, 20x32x7, 24x24x6; FP32 with Kahan terms: 16x16x4, 8x16x4;
 * BF16 and FP16: 16x16x4, 8x16x4, 16x24x8, 24x24x6; FP64: 4x8x4, 8x8x4,
 * 8x16x4, 8x24x6); E_UNSUPPORTED if the shape is not built.  0, 0, 0 selects autotuning at the next step: every
 * built shape is timed on the batch (two interleaved passes of one warm-up
 * and three timed time blocks that follow one another in time) and the
 * fastest kept.  Tiles outside the fast kernel's reach (moving matter,
 * piecewise-linear or narrow-layer profiles, domain ends, one-way sources)
 * either all run in the general kernel, or first pass through a lean kernel
 * that steps those whose window sees one material value during the launch
 * and queues the rest for the general kernel (the uniform-tile split); a
 * shape set here takes the split, autotuning times both ways per shape. */
gfdtd_status gfdtd_set_tuning(gfdtd_ctx* ctx, int cells_per_lane, int time_block, int blocks_per_sm);

typedef struct {
    int cells_per_lane;        /* chosen tile shape */
    int time_block;
    int blocks_per_sm;
    int64_t n_tiles;           /* tiles per time block for the whole batch */
    int64_t kernel_launches;   /* library kernels launched so far (graph nodes counted) */
    int64_t cells;             /* sum of nz */
    int uniform_split;         /* 1: the general lists take the uniform-tile split */
} gfdtd_stats;

gfdtd_status gfdtd_get_stats(const gfdtd_ctx* ctx, gfdtd_stats* out);

/* Space-time capture (the z-t field maps of Fig. 5(a)): after every t_stride
 * steps taken by gfdtd_step, counted from the call, record field `which`
 * (any gfdtd_field, as gfdtd_read_fields defines it, at the state reached) of
 * instance inst at cells z0, z0 + z_stride, ... < z1 as one frame, rounded to
 * FP32 (half = 0) or FP16 (half = 1), in a device buffer of max_frames frames
 * that the context allocates here (through the allocator hooks); frames past
 * max_frames are counted as dropped.  gfdtd_step ends its CUDA-graph chunks at
 * frame steps, so a t_stride below the tile time block shortens the blocks.
 * Frames are not recorded by gfdtd_step_plain, gfdtd_profile_kernels or
 * gfdtd_adjoint.  One capture per context; a new call replaces it (frames
 * discarded), t_stride = 0 turns it off (frames kept).  E_ARG unless
 * 0 <= z0 < z1 <= nz, z_stride, t_stride, max_frames >= 1 and half is 0 or 1;
 * E_UNSUPPORTED for H of moving matter; E_OOM if the buffer cannot be had. */
gfdtd_status gfdtd_set_capture(gfdtd_ctx* ctx, int inst, gfdtd_field which, int64_t z0, int64_t z1,
                               int64_t z_stride, int64_t t_stride, int64_t max_frames, int half);

/* Frames recorded, values per frame and frames dropped so far. */
gfdtd_status gfdtd_capture_info(const gfdtd_ctx* ctx, int64_t* frames, int64_t* cells_per_frame,
                                int64_t* dropped);

/* Copy the recorded frames, frame after frame (n = frames x cells_per_frame),
 * widened to FP64, into host_dst.  Synchronises the context's stream. */
gfdtd_status gfdtd_read_capture(gfdtd_ctx* ctx, double* host_dst, int64_t n);

/* Measurement hook (no counterpart in the paper).  Advances every instance by
 * n_steps exactly as gfdtd_step does (same kernels, same results), but
 * launches them one by one outside CUDA graphs, brackets each batched-kernel
 * launch with CUDA events on the context's stream and waits for the stream
 * at the end.  Index 0 of each array is the general moving-perturbation
 * kernel, 1 the general moving-matter kernel, 2 the fast interior kernel:
 * launches, their summed device time in ms, and the cell-updates they
 * produced (exact output cells of their tiles x steps).  out is written on
 * success only.  Errors as gfdtd_step; E_ARG for a NULL out. */
typedef struct {
    int64_t launches[3];
    double ms[3];
    int64_t cell_updates[3];
} gfdtd_kernel_times;

gfdtd_status gfdtd_profile_kernels(gfdtd_ctx* ctx, int64_t n_steps, gfdtd_kernel_times* out);

/* Measurement hook (no counterpart in the paper): the launch structure of
 * gfdtd_step_plain without its arithmetic, the throughput bound of the
 * one-instance, one-step-per-launch form.  Enqueues n_steps replays of a CUDA
 * graph holding, in instance order on the context's stream, one launch per
 * instance with the plain kernel's grid, in which every thread reads its
 * cell's B and D and the block's output cells are written back unchanged
 * (16 bytes per cell in FP32, the plain kernel's algorithmic traffic), plus
 * the plain path's per-step counter launch.  Fields, probes and the step count
 * are left as they were.  Asynchronous: time it with events on the context's
 * stream.  E_UNSUPPORTED where gfdtd_step_plain is. */
gfdtd_status gfdtd_plain_floor(gfdtd_ctx* ctx, int64_t n_steps);

/* ---- batched parameter sweeps (context-free, GPU, FP64) ----
 *
 * Von Neumann stability map (Sec. 5 and App. A): for each point i, the
 * largest eigenvalue modulus of the one-step amplification matrix of a
 * uniform medium (eps_r[i], mu_r[i]) under the scheme of Sec. 4 / Table 1
 * with Courant number S[i] and velocity beta[i] (kind[i]: GFDTD_PERTURBATION
 * or GFDTD_MATTER), maximised over kz dz = pi (j + 1) / n_theta,
 * j = 0 .. n_theta - 1.  The scheme is stable for a medium where the result
 * is <= 1 (to rounding).  S, beta, eps_r, mu_r, kind and out are DEVICE
 * arrays of n elements owned by the caller; the call only enqueues the work
 * on cuda_stream (NULL: the legacy default stream) and returns.  Valid inputs
 * are those of gfdtd_stability (0 < S <= 1, |beta| < 1, eps_r, mu_r > 0);
 * others give unspecified values.  E_ARG for n < 0, n_theta < 1 or a NULL
 * array (n > 0); E_CUDA if the launch fails.  n == 0 does nothing. */
gfdtd_status gfdtd_stability_map(int64_t n, const double* S, const double* beta, const double* eps_r,
                                 const double* mu_r, const int* kind, int n_theta, double* out,
                                 void* cuda_stream);

/* Star transfer-matrix scattering of moving layered stacks (App. B.3, with
 * the matrices derived from Eq. cont and Eq. star): stack s has the layers
 * layer_off[s] .. layer_off[s+1]-1 (at least two), the first and last being
 * the semi-infinite media, all moving at beta[s] (moving perturbation, c = 1,
 * lengths in cells).  eps_r, mu_r: per layer; thick: per layer, the length in
 * the moving frame (read for the inner layers only).  For each incident lab
 * frequency omega[f] (a +z wave in the first medium) it writes the
 * transmission T and reflection Gamma as ratios of physical E amplitudes,
 * complex, interleaved (re, im), at index s * n_freq + f.  All arrays are
 * DEVICE arrays owned by the caller (layer_off: n_stacks + 1 entries; T and
 * Gamma: 2 n_stacks n_freq doubles); asynchronous on cuda_stream.  A stack
 * with fewer than two layers gets NaN.  E_ARG for negative counts or a NULL
 * array (nonzero counts); E_CUDA if the launch fails. */
gfdtd_status gfdtd_star_tmm(int64_t n_stacks, const int64_t* layer_off, const double* eps_r,
                            const double* mu_r, const double* thick, const double* beta, int64_t n_freq,
                            const double* omega, double* T, double* Gamma, void* cuda_stream);

/* Runtime stability watchdog.  The scheme is unstable where n|beta| > 1
 * (Sec. 5, App. A: the amplification factor of some mode exceeds one), and
 * an instance run there (allow_unstable) grows until it overflows.  At the
 * end of every chunk of at most 1024 steps of gfdtd_step, gfdtd_step_plain
 * and gfdtd_profile_kernels, a scan of the state records, per instance, the
 * largest |B| and |D| (rounded to FP32) and whether any value is not finite;
 * gfdtd_adjoint and the autotuner's trial launches record nothing.  This call
 * synchronises the
 * stream and writes, for each instance i, flags[i] (bit 0: a non-finite value
 * was written; bit 1: the largest magnitude exceeded `limit` > 0, a
 * non-finite value counting as infinite) and amax[i] (the largest magnitude,
 * +inf once a non-finite value was written); either array may be NULL
 * (n_inst entries each); with reset != 0 the record then starts again from
 * zero.  The record covers every time block since the context was created or
 * last reset.  Returns E_UNSTABLE when some instance is flagged, else OK. */
gfdtd_status gfdtd_watchdog(gfdtd_ctx* ctx, double limit, int reset, int* flags, double* amax);

/* Test hook for the bounded waits (no counterpart in the paper).  With on != 0
 * the fast kernel's warps arm the barrier of each tile copy but start no copy,
 * so each wait gives up after its limit (about one second of device time per
 * warp); the step then reports E_TIMEOUT through gfdtd_synchronize and the
 * affected steps are not valid.  No copy is ever in flight, so nothing lands
 * after a block has exited.  on = 0 restores normal operation.  Takes effect
 * at the next step. */
gfdtd_status gfdtd_test_stall(gfdtd_ctx* ctx, int on);

/* Wait for all work queued on the context's stream; returns E_TIMEOUT (once)
 * if a kernel reported that a bounded wait gave up since the last check.
 * gfdtd_read_fields and gfdtd_read_spectrum report it the same way. */
gfdtd_status gfdtd_synchronize(gfdtd_ctx* ctx);

/* Text of the last error on this context (or of the last failed create when
 * ctx is NULL).  Valid until the next call on the context. */
const char* gfdtd_last_error(const gfdtd_ctx* ctx);

/* Allocation-free stepping (the paper has no counterpart).  For callers that
 * cannot allocate device memory: a process whose GPU memory another
 * framework's caching pool has reserved up front, so that cudaMalloc fails or
 * would fragment that pool; a plugin host that hands its plugins buffers but
 * no allocator; a loop with a fixed memory budget that must not risk an
 * allocation failing half way through a run.  Advances ONE instance held in
 * caller-owned device buffers B and D (FP32, nz elements each, the state
 * (B^n, D^{n+1/2}) with n = n_done) by n_steps steps, with the medium given as
 * in gfdtd_set_medium, no sources and no probes, using the same kernels and
 * tile shape (16 cells per lane, 16 steps per time block) as gfdtd_step.
 * Every working buffer lives in one statically allocated device array of
 * about 4.4 MB that each GPU loading this library keeps until the process
 * exits; no call allocates or frees memory.  Limits: 1 <= nz <= 2^18 and
 * n <= 1024 profile values, otherwise E_ARG.  The first call on each device
 * sets up: it looks up the array's device address (cudaGetSymbolAddress), so
 * make that first call before any stream capture.  All calls share the array,
 * which keeps the last call's contents (each call clears what has to start at
 * zero): calls whose work overlaps on the GPU (other streams, other threads)
 * race and corrupt each other.  The call synchronises cuda_stream before it
 * returns; when a kernel's bounded wait gave up it returns E_TIMEOUT and
 * leaves B and D as they were. */
gfdtd_status gfdtd_step_noalloc(int64_t nz, double S, gfdtd_kind kind, double beta,
                                gfdtd_interp interp, int n, const double* z, const double* eps_r,
                                const double* mu_r, float* B, float* D, int64_t n_done,
                                int64_t n_steps, void* cuda_stream);

/* ---- 2D TE generalized scheme (oblique incidence, slanted moving layers) ----
 *
 * Sec. 3 and Sec. 4 before their 1D reduction, for moving perturbation in the
 * x-z plane (d/dy = 0, motion along z, E = E_y y^, B = (B_x, 0, B_z),
 * D = D_y y^).  Eq. star and Eq. const_3d give E*_y = D_y/eps + v B_x,
 * H*_x = B_x/mu + v D_y, H*_z = B_z/mu (E*_y is tangential to every boundary
 * in the x-z plane, Eq. EHstar_comp), and Eq. Maxwell_star, with
 * curl(v x F) = -v dF/dz for a uniform velocity and divergence-free F, gives
 *     dB_x/dt = dE*_y/dz - v dB_x/dz,   dB_z/dt = -dE*_y/dx - v dB_z/dz,
 *     dD_y/dt = dH*_x/dz - dH*_z/dx - v dD_y/dz.
 * Along z these are discretized exactly as the 1D scheme (Table 1 averages in
 * E*_y and H*_x, upwind differences of every component; with b = -B_x the
 * z-part is the 1D update), along x with plain Yee differences.  Grid: D_y at
 * (i, k), B_x at (i, k + 1/2), B_z at (i + 1/2, k); x spacing dx in units of
 * the z cell, S = dt/dz; periodic over the nx columns, every field zero
 * beyond the z ends.  The medium is moving-perturbation layers of the moving
 * coordinate xi = z - beta t - slope x (boundary j at xi = z_j; slope != 0:
 * boundaries slanted against the motion, n not parallel to v), sampled per
 * node exactly in 32.32 fixed point: xi = z 2^32 - round(beta S 2^31) h -
 * round(x slope 2^32) at half level h.  Fields are stored [i][k] (nx rows of
 * nz values) in FP32 or FP64.  The GPU holds all nx <= 32 columns of a
 * z-tile in one block (one warp per column). */
typedef struct gfdtd2d_ctx gfdtd2d_ctx;

/* Create a 2D context: 1 <= nx <= 32 columns, 1 <= nz <= 2^26 cells along z,
 * dx > 0, S in (0, 1] with S^2 (1 + 1/dx^2) <= 1 (the 2D Yee limit in vacuum),
 * prec F32 or F64 (E_UNSUPPORTED otherwise), on cuda_stream.  Vacuum at rest,
 * fields zero.  Device memory from cudaMalloc. */
gfdtd_status gfdtd2d_create(gfdtd2d_ctx** out, int nx, int64_t nz, double dx, double S, gfdtd_prec prec,
                            void* cuda_stream);

/* Moving layers: velocity beta (|beta| S < 1), slope of the boundaries, n >= 1
 * layers with values eps_r[], mu_r[] > 0 and n - 1 increasing boundaries z[]
 * (moving frame at t = 0, at x = 0).  E_UNSTABLE when a layer has n|beta| > 1
 * (the 1D von Neumann limit of the scheme, Sec. 5) unless allow_unstable. */
gfdtd_status gfdtd2d_set_medium(gfdtd2d_ctx* ctx, double beta, double slope, int n, const double* z,
                                const double* eps_r, const double* mu_r, int allow_unstable);

/* Soft line source at z node k: after the D update of step n,
 * D_y(i, k) += amp sin(omega0 (t - t0)) exp(-((t - t0)/tau)^2) cos(kx i dx),
 * t = (n + 1/2) S (Eq. spectrum_incident with a transverse wavenumber kx:
 * waves at the angles +-asin(kx / (n omega))).  E_ARG past 32 sources. */
gfdtd_status gfdtd2d_add_source(gfdtd2d_ctx* ctx, int64_t k, double kx, double omega0, double tau, double t0,
                                double amp);

/* DFT probe of E_y = D_y / eps at node (i, k): every step adds
 * E_y exp(+i omega t) S to each of its n_bins bins (FP64), t = (n + 1/2) S.
 * E_ARG past 32 probes. */
gfdtd_status gfdtd2d_add_probe(gfdtd2d_ctx* ctx, int i, int64_t k, int n_bins, const double* omega,
                               int* probe_id);

/* Tile shape: cells per lane along z and steps per time block; built: FP32
 * 8x8 and 8x16 (the default), FP64 8x8 (the default); E_UNSUPPORTED
 * otherwise. */
gfdtd_status gfdtd2d_set_tuning(gfdtd2d_ctx* ctx, int cells_per_lane, int time_block);

/* Advance n_steps >= 0 steps (asynchronous on the stream). */
gfdtd_status gfdtd2d_step(gfdtd2d_ctx* ctx, int64_t n_steps);

/* Copy field which (0: D_y, 1: B_x, 2: B_z) to / from host_dst[i * nz + k]
 * as doubles, n == nx * nz (written fields rounded to the storage precision).
 * Both synchronise the stream. */
gfdtd_status gfdtd2d_read_fields(gfdtd2d_ctx* ctx, int which, double* host_dst, int64_t n);
gfdtd_status gfdtd2d_write_fields(gfdtd2d_ctx* ctx, int which, const double* host_src, int64_t n);

/* FP64 DFT accumulators of probe probe_id; synchronises the stream. */
gfdtd_status gfdtd2d_read_spectrum(gfdtd2d_ctx* ctx, int probe_id, double* re, double* im);

gfdtd_status gfdtd2d_synchronize(gfdtd2d_ctx* ctx);
const char* gfdtd2d_last_error(const gfdtd2d_ctx* ctx);
void gfdtd2d_destroy(gfdtd2d_ctx* ctx);

/* Release the context and all its device memory.  NULL is ignored. */
void gfdtd_destroy(gfdtd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GFDTD_H */
