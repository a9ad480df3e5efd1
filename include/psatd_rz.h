/*
 * psatd_rz.h -- C ABI of the GB300 quasi-cylindrical arbitrary-order PSATD PIC cycle.
 *
 * Paper: S. Jalas et al., "Accurate modeling of plasma acceleration with arbitrary
 * order pseudo-spectral particle-in-cell methods", arXiv:1611.05712.
 *   - Cartesian PSATD update: Eq. psatd-eqE / psatd-eqB (section "Finite order
 *     pseudo-spectral solvers").
 *   - Quasi-cylindrical form: fields split into azimuthal modes m on separate (z, r)
 *     grids, Hankel transform along r and Fourier transform along z, operators of the
 *     table that follows Eq. psatd-eqB ("qcyl-ops").
 *   - Arbitrary order: k_z replaced by the modified wavenumber [k_z] of the order-2n
 *     centred stencil (Eq. finite_difference and the [k_z] equation), including inside
 *     k, C and S.
 *
 * Conventions (fixed by this library where the paper is silent):
 *   - SI units.  Grid nodes z_i = i*dz (periodic, i < Nz) and r_j = (j+1/2)*dr (j < Nr).
 *   - F(r,theta,z) = Re[F_0 + 2 sum_{m>=1} F_m e^{-i m theta}];  F_+/- = (F_r -/+ i F_theta)/2.
 *   - Complex grids are interleaved (re, im) pairs, layout [comp][m][r][z] with z fastest.
 *     Real-space vector comps are (r, theta, z); spectral comps are (+, -, z).  Spectral
 *     grids use the index n of the radial wavenumber k_{m,n} in place of r and the FFT
 *     order of k_z in place of z.
 *   - Particles are electrons-like macroparticles of one species (charge q, mass m given
 *     in pic_config), SoA float64 x, y, z [m], ux, uy, uz [m/s, u = gamma v], w
 *     (physical particles per macroparticle) plus an int32 id that follows the sort.
 *
 * Ownership: the caller allocates ONE device workspace of pic_required_bytes() bytes
 * (e.g. a torch uint8 tensor) and passes its pointer and a cudaStream_t; the library
 * carves every grid, table and particle array out of it and never allocates or frees
 * device memory itself (the moving window takes a second caller workspace, see
 * pic_window_setup).  It owns only the opaque host handle (freed by pic_destroy).
 *
 * Errors: every call returns a pic_status; no exception, abort or exit crosses the ABI.
 * pic_last_error() returns a thread-local text for the last failure.  Device-side
 * checks (non-finite or out-of-range particle coordinates, iteration caps) raise a
 * device error word that the synchronising calls report as PIC_ERR_NUMERIC or
 * PIC_ERR_TIMEOUT.
 *
 * Asynchrony: all calls enqueue work on the handle's stream and return, except
 * pic_init (synchronises during set-up: after each sweep of the Hankel matrices' Jacobi SVD
 * and at its end), pic_diagnostics, pic_read_particles,
 * pic_copy_buffer with a host destination, and pic_sync.
 */
#ifndef PSATD_RZ_H
#define PSATD_RZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PIC_OK = 0,
  PIC_ERR_ARG = 1,      /* invalid argument or configuration                       */
  PIC_ERR_CUDA = 2,     /* a CUDA runtime call failed (text in pic_last_error)      */
  PIC_ERR_OOM = 3,      /* workspace smaller than pic_required_bytes()              */
  PIC_ERR_TIMEOUT = 4,  /* a device loop hit its iteration cap                      */
  PIC_ERR_NUMERIC = 5,  /* non-finite or out-of-range values detected on the device */
  PIC_ERR_STATE = 6     /* call out of order (e.g. stepping before particles exist) */
} pic_status;

typedef enum {
  PIC_FP64 = 0,          /* every stage in float64                                           */
  PIC_MIXED_TF32X3 = 1,  /* float32 grids, FP32 particles relative to their cell (momenta as
                            float pairs), DHT as 3-term TF32 tcgen05 products with float32
                            accumulation; FP64 setup and diagnostics                         */
  PIC_MIXED_BF16X6 = 2   /* as PIC_MIXED_TF32X3 but the DHT splits each float into three
                            BF16 pieces and sums the six products of order <= 2 on tcgen05
                            (float32 accumulation); DHT row tiles of at most 128             */
} pic_precision;

typedef struct pic_config {
  int32_t Nz;          /* z nodes (FFT length), 8 <= Nz <= 4096 (FP64) / 8192 (mixed); a length
                          that is not 7-smooth goes through Bluestein rows of the next power of
                          two >= 2 Nz - 1, which caps it at 2048 (FP64) / 4096 (mixed)      */
  int32_t Nr;          /* r nodes, 4 <= Nr <= 1024                                          */
  int32_t Nm;          /* azimuthal modes m = 0..Nm-1, 1 <= Nm <= 4                         */
  int32_t order_p;     /* stencil order p = 2n (even, 2..512); 0 = infinite order           */
  double dz, dr, dt;   /* [m], [m], [s]                                                     */
  int32_t filter;      /* 1: binomial source filter cos^2(k_z dz/2) cos^2(k_perp dr/2)      */
  int32_t precision;   /* pic_precision                                                     */
  int64_t np_capacity; /* maximum number of macroparticles                                  */
  double q, mass;      /* species charge [C] and mass [kg]                                  */
} pic_config;

typedef struct pic_sim pic_sim;   /* opaque */

/* Beam-quality diagnostics of one beam (section "Accurate modeling ...": transverse
 * emittance and slice energy spread over 0.5 um slices within +/- 3 sigma_z). */
typedef struct pic_diag {
  double W;                  /* sum of weights                                           */
  double x_mean, y_mean, z_mean, sigma_z, gamma_mean;
  double emit_nx, emit_ny;   /* normalised rms emittance sqrt(<dx^2><dux^2>-<dx dux>^2)/c */
  double sigma_gamma_mean;   /* mean over non-empty slices of the weighted std of gamma  */
  int32_t n_slices;          /* non-empty slices                                         */
  int32_t n_particles;       /* particles with id in [id_lo, id_hi)                     */
} pic_diag;

/* Buffer identifiers for pic_copy_buffer / pic_load_buffer / pic_buffer_bytes.
 * Element type is float64 (complex = 2 x float64) in PIC_FP64 mode and float32 in
 * mixed mode for grids; tables (KPERP, HANKEL_*, KZ_MOD) are float64 in both modes. */
typedef enum {
  PIC_BUF_E = 0,          /* real-space E  [3 (r,th,z)][Nm][Nr][Nz] complex            */
  PIC_BUF_B = 1,          /* real-space B  [3][Nm][Nr][Nz] complex                      */
  PIC_BUF_EH = 2,         /* spectral E    [3 (+,-,z)][Nm][Nr][Nz] complex              */
  PIC_BUF_BH = 3,         /* spectral B    [3 (+,-,z)][Nm][Nr][Nz] complex              */
  PIC_BUF_DEP = 4,        /* real-space deposit [4 (rho, J_r, J_th, J_z)][Nm][Nr][Nz]  */
  PIC_BUF_SRC_H = 5,      /* spectral sources   [4 (rho, J_+, J_-, J_z)][Nm][Nr][Nz]   */
  PIC_BUF_RHO_PREV_H = 6, /* filtered spectral rho^n [Nm][Nr][Nz] complex              */
  PIC_BUF_RHO_ION = 7,    /* real-space immobile background [Nm][Nr][Nz] complex       */
  PIC_BUF_KPERP = 8,      /* k_{m,n} [Nm][Nr] float64                                   */
  PIC_BUF_HANKEL_INV = 9, /* B_p[j][n] = J_p(k_{m,n} r_j), [Nm][3 (p=m-1,m,m+1)][Nr][Nr]  */
  PIC_BUF_HANKEL_FWD = 10,/* pseudo-inverses M_p[n][j], same shape                      */
  PIC_BUF_KZ_MOD = 11,    /* [k_z]_p per FFT bin [Nz] float64                           */
  PIC_BUF_KEYS = 12,      /* int32 cell keys iz*Nr+ir of the last sort [np] (>=Nz*Nr: w=0) */
  PIC_BUF_PERM = 13,      /* int32 stable sort permutation of the last sort [np]        */
  PIC_BUF_COUNT_ = 14
} pic_buffer_id;

/* Deposit selectors for pic_deposit. */
#define PIC_DEP_RHO 1   /* rho at the current positions, plus the ion background */
#define PIC_DEP_J   2   /* J at the current positions with v = u/gamma           */

/* ---- lifecycle ------------------------------------------------------------------ */

/* Bytes of device workspace a configuration needs.  Errors: PIC_ERR_ARG. */
pic_status pic_required_bytes(const pic_config* cfg, size_t* bytes);

/* Validate cfg, carve the workspace and run the setup stage on the GPU (FP64, once):
 * Bessel zeros alpha_{m,n} (Newton from McMahon's expansion), Hankel matrices
 * B_p = J_p(k_{m,n} r_j), their pseudo-inverses (one-sided Jacobi SVD, singular values
 * <= 1e-3 sigma_max dropped), [k_z]_p (Eq. finite_difference / [k_z]) and the PSATD
 * coefficient tables C, S/K, (1-C)/K^2, ... (Eq. psatd-eqE/eqB with [k_z]).
 * workspace: device pointer, >= pic_required_bytes, 256-byte aligned.  stream: a
 * cudaStream_t (NULL = legacy default stream).  Fields start at zero, no particles.
 * Errors: PIC_ERR_ARG, PIC_ERR_OOM, PIC_ERR_CUDA, PIC_ERR_TIMEOUT (SVD did not converge). */
pic_status pic_init(const pic_config* cfg, void* workspace, size_t workspace_bytes,
                    void* stream, pic_sim** out);

/* Free the host handle (the workspace stays the caller's). */
pic_status pic_destroy(pic_sim* sim);

/* Text of the last error on this thread ("" if none).  Never NULL. */
const char* pic_last_error(void);

/* ---- particles and initial state ----------------------------------------------- */

/* Copy n particles in (replacing all): soa[0..6] = x, y, z, ux, uy, uz, w (float64),
 * id (int32).  on_host != 0: the pointers are host memory (copied synchronously);
 * else device pointers (stream-ordered copy).  z must lie in [0, Nz dz) and
 * x^2 + y^2 < (Nr dr)^2.  Errors: PIC_ERR_ARG (n > capacity or negative). */
pic_status pic_write_particles(pic_sim* sim, const double* const soa[7], const int32_t* id,
                               int64_t n, int32_t on_host);

/* Copy the current particles out in the current (sorted) order, same layout. Synchronises. */
pic_status pic_read_particles(pic_sim* sim, double* const soa[7], int32_t* id, int64_t n,
                              int32_t on_host);

/* Number of particles currently held. */
pic_status pic_num_particles(pic_sim* sim, int64_t* n);

/* Staged particle input (data movement only, no step of the method): the host-to-device
 * copy of the next particle set runs on an internal copy stream while the cycles queued
 * before it compute, for callers that hand the library a new particle set every cycle.
 *
 * pic_stage_bytes: device bytes a staging buffer for n particles needs (7 float64 arrays
 * and the int32 ids, each array padded to a multiple of 32 elements).  Errors: PIC_ERR_ARG.
 *
 * pic_stage_particles: start copying n particles (layout of pic_write_particles; soa and
 * id in host memory, page-locked for the copy to be asynchronous) into `staging`, a device
 * buffer of >= pic_stage_bytes(n) bytes, 256-byte aligned, owned by the caller and left
 * untouched by it until pic_take_particles has returned.  Returns without waiting; the copy
 * starts once the previous pic_take_particles of this handle has read its staging buffer.
 * The host arrays must stay valid and unchanged until pic_take_particles returns.
 * Errors: PIC_ERR_ARG (n < 0 or > capacity, NULL pointers, staging too small or misaligned),
 * PIC_ERR_STATE (a staged set is waiting to be taken), PIC_ERR_CUDA.
 *
 * pic_take_particles: wait on the host for the staged copy, then replace all particles by
 * the staged set, stream-ordered on the handle's stream (the mixed forms convert straight
 * from the staging buffer), exactly as pic_write_particles with the same arrays would.
 * Errors: PIC_ERR_STATE (nothing staged), PIC_ERR_CUDA. */
pic_status pic_stage_bytes(int64_t n, size_t* bytes);
pic_status pic_stage_particles(pic_sim* sim, const double* const soa[7], const int32_t* id, int64_t n,
                               void* staging, size_t staging_bytes);
pic_status pic_take_particles(pic_sim* sim);

/* Immobile neutralising background: rho_ion = -rho(particles with id < n_neutral). */
pic_status pic_init_background(pic_sim* sim, int32_t n_neutral);

/* Add the space-charge fields of the particles with id in [id_lo, id_hi), moving along
 * +z with Lorentz factor gamma, to the spectral E and B: relativistic Poisson solve
 * phi = rho/(eps0 (k_perp^2 + K_z^2/gamma^2)), E = -grad-like, B = curl(0,0,beta phi/c). */
pic_status pic_add_beam_fields(pic_sim* sim, int32_t id_lo, int32_t id_hi, double gamma);

/* Deposit rho^0 (+ background), transform and filter it into rho^n, and inverse-
 * transform the spectral E, B into the real-space grids.  Call once before stepping. */
pic_status pic_init_fields(pic_sim* sim);

/* ---- the PIC cycle ------------------------------------------------------------ */

/* a1: cell keys iz*Nr+ir (iz = floor(z/dz), ir = floor(sqrt(x*x+y*y)/dr), clamped) and a
 * stable counting sort of every particle array by key (ties keep the input order).
 * Inactive particles (w = 0; see the moving window) take keys from Nz*Nr up and end up, in
 * no particular order, after all active ones. */
pic_status pic_sort(pic_sim* sim);

/* a4 at the current positions (no move): what = PIC_DEP_RHO and/or PIC_DEP_J.
 * Linear weights in z and r, ghost node r_{-1} folded into node 0 with sign (-1)^m
 * (scalars, z) or (-1)^{m+1} (r, theta), node Nr dropped, volume 2 pi r_j dr dz,
 * mode weight e^{+i m theta}.  Results in PIC_BUF_DEP (the J part is zeroed/overwritten
 * only when selected). */
pic_status pic_deposit(pic_sim* sim, int32_t what);

/* a2 + a3: gather E^n, B^n at x^n (mode sum, linear weights), relativistic Boris push
 * u^{n-1/2} -> u^{n+1/2}, x^n -> x^{n+1/2} -> x^{n+1} (periodic z, specular reflection at
 * r >= R).  fuse_current != 0 also deposits J^{n+1/2} at x^{n+1/2} into PIC_BUF_DEP. */
pic_status pic_gather_push(pic_sim* sim, int32_t fuse_current);

/* a5..a9: forward z-FFT + DHT of PIC_BUF_DEP, PSATD update with [k_z]_p (filter,
 * global spectral current correction), rho^n <- rho^{n+1}, inverse DHT + z-FFT into
 * PIC_BUF_E / PIC_BUF_B.  order_p >= 0 selects the stencil order (0 = infinite),
 * rebuilding the coefficient tables when it differs from the current one; -1 keeps it. */
pic_status pic_field_step(pic_sim* sim, int32_t order_p);

/* Stage pieces of pic_field_step, for stage-wise checking:
 *   pic_forward_transform: PIC_BUF_DEP -> PIC_BUF_SRC_H (a5, a6)
 *   pic_psatd:             PIC_BUF_SRC_H, EH, BH, RHO_PREV_H -> EH, BH, RHO_PREV_H (a7)
 *   pic_inverse_transform: PIC_BUF_EH, BH -> PIC_BUF_E, B (a8, a9) */
pic_status pic_forward_transform(pic_sim* sim);
pic_status pic_psatd(pic_sim* sim);
pic_status pic_inverse_transform(pic_sim* sim);

/* n full cycles: gather_push(fused J) -> sort -> deposit(rho) -> field_step. */
pic_status pic_step(pic_sim* sim, int32_t n_steps);

/* Stages of one cycle, in order, as timed by pic_step_timed. */
typedef enum {
  PIC_STAGE_GATHER_LAYOUT = 0, /* mixed forms: E, B copied node-major for the gather (FP64: empty) */
  PIC_STAGE_GATHER_PUSH = 1,  /* a2 + a3 + a4 (J at x^{n+1/2}; mixed forms: and rho at x^{n+1}) */
  PIC_STAGE_SORT = 2,         /* a1                                     */
  PIC_STAGE_DEPOSIT = 3,      /* a4 (rho at x^{n+1}, FP64 form)         */
  PIC_STAGE_FFT_FWD = 4,      /* a5                                     */
  PIC_STAGE_DHT_FWD = 5,      /* a6                                     */
  PIC_STAGE_PSATD = 6,        /* a7                                     */
  PIC_STAGE_DHT_INV = 7,      /* a8                                     */
  PIC_STAGE_FFT_INV = 8,      /* a9                                     */
  PIC_NSTAGES = 9
} pic_stage;

/* pic_step with CUDA events recorded on the handle's stream between the stages.
 * stage_ms[PIC_NSTAGES + 1] (host) receives the summed device time of each stage over the
 * n_steps cycles and, in stage_ms[PIC_NSTAGES], the time from the first to the last event.
 * 1 <= n_steps <= 4096.  Synchronises. */
pic_status pic_step_timed(pic_sim* sim, int32_t n_steps, double* stage_ms);

/* ---- batched scan (many independent simulations) ---------------------------------
 * The paper's results come from scans over stencil order, resolution, charge and
 * propagation length (section "Accurate modeling of plasma accelerators in finite order
 * PSATD").  pic_batch_create captures cycles_per_launch full cycles of every simulation
 * into ONE CUDA graph: each simulation runs on its own stream (given at its pic_init; must
 * not be the default stream), forked from and joined back to origin_stream (a created
 * stream), so uneven simulations run concurrently.  cycles_per_launch must be even (the
 * particle double buffers return to their starting parity).  The handles must have been
 * brought to their initial state (pic_init_fields) and must not be stepped through other
 * calls while the batch exists.  pic_batch_launch enqueues n graph launches on
 * origin_stream (asynchronous).  Errors: PIC_ERR_ARG, PIC_ERR_CUDA, PIC_ERR_OOM. */
typedef struct pic_batch pic_batch;
pic_status pic_batch_create(pic_sim* const* sims, int32_t n_sims, int32_t cycles_per_launch,
                            void* origin_stream, pic_batch** out);
pic_status pic_batch_launch(pic_batch* batch, int32_t n_launches);
pic_status pic_batch_info(pic_batch* batch, int32_t* cycles_per_launch, int64_t* kernels_per_launch);
pic_status pic_batch_destroy(pic_batch* batch);

/* ---- domain decomposition along z ---------------------------------------------------
 * A stencil of finite order p reaches only a finite number of cells (section "Finite order
 * pseudo-spectral solvers", unit-pulse figure; "Conclusion": about 60 guard cells at
 * p = 32), so a z subdomain extended by that many guard cells on each side can be advanced
 * with its own Fourier transform and reproduce the global update in its interior.  These
 * two calls let a caller build that scheme from several handles of equal Nr, Nm and
 * precision (one per subdomain, Nz = interior + 2 guards).
 *
 * pic_fields_to_spectral: Eh, Bh <- forward transforms (z-FFT, then the DHT of orders m+1,
 * m-1, m per mode) of the real-space E, B buffers, with F_+- = (F_r -/+ i F_theta)/2.  The
 * counterpart of pic_inverse_transform; it sets the spectral field state from real-space
 * fields loaded with pic_load_buffer or pic_copy_window.  Asynchronous.
 *
 * pic_copy_window: for every (component, mode, r) row of a real-space grid buffer
 * (PIC_BUF_E, PIC_BUF_B, PIC_BUF_DEP or PIC_BUF_RHO_ION),
 *     dst[row][(dst_z0 + t) mod dst.Nz] = src[row][(src_z0 + t) mod src.Nz],  0 <= t < nz,
 * i.e. a periodic window of the source written, periodically, into the destination.
 * 0 <= nz <= both Nz.  The copy runs on the destination's stream: order it after work on
 * the source's stream (same stream, or synchronise first).  Errors: PIC_ERR_ARG
 * (another buffer, unequal Nr / Nm / precision, nz out of range), PIC_ERR_CUDA. */
pic_status pic_fields_to_spectral(pic_sim* sim);
pic_status pic_copy_window(pic_sim* src, int32_t buffer_id, int32_t src_z0, int32_t nz, pic_sim* dst,
                           int32_t dst_z0);

/* ---- moving window ---------------------------------------------------------------
 * The paper follows its beams in the co-moving frame zeta = z - c t over 35 mm of
 * propagation (section "Accurate modeling of plasma accelerators in finite order PSATD",
 * Fig. ez) and does not state how the window is implemented.  This library moves it on
 * a ring of z columns: nothing is copied, the window's back column after k shifts is
 * k mod Nz and its back edge lies at (k mod Nz) dz.  Once set up, every pic_step cycle
 *   1. pushes as usual, except that inactive particles (w = 0) are skipped, and then
 *      removes every active particle whose window coordinate
 *        zeta = ((z^n - back edge) mod L) + (its z displacement in the step) - s dz
 *      is negative (s = 1 if the window moves at the end of this cycle, else 0): its
 *      weight and momentum become 0.  Its current of this step is still deposited;
 *   2. if the window moves: loads the template of the departing column c (the plasma
 *      particles that lay in column c at set-up, in increasing id order) at rest into the
 *      inactive particles, smallest id first, each keeping its id; template particles
 *      beyond the number of inactive particles are dropped and counted;
 *   3. sorts, deposits rho and advances the fields as usual;
 *   4. if the window moves: zeroes column c of the real-space E and B and subtracts the
 *      forward transform (z-FFT, DHT of orders m+1, m-1, m) of that column from the
 *      spectral E and B; rho^n and the ion background are left as they are.
 * The window moves at the end of every period-th cycle after set-up (period = 1 gives a
 * window at c when c dt = dz).  The ion background is fixed per array column and the
 * template reloads each column's initial plasma, so the front stays neutral.  The stage
 * entry points (pic_gather_push, pic_sort, ...) do not move the window, pic_write_particles
 * switches it off, and pic_batch_create refuses handles that have it on.
 * While the window is on, pic_diagnostics measures z from the back edge ((z - back edge)
 * mod L).
 *
 * pic_window_required_bytes: device workspace bytes for a template of n_plasma particles
 * on this handle (n_plasma >= 0).
 * pic_window_setup: take the particles held with id < n_plasma as the template (their
 * positions and weights as they are now), append n_reserve inactive particles (w = u = 0;
 * reserve particle k gets id np + k and sits at the centre of cell (k mod Nz,
 * (k div Nz) mod Nr) on the x axis), and switch the window on.  The ids held must be
 * exactly 0 .. np-1 and np + n_reserve <= np_capacity.  workspace: device pointer of
 * >= pic_window_required_bytes, 256-byte aligned, owned by the caller and kept alive
 * while the handle lives.  Synchronises.  Errors: PIC_ERR_ARG (period < 1, n_plasma or
 * n_reserve out of range, ids not 0 .. np-1, workspace too small or misaligned, window
 * already on), PIC_ERR_CUDA, PIC_ERR_OOM (host scratch).
 * pic_window_state: cycles since set-up, shifts so far, the current back column and the
 * number of template particles dropped for want of inactive slots (any output may be
 * NULL).  Synchronises.  Errors: PIC_ERR_STATE (window not set up). */
typedef struct pic_window_info {
  int64_t cycles;
  int64_t shifts;
  int32_t back_column;
  int32_t period;
  int64_t dropped;
  int64_t n_template;
} pic_window_info;
pic_status pic_window_required_bytes(pic_sim* sim, int64_t n_plasma, size_t* bytes);
pic_status pic_window_setup(pic_sim* sim, int64_t n_plasma, int32_t period, int64_t n_reserve,
                            void* workspace, size_t workspace_bytes);
pic_status pic_window_state(pic_sim* sim, pic_window_info* out);

/* ---- tile tuning -----------------------------------------------------------------
 * The paper gives no kernel tiling; these choices belong to this library.  Two tile sizes
 * of the mixed forms (PIC_MIXED_TF32X3, PIC_MIXED_BF16X6) are tunable:
 *   dht_n_tile: rows of the Hankel matrix per tensor-core tile of the DHT (16..256, a
 *               multiple of 16, capped at 128 in the BF16 form; 0 = the built-in rule: Nr
 *               split into the fewest tiles of <= 256 (TF32) or <= 128 (BF16) rows);
 *   band_chunk: cell-sorted particles per CTA of the deposit kernels (512, 1024 or 2048),
 *               which also sets how many grid rows a CTA's shared-memory band covers.
 * Neither changes the arithmetic of a DHT output (same K order, bit-identical results);
 * band_chunk changes the order of the float additions to the global grid only.
 * pic_autotune times the candidates (n tiles of 256, 128, 64 rows; chunks of 512, 1024,
 * 2048) on the handle's own data: the forward and inverse DHT of the current spectral
 * state and the current deposit of the current particles, each after one warm-up launch,
 * best of 3, and keeps the fastest.  It overwrites only buffers that every cycle rewrites
 * before reading (the transform scratch, the spectral sources and the deposit grid), so it
 * may be called between cycles; call it before pic_batch_create.  Synchronises.  In the
 * FP64 form it leaves the (untuned) defaults.  out (host, may be NULL) receives the
 * choice.  Errors: PIC_ERR_ARG, PIC_ERR_CUDA, PIC_ERR_TIMEOUT. */
typedef struct pic_tuning {
  int32_t dht_n_tile;
  int32_t band_chunk;
  double dht_ms;       /* pic_autotune: forward + inverse DHT time of the choice [ms] */
  double deposit_ms;   /* pic_autotune: J deposit time of the choice [ms]             */
} pic_tuning;
pic_status pic_autotune(pic_sim* sim, pic_tuning* out);
/* Set the tile sizes (dht_n_tile, band_chunk; the time fields are ignored).  Errors:
 * PIC_ERR_ARG (a value outside the ranges above), PIC_ERR_CUDA. */
pic_status pic_set_tuning(pic_sim* sim, const pic_tuning* tuning);
pic_status pic_get_tuning(pic_sim* sim, pic_tuning* out);

/* Transform arithmetic of the FP64 form (no counterpart in the paper; the paper's Hankel and
 * Fourier transforms are the operations, this chooses how their float64 results are
 * computed).  The DHT path:
 *   PIC_DHT_AUTO        sliced tensor-core product when Nr <= 256, else the SIMT GEMM
 *                       (the default);
 *   PIC_DHT_F64_GEMM    FP64 SIMT GEMM on the FP64 units, and the z-FFT rows in IEEE float64
 *                       too (the reference arithmetic for studies of rounding floors);
 *   PIC_DHT_F64_SLICED  every row of the matrix and column of the panel scaled by a power
 *                       of two and cut into seven 7-bit slices (exact BF16 numbers); the
 *                       slice products accumulate exactly in FP32 on the tensor cores and
 *                       are combined in FP64: agrees with the FP64 product to about 2^-49
 *                       of (row max x column max x Nr).  Needs Nr <= 256.
 * With AUTO and SLICED the power-of-two z-FFT rows run in double words (each value a sum
 * of two floats, about 48 bits, on the float32 units; rows stay float64 in memory): the
 * pairs hold about 48 bits relative to a row's largest value while that lies between
 * about 2^-100 and 2^127 (the low parts' absolute resolution is 2^-149); values below
 * 2^-126 enter as zero and values from 2^128 on overflow; SI grids of plasma runs lie
 * well inside.  With them the inverse rows also leave a double-word copy of PIC_BUF_E and
 * PIC_BUF_B in the workspace, kept current by every call that writes those buffers, and
 * pic_gather_push reads that copy and forms the mode sum in double words too (error a few
 * 2^-48 of the sum of the weighted terms' magnitudes); with F64_GEMM, or an Nz that is not
 * a power of two, the gather reads the float64 grids.
 * Errors: PIC_ERR_ARG (unknown path, or SLICED with Nr > 256 or a mixed form). */
typedef enum { PIC_DHT_AUTO = 0, PIC_DHT_F64_GEMM = 1, PIC_DHT_F64_SLICED = 2 } pic_dht_path;
pic_status pic_set_dht_path(pic_sim* sim, int32_t path);
pic_status pic_get_dht_path(pic_sim* sim, int32_t* path);

/* Sort interval (no counterpart in the paper): pic_step runs the cell sort (a1) on every
 * interval-th cycle only (1 = every cycle, the default; 1 <= interval <= 16).  The sort
 * changes no particle's state; it orders the particles so that the deposit bands of the
 * mixed forms and the gathers stay local.  Particles move at most about a cell per cycle,
 * so the order a few cycles old is still nearly sorted.  What changes is the order of the
 * float (FP64 form: double) additions of the deposits across CTAs, i.e. their rounding.
 * The stage entry point pic_sort always sorts.  Errors: PIC_ERR_ARG. */
pic_status pic_set_sort_interval(pic_sim* sim, int32_t interval);
pic_status pic_get_sort_interval(pic_sim* sim, int32_t* interval);

/* a10: FP64 beam diagnostics of the particles with id in [id_lo, id_hi) (section
 * "Accurate modeling of plasma accelerators in finite order PSATD": normalised rms
 * emittance and slice energy spread; the fields of pic_diag).  Slices are 0.5 um long from
 * z_mean - 3 sigma_z, covering particles with 0 <= z - z_mean + 3 sigma_z < 6 sigma_z;
 * per non-empty slice the weighted std of gamma.  With the moving window on, z is measured
 * from the window's back edge.  slice_sigma (host, may be NULL) receives the first
 * min(n_slices, max_slices) per-slice values; sigma_gamma_mean is their mean over all
 * non-empty slices.  No selected particle or zero total weight: only n_particles and W are
 * set.  sigma_z = 0: no slices.  More than 65,536 slices: PIC_ERR_ARG.  The passes keep a
 * compacted float64 copy of the selection in scratch memory that holds no state between
 * calls.  Synchronises the handle's stream. */
pic_status pic_diagnostics(pic_sim* sim, int32_t id_lo, int32_t id_hi, pic_diag* out,
                           double* slice_sigma, int32_t max_slices);

/* ---- buffers ------------------------------------------------------------------- */
pic_status pic_buffer_bytes(pic_sim* sim, int32_t buffer_id, size_t* bytes);
pic_status pic_copy_buffer(pic_sim* sim, int32_t buffer_id, void* dst, size_t bytes,
                           int32_t dst_on_host);
pic_status pic_load_buffer(pic_sim* sim, int32_t buffer_id, const void* src, size_t bytes,
                           int32_t src_on_host);

/* Wait for the stream and report any device error word.  The word is sticky: it stays
 * set (and keeps being reported) until pic_clear_error.  Errors: PIC_ERR_CUDA,
 * PIC_ERR_NUMERIC, PIC_ERR_TIMEOUT. */
pic_status pic_sync(pic_sim* sim);

/* Clear the device error word (asynchronous).  Errors: PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_clear_error(pic_sim* sim);

/* Health check of the failure path (no counterpart in the paper): one CTA waits, with a
 * cap of max_polls polls (1 <= max_polls <= 2^24), on an mbarrier that nothing arrives on,
 * the same bounded wait the tensor-core kernels use, then raises the timeout bit of the
 * device error word and returns.  The next pic_sync reports PIC_ERR_TIMEOUT and the
 * handle stays usable after pic_clear_error.  Asynchronous.  Errors: PIC_ERR_ARG,
 * PIC_ERR_CUDA. */
pic_status pic_selftest_wait_timeout(pic_sim* sim, int32_t max_polls);

/* Number of kernels this handle has launched so far (host-side count, for accounting). */
pic_status pic_launch_count(pic_sim* sim, int64_t* launches);

/* ---- allocation-free variant ----------------------------------------------------
 * The paper has no counterpart to this entry point.  It exists for callers that cannot
 * allocate device memory when they need the sort: applications that give this library a
 * fixed memory budget at start-up and forbid allocation afterwards, or hosts whose own
 * allocator owns the device and keeps cudaMalloc away from the libraries they load.
 * It computes the cell keys iz*Nr+ir and the stable permutation of pic_sort on a
 * PIC_FP64 handle without a moving window (the same float64 key arithmetic), but takes
 * the particle coordinates and the output arrays as plain device pointers and needs no
 * pic_sim workspace.  Differences from pic_sort: non-finite coordinates get key 0
 * silently (pic_sort also raises PIC_ERR_NUMERIC on its handle); the mixed-precision
 * handles compute their keys from cell-relative float32 positions, and a moving window
 * gives inactive particles keys past the cells, neither of which applies here.
 *   x, y, z: device float64 [n]; keys, perm: device int32 [n] (outputs, caller-owned).
 *   Limits: 0 <= n <= 262144 and Nz*Nr <= 65536; larger sizes return PIC_ERR_ARG with a
 *   message.  dz, dr > 0.  stream: cudaStream_t (NULL = legacy default stream).
 * Cost: O(n) plus the ordering of each cell's entries, at most 128^2/32 comparisons per
 * lane for cells of up to 128 entries and an O(c log c) CTA sort for larger ones, so a
 * cell holding all n particles stays a few passes over them.
 * Its scratch (1.84 MB) is a fixed __device__ array inside the library: every GPU that
 * loads the library holds it until the process exits.  The call allocates nothing
 * (no cudaMalloc/cudaFree, no allocating library routine).  All calls share that array
 * and the counts are cleared at the start of each call, so calls whose kernels overlap
 * on the GPU (different streams, or different host threads on one device) race and must
 * be serialised by the caller.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current and keeps it for the
 * life of the process: do not use the call across a reset of the device
 * (cudaDeviceReset) in the same process.  Asynchronous on the stream; after that first
 * call it enqueues kernels only, so it may be captured into a CUDA graph.  Errors:
 * PIC_ERR_ARG, PIC_ERR_CUDA. */
pic_status pic_sort_keys_noalloc(const double* x, const double* y, const double* z, int64_t n,
                                 int32_t Nz, int32_t Nr, double dz, double dr, int32_t* keys,
                                 int32_t* perm, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* PSATD_RZ_H */
