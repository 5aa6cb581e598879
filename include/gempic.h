/*
 * gempic.h -- C-ABI of the GB300 GEM-PIC hot path (Galilean electromagnetic particle-in-cell,
 * Pukhov, Elkina, Wilson, arXiv 2509.16793).
 *
 * One simulation = one persistent spectral field state on the device plus its particle
 * stores.  Each s-step (slow coordinate, step Delta) marches the zeta-slices from the front
 * of the window to the back (Sec. 4.1): fresh plasma is injected at the front (Sec. 5.1,
 * Q_f = q n h_x h_y Delta), particles are gathered, pushed along zeta with the GT2
 * characteristics (Sec. 5, Eqs. after Vlasov2, trap2) and deposited, and the
 * universal reduced Maxwell system (Eqs. RxGu..EzGu) is advanced slice by slice with the
 * semi-implicit scheme of Sec. 4.1 (Eqs. RxN..eqall, closed form of App. B).  Particles that
 * pass the back boundary are removed; particles whose slow-coordinate budget is used up stay
 * in the box as stored (trapped) particles and are pushed along s.
 *
 * Conventions
 *   - Units: the paper's normalisation (Sec. 3): c = 1, lengths in c/omega_0, time in
 *     1/omega_0, fields in m c omega_0/e, densities in n_cr.
 *   - Grid: nx x ny transverse nodes x_i = i hx, y_j = j hy (periodic), nzeta slices
 *     zeta_n = n h, n = 0..nzeta-1, plus a field-free ghost slice zeta_nzeta at the front.
 *     ny == 1 selects the 2-D (x, zeta) slab.  nx, ny powers of two (ny may be 1),
 *     nx in [8, 1024], ny <= 1024.
 *   - Ownership: every device buffer belongs to the library.  Pointers passed in are
 *     borrowed for the duration of the call only.  No call keeps a caller pointer.
 *   - Errors: every call returns a gempic_status; no C++ exception crosses this boundary.
 *     After a CUDA or device-side error the simulation is sticky-failed: later calls return
 *     GEMPIC_ESTATE until gempic_destroy.
 *   - Threading: one simulation per host thread at a time.  Calls on one simulation are
 *     issued on its CUDA stream (gempic_config.cuda_stream, NULL = legacy default stream).
 */
#ifndef GEMPIC_H
#define GEMPIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque handle of one simulation (created by gempic_create, released by gempic_destroy). */
struct gempic_sim;

typedef enum {
  GEMPIC_OK = 0,
  GEMPIC_EINVAL = -1,     /* bad argument or unsupported size                              */
  GEMPIC_ENOMEM = -2,     /* device or host allocation failed                               */
  GEMPIC_ECUDA = -3,      /* a CUDA runtime call failed                                     */
  GEMPIC_EUNSTABLE = -4,  /* Delta h omega_p^2 > 4, outside the stability bound (Sec. 4.2)   */
  GEMPIC_ETIMEOUT = -5,   /* a bounded device-side wait gave up                             */
  GEMPIC_ESTATE = -6,     /* simulation failed earlier, or call not valid in this state     */
  GEMPIC_EOVERFLOW = -7,  /* a fixed-capacity particle store overflowed (particles dropped) */
  GEMPIC_ENONFINITE = -8  /* watchdog: a NaN or infinity reached the FP64 field or kinetic
                             energy sums (needs GEMPIC_FLAG_DIAG), or a particle moved more
                             than 256 cells across one slice                                */
} gempic_status;

/* Transverse grid and slices (Sec. 4.1: large step Delta in s, fine step h in zeta). */
typedef struct {
  int32_t nx, ny, nzeta;
  double hx, hy, h;       /* 2-D: hy is the per-unit-length depth, normally 1 */
} gempic_grid;

/* A background species swept by the window and injected fresh at the front each s-step
 * (Sec. 5.1, Q_f = q n h_x h_y Delta, split over ppc macroparticles per transverse cell,
 * cold, at uniform random in-cell offsets drawn from a counter-based SplitMix64 stream keyed
 * by (seed, s-step, particle)). */
typedef struct {
  double charge, mass;    /* in e and m_e */
  double density;         /* in n_cr */
  int32_t ppc;
  int32_t reserved;
} gempic_species;

/* Laser driver at s = 0: E = e_pol a0 cos(phi) exp(-phi^2/T^2) exp(-r^2/R^2),
 * phi = zeta - zeta_center (Eq. E_laser), laid as a forward wave R = 2E, L = 0 (Eqs. Rx, Ry),
 * centred on the middle transverse node. */
typedef struct {
  double a0, waist, duration, zeta_center;
  int32_t pol;            /* 0 = x, 1 = y */
  int32_t reserved;
  /* > 0: the full width at half maximum of the intensity |E|^2 on the axis; the library takes
   * T = fwhm_intensity / sqrt(2 ln 2) (intensity ~ exp(-2 phi^2/T^2)) and ignores duration.
   * 0: duration is T itself. */
  double fwhm_intensity;
} gempic_laser;

/* Gaussian particle bunch placed in the box at creation (a PWFA-style driver; Sec. 5.1: a
 * particle inside the box carries a charge Q_b and is pushed along s as a beam particle).
 * Its density is n_peak exp(-r^2/(2 sigma_r^2) - (zeta - zeta_center)^2/(2 sigma_z^2)),
 * r measured from the window's middle node (x_c, y_c) = (nx hx/2, ny hy/2) (2-D: |x - x_c|,
 * a sheet uniform in y).  It is sampled on the device with n_macro equal-charge macro-
 * particles, Q = charge n_peak (2 pi)^(3/2) sigma_r^2 sigma_z / n_macro (2-D, per unit depth:
 * charge n_peak 2 pi sigma_r sigma_z / n_macro), cold (u_x = u_y = 0) and moving along +z with
 * gamma_i = gamma (1 + rel_spread g_3), u_z = sqrt(max(gamma_i^2 - 1, 0)).
 * Sampling: macroparticle i draws the uniforms v_j = ((o >> 11) + 1) 2^-53 in (0, 1] from
 * outputs o = 4 i + j (j = 0..3) of the counter-based SplitMix64 stream of `seed`, and the
 * normal pairs (g_0, g_1), (g_2, g_3) by the Box-Muller transform
 * (sqrt(-2 ln v_0) cos(2 pi v_1), sqrt(-2 ln v_0) sin(2 pi v_1)), likewise from (v_2, v_3);
 * x = x_c + sigma_r g_0, y = y_c + sigma_r g_1 (wrapped into the periodic box; 2-D: y = 0),
 * zeta = zeta_center + sigma_z g_2.  Macroparticles outside 0 < zeta <= window length are
 * dropped (their charge is not redistributed).  The bunch uses the species of equal charge
 * and mass if the config has one, else an extra species slot that is never injected fresh
 * (nspecies + 1 must then stay <= 4).  n_peak may have either sign with charge; sigma_r,
 * sigma_z > 0, gamma >= 1, rel_spread >= 0, n_macro >= 0, else gempic_create returns
 * GEMPIC_EINVAL. */
typedef struct {
  double charge, mass;    /* in e and m_e */
  double n_peak;          /* in n_cr */
  double sigma_r, sigma_z, zeta_center;
  double gamma, rel_spread;
  int64_t n_macro;
  uint64_t seed;          /* SplitMix64 stream of the bunch (independent of the fresh plasma's) */
} gempic_beam;

/* Transverse plasma channel (Sec. 6, Eq. n_plasma): the density of every species is
 * n(r) = n [1 + (n1/n0 - 1) exp(-r^2 / R_ch^2)], r the transverse distance from the window's
 * middle node (x_c, y_c) = (nx hx / 2, ny hy / 2); in 2-D r = |x - x_c|.  A fresh
 * macroparticle takes the charge Q_f n(r)/n at its injection position.  n1_over_n0 >= 0 and
 * radius > 0, else gempic_create returns GEMPIC_EINVAL.  Immobile ions carry no current in
 * the slice equations, so the profile enters through the injected charge alone. */
typedef struct {
  double n1_over_n0;      /* density on the axis over the density far from it */
  double radius;          /* R_ch */
} gempic_channel;

/* Flags */
#define GEMPIC_FLAG_DIAG      1u  /* FP64 diagnostics every s-step (default on)           */
#define GEMPIC_FLAG_SNAPSHOT  2u  /* keep real-space E, B, j of the last s-step of a call */
/* Particle law GT1 (Sec. 5, Eq. trap1): the s-budget of a particle is the lab time,
 * ds = |dzeta|/(1 - v_z), a streaming step is at most (Delta - sigma)(1 - v_z), a stored
 * particle advances by the lab time Delta and rejoins when Delta (1 - v_z) >= h.  Default
 * (flag clear): GT2 (Eq. trap2), ds~ = v_z |dzeta|/(1 - v_z), the s-step is the propagation
 * distance Delta.  Under GT1 with Delta shorter than the window every fresh particle stops
 * inside it (the paper's stitches), so the stored buckets need room for a full layer. */
#define GEMPIC_FLAG_GT1       4u
/* Verification mode: the discrete continuity residual of the deposit and the Gauss residual
 * (gempic_diag.continuity_residual, gauss_residual), 2-D and 3-D.  Three more shared-memory
 * planes of the band's rows (taken from the particle headroom), three CIC reductions per push
 * (into the owner CTA of each row) and, in 3-D, two more cluster barriers per slice; runs take
 * the generic kernel.  The fields and particles are those of a run without the flag. */
#define GEMPIC_FLAG_RESIDUAL  8u
/* Keep the current j of the last s-step of each call (gempic_get_current), e.g. to train the
 * denoiser on pairs of runs. */
#define GEMPIC_FLAG_CURRENT   16u

typedef struct {
  gempic_grid grid;
  double delta;                  /* s-step Delta (Sec. 4.1) */
  int32_t precision;             /* 32 or 64: arithmetic of push, deposit and field update */
  uint32_t flags;
  uint64_t seed;
  int32_t nspecies;              /* 1..4 */
  int32_t cluster_ctas;          /* CTAs per slice march (thread-block cluster); 0 = auto */
  const gempic_species* species; /* nspecies entries, copied at create */
  const gempic_laser* laser;     /* NULL: no driver */
  int32_t stored_bucket_capacity;/* stored particles per zeta-cell and s-level; 0 = auto */
  int32_t particle_headroom;     /* extra streaming slots per CTA for rejoining particles; 0 = auto */
  int32_t pipeline_depth;        /* s-steps marched concurrently (wavefront); 0 = auto, 1 = none */
  int32_t reserved;
  void* cuda_stream;             /* cudaStream_t; NULL = legacy default stream */
  const gempic_channel* channel; /* NULL: uniform density; copied at create */
  /* Variable zeta-step (Sec. 6 refines the back of the window): nzeta slab thicknesses, slab
   * n lying between planes n and n+1, plane 0 at the back; every step-dependent part of the
   * scheme (slice equations, particle step, deposit normalisation, energies, stored
   * particles' slabs) takes the thickness of the slab it concerns.  NULL: grid.h everywhere.
   * The profile should vary smoothly (second order needs h_{n+1} - h_n = O(h^2)).  Copied at
   * create; GEMPIC_EINVAL for a non-positive or non-finite entry; the stability bound uses
   * the largest slab.  gempic_step_noalloc does not take a table (GEMPIC_EINVAL). */
  const double* hz;
  /* NULL: no bunch.  Copied at create; sampled into the stored set of level 0 by the first
   * call that initialises the simulation (before the consistency march).  With
   * stored_bucket_capacity = 0 the buckets are sized for the bunch's densest slab. */
  const gempic_beam* beam;
} gempic_config;

/* Per-s-step diagnostics, accumulated on the device in FP64. */
typedef struct {
  int64_t step;                 /* s-steps completed */
  double field_energy;          /* 1/2 sum (E^2 + B^2) hx hy h over the box at the new level */
  double kinetic_energy;        /* streaming: sum N m (gamma-1) dt/Delta per crossing;
                                   stored: sum N m (gamma-1); N = Q/q physical particles     */
  double charge_flux;           /* sum over slice planes of (rho - j_z) hx hy h              */
  int64_t n_trapped;            /* streaming particles whose s-budget ran out this step     */
  int64_t n_stored;             /* stored particles at the new level                         */
  int64_t n_rejoined;           /* stored particles that rejoined the zeta march this step   */
  int64_t pushes;               /* streaming crossings performed this step                   */
  double continuity_residual;   /* with GEMPIC_FLAG_RESIDUAL: max over slabs and nodes of
                                   |(D_start - D_end)/h - div j_perp| (backward differences:
                                   j_x on x-edges, j_y on y-edges), D the CIC density of the
                                   weights at the start and end of every move of the step
                                   (Sec. 5.1: rho - j_z is carried through the planes);
                                   round-off for the charge-conserving deposit.  -1 otherwise */
  double gauss_residual;        /* with GEMPIC_FLAG_RESIDUAL: max over the slice planes and
                                   nodes of |d_x L_x + d_y L_y - (rho - j_z)|: Gauss's law with
                                   d E_z/d zeta from Eq. EzGu, L_x = E_x - B_y, L_y = E_y + B_x,
                                   central differences across; rho - j_z = the CIC density of
                                   the weights of the particles reaching the plane plus the
                                   neutralising background -sum_s q_s n_s f(r) (stored particles,
                                   rho - j_z = Q (1 - v_z) ~ 0, are not counted).  Not a
                                   round-off quantity: the scheme conserves it only while
                                   dR/ds = 0.  -1 otherwise */
  double stored_kinetic_energy; /* the stored set's part of kinetic_energy */
} gempic_diag;

/* Create a simulation: validates the config (GEMPIC_EUNSTABLE if Delta h omega_p^2 > 4),
 * allocates the device state, lays the laser into the spectral state, and runs the Delta = 0
 * consistency march that fills E_z, B_z and L from R at s = 0.  *out receives the handle. */
gempic_status gempic_create(const gempic_config* cfg, struct gempic_sim** out);

/* Place macroparticles inside the box at the current level (beam / driver particles,
 * Sec. 5.1 Q_b): absolute positions, momenta u = p/(m c) and charge Q (host FP64 arrays of
 * length n, species[i] < nspecies).  Valid only before the first gempic_step. */
gempic_status gempic_add_particles(struct gempic_sim* sim, int64_t n, const double* x,
                                   const double* y, const double* zeta, const double* ux,
                                   const double* uy, const double* uz, const double* weight,
                                   const int32_t* species);

/* Advance n s-steps (one persistent device launch), then wait and check the device status. */
gempic_status gempic_step(struct gempic_sim* sim, int32_t n);

/* Same, without waiting: launches on the simulation's stream and returns. */
gempic_status gempic_step_async(struct gempic_sim* sim, int32_t n);

/* Change the s-step Delta for the s-steps launched after this call (Sec. 6 varies Delta along
 * the run; the field update of Sec. 4.1, the fresh weight Q_f = q n h_x h_y Delta/ppc and the
 * s-budget of each particle all take the new value; particles already stored keep their
 * charge).  The stored set is advanced to the next level at the end of each s-step, with
 * that s-step's fields and Delta, so after a change it lags the new Delta by one s-step.
 * Initialises the simulation first if no step has run, so that the level-0 set-up uses the
 * Delta of gempic_create.  GEMPIC_EINVAL for delta < 0 or non-finite,
 * GEMPIC_EUNSTABLE above the stability bound (the simulation keeps its old Delta), GEMPIC_ESTATE
 * after a failure.  Launches already issued are not affected. */
gempic_status gempic_set_delta(struct gempic_sim* sim, double delta);

/* Bounded device waits: when several s-steps march concurrently (pipeline_depth > 1) each
 * march polls the progress word of the march ahead of it; after `polls` polls (about 200 ns
 * apart) without progress it gives up, sets the timeout bit of the device status word and
 * finishes its march on whatever data it has, so the launch always completes and the next
 * gempic_sync returns GEMPIC_ETIMEOUT (then the simulation is failed: GEMPIC_ESTATE).  The
 * default is 2e7 polls (a few seconds).  Takes effect for the launches after this call.
 * GEMPIC_EINVAL for polls < 0; GEMPIC_ESTATE after a failure. */
gempic_status gempic_set_wait_limit(struct gempic_sim* sim, int64_t polls);

/* Wait for the stream and check the device status word of the simulation. */
gempic_status gempic_sync(struct gempic_sim* sim);

/* End-to-end step through host buffers: copy the spectral state in from host memory, advance
 * n s-steps, copy the state back out and return the diagnostics of the last step.  state_in
 * may be NULL (keep the device state); state_out may be NULL.  Both use the layout of
 * gempic_get_state; pinned host memory gives the fastest copies. */
gempic_status gempic_step_host(struct gempic_sim* sim, int32_t n, const void* state_in,
                               void* state_out, size_t state_bytes, gempic_diag* diag_out);

/* End-to-end s-steps with the state streamed through host memory while the marches run.
 * The n s-steps march as the wavefront of gempic_step (pipeline_depth marches in flight);
 * each s-step reads its old level from a device input buffer and writes its new level to a
 * device output buffer (both in the layout of gempic_get_state), and the library moves the
 * levels through host_state slice group by slice group: the slices a march has finished are
 * copied out to host_state, copied back in as the next s-step's input, and released to that
 * march.  So every s-step's input comes in from host memory and its result goes out to host
 * memory (gempic_state_bytes each way), and the copies overlap the marches.
 *   host_state   the input of the first s-step on entry, the result of the last on return;
 *                layout of gempic_get_state, bytes >= gempic_state_bytes.  Page-locked
 *                memory (cudaHostAlloc, cudaHostRegister) lets the copies run asynchronously;
 *                pageable memory works but serialises them.
 *   diag_out     NULL or n records: the diagnostics of each s-step, in order.
 * The calling thread drives the copies and returns when all s-steps are done; the device
 * state is then the last result (gempic_get_state returns it).  The marches wait for their
 * input slices with the bounded waits of gempic_set_wait_limit (GEMPIC_ETIMEOUT if one gives
 * up; the calling thread also gives up after 120 s without progress).  The library keeps two
 * device state buffers and a few words of mapped host memory for it, allocated at the first
 * call.  GEMPIC_ESTATE with a denoiser set or after a failure; GEMPIC_EINVAL for n < 0, a NULL
 * host_state or too few bytes. */
gempic_status gempic_step_streamed(struct gempic_sim* sim, int32_t n, void* host_state,
                                   size_t bytes, gempic_diag* diag_out);

/* Size in bytes of the spectral state of gempic_get_state. */
size_t gempic_state_bytes(const struct gempic_sim* sim);

/* Copy the spectral field state (Sec. 4.1: what the scheme needs at s^0): complex values in
 * the simulation's precision, layout [6][nzeta][ny][nx/2] for R_x, R_y, E_z, B_z on the
 * slices and j_x, j_y on the half-slices (index n <-> zeta_{n+1/2}); kx = 2 pi m/(nx hx),
 * m = 0..nx/2-1; ky in FFT order.  dst_is_device selects a device or host destination. */
gempic_status gempic_get_state(struct gempic_sim* sim, void* dst, size_t bytes,
                               int32_t dst_is_device);

/* Replace the spectral state (same layout as gempic_get_state). */
gempic_status gempic_set_state(struct gempic_sim* sim, const void* src, size_t bytes,
                               int32_t src_is_device);

/* Real-space fields of the last s-step of the last call (needs GEMPIC_FLAG_SNAPSHOT):
 * comp 0..5 = E_x, E_y, E_z, B_x, B_y, B_z on the slices, 6..8 = j_x, j_y, j_z on the
 * half-slices (j_x at x + hx/2; in 3-D j_y at y + hy/2); layout [nzeta][ny][nx] in the
 * simulation's precision. */
gempic_status gempic_get_fields(struct gempic_sim* sim, int32_t comp, void* dst, size_t bytes,
                                int32_t dst_is_device);

/* Stored (trapped / beam) particles.  kind 0: particles at the next level, already pushed
 * along s with the fields of the current level; kind 1: particles queued to rejoin the next
 * zeta march.  On entry *n_inout is the capacity of the host FP64 arrays; on return the
 * number of particles (if larger than the capacity nothing is copied and GEMPIC_EINVAL is
 * returned).  Any array pointer may be NULL. */
gempic_status gempic_get_particles(struct gempic_sim* sim, int32_t kind, int64_t* n_inout,
                                   double* x, double* y, double* zeta, double* ux, double* uy,
                                   double* uz, double* weight, int32_t* species);

/* Diagnostics of the last completed s-step. */
gempic_status gempic_get_diagnostics(struct gempic_sim* sim, gempic_diag* out);

/* On-axis E_z(zeta_n), n = 0..nzeta-1, of the last completed s-step (FP64 host array). */
gempic_status gempic_get_onaxis_ez(struct gempic_sim* sim, double* dst, int32_t n);

/* Device kernels this library launched since create (for launch accounting). */
int64_t gempic_launch_count(const struct gempic_sim* sim);

/* Launch shape chosen at create: CTAs per cluster, threads per CTA, dynamic shared bytes,
 * s-steps marched concurrently. */
gempic_status gempic_launch_shape(const struct gempic_sim* sim, int32_t* cluster_ctas,
                                  int32_t* threads, int32_t* smem_bytes, int32_t* pipeline);

/* ---- Batched parameter scan ------------------------------------------------------------
 * Independent simulations stepped together (the paper has no counterpart: a scan over grids,
 * drivers and densities).  A step call of n s-steps is one persistent launch (one CTA per SM,
 * recorded once per n as a CUDA graph with the upload of the launch parameters and replayed)
 * whose CTAs take work items (simulation, s-step) from a queue: s-step by s-step, the costliest
 * simulations first.  The march of a simulation's s-step waits slice by slice (bounded) for
 * its previous s-step, so a large simulation marches up to 16 s-steps at once while small ones
 * fill the other SMs.  The costs come from an autotuner run at creation: for each size class
 * (grid, precision, particles per cell, flags) it times one s-step of a throw-away simulation
 * at 256 and at 512 threads per CTA, launches the batch at the CTA size with the smaller
 * total and orders the items by the measured per-class times (gempic_batch_tuning).  All
 * simulations share the batch's stream and must have the same precision; beams, channels and
 * the other config fields work as in gempic_create, denoisers do not. */
typedef struct gempic_batch gempic_batch;

/* Create n >= 1 instances from cfgs[0..n-1], each validated like gempic_create (GEMPIC_EINVAL
 * also for mixed precisions); cuda_stream and pipeline_depth of the configs are ignored.
 * Runs the autotuner (a few s-steps of one throw-away simulation per size class).  On a
 * failure nothing is kept and the first failing status is returned. */
gempic_status gempic_batch_create(const gempic_config* cfgs, int32_t n, gempic_batch** out);

/* Launch n s-steps of every instance (one persistent launch per 16 s-steps) and return. */
gempic_status gempic_batch_step_async(gempic_batch* b, int32_t n);

/* Wait for the batch and check every instance's device status word; the first error is
 * returned. */
gempic_status gempic_batch_sync(gempic_batch* b);

/* gempic_batch_step_async then gempic_batch_sync. */
gempic_status gempic_batch_step(gempic_batch* b, int32_t n);

/* Number of instances (0 for NULL). */
int32_t gempic_batch_size(const gempic_batch* b);

/* Instance i, owned by the batch: use it with the gempic_get_* and gempic_add_particles
 * calls, never with gempic_destroy.  NULL if i is out of range. */
struct gempic_sim* gempic_batch_sim(gempic_batch* b, int32_t i);

/* The cudaStream_t the batch launches on (the same for every i; for events and
 * interoperation); NULL if i is out of range. */
void* gempic_batch_stream(gempic_batch* b, int32_t i);

/* The autotuner's choice: the launch's threads per CTA and the measured ms per s-step of
 * instance i's size class at that size. */
gempic_status gempic_batch_tuning(const gempic_batch* b, int32_t i, int32_t* nthreads,
                                  double* ms_per_step);

/* Destroy every instance and the batch (waits for it first). */
void gempic_batch_destroy(gempic_batch* b);

/* Allocation-free s-step.  The paper has no counterpart: this entry point is for callers that
 * cannot allocate device memory -- for example code whose host application owns every device
 * allocation under a fixed budget, or a plug-in that is not allowed to call cudaMalloc.
 * It advances the caller's spectral state by the s-step numbered `step` (0 for the first
 * s-step; it selects the fresh-particle offsets) and calls no cudaMalloc, cudaFree or other
 * allocating routine.
 *   state        device memory owned by the caller, layout of gempic_get_state, updated in
 *                place; state_bytes must cover it.  There is no laser set-up here: pass a
 *                state prepared elsewhere (e.g. copied out with gempic_get_state).
 *   cfg          used: grid, delta, precision, seed, nspecies, species, channel,
 *                cluster_ctas, cuda_stream and, of the flags, GEMPIC_FLAG_GT1.  Ignored:
 *                laser, stored_bucket_capacity, particle_headroom, pipeline_depth and
 *                GEMPIC_FLAG_DIAG (the diagnostics are always computed).  Rejected with
 *                GEMPIC_EINVAL: a zeta-step table (hz), a bunch (beam), GEMPIC_FLAG_SNAPSHOT
 *                and GEMPIC_FLAG_RESIDUAL (this call has no buffers for them).
 *   diag_out     host, may be NULL: diagnostics of the step (continuity_residual = -1).
 *   onaxis_out   host, may be NULL: nzeta doubles of on-axis E_z.
 * Working memory: one array of 248 320 bytes in device memory, declared at file scope in the
 * library; every GPU that loads the library holds it until the process exits.  Limits:
 * nzeta <= 4096; nx <= 1024; at most 16 CTAs per cluster with (nx/2) ny / C <= 512 spectral
 * modes per CTA and, in 3-D, at least two rows (ny / C >= 2) per CTA; one band's fresh
 * particles, fields and spectra must fit the shared memory of one CTA.  Larger sizes return
 * GEMPIC_EINVAL before any work.  The first call on a device looks up the array's device
 * address (set-up); make that first call before any stream capture.  All calls share the
 * array and it keeps the last call's contents (each call clears what must start at zero):
 * calls that overlap on the GPU, from several streams or threads, race -- serialise them.
 * GEMPIC_EOVERFLOW has two causes, and in both the state is still advanced: a particle
 * trapped during the step (there is no stored-particle store: the trapped particle is
 * dropped), or a band whose streaming slots overflow when particles move in from other bands
 * (the extra particles are dropped).  GEMPIC_ENONFINITE: the watchdog of the FP64 sums.  The
 * call waits for its stream. */
gempic_status gempic_step_noalloc(const gempic_config* cfg, int64_t step, void* state,
                                  size_t state_bytes, gempic_diag* diag_out, double* onaxis_out);

/* ---- Learned current denoiser -----------------------------------------------------------
 * The paper has no counterpart.  With few particles per cell the deposited current is noisy;
 * a small 3-D convolutional net trained on pairs of runs of this method (few versus many
 * particles per cell) maps the current of a sparse run towards that of a dense one, so that
 * the sparse run can stand in for the dense one.  Net: x0 = j/scale, h1 = relu(conv1(x0)),
 * h2 = relu(conv2(h1)), r = conv3(h2), denoised j = j + scale r; every conv is 3x3x3 (taps
 * dz, dy, dx in {-1, 0, 1}, periodic across, zero outside the window along zeta) with 16
 * hidden channels; activations and weights in BF16, accumulation in FP32 on the tensor cores.
 * Currents are device FP32 arrays [nz][3][ny][nx] (j_x on x-edges, j_y on y-edges in 3-D, j_z
 * on nodes, every plane a half-slice), the layout of gempic_get_current.
 * Parameters: one FP32 vector of gempic_denoiser_param_count() entries, W1 [27][3][16], b1 [16],
 * W2 [27][16][16], b2 [16], W3 [27][16][3], b3 [3] (tap index (dz+1) 9 + (dy+1) 3 + (dx+1),
 * then input channel, then output channel).  All calls use the current device; they wait
 * for their stream.  GEMPIC_ETIMEOUT if a bounded tensor-core wait gave up. */
typedef struct gempic_denoiser gempic_denoiser;

size_t gempic_denoiser_param_count(void);

/* params: host FP32 vector, or NULL for all zeros (the identity on j); scale > 0 normalises
 * the current (e.g. |q n0|). */
gempic_status gempic_denoiser_create(const float* params, double scale, gempic_denoiser** out);

/* Replace or read the parameters (host vectors of n = gempic_denoiser_param_count() floats);
 * setting them also resets the optimiser. */
gempic_status gempic_denoiser_set_params(gempic_denoiser* d, const float* params, size_t n);
gempic_status gempic_denoiser_get_params(gempic_denoiser* d, float* params, size_t n);

/* j_out = denoised j_in (device arrays, may not alias). */
gempic_status gempic_denoiser_apply(gempic_denoiser* d, const float* j_in, float* j_out,
                                    int32_t nx, int32_t ny, int32_t nz, void* cuda_stream);

/* Loss mean((j_in/scale + r - j_target/scale)^2) over the planes z_margin .. nz-1-z_margin
 * and its gradient with respect to the parameters (host vector grad_host, may be NULL). */
gempic_status gempic_denoiser_grad(gempic_denoiser* d, const float* j_in, const float* j_target,
                                   int32_t nx, int32_t ny, int32_t nz, int32_t z_margin,
                                   double* loss, float* grad_host, void* cuda_stream);

/* gempic_denoiser_grad followed by one Adam step (Kingma and Ba 2015: beta1 = 0.9,
 * beta2 = 0.999, eps = 1e-8, bias-corrected) with learning rate lr; loss is the pre-step loss. */
gempic_status gempic_denoiser_train_step(gempic_denoiser* d, const float* j_in,
                                         const float* j_target, int32_t nx, int32_t ny,
                                         int32_t nz, int32_t z_margin, double lr, double* loss,
                                         void* cuda_stream);

void gempic_denoiser_destroy(gempic_denoiser* d);

/* Denoised s-steps (FP32 simulations): with d set, every s-step of gempic_step runs in two
 * passes.  The first marches the particles with the plain deposit and keeps its current (the
 * plain deposit stays the fallback and the reference); the denoiser maps that current; the second
 * recomputes the new level from the old one with the denoised current (the denoiser acts on j
 * before the field update) and pushes the stored set with those fields.  The pushes of the
 * s-step saw the first pass's fields: the net needs the current of half-slices on both sides
 * of each one, which the march produces only one at a time.  The n s-steps of a call run as
 * one chain of 2n marches in one launch, each following the one before it slice by slice; up
 * to min(7, pipeline_depth) in flight, or, with pipeline_depth 0, as many as leave a third of
 * the SMs to the net.  The calling thread runs the net on groups of half-slices as soon as the
 * first pass has written them and the three half-slices beyond, on a stream of its own, and
 * releases each group to the second pass, which waits for it (bounded).  The call waits for
 * its stream.  The diagnostics combine both passes: the field energy, on-axis E_z and stored
 * set are the second pass's, the streaming particles' energy, flux and counts the first's.
 * d = NULL returns to plain steps.  The denoiser is borrowed: it must outlive its use.
 * GEMPIC_EINVAL for an FP64 simulation. */
gempic_status gempic_set_denoiser(struct gempic_sim* sim, gempic_denoiser* d);

/* The plain current of the last s-step (needs GEMPIC_FLAG_CURRENT or a denoiser): [nzeta][3]
 * [ny][nx] in the simulation's precision, j_x at x + hx/2, j_y at y + hy/2 (3-D), plane n the
 * half-slice n + 1/2, beam current included.  GEMPIC_ESTATE before the first s-step. */
gempic_status gempic_get_current(struct gempic_sim* sim, void* dst, size_t bytes,
                                 int32_t dst_is_device);

/* FP32 FMA throughput probe (measurement only; the paper has no counterpart): the measured
 * denominator of the ALU roofline that the FP32 particle push is reported against.  Launches a
 * short warm-up and then one timed kernel of 4 CTAs x 512 threads per SM, each thread running
 * 16 independent FMA chains for `iters` iterations (2 FLOP per FMA), on cuda_stream (NULL =
 * legacy default stream), timed with CUDA events.  *tflops receives the achieved TFLOP/s,
 * *ms (may be NULL) the kernel's time.  Allocates no device memory.  GEMPIC_EINVAL for
 * iters < 1 or tflops NULL, GEMPIC_ECUDA if a CUDA call fails.  Waits for its stream. */
gempic_status gempic_probe_fp32_fma(void* cuda_stream, int32_t iters, double* tflops, double* ms);

const char* gempic_strerror(gempic_status s);

void gempic_destroy(struct gempic_sim* sim);

#ifdef __cplusplus
}
#endif

#endif /* GEMPIC_H */
