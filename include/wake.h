/*
 * wake.h -- C ABI of the GB300 gridless quasistatic wake solver (libwake.so).
 *
 * The solver advances the plasma-electron ring macroparticles of an
 * axisymmetric plasma column through the co-moving window, one slice of
 * thickness dxi at a time, as in Sec. II-III of arXiv 2603.16623 (gridless
 * quasistatic model): per slice it sorts the rings by radius, forms the radial
 * prefix sums of their charge and current, evaluates psi, d_rho psi,
 * d_zeta psi, the beam field B_theta^(b) and the plasma field B_theta^(p)
 * (Eq. ai_bi / App. A), the fields on the beam macroparticles of the slice,
 * and advances ring radii and momenta with second-order Adams-Bashforth.
 *
 * Units: the paper's normalised plasma units (lengths k_p^-1, densities n0,
 * fields m_e c omega_p / e).  xi = -zeta, xi = 0 is the head of the window;
 * slice s covers xi in [(s-1/2) dxi, (s+1/2) dxi).  Plasma electrons
 * (q = -1, m = 1) move over an immobile uniform ion column of density
 * `density` filling rho <= r_edges[n_rings].
 *
 * Conventions for every entry point:
 *   - Return value: a wake_status; nothing throws across the ABI.  On error
 *     wake_last_error() returns a thread-local message.
 *   - Ownership: the caller owns every array it passes.  wake_init copies its
 *     inputs to the device; afterwards the handle owns all device state until
 *     wake_destroy.  Output arrays are written, never kept.
 *   - Streams: work is enqueued on the CUDA stream given to wake_init
 *     (cudaStream_t passed as void*, NULL = legacy default stream).  Calls that
 *     return data to host memory synchronise that stream.
 *   - Precision: WAKE_FP64 computes everything in double and returns double
 *     arrays; WAKE_MIXED computes pushes and field evaluation in float with
 *     compensated (float-float) prefix sums and returns float arrays.
 *     "real" below means double for WAKE_FP64 and float for WAKE_MIXED.
 */
#ifndef GBWAKE_WAKE_H
#define GBWAKE_WAKE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int wake_status;
enum {
    WAKE_OK = 0,
    WAKE_EINVAL = 1,      /* bad argument or unsupported size                 */
    WAKE_ENOMEM = 2,      /* device allocation failed                         */
    WAKE_ECUDA = 3,       /* a CUDA call failed                               */
    WAKE_ENONFINITE = 4,  /* a slice produced psibar <= 0 or a non-finite field;
                             the wake stopped there (see wake_get_progress)   */
    WAKE_ETIMEOUT = 5,    /* a bounded device-side wait gave up: the wake
                             stopped at that slice (wake_get_progress)      */
    WAKE_EBUSY = 6        /* admission refused (memory budget / capacity)     */
};

enum { WAKE_FP64 = 0, WAKE_MIXED = 1 };

/* ring integrators (wake_config.integrator) */
enum {
    WAKE_AB2 = 0,  /* second-order Adams-Bashforth, forward Euler start (Sec. III) */
    WAKE_RK4 = 1   /* classical fourth-order Runge-Kutta, the alternative Sec. II
                      names: four field evaluations per slice, the beam source at
                      the half step the mean of the two slices; a stage state
                      below the axis is evaluated mirrored.  Electron-only wakes
                      (no mobile ions) of at most 16384 rings, on the global-
                      memory march: one block per wake, or a thread-block
                      cluster of cluster_ctas (1..8) blocks that split the
                      sorted rings (block 0 sorts the state and the stage
                      states); 0 = automatic, the fewest blocks (at most 8)
                      that hold at most 2 rings per thread.  rings_per_thread
                      must be 0. */
};

/* flags of wake_config */
enum {
    WAKE_DUMP_RING_R = 1,      /* keep ring radii at the start of every slice  */
    WAKE_DUMP_RING_FIELDS = 2, /* keep psi, d_rho psi, d_zeta psi, B^(p), B^(b)
                                  and u_r at every ring and slice (tests)      */
    WAKE_INIT_ASYNC = 4,       /* wake_init returns without waiting for the
                                  device: a slice denser than
                                  wake_max_slice_particles() is reported by
                                  wake_get_progress as status WAKE_EINVAL     */
    WAKE_TEST_STALL_STAGE = 8, /* test only (mixed, on-chip march): of each
                                  march launch, the bulk copies that stage the
                                  first beam slice after the launch's first
                                  slice are never issued, so the march's
                                  bounded wait for them runs out (~0.25 s) and
                                  the wake stops with status WAKE_ETIMEOUT
                                  before that slice: exercises the timeout
                                  path without any fault or hang             */
    WAKE_NO_STAGE = 16         /* mixed, on-chip march: read each slice's beam
                                  arrays from global memory instead of
                                  staging them in shared memory with bulk
                                  copies (the same results, bitwise; for
                                  comparison)                               */
};

/* Plasma column (Sec. II, ring macroparticles): ring j fills the cell
   [r_edges[j], r_edges[j+1]); it starts at the cell centre with u_r = 0 and
   weight density * centre * width (Eq. macroparticle_weight).

   Mobile ions (Sec. II, multiple plasma species): with ion_charge Z > 0 the
   ions are a second ring species of charge Z and mass ion_mass M (electron
   masses) on the same cells, of density density / Z (neutral), instead of
   the immobile column.  Each species' psi, d_rho psi and d_zeta psi are
   solved on its own rings and reach the other species' rings by linear
   interpolation between its ring values; B_theta^(p) comes from the
   electrons only; ions move with q/m = Z/M.  A wake then has 2 n_rings
   rings: ids 0..n_rings-1 electrons, n_rings..2 n_rings-1 ions, in every
   per-ring array of this interface (ring state, dumps).  n_rings <= 4096;
   rings_per_thread must be 0, and cluster_ctas (0..8) sets the thread
   blocks of the march: one block per wake, or a thread-block cluster whose
   blocks split each species' sorted rings in rank order (scans folded over
   the cluster, cluster barriers between the phases).  0 = automatic: the
   fewest blocks (at most 8) that hold at most 2 rings of each species per
   thread (one block up to 1024 cells at 512 threads).
   ion_mass = +inf gives ion rings that never move.

   Radial density profile (Sec. II, arbitrary profiles): cell_density (host,
   n_rings values > 0, uniform within each cell; NULL = `density`
   everywhere) sets both species' ring weights; it needs ion rings
   (ion_charge > 0), which carry the profile of the background. */
typedef struct {
    int32_t n_rings;          /* 1 <= n_rings <= wake_max_rings() (4096 with
                                 mobile ions)                                   */
    const double *r_edges;    /* host, n_rings+1 values, r_edges[0] = 0,
                                 strictly increasing                            */
    double density;           /* uniform electron density (= ion column
                                 charge density), > 0                           */
    double ion_charge;        /* 0: immobile ion column; > 0: mobile ions, Z   */
    double ion_mass;          /* mobile ions: M in electron masses, > 0 or +inf */
    const double *cell_density; /* NULL, or n_rings cell densities (ion rings) */
} wake_plasma_desc;

/* A beam species (ultra-relativistic, frozen during a wake solve, Sec. II).
   Each macroparticle is a charged ring of `w` real particles in the slice
   nearest to its xi; its B_theta^(b) is that of the enclosed charge. */
typedef struct {
    int64_t n;                /* macroparticles (>= 0)                          */
    const double *xi;         /* host [n]                                       */
    const double *r;          /* host [n], >= 0                                 */
    const double *w;          /* host [n], weights (real particles, n0 k_p^-3)  */
    double q;                 /* charge sign of the species, e.g. -1            */
} wake_beam_desc;

typedef struct {
    double dxi;               /* slice thickness, > 0                            */
    int32_t n_steps;          /* slices in the window, 1..12288                  */
    int32_t precision;        /* WAKE_FP64 or WAKE_MIXED                         */
    int32_t flags;            /* WAKE_DUMP_* bits                                */
    int32_t block_threads;    /* FP64, mobile ions, RK4: threads per wake
                                 (multiple of 32, 64..512); 0 = library
                                 default (256; 512 with mobile ions or RK4)    */
    int32_t rings_per_thread; /* MIXED: 2, 4 or 8 rings per thread; 0 = auto  */
    int32_t cluster_ctas;     /* MIXED: CTAs per wake, 1..16 (> 1: a thread-
                                 block cluster); 0 = automatic.  The threads
                                 per CTA follow: ceil(n / (rings_per_thread x
                                 cluster_ctas)) rounded up to a multiple of 32,
                                 at most 512, and no CTA may be left empty.
                                 Both must be 0 for WAKE_FP64.  Automatic
                                 (both 0): see wake_launch_shape.  With
                                 mobile ions, RK4 or beam grids (FP64 or
                                 MIXED) cluster_ctas is 0..8 and
                                 rings_per_thread 0 (see above and grid_nr). */
    int32_t integrator;       /* WAKE_AB2 (0) or WAKE_RK4                        */
    int32_t grid_nr;          /* 0: gridless beam coupling (fields at each beam
                                 particle); 1..1024: adaptive beam grids
                                 (Sec. IV): per beam species grid_nr radial
                                 cells out to (1 + 1/grid_nr) x its largest
                                 radius, one node line per slice; B^(b) at
                                 the rings from the grids (B_N r_N / rho
                                 beyond), beam-particle fields interpolated
                                 from the nodes.  WAKE_AB2, no mobile ions,
                                 at most 8 beam species, at most 16384
                                 rings; both precisions.  One block per wake
                                 or a thread-block cluster (cluster_ctas
                                 0..8; 0 = automatic: the fewest blocks, at
                                 most 8, that hold at most 4 rings per
                                 thread); block 0 sorts the rings and sums
                                 the node charges. */
    double grid_rmax;         /* with grid_nr > 0: 0 = adaptive extents; > 0 =
                                 every grid spans [0, grid_rmax] (the regular
                                 intermediate grid).  Every beam particle must
                                 lie below it: EINVAL at wake_init and
                                 wake_reset with new beams; a push that moves
                                 one beyond makes the next preparation stop
                                 the wake with status EINVAL. */
} wake_config;

typedef struct wake_handle wake_handle;

/* Copies the plasma and the beams to the device, initialises the rings
   (Sec. II: cell centres, weights, self weights) and bins and radially sorts
   the beam macroparticles by slice (once per solve: the beam is frozen).
   Beams are concatenated in order; "beam particle k" below indexes that
   concatenation.  Errors: EINVAL (bad sizes, edges, dxi, a slice holding
   more than wake_max_slice_particles() particles), ENOMEM, ECUDA.
   On success *out receives a handle at slice 0. */
wake_status wake_init(const wake_config *cfg, const wake_plasma_desc *plasma,
                      const wake_beam_desc *beams, int32_t n_beams,
                      void *cuda_stream, wake_handle **out);

/* Puts the wake back at slice 0 without reallocating: if beams is not NULL,
   first uploads a new set of beam macroparticles from host arrays (same
   number of species and the same particle counts as at wake_init; the
   charge signs may change), then re-initialises the rings and re-bins and
   re-sorts the beam on the device (the same a0/a1 preparation as wake_init).
   Asynchronous on the handle's stream; the host arrays must stay valid until
   the stream reaches this point (use pinned memory for overlap).  A slice
   holding more than wake_max_slice_particles() particles is reported later
   by wake_get_progress as status WAKE_EINVAL (the march does not run).
   Errors: EINVAL (different species count or sizes), ECUDA. */
wake_status wake_reset(wake_handle *h, const wake_beam_desc *beams, int32_t n_beams);

/* wake_reset of n wakes at once (a0/a1 of Sec. II for each), the wakes'
   preparations running concurrently on the library's auxiliary streams,
   ordered after the work already queued on the handles' (common) stream and
   joined back into it.  beams[i] (may be NULL, or beams itself NULL) gives
   wake i new beam arrays with n_beams[i] species, under wake_reset's rules;
   they are counted into slices on the device only (the per-slice sort sizes
   itself there), so the call does not wait for the device.
   Errors: EINVAL (NULL handle, different streams, bad beams), ECUDA. */
wake_status wake_batch_reset(int32_t n, wake_handle *const *handles, const wake_beam_desc *const *beams,
                             const int32_t *n_beams);

/* Advances the wake by up to n_slices slices (fewer at the end of the
   window); for each slice: sort, B^(b) at the rings, psi and its derivatives
   (Eqs. dpsi_dr, psi, dpsi_dzeta), u_z and gamma, B^(p) (Eq. ai_bi), fields
   at that slice's beam particles, then the AB2 push to the next slice.
   Asynchronous on the handle's stream; resumable.  A slice that fails the
   guard (psibar <= 0 or a non-finite field) stops the wake: its beam fields
   are written, no push is done, and wake_get_progress reports
   WAKE_ENONFINITE.  The on-chip march stages each slice's beam arrays in
   shared memory with bulk asynchronous copies issued during the previous
   slice; if its bounded wait for them gives up, the wake stops before that
   slice and wake_get_progress reports WAKE_ETIMEOUT.  Errors: EINVAL, ECUDA. */
wake_status wake_step_slices(wake_handle *h, int32_t n_slices);

/* Fields at the current slice (the one the next wake_step_slices would
   solve) at n arbitrary radii r (Eqs. b_theta_plasma..dpsi_dzeta sampled off
   the rings): ez = E_z = -d_zeta psi, wr = E_r - B_theta = -d_rho psi,
   bt = B_theta^(p) + B_theta^(b), psi.  The ring state is not advanced.
   The fields are the gridless sums at r also for wakes with beam grids
   (the plasma answering the grids' B^(b), the beam's own B^(b) at r from
   its particles); with mobile ions, the sums of both species.
   r and the outputs are host arrays (device_ptrs = 0) or device arrays
   (device_ptrs = 1); outputs are "real"; any output may be NULL.
   Errors: EINVAL (n < 0, or the window is finished: no slice is left to
   sample), ENONFINITE (the wake stopped), ECUDA. */
wake_status wake_fields_at(wake_handle *h, int64_t n, const double *r, void *ez, void *wr,
                           void *bt, void *psi, int32_t device_ptrs);

/* Fields on every beam particle at its own slice (filled as slices are
   solved; 0 for particles outside the window or not yet reached), in the
   caller's beam order: E_z, W_r = E_r - B_theta, B_theta, psi ("real",
   NULL = skip).  Host (device_ptrs = 0) or device (1) arrays.
   Errors: EINVAL, ECUDA. */
wake_status wake_get_beam_fields(wake_handle *h, void *ez, void *wr, void *bt, void *psi,
                                 int32_t device_ptrs);

/* wake_get_beam_fields of n wakes sharing one stream: E_z and W_r only
   (ez[i], wr[i] may be NULL; ez or wr itself may be NULL), all copies
   queued, then one synchronisation for host arrays.  Errors: EINVAL,
   ENOMEM, ECUDA. */
wake_status wake_batch_get_beam_fields(int32_t n, wake_handle *const *handles, void *const *ez, void *const *wr,
                                       int32_t device_ptrs);

/* Runs the rest of the window and returns E_z and W_r per beam particle in
   caller order (host arrays of "real", NULL = skip) and, if the handle was
   created with WAKE_DUMP_RING_R and ring_r is not NULL, the ring radii at
   the start of every slice, [n_steps][n_rings] by ring index ("real").
   Returns ENONFINITE if the wake stopped early at the guard (outputs still
   written), ETIMEOUT if it stopped because a bounded device wait gave up. */
wake_status wake_run(wake_handle *h, void *beam_ez, void *beam_wr, void *ring_r);

/* Runs the rest of the window of n handles: one launch per kernel
   configuration (launch shape, block size, mobile ions or not), run
   concurrently (one thread block, or cluster, walks one wake; blocks take
   wakes largest-first).  All handles must share precision and stream.
   Returns OK when the launches were enqueued; per-wake outcome via
   wake_get_progress. */
wake_status wake_batch_run(int32_t n, wake_handle *const *handles);

/* wake_batch_reset(n, handles, NULL, NULL) followed by wake_batch_run, as
   one pipelined submission: wake_batch_solve(n, handles, NULL, NULL). */
wake_status wake_batch_reset_run(int32_t n, wake_handle *const *handles);

/* Solves n wakes through their whole window in one pipelined submission:
   for each wake, in order of its predicted march time (longest first), the
   upload of its new beams (beams[i] not NULL: host arrays under
   wake_reset's rules, copied on the library's preparation streams, so pinned
   memory overlaps everything else), its a0/a1 preparation (Sec. II: rings,
   nearest-slice binning, per-slice radial sort) and then, as soon as the
   wakes of its launch are prepared, the march.  Nothing waits for the
   device: the per-slice sort sizes itself on the device.  The same results
   as wake_batch_reset followed by wake_batch_run.  All handles share
   precision and stream; beams may be NULL (no new beams for any wake).
   Errors: EINVAL (NULL handle, mixed precision or stream, bad beams),
   ECUDA; per-wake outcome via wake_get_progress. */
wake_status wake_batch_solve(int32_t n, wake_handle *const *handles, const wake_beam_desc *const *beams,
                             const int32_t *n_beams);

/* Advances every wake by up to max_slices slices (fewer at the end of a
   window or after a stop), in the launches of wake_batch_run.  With
   time_budget_ns > 0 each wake's launch also stops at the first slice
   boundary at least that long after its start (it always does one slice):
   the step of a continuous-batching loop, whose wakes of different sizes
   then finish a step together.  Asynchronous on the handles' stream.
   Errors: EINVAL (NULL handle, mixed precision or stream, negative
   limits), ECUDA. */
wake_status wake_batch_step(int32_t n, wake_handle *const *handles, int32_t max_slices,
                            int64_t time_budget_ns);

/* Next slice and status (0, or the WAKE_* code that stopped the wake) of n
   wakes sharing one stream, with one gather and one synchronisation of that
   stream.  Errors: EINVAL, ECUDA. */
wake_status wake_batch_progress(int32_t n, wake_handle *const *handles, int32_t *next_slice,
                                int32_t *status);

/* Device bytes the handle holds (for admission by a memory budget): every
   allocation wake_init and wake_set_beam_phase_space made for it.  Host
   call, no device work.  Errors: EINVAL (NULL handle or bytes). */
wake_status wake_get_device_bytes(wake_handle *h, int64_t *bytes);

/* Device times of the last march launch that advanced this wake
   (synchronises its stream): the GPU's global timer, in ns, when the
   launch began on the wake and when it finished with it (0, 0 before any
   march).  The time a batched wake waited for a free SM is its begin
   minus that of the batch's first wake; serving and launch-shape tuning
   read per-wake device latency from it.  Errors: EINVAL (NULL handle),
   ECUDA. */
wake_status wake_get_march_times(wake_handle *h, int64_t *begin_ns, int64_t *end_ns);

/* Progress of a wake (synchronises its stream): next slice to solve,
   status (OK, ENONFINITE, or EINVAL for a slice denser than
   wake_max_slice_particles() after an asynchronous preparation) and the
   failing slice (-1 if none); any output may be NULL.  Errors: EINVAL
   (NULL handle), ECUDA. */
wake_status wake_get_progress(wake_handle *h, int32_t *next_slice, int32_t *status,
                              int32_t *fail_slice);

/* Ring state by ring index (synchronises): radii, radial momenta and the
   AB2 history (d rho/d xi and d u_r/d xi of the previous slice) at the
   current slice, as double host arrays of n_rings (NULL = skip).  Together
   with wake_get_progress this is a checkpoint of a resumable solve. */
wake_status wake_get_ring_state(wake_handle *h, double *rho, double *ur, double *f_rho,
                                double *f_ur);

/* Restores a checkpoint: the wake continues from `slice` (0 <= slice <=
   n_steps) with the given ring state by ring index (double host arrays of
   n_rings; rho >= 0).  f_rho and f_ur are the AB2 history; pass both NULL
   to start the next step with forward Euler.  Clears the stopped status.
   Errors: EINVAL, ENOMEM, ECUDA. */
wake_status wake_set_ring_state(wake_handle *h, int32_t slice, const double *rho, const double *ur,
                                const double *f_rho, const double *f_ur);

/* Dumps kept with WAKE_DUMP_RING_FIELDS, [n_steps][n_rings] by ring index,
   "real" host arrays (NULL = skip). */
wake_status wake_get_ring_dumps(wake_handle *h, void *r, void *ur, void *psi, void *dpsidr,
                                void *dpsidz, void *bp, void *bb);

/* How the march kernels serve this wake: threads per block, rings per
   thread (on the global-memory marches: ceil(rings / (threads x blocks)),
   both species counted with mobile ions), and thread blocks per wake (> 1: a thread-
   block cluster).  For batched launches, wakes of the same march (on-chip,
   plain, two-species, RK4, beam grids) with equal triples share one
   launch. */
wake_status wake_get_launch_config(wake_handle *h, int32_t *threads, int32_t *rings_per_thread,
                                   int32_t *blocks_per_wake);


/* Beam push between wake solves (Sec. V: the beam moves over a time step in
   the fields the wake gave at each particle; Boris method).  The beam needs
   a full phase space for it: x, y, u_x, u_y, u_z (u = p/(m c)) per beam
   particle in the concatenated order of wake_init, host double arrays of
   the total particle count; the radius the wake bins by becomes |(x, y)|
   and xi stays as given.  Beam species must be electrons or positrons
   (q = -1 or +1, electron mass).  Synchronises the
   handle's stream.  Errors: EINVAL (NULL arrays, non-finite values), ENOMEM,
   ECUDA. */
wake_status wake_set_beam_phase_space(wake_handle *h, const double *x, const double *y, const double *ux,
                                      const double *uy, const double *uz);

/* The beam's current x, y, xi, r (the radius the next wake_reset bins by),
   u_x, u_y, u_z (host double arrays, any may be NULL).  Errors: EINVAL (no
   phase space set and x, y or u asked for), ECUDA. */
wake_status wake_get_beam_phase_space(wake_handle *h, double *x, double *y, double *xi, double *r, double *ux,
                                      double *uy, double *uz);

/* One time step dt (> 0, in 1/omega_p) of every beam particle in the fields
   of the last march (particles outside the window see none): u is updated
   by the Boris method with E = (E_r x/r, E_r y/r, E_z), E_r = W_r + B_theta,
   B = (-B_theta y/r, B_theta x/r, 0), then x, y move by dt u/gamma and xi by
   dt (1 - u_z/gamma).  The next wake_reset(h, NULL) bins the moved beam, and
   a march then solves the wake it drives.  FP64 wakes push in FP64; mixed
   wakes add FP32 increments (~1e-7 of themselves) to the FP64 phase space.
   Asynchronous on the handle's stream.  Errors: EINVAL (dt <= 0, no phase
   space, unsupported species), ENOMEM, ECUDA. */
wake_status wake_push_beam(wake_handle *h, double dt);

/* wake_push_beam of n wakes sharing one stream and one precision, as one
   kernel launch on that stream.  Errors: as wake_push_beam, and EINVAL for
   handles on different streams or of different precisions. */
wake_status wake_batch_push_beam(int32_t n, wake_handle *const *handles, double dt);

/* wake_fields_at without any allocation.  The paper has no counterpart:
   this entry exists for callers that cannot allocate while they run -- a
   host code that owns the device's memory through its own pool allocator,
   or a latency-critical loop that must not let cudaMalloc/cudaFree
   synchronise the device.  Same fields, same kernels and same results as
   wake_fields_at at the current slice; r and the outputs are HOST arrays
   ("real" outputs, any may be NULL), n <= WAKE_STATIC_MAX_QUERIES.
   The per-call scratch (query radii, outputs, launch descriptor, about
   2.5 MiB) is one static device array of the library, not memory of the
   handle or of the caller.  The first call on each device looks up its
   address with cudaGetSymbolAddress, so make one call (n = 0 does only
   this set-up) before any stream capture.  The handle's device must be
   current.  There is one scratch array per device and process: calls that
   overlapped would race on it, so a call made while another is in
   progress in this process returns WAKE_EBUSY.  Synchronises the handle's
   stream before returning.
   Errors: EINVAL (n < 0 or n > WAKE_STATIC_MAX_QUERIES, NULL r, handle on
   another device, window finished), EBUSY, ENONFINITE (the wake stopped),
   ECUDA. */
#define WAKE_STATIC_MAX_QUERIES 65536
wake_status wake_fields_at_static(wake_handle *h, int64_t n, const double *r, void *ez, void *wr,
                                  void *bt, void *psi);

/* Releases the handle; its device memory returns to the library's pool in
   stream order (after the work already queued on the handle's stream), so
   the call does not wait for the device. */
void wake_destroy(wake_handle *h);

/* Debug builds only (compiled with -DWAKE_BOUNDS_CHECK: python -m
   paper_2603_16623_gb300.build --bounds-check): how many swizzled
   shared-memory positions and DSMEM peer ranks out of range the on-chip
   marches met since the last call (each was replaced by 0, an index in
   range, and counted), and resets the count.  -1 in a build without the
   checks, -2 if the counters could not be read (a CUDA error). */
int64_t wake_debug_bounds_violations(void);

const char *wake_last_error(void);
int32_t wake_max_rings(int32_t precision);          /* rings per wake supported */
int64_t wake_max_slice_particles(int32_t precision); /* beam particles per slice */

/* The launch shape wake_init gives the on-chip march (mixed precision,
   electrons over the ion column, no beam grids) for a wake of n_rings rings
   and n_steps slices and the config's rings_per_thread and cluster_ctas,
   computed on the host: no device, no handle, nothing allocated.  Both 0:
   the automatic shape, which is the batch shape (one CTA of up to 512
   threads x 2 rings up to 1024 rings, x 4 rings up to 2048 rings; up to
   16,384 rings a cluster of ceil(n / 1024) CTAs of 4 rings per thread; up
   to 32,768 ceil(n / 2048) CTAs; beyond, 8 rings per thread), or, when its
   predicted march time is at least wake_get_latency_shape_ms(), the latency
   shape (wake_launch_shape_latency).  n_steps 0: the batch shape.  Outputs
   (each may be NULL): threads per CTA, rings per thread and CTAs per wake
   (> 1: a thread-block cluster); all three 0 when the wake runs on a
   one-CTA march instead (FP64, or the automatic shape beyond the on-chip
   march's 65,536 rings).  The launch-shape autotuner enumerates its
   candidates with it.  Errors: EINVAL for a precision other than WAKE_FP64
   or WAKE_MIXED, n_rings outside [1, wake_max_rings(precision)], a negative
   n_steps, or the shape wake_init would refuse (rings_per_thread not 0, 2,
   4 or 8; cluster_ctas outside [0, 16]; more than 512 threads per CTA; an
   empty last CTA; either field set with FP64). */
wake_status wake_launch_shape(int32_t precision, int32_t n_rings, int32_t n_steps, int32_t rings_per_thread,
                              int32_t cluster_ctas, int32_t *threads, int32_t *rings_per_thread_out,
                              int32_t *blocks_per_wake);

/* The latency shape of an automatic-shape wake of n_rings rings (mixed
   precision), computed on the host: 2 rings per thread, the shortest time
   per slice (about 0.7x the batch shape's per slice on clusters) for about
   1.3x its SM time.  Up to 1024 rings one CTA of ceil(n / 2) threads
   (rounded up to a multiple of 32); up to 8192 rings a cluster of
   ceil(n / 512) CTAs of at most 256 threads; up to 16,384 rings
   ceil(n / 1024) CTAs of at most 512 threads; beyond, the batch shape.
   Outputs as wake_launch_shape (all 0 for WAKE_FP64).  Errors: EINVAL as
   wake_launch_shape. */
wake_status wake_launch_shape_latency(int32_t precision, int32_t n_rings, int32_t *threads,
                                      int32_t *rings_per_thread_out, int32_t *blocks_per_wake);

/* The threshold, in milliseconds of predicted march time, at and above
   which wake_init gives an automatic-shape wake its latency shape rather
   than its batch shape (process-wide; default INFINITY: none; 0: every
   wake).  Alone, the latency shape marches a wake 10-35 % faster; in a
   batch that fills the GPU its larger clusters are placed late and the
   batch takes longer, hence the default.  The prediction is the library's model of the on-chip
   march's time per slice on GB300 for the batch shape x n_steps.  A
   wake's shape is fixed when it is created, so a wake gives the same
   results alone and in any batch.  Errors: EINVAL for a negative value or
   NaN. */
wake_status wake_set_latency_shape_ms(double ms);
double wake_get_latency_shape_ms(void);

/* the global-memory marches whose wakes also run on thread-block clusters */
enum { WAKE_GM_IONS = 1, WAKE_GM_RK4 = 2, WAKE_GM_GRID = 3 };

/* The launch shape wake_init gives a wake of the two-species march
   (WAKE_GM_IONS: n_cells per species), the RK4 march (WAKE_GM_RK4) or a
   beam-grid wake (WAKE_GM_GRID: n_cells rings), computed on the host from
   the config's block_threads (0: the default, 512 for ions and RK4, 256 for
   grids) and cluster_ctas (0: automatic, the fewest blocks, at most 8, that
   hold at most 2 rings of each species (ions), 2 rings (RK4) or 4 rings
   (grids) per thread).  Outputs (each may be NULL): threads per block,
   rings per thread (both species counted with ions) and blocks per wake,
   as wake_get_launch_config reports them.  Errors: EINVAL for an unknown
   march, n_cells outside [1, 4096] (ions) or [1, 16384], block_threads not
   0 or a multiple of 32 in [64, 512], cluster_ctas outside [0, 8]. */
wake_status wake_gm_launch_shape(int32_t march, int32_t n_cells, int32_t block_threads, int32_t cluster_ctas,
                                 int32_t *threads, int32_t *rings_per_thread, int32_t *blocks_per_wake);


#ifdef __cplusplus
}
#endif
#endif /* GBWAKE_WAKE_H */
