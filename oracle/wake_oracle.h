/*
 * wake_oracle.h -- FP64 CPU oracle of the gridless quasistatic wake model.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, sequential reference
 * that the CUDA path is checked against.  Only tests, the smoke check and the
 * benchmark's CPU-baseline/reference legs may load it; the product library
 * never links or calls it, and it shares no code with the CUDA sources.
 *
 * Model: Sec. II of the paper (gridless quasistatic model), no laser; xi =
 * -zeta, one step advances xi by dxi.
 *   orc_run: electrons (q = -1, m = 1) over an immobile uniform ion column of
 *     density n filling rho <= rho_max = edges[N] (the Baxevanis-Stupakov
 *     limit named at the end of Sec. II); the ring integrator AB2 (Sec. III)
 *     or RK4; the beam fields gridless (a9) or through adaptive beam grids
 *     (Sec. IV, AB2 only).
 *   orc_run_ions: electrons and mobile ions as two ring species (Sec. II,
 *     multiple plasma species), with an optional radial density profile.
 * The beam push between solves is oracle/beam_push.py.
 */
#ifndef WAKE_ORACLE_H
#define WAKE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 2, ORC_ENONFINITE = 4 };
enum { ORC_AB2 = 0, ORC_RK4 = 1 };

typedef struct {
    int32_t n_rings;          /* N >= 1 */
    const double *edges;      /* N+1 cell edges, edges[0]=0, strictly increasing */
    double density;           /* uniform n of electrons and of the ion column */
    int64_t n_beam;           /* beam macroparticles (all beams concatenated) */
    const double *beam_xi;    /* [n_beam] */
    const double *beam_r;     /* [n_beam] >= 0 */
    const double *beam_qw;    /* [n_beam] charge sign x weight */
    double dxi;               /* step in xi (> 0) */
    int32_t n_steps;          /* slices in the window */
    /* radial density profile: density of each cell [n_rings] (> 0), uniform
       within a cell; NULL = `density` everywhere.  orc_run_ions only (the
       ion rings carry the profile; orc_run's column is uniform). */
    const double *cell_density;
    /* ring integrator of orc_run: ORC_AB2 (Sec. III) or ORC_RK4 (the
       Runge-Kutta alternative Sec. II names) */
    int32_t integrator;
    /* beam-plasma coupling through adaptive beam grids (Sec. IV; orc_run
       with ORC_AB2): grid_nr > 0 radial cells per beam species, whose
       extent covers all its particles; 0 = gridless (a9).  beam_species
       [n_beam] gives each particle's species (NULL: all 0), n_species. */
    int32_t grid_nr;
    const int32_t *beam_species;
    int32_t n_species;
    /* grid_rmax > 0: every species' grid spans [0, grid_rmax] (the regular
       intermediate grid); every beam particle must lie below it (else
       ORC_EINVAL).  0: the adaptive extent. */
    double grid_rmax;
    /* initial ring state by ring id (orc_run only; NULL: the rings start
       at rest at their cell centres, Sec. II): radii (>= 0) and radial
       momenta, and optionally the AB2 history (the previous slice's
       d rho/dxi and d u_r/dxi; NULL: the first step is forward Euler).
       The counterpart of a checkpoint restored on the GPU path. */
    const double *init_r, *init_ur, *init_fr, *init_fu;
} orc_problem;

typedef struct {
    /* per beam particle, caller order (NULL: skip).  Particles whose
       nearest slice is outside the window get 0. */
    double *ez, *wr, *bt, *psi;
    /* per slice and ring id, [n_steps][n_rings] (NULL: skip); values at the
       start of the slice (before the push). */
    double *ring_r, *ring_ur, *ring_psi, *ring_dpsidr, *ring_dpsidz, *ring_bp,
           *ring_bb, *ring_psibar, *ring_gamma, *ring_uz;
    /* AB2 history at the start of each slice (the previous slice's
       d rho/dxi and d u_r/dxi; 0 at slice 0), [n_steps][n_rings] by id */
    double *ring_frprev, *ring_fuprev;
    /* ring state by id after the last slice run (NULL: skip) */
    double *final_r, *final_ur;
    int32_t status;       /* ORC_OK or ORC_ENONFINITE */
    int32_t fail_slice;   /* first slice whose fields failed the guard, else -1 */
    int32_t slices_run;
    /* orc_run: the ring dumps above at n_snap chosen slices only (snapshots
       of long windows): snap [n_snap][ORC_SNAP_FIELDS][n_rings] by ring id,
       the fields in the order r, ur, psi, dpsidr, dpsidz, bp, bb, frprev,
       fuprev; rows of slices not reached stay as they are. */
    int32_t n_snap;
    const int32_t *snap_slice;
    double *snap;
} orc_outputs;

enum { ORC_SNAP_FIELDS = 9 };

/* Fields of one slice for a given ring state; everything per ring is indexed
   by ring id, per-region coefficients in radius order. */
typedef struct {
    double *psi, *dpsidr, *dpsidz, *psibar, *gamma, *uz, *bb, *A, *B, *C, *bp;
    double *a, *b;            /* [N+1] B_theta^(p) = a_k rho + b_k / rho in region k */
    int32_t *order;           /* [N] ring ids in radius order */
    /* optional query points */
    int64_t nq;
    const double *rq;
    double *q_ez, *q_wr, *q_bt, *q_psi, *q_bp, *q_bb, *q_dpsidr, *q_dpsidz;
} orc_slice_out;

/* Ring initialisation (Sec. II, ring macroparticles and Eq. macroparticle_weight;
   the self weight of the "key algorithmic adjustments"). */
void orc_ring_init(int32_t n, const double *edges, double density,
                   double *rho0, double *drho, double *w, double *what);

/* One slice: fields at every ring and (optionally) at query radii. */
int orc_slice_fields(int32_t n, const double *rho, const double *ur,
                     const double *w, const double *what, double density, double rho_max,
                     int64_t m, const double *beam_r, const double *beam_qw, double dxi,
                     orc_slice_out *out);

/* App. A shooting solve of the B_theta^(p) recursion (Eq. ai_bi): rings in
   radius order (rho[0] < ... < rho[n-1]); returns a[0..n], b[0..n]. */
int orc_bp_shooting(int32_t n, const double *rho, const double *A, const double *B,
                    const double *C, double *a, double *b);

/* The same system solved directly (banded elimination with partial
   pivoting); this is what the oracle's slices use: it stays accurate on wide
   plasma columns where the shooting loses digits to the growing mode. */
int orc_bp_solve(int32_t n, const double *rho, const double *A, const double *B,
                 const double *C, double *a, double *b);

/* Whole window (or its first max_slices slices when max_slices > 0). */
int orc_run(const orc_problem *p, int32_t max_slices, orc_outputs *out);

/* The same with mobile ions of charge Z > 0 and mass M > 0 (electron
   masses; M = +inf: ions that never move) as a second ring species on the
   same edges, in place of the immobile column (Sec. II, multiple plasma
   species): ring outputs are [n_steps][2 N] and final_r, final_ur [2 N],
   electrons by id 0..N-1, ions N..2N-1.  Both species follow the density
   profile (p->cell_density, ions at 1/Z of it). */
int orc_run_ions(const orc_problem *p, double ion_z, double ion_m, int32_t max_slices,
                 orc_outputs *out);

#ifdef __cplusplus
}
#endif
#endif
