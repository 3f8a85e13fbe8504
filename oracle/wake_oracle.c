/*
 * wake_oracle.c -- FP64 CPU oracle of the gridless quasistatic wake model.
 *
 * TEST INFRASTRUCTURE ONLY (see wake_oracle.h).  Plain sequential C: one
 * stable merge sort, sequential sums, the App. A shooting recursion and the
 * second-order Adams-Bashforth push, in the order of Sec. III (sort, gather
 * sources, psi and its derivatives, u_z and gamma, B_theta^(p), evolve).
 *
 * Conventions (electrons q = -1, m = 1, so psibar = 1 + psi):
 *   ring i in radius order, weight w_i, self weight what_i;
 *   S(rho) = sum_{rho_j < rho} w_j                      (Eq. dpsi_dr)
 *   I(rho) = n min(rho, rho_max)^2 / 2                  (ion column, enclosed)
 *   d_rho psi  = (S - I) / rho                          (Eq. dpsi_dr + ions)
 *   psi(rho)   = sum_j w_j ln max(rho, rho_j) + psi_ion (Eq. psi + ions)
 *   d_zeta psi = -sum_{rho_j > rho} w_j u_j / (rho_j psibar_j)
 *                (the zeta derivative of Eq. psi at fixed rho, using
 *                 Eq. plasma_particle_motion_2; see the note at
 *                 zeta_derivative() on the sign of Eq. dpsi_dzeta)
 * At a ring the partial sums use the self weight what_i in place of w_i
 * (Sec. II, "key algorithmic adjustments").
 */
#include "wake_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_2PI 6.283185307179586476925286766559

/* ---------------------------------------------------------------------- */
/* ion column: uniform density n on rho <= rho_max, immobile               */
/* ---------------------------------------------------------------------- */

/* Ion charge enclosed within rho (per unit length and per 2 pi). */
static double ion_enclosed(double rho, double n, double rho_max)
{
    double c = rho < rho_max ? rho : rho_max;
    return 0.5 * n * c * c;
}

/* Ion-column part of psi: Eq. psi applied to the continuous ion column,
   normalised so that psi -> 0 at infinity once the (neutralising) electron
   sum is added: d/drho psi_ion = -I(rho)/rho, psi_ion ~ -(n rho_max^2/2) ln rho
   outside the column. */
static double ion_psi(double rho, double n, double rho_max)
{
    double q = 0.5 * n * rho_max * rho_max;
    if (rho <= rho_max)
        return 0.25 * n * (rho_max * rho_max - rho * rho) - q * log(rho_max);
    return -q * log(rho);
}

/* ---------------------------------------------------------------------- */
/* small helpers                                                           */
/* ---------------------------------------------------------------------- */

/* First index i in the increasing array a[0..n) with a[i] >= x. */
static int64_t lower_bound(const double *a, int64_t n, double x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

/* Stable bottom-up merge sort of ids[0..n) by key[id]; equal keys keep
   their input order (the previous slice's order, Sec. III). */
static void stable_sort_ids(int32_t n, int32_t *ids, const double *key, int32_t *tmp)
{
    int32_t *src = ids, *dst = tmp;
    for (int32_t width = 1; width < n; width *= 2) {
        for (int32_t lo = 0; lo < n; lo += 2 * width) {
            int32_t mid = lo + width < n ? lo + width : n;
            int32_t hi = lo + 2 * width < n ? lo + 2 * width : n;
            int32_t i = lo, j = mid, k = lo;
            while (i < mid && j < hi)
                dst[k++] = (key[src[j]] < key[src[i]]) ? src[j++] : src[i++];
            while (i < mid)
                dst[k++] = src[i++];
            while (j < hi)
                dst[k++] = src[j++];
        }
        int32_t *t = src;
        src = dst;
        dst = t;
    }
    if (src != ids)
        memcpy(ids, src, (size_t)n * sizeof(int32_t));
}

/* Beam particles of one slice sorted by (r, index), with the exclusive
   prefix P[p] = sum_{q < p} qw[q] (P has m+1 entries).  The enclosed beam
   charge strictly below rho is P[lower_bound(r, rho)]. */
typedef struct {
    int64_t m;
    double *r, *P;
    int64_t *idx;
} beam_slice;

/* a beam particle of one slice: radius, charge x weight, caller index */
typedef struct { double r; double qw; int64_t idx; } bpart;

static int bpart_cmp(const void *x, const void *y)
{
    const bpart *a = (const bpart *)x, *b = (const bpart *)y;
    if (a->r < b->r) return -1;
    if (a->r > b->r) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

static int beam_slice_build(beam_slice *bs, int64_t m, const bpart *parts_in)
{
    bs->m = m;
    bs->r = (double *)malloc((size_t)(m + 1) * sizeof(double));
    bs->P = (double *)malloc((size_t)(m + 1) * sizeof(double));
    bs->idx = (int64_t *)malloc((size_t)(m + 1) * sizeof(int64_t));
    bpart *parts = (bpart *)malloc((size_t)(m + 1) * sizeof(bpart));
    if (!bs->r || !bs->P || !bs->idx || !parts) {
        free(parts);
        return ORC_ENOMEM;
    }
    if (m > 0)
        memcpy(parts, parts_in, (size_t)m * sizeof(bpart));
    qsort(parts, (size_t)m, sizeof(bpart), bpart_cmp);
    double acc = 0.0;
    for (int64_t p = 0; p < m; ++p) {
        bs->r[p] = parts[p].r;
        bs->idx[p] = parts[p].idx;
        bs->P[p] = acc;
        acc += parts[p].qw;
    }
    bs->P[m] = acc;
    free(parts);
    return ORC_OK;
}

static void beam_slice_free(beam_slice *bs)
{
    free(bs->r);
    free(bs->P);
    free(bs->idx);
    bs->r = bs->P = NULL;
    bs->idx = NULL;
}

/* Beam field (Sec. II, the B_theta^(b) equation integrated from the axis):
   rho B^(b) = int_0^rho q n_b rho' drho'; a beam macroparticle of weight W in
   a slice of thickness dxi is a ring of density W / (2 pi rho dxi) delta, so
   B^(b)(rho) = Q(rho) / (2 pi dxi rho) with Q the charge strictly below rho. */
static double beam_field(const beam_slice *bs, double rho, double dxi)
{
    if (bs->m == 0 || !(rho > 0.0))
        return 0.0;
    double Q = bs->P[lower_bound(bs->r, bs->m, rho)];
    return Q / (ORC_2PI * dxi * rho);
}

/* ---------------------------------------------------------------------- */
/* ring initialisation                                                     */
/* ---------------------------------------------------------------------- */

/* Sec. II: rho_j0 = sum_{k<j} drho_k + drho_j/2 (cell centre), weight
   w_j = n rho_j0 drho_j (Eq. macroparticle_weight) and the self weight
   what_j = n (rho_j0 drho_j / 2 - drho_j^2 / 8), the charge of the cell below
   the ring ("key algorithmic adjustments"; with n = 1 it is w_j/2 - drho_j^2/8). */
void orc_ring_init(int32_t n, const double *edges, double density,
                   double *rho0, double *drho, double *w, double *what)
{
    for (int32_t j = 0; j < n; ++j) {
        double d = edges[j + 1] - edges[j];
        double c = 0.5 * (edges[j] + edges[j + 1]);
        if (rho0) rho0[j] = c;
        if (drho) drho[j] = d;
        if (w) w[j] = density * c * d;
        if (what) what[j] = density * (0.5 * c * d - 0.125 * d * d);
    }
}

/* ---------------------------------------------------------------------- */
/* App. A: shooting solution of the B^(p) recursion                        */
/* ---------------------------------------------------------------------- */

/* Eq. ai_bi with b_0 = 0, a_N = 0, solved as in App. A: a_i = K_i a_0 + T_i,
   b_i = U_i a_0 + P_i, (K,U,T,P)_0 = (1,0,0,0), both pairs advanced by the
   matrix of Eq. ai_bi (the (T,P) pair also by its source vector), then
   a_0 = -T_N / K_N (Eq. app1_a0).  Ring i (1-based in the paper) is rho[i-1]
   here; region k lies between rings k and k+1. */
int orc_bp_shooting(int32_t n, const double *rho, const double *A, const double *B,
                    const double *C, double *a, double *b)
{
    double *K = (double *)malloc((size_t)(n + 1) * 4 * sizeof(double));
    if (!K)
        return ORC_ENOMEM;
    double *U = K + (n + 1), *T = U + (n + 1), *P = T + (n + 1);
    K[0] = 1.0; U[0] = 0.0; T[0] = 0.0; P[0] = 0.0;
    for (int32_t i = 1; i <= n; ++i) {
        double r = rho[i - 1], Ai = A[i - 1], Bi = B[i - 1], Ci = C[i - 1];
        double m11 = 1.0 + 0.5 * Ai * r;
        double m12 = 0.5 * Ai / r;
        double m21 = -0.5 * Ai * r * r * r;
        double m22 = 1.0 - 0.5 * Ai * r;
        double s1 = 0.25 * (2.0 * Bi + Ai * Ci);
        double s2 = 0.25 * r * (4.0 * Ci - 2.0 * Bi * r - Ai * Ci * r);
        K[i] = m11 * K[i - 1] + m12 * U[i - 1];
        U[i] = m21 * K[i - 1] + m22 * U[i - 1];
        T[i] = m11 * T[i - 1] + m12 * P[i - 1] + s1;
        P[i] = m21 * T[i - 1] + m22 * P[i - 1] + s2;
    }
    double a0 = -T[n] / K[n];
    for (int32_t k = 0; k <= n; ++k) {
        a[k] = K[k] * a0 + T[k];
        b[k] = U[k] * a0 + P[k];
    }
    free(K);
    return ORC_OK;
}

/* Banded Gaussian elimination with partial pivoting (the textbook band LU,
   e.g. Golub & Van Loan, Sec. 4.3): n unknowns, kl sub- and ku
   super-diagonals; row r keeps columns [r - kl, r + ku + kl] (room for the
   fill-in of row swaps) at ab[r * W + (c - r + kl)], W = 2 kl + ku + 1.
   Solves in place: x returned in rhs.  Returns ORC_EINVAL if singular. */
static int band_solve(int64_t n, int kl, int ku, double *ab, double *rhs)
{
    const int W = 2 * kl + ku + 1;
#define AB(r, c) ab[(r) * W + ((c) - (r) + kl)]
    for (int64_t k = 0; k < n; ++k) {
        int64_t last_r = k + kl < n - 1 ? k + kl : n - 1;
        int64_t last_c = k + kl + ku < n - 1 ? k + kl + ku : n - 1;
        int64_t p = k;
        double best = fabs(AB(k, k));
        for (int64_t r = k + 1; r <= last_r; ++r)
            if (fabs(AB(r, k)) > best) {
                best = fabs(AB(r, k));
                p = r;
            }
        if (!(best > 0.0))
            return ORC_EINVAL;
        if (p != k) {
            for (int64_t c = k; c <= last_c; ++c) {
                double t = AB(k, c);
                AB(k, c) = AB(p, c);
                AB(p, c) = t;
            }
            double t = rhs[k];
            rhs[k] = rhs[p];
            rhs[p] = t;
        }
        for (int64_t r = k + 1; r <= last_r; ++r) {
            double f = AB(r, k) / AB(k, k);
            if (f == 0.0)
                continue;
            AB(r, k) = 0.0;
            for (int64_t c = k + 1; c <= last_c; ++c)
                AB(r, c) -= f * AB(k, c);
            rhs[r] -= f * rhs[k];
        }
    }
    for (int64_t k = n - 1; k >= 0; --k) {
        int64_t last_c = k + kl + ku < n - 1 ? k + kl + ku : n - 1;
        double sum = rhs[k];
        for (int64_t c = k + 1; c <= last_c; ++c)
            sum -= AB(k, c) * rhs[c];
        rhs[k] = sum / AB(k, k);
    }
#undef AB
    return ORC_OK;
}

/* Eq. ai_bi with b_0 = 0 and a_N = 0, solved directly as the linear system
   it defines (unknowns a_0, b_0, ..., a_N, b_N; rows: b_0 = 0, the two rows
   of Eq. ai_bi for each ring, a_N = 0) by banded elimination.  Same
   solution as the App. A shooting, which amplifies rounding by the growth
   of the homogeneous solution (~e^rho_max) and loses digits on wide
   plasma columns. */
int orc_bp_solve(int32_t n, const double *rho, const double *A, const double *B,
                 const double *C, double *a, double *b)
{
    const int64_t m = 2 * (int64_t)n + 2;
    const int kl = 2, ku = 1, W = 2 * kl + ku + 1;
    double *ab = (double *)calloc((size_t)(m * W), sizeof(double));
    double *x = (double *)calloc((size_t)m, sizeof(double));
    if (!ab || !x) {
        free(ab);
        free(x);
        return ORC_ENOMEM;
    }
#define SET(r, c, v) ab[(r) * W + ((c) - (r) + kl)] = (v)
    SET(0, 1, 1.0);  /* b_0 = 0 */
    for (int32_t i = 1; i <= n; ++i) {
        double r = rho[i - 1], Ai = A[i - 1], Bi = B[i - 1], Ci = C[i - 1];
        int64_t ra = 2 * (int64_t)i - 1, rb = 2 * (int64_t)i;
        int64_t ca0 = 2 * (int64_t)(i - 1), cb0 = ca0 + 1, ca1 = ca0 + 2, cb1 = ca0 + 3;
        /* a_i - (1 + A r/2) a_{i-1} - (A/(2r)) b_{i-1} = (2B + AC)/4 */
        SET(ra, ca0, -(1.0 + 0.5 * Ai * r));
        SET(ra, cb0, -(0.5 * Ai / r));
        SET(ra, ca1, 1.0);
        x[ra] = 0.25 * (2.0 * Bi + Ai * Ci);
        /* b_i + (A r^3/2) a_{i-1} - (1 - A r/2) b_{i-1} = r (4C - 2Br - ACr)/4 */
        SET(rb, ca0, 0.5 * Ai * r * r * r);
        SET(rb, cb0, -(1.0 - 0.5 * Ai * r));
        SET(rb, cb1, 1.0);
        x[rb] = 0.25 * r * (4.0 * Ci - 2.0 * Bi * r - Ai * Ci * r);
    }
    SET(m - 1, m - 2, 1.0);  /* a_N = 0 */
#undef SET
    int rc = band_solve(m, kl, ku, ab, x);
    if (!rc)
        for (int32_t k = 0; k <= n; ++k) {
            a[k] = x[2 * k];
            b[k] = x[2 * k + 1];
        }
    free(ab);
    free(x);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* one slice                                                               */
/* ---------------------------------------------------------------------- */

/* Work arrays of a slice, all in radius order (index i = sorted position). */
typedef struct {
    int32_t n;
    double *r, *u, *w, *wh;          /* ring state and weights */
    double *S, *L, *T;               /* exclusive prefix sums, [n+1] */
    double *t;                       /* w u / (rho psibar) */
    double *psi, *dpr, *dpz, *psib, *gam, *uz, *bb, *A, *B, *C, *bp;
    double *a, *b;                   /* [n+1] */
    double Wtot, Ltot, Ttot;
    int32_t *tmp;
} slice_ws;

static int ws_alloc(slice_ws *s, int32_t n)
{
    memset(s, 0, sizeof(*s));
    s->n = n;
    size_t m = (size_t)n + 1;
    double *blk = (double *)calloc(m * 22, sizeof(double));
    s->tmp = (int32_t *)malloc(m * sizeof(int32_t));
    if (!blk || !s->tmp) {
        free(blk);
        free(s->tmp);
        return ORC_ENOMEM;
    }
    double **fields[] = {&s->r, &s->u, &s->w, &s->wh, &s->S, &s->L, &s->T, &s->t,
                         &s->psi, &s->dpr, &s->dpz, &s->psib, &s->gam, &s->uz,
                         &s->bb, &s->A, &s->B, &s->C, &s->bp, &s->a, &s->b};
    for (size_t f = 0; f < sizeof(fields) / sizeof(fields[0]); ++f)
        *fields[f] = blk + f * m;
    return ORC_OK;
}

static void ws_free(slice_ws *s)
{
    free(s->r);
    free(s->tmp);
    memset(s, 0, sizeof(*s));
}

/* Eq. dpsi_dzeta.  Differentiating Eq. psi in zeta at fixed rho with
   d rho_i / d zeta = -u_i / psibar_i (Eq. plasma_particle_motion_2) gives
   d_zeta psi = + sum_i q_i w_i u_i/(rho_i psibar_i)
                - sum_{rho_i<rho} q_i w_i u_i/(rho_i psibar_i),
   the printed equation with the opposite overall sign.  The true partial
   derivative is used (it is what E_z = -d_zeta psi of Eq. lorentz_gauge_1 and
   the B_i coefficient of Eq. b_coeffs_2 need).  With q = -1 this is
   -sum_{rho_j >= rho} t_j, t_j = w_j u_j / (rho_j psibar_j); at ring i the
   ring's own term enters the partial sum with what_i / w_i. */
static double zeta_derivative(double suffix_above, double t_self, double w_self,
                              double wh_self)
{
    return -(suffix_above + (1.0 - wh_self / w_self) * t_self);
}

/* The adaptive beam grids of one slice (Sec. IV): species b has nr radial
   cells of width R[b] / nr; B[b (nr + 1) + j] is its B^(b) at node r_j =
   j R[b] / nr: the slice's charge of species b strictly inside r_j over
   2 pi dxi r_j (0 on the axis). */
typedef struct {
    int32_t nsp, nr;
    const double *R;
    double *B;
} ag_slice;

/* Node index j with r_j <= x < r_{j+1} for x >= 0 (nodes j dr, the
   comparison as written: j dr <= x), clamped to [0, nr - 1]. */
static int32_t ag_cell(double x, double dr, int32_t nr)
{
    int32_t j = (int32_t)floor(x / dr);
    if (j > nr - 1) j = nr - 1;
    if (j < 0) j = 0;
    while (j > 0 && (double)j * dr > x) --j;
    while (j < nr - 1 && (double)(j + 1) * dr <= x) ++j;
    return j;
}

/* B^(b) of species b at radius rho from its grid: linear between the nodes
   inside the grid, B_N r_N / rho beyond it (Sec. IV). */
static double ag_species_field(const ag_slice *g, int32_t b, double rho)
{
    const double *B = g->B + (size_t)b * (g->nr + 1);
    double R = g->R[b], dr = R / g->nr;
    if (rho >= R)
        return B[g->nr] * R / rho;
    int32_t j = ag_cell(rho, dr, g->nr);
    double t = (rho - (double)j * dr) / dr;
    return (1.0 - t) * B[j] + t * B[j + 1];
}

static double ag_field(const ag_slice *g, double rho)
{
    double v = 0.0;
    for (int32_t b = 0; b < g->nsp; ++b)
        v += ag_species_field(g, b, rho);
    return v;
}

/* All ring fields of one slice (Sec. III order: sources, psi and its
   derivatives, u_z and gamma, B_theta^(p)).  order[] holds the previous
   radius order on entry and the new one on exit.  The beam source is
   w1 x (the field of slice bs) + w2 x (that of bs2, if given): the RK4
   stages between two slices take the mean of both; with beam grids (ag)
   the grids' field instead. */
static int slice_core(slice_ws *s, int32_t *order, const double *rho_id,
                      const double *ur_id, const double *w_id, const double *wh_id,
                      double dens, double rho_max, const beam_slice *bs, const beam_slice *bs2,
                      double w1, double w2, const ag_slice *ag, double dxi)
{
    int32_t n = s->n;
    /* sort by radius, stable w.r.t. the previous order */
    stable_sort_ids(n, order, rho_id, s->tmp);
    for (int32_t i = 0; i < n; ++i) {
        int32_t id = order[i];
        s->r[i] = rho_id[id];
        s->u[i] = ur_id[id];
        s->w[i] = w_id[id];
        s->wh[i] = wh_id[id];
    }
    /* gather the beam source at the rings */
    for (int32_t i = 0; i < n; ++i) {
        if (ag) {
            s->bb[i] = ag_field(ag, s->r[i]);
            continue;
        }
        s->bb[i] = w1 * beam_field(bs, s->r[i], dxi);
        if (bs2)
            s->bb[i] += w2 * beam_field(bs2, s->r[i], dxi);
    }
    /* radial prefix sums of charge and of charge x ln rho (Eqs. dpsi_dr, psi) */
    double accS = 0.0, accL = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        s->S[i] = accS;
        s->L[i] = accL;
        accS += s->w[i];
        accL += s->w[i] * log(s->r[i]);
    }
    s->S[n] = accS;
    s->L[n] = accL;
    s->Wtot = accS;
    s->Ltot = accL;
    /* psi, d_rho psi (self weight), psibar, gamma, u_z
       (Eqs. psi, dpsi_dr, plasma_particle_motion_3/4) */
    for (int32_t i = 0; i < n; ++i) {
        double r = s->r[i], u = s->u[i];
        s->psi[i] = (s->Ltot - s->L[i]) + s->S[i] * log(r) + ion_psi(r, dens, rho_max);
        s->dpr[i] = (s->S[i] + s->wh[i] - ion_enclosed(r, dens, rho_max)) / r;
        double pb = 1.0 + s->psi[i];
        s->psib[i] = pb;
        s->gam[i] = (1.0 + u * u + pb * pb) / (2.0 * pb);
        s->uz[i] = (1.0 + u * u - pb * pb) / (2.0 * pb);
        s->t[i] = s->w[i] * u / (r * pb);
    }
    /* current prefix sum and d_zeta psi (Eq. dpsi_dzeta, see zeta_derivative) */
    double accT = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        s->T[i] = accT;
        accT += s->t[i];
    }
    s->T[n] = accT;
    s->Ttot = accT;
    for (int32_t i = 0; i < n; ++i) {
        double above = s->Ttot - s->T[i + 1];
        s->dpz[i] = zeta_derivative(above, s->t[i], s->w[i], s->wh[i]);
    }
    /* coefficients A_i, B_i, C_i (Eqs. b_coeffs_1..3 with q = -1, m = 1, no
       laser); the beam field enters B_i, the plasma field is the unknown */
    for (int32_t i = 0; i < n; ++i) {
        double r = s->r[i], u = s->u[i], w = s->w[i], pb = s->psib[i];
        double g = s->gam[i], dpr = s->dpr[i], dpz = s->dpz[i];
        double wr = w / r;
        s->A[i] = wr / pb;
        s->B[i] = -wr * g * dpr / (pb * pb)
                  + wr * s->bb[i] / pb
                  + (w / (r * r)) * u * u / (pb * pb)
                  + wr * u * u * dpr / (pb * pb * pb)
                  - wr * u * dpz / (pb * pb);
        s->C[i] = -wr * (g / pb - 1.0 - u * u / (pb * pb));
    }
    /* B_theta^(p): the system of Eq. ai_bi with its two boundary conditions
       (orc_bp_solve), then the field at each ring.  B^(p) jumps across a ring
       (the C_i term makes rho B jump by C_i rho_i); the matrix and source
       vector of Eq. ai_bi follow from the jump conditions exactly when the
       ring sees the mean of the two one-sided values, which is the value
       used for the ring itself. */
    int rc = orc_bp_solve(n, s->r, s->A, s->B, s->C, s->a, s->b);
    if (rc)
        return rc;
    for (int32_t i = 0; i < n; ++i) {
        double r = s->r[i];
        s->bp[i] = 0.5 * ((s->a[i] + s->a[i + 1]) * r + (s->b[i] + s->b[i + 1]) / r);
    }
    return ORC_OK;
}

/* Fields at an arbitrary radius x (Eqs. b_theta_plasma..dpsi_dzeta sampled
   off the rings, the "arbitrary radial resolution" remark of Sec. II): no
   self weight, region k = number of rings strictly below x. */
static void fields_at(const slice_ws *s, const beam_slice *bs, double dens,
                      double rho_max, double dxi, double x,
                      double *psi, double *dpr, double *dpz, double *bp, double *bb)
{
    int64_t k = lower_bound(s->r, s->n, x);
    if (!(x > 0.0)) {
        /* on the axis: every ring is outside, d_rho psi and B vanish */
        *psi = s->Ltot + ion_psi(0.0, dens, rho_max);
        *dpr = 0.0;
        *dpz = -(s->Ttot - s->T[0]);
        *bp = 0.0;
        *bb = 0.0;
        return;
    }
    double S = s->S[k];
    *psi = (s->Ltot - s->L[k]) + S * log(x) + ion_psi(x, dens, rho_max);
    *dpr = (S - ion_enclosed(x, dens, rho_max)) / x;
    *dpz = -(s->Ttot - s->T[k]);
    *bp = s->a[k] * x + s->b[k] / x;
    *bb = beam_field(bs, x, dxi);
}

static int ring_fields_ok(const slice_ws *s)
{
    for (int32_t i = 0; i < s->n; ++i) {
        if (!(s->psib[i] > 0.0) || !isfinite(s->psi[i]) || !isfinite(s->dpr[i]) ||
            !isfinite(s->dpz[i]) || !isfinite(s->bp[i]) || !isfinite(s->bb[i]) ||
            !isfinite(s->gam[i]))
            return 0;
    }
    return 1;
}

int orc_slice_fields(int32_t n, const double *rho, const double *ur,
                     const double *w, const double *what, double density, double rho_max,
                     int64_t m, const double *beam_r, const double *beam_qw, double dxi,
                     orc_slice_out *out)
{
    if (n < 1 || !rho || !ur || !w || !what || !out || !(dxi > 0.0))
        return ORC_EINVAL;
    slice_ws s;
    if (ws_alloc(&s, n))
        return ORC_ENOMEM;
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    bpart *parts = (bpart *)malloc((size_t)(m + 1) * sizeof(bpart));
    beam_slice bs = {0, NULL, NULL, NULL};
    if (!order || !parts) {
        free(order);
        free(parts);
        ws_free(&s);
        return ORC_ENOMEM;
    }
    for (int64_t p = 0; p < m; ++p) {
        parts[p].r = beam_r[p];
        parts[p].qw = beam_qw[p];
        parts[p].idx = p;
    }
    int rc = beam_slice_build(&bs, m, parts);
    free(parts);
    if (!rc) {
        for (int32_t i = 0; i < n; ++i)
            order[i] = i;
        rc = slice_core(&s, order, rho, ur, w, what, density, rho_max, &bs, NULL, 1.0, 0.0, NULL, dxi);
    }
    if (!rc) {
        for (int32_t i = 0; i < n; ++i) {
            int32_t id = order[i];
            if (out->order) out->order[i] = id;
            if (out->psi) out->psi[id] = s.psi[i];
            if (out->dpsidr) out->dpsidr[id] = s.dpr[i];
            if (out->dpsidz) out->dpsidz[id] = s.dpz[i];
            if (out->psibar) out->psibar[id] = s.psib[i];
            if (out->gamma) out->gamma[id] = s.gam[i];
            if (out->uz) out->uz[id] = s.uz[i];
            if (out->bb) out->bb[id] = s.bb[i];
            if (out->A) out->A[id] = s.A[i];
            if (out->B) out->B[id] = s.B[i];
            if (out->C) out->C[id] = s.C[i];
            if (out->bp) out->bp[id] = s.bp[i];
        }
        for (int32_t k = 0; k <= n; ++k) {
            if (out->a) out->a[k] = s.a[k];
            if (out->b) out->b[k] = s.b[k];
        }
        for (int64_t q = 0; q < out->nq; ++q) {
            double psi, dpr, dpz, bp, bb;
            fields_at(&s, &bs, density, rho_max, dxi, out->rq[q], &psi, &dpr, &dpz, &bp, &bb);
            if (out->q_ez) out->q_ez[q] = -dpz;
            if (out->q_wr) out->q_wr[q] = -dpr;
            if (out->q_bt) out->q_bt[q] = bp + bb;
            if (out->q_psi) out->q_psi[q] = psi;
            if (out->q_bp) out->q_bp[q] = bp;
            if (out->q_bb) out->q_bb[q] = bb;
            if (out->q_dpsidr) out->q_dpsidr[q] = dpr;
            if (out->q_dpsidz) out->q_dpsidz[q] = dpz;
        }
        if (!ring_fields_ok(&s))
            rc = ORC_ENONFINITE;
    }
    beam_slice_free(&bs);
    free(order);
    ws_free(&s);
    return rc;
}

/* ---------------------------------------------------------------------- */
/* the whole window                                                        */
/* ---------------------------------------------------------------------- */

/* Nearest slice of a beam particle (the beam-grid spacing equals the solver
   step, Sec. III): s = floor(xi/dxi + 1/2). */
static int64_t nearest_slice(double xi, double dxi)
{
    return (int64_t)floor(xi / dxi + 0.5);
}

/* One step of a ring's radius and radial momentum to the next slice
   (Eqs. plasma_particle_motion_1,2 with xi = -zeta), second-order
   Adams-Bashforth (Sec. III) with forward Euler when there is no previous
   slice (have_prev = 0): from (r, u) with the derivatives (fr, fu) of this
   slice and the previous slice's (*frp, *fup); *frp, *fup become this
   slice's.  A ring pushed below the axis reappears at -rho moving the
   other way; f_rho and f_u are odd in (rho, u_r), so its history is
   negated too.  Both marches (one species, two species) step with it. */
static void ab2_step(double r, double u, double fr, double fu, int have_prev, double dxi, double *rho, double *ur,
                     double *frp, double *fup)
{
    if (have_prev) {
        *rho = r + dxi * (1.5 * fr - 0.5 * *frp);
        *ur = u + dxi * (1.5 * fu - 0.5 * *fup);
    } else {
        *rho = r + dxi * fr;
        *ur = u + dxi * fu;
    }
    *frp = fr;
    *fup = fu;
    if (*rho < 0.0) {
        *rho = -*rho;
        *ur = -*ur;
        *frp = -*frp;
        *fup = -*fup;
    }
}

int orc_run(const orc_problem *p, int32_t max_slices, orc_outputs *out)
{
    if (!p || !out || p->n_rings < 1 || !p->edges || !(p->dxi > 0.0) || p->n_steps < 0 ||
        p->cell_density || (p->integrator != ORC_AB2 && p->integrator != ORC_RK4) ||
        p->grid_nr < 0 || (p->grid_nr > 0 && (p->integrator != ORC_AB2 || p->n_species < 1)) ||
        (p->n_beam > 0 && (!p->beam_xi || !p->beam_r || !p->beam_qw)))
        return ORC_EINVAL;
    if (p->grid_nr > 0 && p->beam_species)
        for (int64_t k = 0; k < p->n_beam; ++k)
            if (p->beam_species[k] < 0 || p->beam_species[k] >= p->n_species)
                return ORC_EINVAL;
    for (int32_t j = 0; j < p->n_rings; ++j)
        if (!(p->edges[j + 1] > p->edges[j]))
            return ORC_EINVAL;
    if (p->edges[0] != 0.0)
        return ORC_EINVAL;
    if (p->init_r)
        for (int32_t j = 0; j < p->n_rings; ++j)
            if (!(p->init_r[j] >= 0.0))
                return ORC_EINVAL;
    int32_t n = p->n_rings, ns = p->n_steps;
    int32_t nrun = (max_slices > 0 && max_slices < ns) ? max_slices : ns;
    double rho_max = p->edges[n], dens = p->density, dxi = p->dxi;
    out->status = ORC_OK;
    out->fail_slice = -1;
    out->slices_run = 0;

    /* state by ring id; RK4 scratch: stage state, derivatives, stage order */
    double *st = (double *)calloc((size_t)n * 6, sizeof(double));
    double *rk = (double *)calloc((size_t)n * 7, sizeof(double));
    int32_t *order = (int32_t *)malloc((size_t)n * 2 * sizeof(int32_t));
    int64_t *cnt = (int64_t *)calloc((size_t)ns + 2, sizeof(int64_t));
    bpart *parts = (bpart *)malloc((size_t)(p->n_beam + 1) * sizeof(bpart));
    slice_ws s;
    int rc = ws_alloc(&s, n);
    if (!st || !rk || !order || !cnt || !parts || rc) {
        free(st); free(rk); free(order); free(cnt); free(parts);
        if (!rc) ws_free(&s);
        return ORC_ENOMEM;
    }
    double *rho = st, *ur = st + n, *w = st + 2 * n, *wh = st + 3 * n;
    double *fr_prev = st + 4 * n, *fu_prev = st + 5 * n;
    /* RK4: stage state (rs, us, mirror sign sg), the last stage's
       derivatives (ksr, ksu) and the weighted sums k1 + 2 k2 + 2 k3 + k4 */
    double *rs = rk, *us = rk + n, *sg = rk + 2 * n, *ksr = rk + 3 * n, *ksu = rk + 4 * n;
    double *sum_r = rk + 5 * n, *sum_u = rk + 6 * n;
    int32_t *ord_s = order + n;
    orc_ring_init(n, p->edges, dens, rho, NULL, w, wh);
    for (int32_t j = 0; j < n; ++j)
        order[j] = j;
    int have_prev = 0;
    if (p->init_r) {
        /* a given starting state (weights stay those of the cells) */
        for (int32_t j = 0; j < n; ++j) {
            rho[j] = p->init_r[j];
            ur[j] = p->init_ur ? p->init_ur[j] : 0.0;
        }
        if (p->init_fr && p->init_fu) {
            memcpy(fr_prev, p->init_fr, (size_t)n * sizeof(double));
            memcpy(fu_prev, p->init_fu, (size_t)n * sizeof(double));
            have_prev = 1;
        }
    }

    /* bin the beam by nearest slice (counting sort, stable in caller order) */
    for (int64_t k = 0; k < p->n_beam; ++k) {
        int64_t sl = nearest_slice(p->beam_xi[k], dxi);
        if (sl >= 0 && sl < ns)
            cnt[sl + 1]++;
    }
    for (int32_t sl = 0; sl < ns; ++sl)
        cnt[sl + 1] += cnt[sl];
    {
        int64_t *fill = (int64_t *)malloc(((size_t)ns + 1) * sizeof(int64_t));
        if (!fill) {
            rc = ORC_ENOMEM;
        } else {
            memcpy(fill, cnt, ((size_t)ns + 1) * sizeof(int64_t));
            for (int64_t k = 0; k < p->n_beam; ++k) {
                int64_t sl = nearest_slice(p->beam_xi[k], dxi);
                if (sl >= 0 && sl < ns) {
                    bpart *bp = &parts[fill[sl]++];
                    bp->r = p->beam_r[k];
                    bp->qw = p->beam_qw[k];
                    bp->idx = k;
                }
            }
            free(fill);
        }
    }
    /* particles outside the window get zero fields */
    for (int64_t k = 0; k < p->n_beam; ++k) {
        if (out->ez) out->ez[k] = 0.0;
        if (out->wr) out->wr[k] = 0.0;
        if (out->bt) out->bt[k] = 0.0;
        if (out->psi) out->psi[k] = 0.0;
    }

    /* the adaptive beam grids (Sec. IV): per species nr cells out to (1 +
       1/nr) x its largest radius, so that every particle lies strictly
       inside; node fields [species][nr + 1][psi, dpr, dpz, bt] */
    const int32_t nr = p->grid_nr, nsp = nr > 0 ? p->n_species : 0;
    double *agR = NULL, *agB = NULL, *agF = NULL;
    ag_slice ag = {nsp, nr, NULL, NULL};
    if (nr > 0 && !rc) {
        agR = (double *)calloc((size_t)nsp, sizeof(double));
        agB = (double *)calloc((size_t)nsp * (nr + 1), sizeof(double));
        agF = (double *)calloc((size_t)nsp * (nr + 1) * 4, sizeof(double));
        if (!agR || !agB || !agF) {
            rc = ORC_ENOMEM;
        } else {
            for (int64_t k = 0; k < p->n_beam; ++k) {
                int32_t b = p->beam_species ? p->beam_species[k] : 0;
                if (p->beam_r[k] > agR[b]) agR[b] = p->beam_r[k];
            }
            for (int32_t b = 0; b < nsp; ++b) {
                if (p->grid_rmax > 0.0) {
                    /* the regular intermediate grid: a fixed extent that every
                       particle must lie below */
                    if (!(agR[b] < p->grid_rmax))
                        rc = ORC_EINVAL;
                    agR[b] = p->grid_rmax;
                } else {
                    agR[b] = (agR[b] > 1e-12 ? agR[b] : 1e-12) * (1.0 + 1.0 / nr);
                }
            }
            ag.R = agR;
            ag.B = agB;
        }
    }

    for (int32_t sl = 0; sl < nrun && !rc; ++sl) {
        beam_slice bs = {0, NULL, NULL, NULL};
        rc = beam_slice_build(&bs, cnt[sl + 1] - cnt[sl], parts + cnt[sl]);
        if (rc)
            break;
        if (nr > 0) {
            /* B^(b) at the grid nodes: each particle's charge reaches the
               nodes strictly above it */
            memset(agB, 0, (size_t)nsp * (nr + 1) * sizeof(double));
            for (int64_t q = 0; q < bs.m; ++q) {
                int32_t b = p->beam_species ? p->beam_species[bs.idx[q]] : 0;
                double dr = agR[b] / nr;
                int32_t j = ag_cell(bs.r[q], dr, nr) + 1;  /* the first node above the particle */
                agB[(size_t)b * (nr + 1) + j] += p->beam_qw[bs.idx[q]];
            }
            for (int32_t b = 0; b < nsp; ++b) {
                double *B = agB + (size_t)b * (nr + 1), acc = 0.0, dr = agR[b] / nr;
                B[0] = 0.0;
                for (int32_t j = 1; j <= nr; ++j) {
                    acc += B[j];
                    B[j] = acc / (ORC_2PI * dxi * ((double)j * dr));
                }
            }
        }
        rc = slice_core(&s, order, rho, ur, w, wh, dens, rho_max, &bs, NULL, 1.0, 0.0, nr > 0 ? &ag : NULL, dxi);
        if (rc) {
            beam_slice_free(&bs);
            break;
        }
        size_t row = (size_t)sl * (size_t)n;
        for (int32_t i = 0; i < n; ++i) {
            int32_t id = order[i];
            if (out->ring_r) out->ring_r[row + id] = s.r[i];
            if (out->ring_ur) out->ring_ur[row + id] = s.u[i];
            if (out->ring_psi) out->ring_psi[row + id] = s.psi[i];
            if (out->ring_dpsidr) out->ring_dpsidr[row + id] = s.dpr[i];
            if (out->ring_dpsidz) out->ring_dpsidz[row + id] = s.dpz[i];
            if (out->ring_bp) out->ring_bp[row + id] = s.bp[i];
            if (out->ring_bb) out->ring_bb[row + id] = s.bb[i];
            if (out->ring_psibar) out->ring_psibar[row + id] = s.psib[i];
            if (out->ring_gamma) out->ring_gamma[row + id] = s.gam[i];
            if (out->ring_uz) out->ring_uz[row + id] = s.uz[i];
            if (out->ring_frprev) out->ring_frprev[row + id] = have_prev ? fr_prev[id] : 0.0;
            if (out->ring_fuprev) out->ring_fuprev[row + id] = have_prev ? fu_prev[id] : 0.0;
        }
        for (int32_t j = 0; j < out->n_snap && out->snap; ++j) {
            if (out->snap_slice[j] != sl)
                continue;
            double *sn = out->snap + (size_t)j * ORC_SNAP_FIELDS * (size_t)n;
            for (int32_t i = 0; i < n; ++i) {
                int32_t id = order[i];
                sn[id] = s.r[i];
                sn[n + id] = s.u[i];
                sn[2 * (size_t)n + id] = s.psi[i];
                sn[3 * (size_t)n + id] = s.dpr[i];
                sn[4 * (size_t)n + id] = s.dpz[i];
                sn[5 * (size_t)n + id] = s.bp[i];
                sn[6 * (size_t)n + id] = s.bb[i];
                sn[7 * (size_t)n + id] = have_prev ? fr_prev[id] : 0.0;
                sn[8 * (size_t)n + id] = have_prev ? fu_prev[id] : 0.0;
            }
        }
        /* fields on the beam particles of this slice: directly (a9), or from
           the grid nodes (the plasma fields evaluated there, B^(b) of all
           grids) by linear interpolation in r */
        if (nr > 0) {
            for (int32_t b = 0; b < nsp; ++b) {
                double dr = agR[b] / nr;
                for (int32_t j = 0; j <= nr; ++j) {
                    double x = (double)j * dr, psi, dpr, dpz, bpv, bbv;
                    fields_at(&s, &bs, dens, rho_max, dxi, x, &psi, &dpr, &dpz, &bpv, &bbv);
                    double *F = agF + ((size_t)b * (nr + 1) + j) * 4;
                    F[0] = psi;
                    F[1] = dpr;
                    F[2] = dpz;
                    F[3] = bpv + (j > 0 ? ag_field(&ag, x) : 0.0);
                }
            }
        }
        for (int64_t q = 0; q < bs.m; ++q) {
            double psi, dpr, dpz, bpv, bbv;
            int64_t k = bs.idx[q];
            if (nr > 0) {
                int32_t b = p->beam_species ? p->beam_species[k] : 0;
                double dr = agR[b] / nr, x = bs.r[q];
                int32_t j = ag_cell(x, dr, nr);
                double t = (x - (double)j * dr) / dr;
                const double *F0 = agF + ((size_t)b * (nr + 1) + j) * 4, *F1 = F0 + 4;
                psi = (1.0 - t) * F0[0] + t * F1[0];
                dpr = (1.0 - t) * F0[1] + t * F1[1];
                dpz = (1.0 - t) * F0[2] + t * F1[2];
                bpv = (1.0 - t) * F0[3] + t * F1[3];
                bbv = 0.0;
            } else {
                fields_at(&s, &bs, dens, rho_max, dxi, bs.r[q], &psi, &dpr, &dpz, &bpv, &bbv);
            }
            if (out->ez) out->ez[k] = -dpz;
            if (out->wr) out->wr[k] = -dpr;
            if (out->bt) out->bt[k] = bpv + bbv;
            if (out->psi) out->psi[k] = psi;
        }
        out->slices_run = sl + 1;
        if (!ring_fields_ok(&s)) {
            beam_slice_free(&bs);
            out->status = ORC_ENONFINITE;
            out->fail_slice = sl;
            break;
        }
        if (p->integrator == ORC_RK4) {
            /* classical RK4 over the slice (the integrator of Sec. II's
               reference model): k1 at (xi_n, y_n) from the fields above,
               k2, k3 at xi_n + dxi/2 with the mean of slices n and n+1 as
               the beam source, k4 at xi_n + dxi with slice n+1's.  A stage
               state below the axis is evaluated mirrored (rho, u -> -rho,
               -u) and its derivative mirrored back: the ring equations are
               odd in (rho, u).  Each stage sorts from the slice's order. */
            beam_slice bsn = {0, NULL, NULL, NULL};
            rc = sl + 1 < ns ? beam_slice_build(&bsn, cnt[sl + 2] - cnt[sl + 1], parts + cnt[sl + 1])
                             : beam_slice_build(&bsn, 0, parts);
            if (rc) {
                beam_slice_free(&bs);
                break;
            }
            for (int32_t i = 0; i < n; ++i) {
                int32_t id = order[i];
                double pb = s.psib[i];
                ksr[id] = s.u[i] / pb;
                ksu[id] = s.gam[i] * s.dpr[i] / pb - (s.bp[i] + s.bb[i]);
                sum_r[id] = ksr[id];
                sum_u[id] = ksu[id];
            }
            static const double cs[3] = {0.5, 0.5, 1.0}, ws[3] = {2.0, 2.0, 1.0};
            int bad = 0;
            for (int stg = 0; stg < 3 && !bad; ++stg) {
                for (int32_t id = 0; id < n; ++id) {
                    double r = rho[id] + cs[stg] * dxi * ksr[id];
                    double u = ur[id] + cs[stg] * dxi * ksu[id];
                    sg[id] = r < 0.0 ? -1.0 : 1.0;
                    rs[id] = sg[id] * r;
                    us[id] = sg[id] * u;
                }
                memcpy(ord_s, order, (size_t)n * sizeof(int32_t));
                if (stg < 2)
                    rc = slice_core(&s, ord_s, rs, us, w, wh, dens, rho_max, &bs, &bsn, 0.5, 0.5, NULL, dxi);
                else
                    rc = slice_core(&s, ord_s, rs, us, w, wh, dens, rho_max, &bsn, NULL, 1.0, 0.0, NULL, dxi);
                if (rc)
                    break;
                if (!ring_fields_ok(&s)) {
                    bad = 1;
                    break;
                }
                for (int32_t i = 0; i < n; ++i) {
                    int32_t id = ord_s[i];
                    double pb = s.psib[i];
                    ksr[id] = sg[id] * (s.u[i] / pb);
                    ksu[id] = sg[id] * (s.gam[i] * s.dpr[i] / pb - (s.bp[i] + s.bb[i]));
                    sum_r[id] += ws[stg] * ksr[id];
                    sum_u[id] += ws[stg] * ksu[id];
                }
            }
            beam_slice_free(&bsn);
            beam_slice_free(&bs);
            if (rc)
                break;
            if (bad) {
                out->status = ORC_ENONFINITE;
                out->fail_slice = sl;
                break;
            }
            for (int32_t id = 0; id < n; ++id) {
                rho[id] += dxi / 6.0 * sum_r[id];
                ur[id] += dxi / 6.0 * sum_u[id];
                if (rho[id] < 0.0) {
                    rho[id] = -rho[id];
                    ur[id] = -ur[id];
                }
            }
            continue;
        }
        beam_slice_free(&bs);
        /* evolve rho, u_r to the next slice (Eqs. plasma_particle_motion_1,2
           with xi = -zeta; second-order Adams-Bashforth, Sec. III; forward
           Euler on the first step) */
        for (int32_t i = 0; i < n; ++i) {
            int32_t id = order[i];
            double pb = s.psib[i];
            double fr = s.u[i] / pb;
            double fu = s.gam[i] * s.dpr[i] / pb - (s.bp[i] + s.bb[i]);
            ab2_step(s.r[i], s.u[i], fr, fu, have_prev, dxi, &rho[id], &ur[id], &fr_prev[id], &fu_prev[id]);
        }
        have_prev = 1;
    }
    if (out->final_r)
        memcpy(out->final_r, rho, (size_t)n * sizeof(double));
    if (out->final_ur)
        memcpy(out->final_ur, ur, (size_t)n * sizeof(double));
    free(agR);
    free(agB);
    free(agF);
    free(st);
    free(rk);
    free(order);
    free(cnt);
    free(parts);
    ws_free(&s);
    return rc;
}

/* ====================================================================== */
/* Mobile ions: two ring species (Sec. II, "key algorithmic adjustments")   */
/* ====================================================================== */
/*
 * Electrons (q = -1, m = 1) and ions (q = +Z, m = M electron masses) are
 * both rings, initialised on the same cell edges from the same density
 * profile (Eq. macroparticle_weight), the ions with density n/Z so that the
 * plasma is neutral.  With the signed charge weight c_j = -q_j w_j
 * (electrons +w_j, ions -w_j for Z w^ion = w^e) the sums of Sec. II are, per
 * species,
 *   psi(rho)      = sum_j c_j ln max(rho, rho_j)                 (Eq. psi)
 *   d_rho psi     = (1/rho) sum_{rho_j < rho} c_j                (Eq. dpsi_dr)
 *   d_zeta psi    = -sum_{rho_j >= rho} c_j u_j / (rho_j psibar_j)
 *                   (Eq. dpsi_dzeta; the sign reading of zeta_derivative())
 *   psibar_j      = 1 - (q_j/m_j) psi_j                           (Eq. cold_plasma_constant)
 * Each species is solved on its own rings (with the self weight at its own
 * ring), and its fields reach the rings of the other species by linear
 * interpolation between its own ring values: at a radius x, j = the last ring
 * of the species below x, F(x) = F_j + (F_{j+1} - F_j)(x - rho_j)/(rho_{j+1} -
 * rho_j).  Below the species' first ring the interpolation runs from the
 * axis value (d_rho psi = 0, B = 0); between its last ring and the plasma's
 * initial outer edge rho_max = edges[N] it runs to the exact value at
 * rho_max (all of the species' charge inside); beyond both the species'
 * field is smooth and is taken exactly.  For an unperturbed uniform species
 * this reproduces the continuous column: its d_rho psi is linear in rho.  B_theta^(p) comes from the electrons only
 * (Eqs. b_coeffs_1..3 over electron rings with the total fields); the ions
 * see it interpolated.  Beam particles see the exact sums of both species.
 * Ions move by Eqs. plasma_particle_motion_1,2 with q/m = Z/M: in xi = -zeta,
 *   d rho / d xi = u / psibar,  d u / d xi = -(q/m) (gamma d_rho psi / psibar - B_theta).
 */

typedef struct {
    int32_t n;
    double qm;                     /* q / m */
    double edge;                   /* the plasma's initial outer edge rho_max */
    double *r, *u, *c, *ch;        /* sorted state, charge weight, self weight */
    double *S, *L, *T;             /* exclusive prefix sums [n+1] */
    double Stot, Ltot, Ttot;
    double *psi_o, *dpr_o, *dpz_o; /* own-species fields at own rings */
    double *psi, *dpr, *dpz;       /* totals at own rings */
    double *psib, *gam, *uz, *t, *bb, *bp;
    int32_t *order, *tmp;
} species_ws;

static int sp_alloc(species_ws *s, int32_t n, double qm, double edge)
{
    memset(s, 0, sizeof(*s));
    s->n = n;
    s->qm = qm;
    s->edge = edge;
    size_t m = (size_t)n + 1;
    double *blk = (double *)calloc(m * 20, sizeof(double));
    s->order = (int32_t *)malloc(m * sizeof(int32_t));
    s->tmp = (int32_t *)malloc(m * sizeof(int32_t));
    if (!blk || !s->order || !s->tmp) {
        free(blk);
        free(s->order);
        free(s->tmp);
        return ORC_ENOMEM;
    }
    double **f[] = {&s->r, &s->u, &s->c, &s->ch, &s->S, &s->L, &s->T, &s->psi_o, &s->dpr_o,
                    &s->dpz_o, &s->psi, &s->dpr, &s->dpz, &s->psib, &s->gam, &s->uz, &s->t,
                    &s->bb, &s->bp};
    for (size_t k = 0; k < sizeof(f) / sizeof(f[0]); ++k)
        *f[k] = blk + k * m;
    for (int32_t j = 0; j < n; ++j)
        s->order[j] = j;
    return ORC_OK;
}

static void sp_free(species_ws *s)
{
    free(s->r);
    free(s->order);
    free(s->tmp);
    memset(s, 0, sizeof(*s));
}

/* Sort the species (stable w.r.t. its previous order), gather the beam
   source and its own psi, d_rho psi at its rings (self weight in d_rho psi). */
static void sp_own_potential(species_ws *s, const double *rho_id, const double *ur_id,
                             const double *c_id, const double *ch_id, const beam_slice *bs, double dxi)
{
    int32_t n = s->n;
    stable_sort_ids(n, s->order, rho_id, s->tmp);
    for (int32_t i = 0; i < n; ++i) {
        int32_t id = s->order[i];
        s->r[i] = rho_id[id];
        s->u[i] = ur_id[id];
        s->c[i] = c_id[id];
        s->ch[i] = ch_id[id];
        s->bb[i] = beam_field(bs, s->r[i], dxi);
    }
    double aS = 0.0, aL = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        s->S[i] = aS;
        s->L[i] = aL;
        aS += s->c[i];
        aL += s->c[i] * log(s->r[i]);
    }
    s->S[n] = aS;
    s->L[n] = aL;
    s->Stot = aS;
    s->Ltot = aL;
    for (int32_t i = 0; i < n; ++i) {
        double r = s->r[i];
        s->psi_o[i] = (s->Ltot - s->L[i]) + s->S[i] * log(r);
        s->dpr_o[i] = (s->S[i] + s->ch[i]) / r;
    }
}

/* The species' own d_zeta psi at its rings (needs psibar, so the totals of
   psi first): T prefix of t = c u / (rho psibar), self weight on the ring's
   own term. */
static void sp_own_dzeta(species_ws *s)
{
    int32_t n = s->n;
    double aT = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        s->T[i] = aT;
        aT += s->t[i];
    }
    s->T[n] = aT;
    s->Ttot = aT;
    for (int32_t i = 0; i < n; ++i) {
        double above = s->Ttot - s->T[i + 1];
        s->dpz_o[i] = -(above + (1.0 - s->ch[i] / s->c[i]) * s->t[i]);
    }
}

/* The species' field outside all its rings at radius x > 0 (which = 0, 1,
   2 for psi, d_rho psi, d_zeta psi; 3 for B^(p), whose outermost region has
   a_N = 0 and b_N = bN). */
static double sp_outside(const species_ws *s, int which, double bN, double x)
{
    if (which == 0) return s->Stot * log(x);
    if (which == 1) return s->Stot / x;
    if (which == 2) return 0.0;
    return bN / x;
}

/* Linear interpolation of a species' ring values F[0..n) (radius order r)
   at radius x (the multi-species gather of Sec. II).  F0: the value on the
   axis; the node beyond the last ring is rho_max with the outside value. */
static double sp_interp(const species_ws *s, const double *F, double F0, int which, double bN,
                        double x)
{
    int32_t n = s->n;
    int64_t k = lower_bound(s->r, n, x);   /* rings strictly below x */
    if (k >= n) {
        double rl = s->r[n - 1];
        if (x >= s->edge || !(s->edge > rl))
            return sp_outside(s, which, bN, x);
        double Fe = sp_outside(s, which, bN, s->edge);
        return F[n - 1] + (Fe - F[n - 1]) * (x - rl) / (s->edge - rl);
    }
    double rl = k > 0 ? s->r[k - 1] : 0.0;
    double Fl = k > 0 ? F[k - 1] : F0;
    double rh = s->r[k], Fh = F[k];
    if (!(rh > rl))
        return Fh;
    return Fl + (Fh - Fl) * (x - rl) / (rh - rl);
}

/* psi, d_rho psi, d_zeta psi of one species alone at an off-ring radius x
   (exact sums, no self weight): what a beam particle sees of it. */
static void sp_exact_at(const species_ws *s, double x, double *psi, double *dpr, double *dpz)
{
    if (!(x > 0.0)) {
        *psi = s->Ltot;
        *dpr = 0.0;
        *dpz = -s->Ttot;
        return;
    }
    int64_t k = lower_bound(s->r, s->n, x);
    *psi = (s->Ltot - s->L[k]) + s->S[k] * log(x);
    *dpr = s->S[k] / x;
    *dpz = -(s->Ttot - s->T[k]);
}

int orc_run_ions(const orc_problem *p, double ion_z, double ion_m, int32_t max_slices,
                 orc_outputs *out)
{
    if (!p || !out || p->n_rings < 1 || !p->edges || !(p->dxi > 0.0) || p->n_steps < 0 ||
        !(ion_z > 0.0) || !(ion_m > 0.0) || p->init_r ||
        (p->n_beam > 0 && (!p->beam_xi || !p->beam_r || !p->beam_qw)))
        return ORC_EINVAL;
    if (p->cell_density)
        for (int32_t j = 0; j < p->n_rings; ++j)
            if (!(p->cell_density[j] > 0.0))
                return ORC_EINVAL;
    for (int32_t j = 0; j < p->n_rings; ++j)
        if (!(p->edges[j + 1] > p->edges[j]))
            return ORC_EINVAL;
    if (p->edges[0] != 0.0)
        return ORC_EINVAL;
    const int32_t n = p->n_rings, ns = p->n_steps, n2 = 2 * n;
    const int32_t nrun = (max_slices > 0 && max_slices < ns) ? max_slices : ns;
    const double dxi = p->dxi;
    out->status = ORC_OK;
    out->fail_slice = -1;
    out->slices_run = 0;

    /* state by ring id: electrons 0..n-1, ions n..2n-1 */
    double *st = (double *)calloc((size_t)n2 * 6, sizeof(double));
    int64_t *cnt = (int64_t *)calloc((size_t)ns + 2, sizeof(int64_t));
    bpart *parts = (bpart *)malloc((size_t)(p->n_beam + 1) * sizeof(bpart));
    double *ab = (double *)malloc(((size_t)n + 1) * 5 * sizeof(double));
    species_ws sp[2];
    int rc = sp_alloc(&sp[0], n, -1.0, p->edges[n]);
    if (!rc) {
        rc = sp_alloc(&sp[1], n, isinf(ion_m) ? 0.0 : ion_z / ion_m, p->edges[n]);
        if (rc) sp_free(&sp[0]);
    }
    if (!st || !cnt || !parts || !ab || rc) {
        free(st); free(cnt); free(parts); free(ab);
        if (!rc) { sp_free(&sp[0]); sp_free(&sp[1]); }
        return ORC_ENOMEM;
    }
    double *rho = st, *ur = st + n2, *cw = st + 2 * n2, *ch = st + 3 * n2;
    double *fr_prev = st + 4 * n2, *fu_prev = st + 5 * n2;
    double *A = ab, *B = ab + (n + 1), *Cc = ab + 2 * (n + 1), *ak = ab + 3 * (n + 1),
           *bk = ab + 4 * (n + 1);
    double *w0 = (double *)malloc((size_t)n * 2 * sizeof(double));
    if (!w0) {
        free(st); free(cnt); free(parts); free(ab);
        sp_free(&sp[0]); sp_free(&sp[1]);
        return ORC_ENOMEM;
    }
    /* Eq. macroparticle_weight with the cell's own density (uniform within
       the cell), and the self weight of the cell below the ring */
    for (int32_t j = 0; j < n; ++j) {
        double dens_j = p->cell_density ? p->cell_density[j] : p->density;
        orc_ring_init(1, p->edges + j, dens_j, rho + j, NULL, w0 + j, w0 + n + j);
    }
    for (int32_t j = 0; j < n; ++j) {
        rho[n + j] = rho[j];
        cw[j] = w0[j];          /* electrons: c = -q w = +w */
        ch[j] = w0[n + j];
        cw[n + j] = -w0[j];     /* ions: w^ion = w / Z, c = -Z w^ion */
        ch[n + j] = -w0[n + j];
    }
    free(w0);

    /* nearest-slice binning of the beam, as orc_run */
    for (int64_t k = 0; k < p->n_beam; ++k) {
        int64_t sl = nearest_slice(p->beam_xi[k], dxi);
        if (sl >= 0 && sl < ns)
            cnt[sl + 1]++;
    }
    for (int32_t sl = 0; sl < ns; ++sl)
        cnt[sl + 1] += cnt[sl];
    {
        int64_t *fill = (int64_t *)malloc(((size_t)ns + 1) * sizeof(int64_t));
        if (!fill) {
            rc = ORC_ENOMEM;
        } else {
            memcpy(fill, cnt, ((size_t)ns + 1) * sizeof(int64_t));
            for (int64_t k = 0; k < p->n_beam; ++k) {
                int64_t sl = nearest_slice(p->beam_xi[k], dxi);
                if (sl >= 0 && sl < ns) {
                    bpart *bp = &parts[fill[sl]++];
                    bp->r = p->beam_r[k];
                    bp->qw = p->beam_qw[k];
                    bp->idx = k;
                }
            }
            free(fill);
        }
    }
    for (int64_t k = 0; k < p->n_beam; ++k) {
        if (out->ez) out->ez[k] = 0.0;
        if (out->wr) out->wr[k] = 0.0;
        if (out->bt) out->bt[k] = 0.0;
        if (out->psi) out->psi[k] = 0.0;
    }

    int have_prev = 0;
    for (int32_t sl = 0; sl < nrun && !rc; ++sl) {
        beam_slice bs = {0, NULL, NULL, NULL};
        rc = beam_slice_build(&bs, cnt[sl + 1] - cnt[sl], parts + cnt[sl]);
        if (rc)
            break;
        species_ws *e = &sp[0], *io = &sp[1];
        /* 1. each species: sort, beam source, own psi and d_rho psi */
        sp_own_potential(e, rho, ur, cw, ch, &bs, dxi);
        sp_own_potential(io, rho + n, ur + n, cw + n, ch + n, &bs, dxi);
        /* 2. totals of psi, d_rho psi at every ring (own + the other species
              interpolated), then psibar, gamma, u_z, t */
        for (int s = 0; s < 2; ++s) {
            species_ws *me = &sp[s], *ot = &sp[1 - s];
            for (int32_t i = 0; i < n; ++i) {
                double x = me->r[i];
                me->psi[i] = me->psi_o[i] + sp_interp(ot, ot->psi_o, ot->Ltot, 0, 0.0, x);
                me->dpr[i] = me->dpr_o[i] + sp_interp(ot, ot->dpr_o, 0.0, 1, 0.0, x);
                double pb = 1.0 - me->qm * me->psi[i];
                double u = me->u[i];
                me->psib[i] = pb;
                me->gam[i] = (1.0 + u * u + pb * pb) / (2.0 * pb);
                me->uz[i] = (1.0 + u * u - pb * pb) / (2.0 * pb);
                me->t[i] = me->c[i] * u / (x * pb);
            }
        }
        /* 3. d_zeta psi: own, then the totals */
        sp_own_dzeta(e);
        sp_own_dzeta(io);
        for (int s = 0; s < 2; ++s) {
            species_ws *me = &sp[s], *ot = &sp[1 - s];
            for (int32_t i = 0; i < n; ++i)
                me->dpz[i] = me->dpz_o[i] + sp_interp(ot, ot->dpz_o, -ot->Ttot, 2, 0.0, me->r[i]);
        }
        /* 4. B_theta^(p) from the electrons (Eqs. b_coeffs_1..3, q = -1, m = 1,
              with the total fields at the electron rings), Eq. ai_bi */
        for (int32_t i = 0; i < n; ++i) {
            double r = e->r[i], u = e->u[i], w = e->c[i], pb = e->psib[i];
            double g = e->gam[i], dpr = e->dpr[i], dpz = e->dpz[i];
            double wr = w / r;
            A[i] = wr / pb;
            B[i] = -wr * g * dpr / (pb * pb) + wr * e->bb[i] / pb + (w / (r * r)) * u * u / (pb * pb) +
                   wr * u * u * dpr / (pb * pb * pb) - wr * u * dpz / (pb * pb);
            Cc[i] = -wr * (g / pb - 1.0 - u * u / (pb * pb));
        }
        rc = orc_bp_solve(n, e->r, A, B, Cc, ak, bk);
        if (rc) {
            beam_slice_free(&bs);
            break;
        }
        for (int32_t i = 0; i < n; ++i) {
            double r = e->r[i];
            e->bp[i] = 0.5 * ((ak[i] + ak[i + 1]) * r + (bk[i] + bk[i + 1]) / r);
        }
        /* the ions see the electrons' B^(p) interpolated */
        for (int32_t i = 0; i < n; ++i)
            io->bp[i] = sp_interp(e, e->bp, 0.0, 3, bk[n], io->r[i]);
        /* ring dumps (ids: electrons 0..n-1, ions n..2n-1) */
        size_t row = (size_t)sl * (size_t)n2;
        for (int s = 0; s < 2; ++s) {
            species_ws *me = &sp[s];
            for (int32_t i = 0; i < n; ++i) {
                int32_t id = me->order[i] + s * n;
                if (out->ring_r) out->ring_r[row + id] = me->r[i];
                if (out->ring_ur) out->ring_ur[row + id] = me->u[i];
                if (out->ring_psi) out->ring_psi[row + id] = me->psi[i];
                if (out->ring_dpsidr) out->ring_dpsidr[row + id] = me->dpr[i];
                if (out->ring_dpsidz) out->ring_dpsidz[row + id] = me->dpz[i];
                if (out->ring_bp) out->ring_bp[row + id] = me->bp[i];
                if (out->ring_bb) out->ring_bb[row + id] = me->bb[i];
                if (out->ring_psibar) out->ring_psibar[row + id] = me->psib[i];
                if (out->ring_gamma) out->ring_gamma[row + id] = me->gam[i];
                if (out->ring_uz) out->ring_uz[row + id] = me->uz[i];
                if (out->ring_frprev) out->ring_frprev[row + id] = have_prev ? fr_prev[id] : 0.0;
                if (out->ring_fuprev) out->ring_fuprev[row + id] = have_prev ? fu_prev[id] : 0.0;
            }
        }
        /* 5. beam particles: exact sums of both species, electron B^(p) */
        for (int64_t q = 0; q < bs.m; ++q) {
            double x = bs.r[q], psi = 0.0, dpr = 0.0, dpz = 0.0, bpv = 0.0;
            for (int s = 0; s < 2; ++s) {
                double a1, a2, a3;
                sp_exact_at(&sp[s], x, &a1, &a2, &a3);
                psi += a1;
                dpr += a2;
                dpz += a3;
            }
            if (x > 0.0) {
                int64_t k = lower_bound(e->r, n, x);
                bpv = ak[k] * x + bk[k] / x;
            }
            double bbv = beam_field(&bs, x, dxi);
            int64_t k = bs.idx[q];
            if (out->ez) out->ez[k] = -dpz;
            if (out->wr) out->wr[k] = -dpr;
            if (out->bt) out->bt[k] = bpv + bbv;
            if (out->psi) out->psi[k] = psi;
        }
        beam_slice_free(&bs);
        out->slices_run = sl + 1;
        /* guard (c11) over both species */
        int ok = 1;
        for (int s = 0; s < 2 && ok; ++s)
            for (int32_t i = 0; i < n; ++i) {
                species_ws *me = &sp[s];
                if (!(me->psib[i] > 0.0) || !isfinite(me->psi[i]) || !isfinite(me->dpr[i]) ||
                    !isfinite(me->dpz[i]) || !isfinite(me->bp[i]) || !isfinite(me->bb[i]) ||
                    !isfinite(me->gam[i])) {
                    ok = 0;
                    break;
                }
            }
        if (!ok) {
            out->status = ORC_ENONFINITE;
            out->fail_slice = sl;
            break;
        }
        /* 6. push both species (AB2, Euler start, axis reflection) */
        for (int s = 0; s < 2; ++s) {
            species_ws *me = &sp[s];
            for (int32_t i = 0; i < n; ++i) {
                int32_t id = me->order[i] + s * n;
                double pb = me->psib[i];
                double fr = me->u[i] / pb;
                double fu = -me->qm * (me->gam[i] * me->dpr[i] / pb - (me->bp[i] + me->bb[i]));
                ab2_step(me->r[i], me->u[i], fr, fu, have_prev, dxi, &rho[id], &ur[id], &fr_prev[id],
                         &fu_prev[id]);
            }
        }
        have_prev = 1;
    }
    if (out->final_r)
        memcpy(out->final_r, rho, (size_t)n2 * sizeof(double));
    if (out->final_ur)
        memcpy(out->final_ur, ur, (size_t)n2 * sizeof(double));
    free(st);
    free(cnt);
    free(parts);
    free(ab);
    sp_free(&sp[0]);
    sp_free(&sp[1]);
    return rc;
}
