// march.cuh -- the per-slice march of one wake per thread block.
//
// One block owns one wake.  Rings live in radius order in the wake's device
// arrays; thread t owns the contiguous chunk [t*K, t*K+K) of sorted
// positions (K = ceil(n / blockDim)).  Each slice runs the chain of Sec. III:
//   a2 sort (check; bitonic sort in shared memory only if out of order)
//   a3 B^(b) at the rings (binary search in the slice's sorted beam radii)
//   a4 block scan of (sum w, sum w ln rho)                   (Eqs. dpsi_dr, psi)
//   a5 psi, d_rho psi (self weight), psibar, gamma            (Eq. plasma_particle_motion_3/4)
//   a6 block scan of t = w u/(rho psibar) -> d_zeta psi        (Eq. dpsi_dzeta)
//   a7 A, B, C                                                (Eqs. b_coeffs_1..3)
//   a8 B^(p): the discrete solution of Eq. ai_bi with b_0 = 0, a_N = 0 from
//            the regular (forward) and decaying (backward) homogeneous
//            solutions and the discrete Green's function; the same solution
//            as App. A's shooting without its growing-mode cancellation
//   a9 fields on the beam particles of the slice
//   a10 AB2 push with axis reflection
#pragma once

#include <cooperative_groups.h>

#include "common.cuh"

namespace gbwake {


enum { MODE_MARCH = 0, MODE_QUERY = 1 };

constexpr int kScanBytes = 33 * 64;  // block-scan scratch (33 values of <= 64 B)
constexpr int kMaxGridSpecies = 8;   // beam species with adaptive grids

template <class P>
struct WakeDev {
    using R = typename P::R;
    using A = typename P::A;
    int32_t n, n_steps, n_pad;
    int32_t stage;  // STAGE_* flags (stage.cuh): bulk-copy staging of the beam arrays
    double dxi, density, rho_max;
    const R* w;   // [n] by ring id
    const R* wh;  // [n] by ring id
    // mixed path: per-ring constants by id, 3 float4 each, split float-float
    // from FP64: {rho0, ln rho0}, {w, what}, {w ln rho0, 0}
    const float4* ctab;
    R* rho[2];
    R* rho_lo;    // low part of rho (mixed path: rho = rho + rho_lo in float-float)
    R* ur[2];
    R* frho[2];
    R* fur[2];
    int32_t* rid[2];
    // per-ring scratch, sorted order
    R *bb, *psib, *gam, *dpr, *tt, *cA, *cB, *cC;
    // per-region arrays [n+1]
    A *regS, *regL;
    R *regT, *ak, *bk, *Ra, *Rb, *Da, *Db;
    // binned beam
    int64_t nb;
    const int32_t* boff;  // [n_steps+1]
    const R *br, *bE, *bQs, *bTot;
    R *out_ez, *out_wr, *out_bt, *out_psi;
    // dumps [n_steps][n] by ring id (nullable)
    R *dump_r, *dump_ur, *dump_psi, *dump_dpr, *dump_dpz, *dump_bp, *dump_bb;
    int32_t* ctl;
    // query mode
    int64_t nq;
    const double* rq;
    R *q_ez, *q_wr, *q_bt, *q_psi;
    // > 0: a march launch stops at the first slice boundary this many ns
    // after its start (on-chip kernels; batched steps of a serving loop)
    int64_t budget_ns;
    // mobile ions (march_ions.cuh): n_ion > 0 rings per species, n = 2 n_ion,
    // electrons at ids [0, n_ion), ions at [n_ion, n); w, wh are the signed
    // charge weights -q w; ion_qm = Z / M; own-species fields per ring
    int32_t n_ion, pad1;
    double ion_qm;
    A *psio, *dpro;
    R* dpzo;
    // RK4 (march_rk4.cuh): stage state (radius hi/lo, u, mirror sign), the
    // last stage's derivatives, the stage's radius order
    R *rk_r, *rk_rlo, *rk_u, *rk_sg, *rk_kr, *rk_ku;
    int32_t* rk_perm;
    // adaptive beam grids (Sec. IV; FP64): grid_nr > 0 radial cells per
    // beam species out to (1 + 1/grid_nr) x the species' largest radius
    // (ag_rmax, from the preparation); species of caller particle k: the
    // last s with sp_begin[s] <= k; bidx: binned -> caller index; qw: the
    // caller's charge x weight; agB: B^(b) at the nodes [species][nr + 1];
    // agF: the node fields [species][nr + 1][psi, d_rho psi, d_zeta psi, B]
    int32_t grid_nr, n_species;
    double grid_rmax;  // > 0: every grid's fixed extent
    int64_t sp_begin[kMaxGridSpecies + 1];
    const int32_t* bidx;
    const double* qw;
    const double* rc;  // the caller's beam radii (FP64)
    const double* ag_rmax;
    R *agB, *agF;
};

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// records when the march launch began (t0) and now finishes a wake
__device__ __forceinline__ void put_march_times(int32_t* ctl, uint64_t t0) {
    reinterpret_cast<unsigned long long*>(ctl + CTL_T_BEGIN)[0] = t0;
    reinterpret_cast<unsigned long long*>(ctl + CTL_T_END)[0] = global_ns();
}

// ion column: enclosed charge n min(x, rho_max)^2 / 2 and its potential
template <class A, class R>
__device__ __forceinline__ A ion_enclosed(R x, R rmax, R half_n, A Imax) {
    if (x < rmax) return acc_mul_r(acc_sq(x), half_n);
    return Imax;
}
template <class A, class R>
__device__ __forceinline__ A ion_psi(R x, R rmax, R quarter_n, A Imax, A c0) {
    if (x <= rmax) return acc_sub(c0, acc_mul_r(acc_sq(x), quarter_n));
    return acc_mul_r(Imax, -real_log(x));
}

// Node index j with j dr <= x < (j + 1) dr for x >= 0, clamped to [0, nr - 1]
// (the comparison as written, so that the two sides agree at the nodes).
__device__ __forceinline__ int ag_cell(double x, double dr, int nr) {
    int j = (int)floor(x / dr);
    if (j > nr - 1) j = nr - 1;
    if (j < 0) j = 0;
    while (j > 0 && (double)j * dr > x) --j;
    while (j < nr - 1 && (double)(j + 1) * dr <= x) ++j;
    return j;
}
template <class P>
__device__ __forceinline__ int ag_species(const WakeDev<P>& W, int64_t k) {
    int s = 0;
    while (s + 1 < W.n_species && k >= W.sp_begin[s + 1]) ++s;
    return s;
}
// the grid extent of species b: (1 + 1/nr) x its largest radius (at least
// 1e-12, for a beam on the axis)
template <class P>
__device__ __forceinline__ double ag_extent(const WakeDev<P>& W, int b) {
    if (W.grid_rmax > 0.0) return W.grid_rmax;  // the regular intermediate grid
    return fmax(W.ag_rmax[b], 1e-12) * (1.0 + 1.0 / W.grid_nr);
}
// B^(b) of species b at rho from its grid: linear between nodes inside,
// B_N r_N / rho beyond (Sec. IV)
template <class P>
__device__ __forceinline__ double ag_species_field(const WakeDev<P>& W, int b, double rho) {
    const int nr = W.grid_nr;
    const double R = ag_extent(W, b), dr = R / nr;
    const typename P::R* B = W.agB + (size_t)b * (nr + 1);
    if (rho >= R) return (double)B[nr] * R / rho;
    const int j = ag_cell(rho, dr, nr);
    const double t = (rho - (double)j * dr) / dr;
    return (1.0 - t) * (double)B[j] + t * (double)B[j + 1];
}
template <class P>
__device__ __forceinline__ double ag_field(const WakeDev<P>& W, double rho) {
    double v = 0.0;
    for (int b = 0; b < W.n_species; ++b) v += ag_species_field(W, b, rho);
    return v;
}

// ---------------------------------------------------------------------------
// precision helpers of the one-CTA marches: in FP64 they are the plain
// operations; the mixed path keeps ring radii float-float (hi in rho, lo in
// rho_lo), takes ln rho as ln rho0 + log1p((rho - rho0) / rho0) and the
// weights float-float from the per-ring table ctab
// ---------------------------------------------------------------------------
// ln rho of ring `id` at radius (r, r_lo) in the accumulator type
__device__ __forceinline__ double ring_log(const float4*, int, double r, double) { return log(r); }
__device__ __forceinline__ ff ring_log(const float4* ctab, int id, float r, float r_lo) {
    const float4 c = ctab[3 * id];  // {rho0 (hi, lo), ln rho0 (hi, lo)}
    const ff r0 = {c.x, c.y};
    const float dl = ff_to_f(ff_acc(ff{r, r_lo}, ff_neg(r0)));
    return ff_add_f(ff{c.z, c.w}, log1pf(dl / c.x));
}
// ln X of an arbitrary radius X (accumulator type), relative to the plasma
// edge whose logarithm ln_e is known to the accumulator's precision
__device__ __forceinline__ double acc_log(double X, double, double, double) { return log(X); }
__device__ __forceinline__ ff acc_log(ff X, ff Xe, ff ln_e, float edge) {
    return ff_add_f(ln_e, log1pf(ff_to_f(ff_acc(X, ff_neg(Xe))) / edge));
}
__device__ __forceinline__ double acc_mul_a(double a, double b) { return a * b; }
__device__ __forceinline__ ff acc_mul_a(ff a, ff b) { return ff_mul(a, b); }
__device__ __forceinline__ double acc_div(double a, double b) { return a / b; }
__device__ __forceinline__ ff acc_div(ff a, ff b) {
    const float q1 = a.hi / b.hi;
    const ff rem = ff_acc(a, ff_neg(ff_mul_f(b, q1)));
    return ff_fast_two_sum(q1, rem.hi / b.hi);
}
// ring radius at sorted position p in the accumulator type
__device__ __forceinline__ double ring_radius(const double* hi, const double*, int p) { return hi[p]; }
__device__ __forceinline__ ff ring_radius(const float* hi, const float* lo, int p) { return ff{hi[p], lo[p]}; }

// rho + d in the state's arithmetic: FP64, or float-float (hi in r, lo in r_lo)
__device__ __forceinline__ void radius_add(double& r, double&, double d) { r += d; }
__device__ __forceinline__ void radius_add(float& r, float& r_lo, float d) {
    const ff s = ff_add_f(ff{r, r_lo}, d);
    r = s.hi;
    r_lo = s.lo;
}

// a radius (hi, lo) in the accumulator type
__device__ __forceinline__ double make_radius(double hi, double) { return hi; }
__device__ __forceinline__ ff make_radius(float hi, float lo) { return ff{hi, lo}; }

// ring id's weight and self weight in the accumulator type: the mixed path
// takes them float-float from the per-ring table ({w, what} = ctab[3 id + 1]),
// since their sum meets the exact ion column and FP32-rounded weights would
// leave ~1e-7 of the enclosed charge
__device__ __forceinline__ void ring_weights(const float4*, const double* w, const double* wh, int id, double& wa,
                                             double& wha) {
    wa = w[id];
    wha = wh[id];
}
__device__ __forceinline__ void ring_weights(const float4* ctab, const float*, const float*, int id, ff& wa, ff& wha) {
    const float4 c = ctab[3 * id + 1];
    wa = ff{c.x, c.y};
    wha = ff{c.z, c.w};
}

__device__ __forceinline__ double acc_add_prod(double a, double x, double y) { return a + x * y; }
__device__ __forceinline__ ff acc_add_prod(ff a, float x, float y) { return ff_add(a, ff_two_prod(x, y)); }

// ---------------------------------------------------------------------------
// The thread blocks of one wake on the global-memory marches: one block (a
// plain launch), or a thread-block cluster whose blocks split the wake's
// sorted positions in rank order.  sync() orders the wake's global-memory
// arrays between all of its threads: a block barrier, or a cluster barrier
// (arrive with release, wait with acquire at cluster scope: every write
// before it, global or shared, is visible to every thread of the cluster
// after it).  The scans below fold the blocks' totals in rank order after a
// block scan; the totals travel through `part` (shared memory, two buffers
// used in turn, so that a buffer is written again only after a later call's
// barrier, which every block passes only after it read the buffer).
// ---------------------------------------------------------------------------
constexpr int kMaxWakeCtas = 8;
constexpr int kPartSlot = 64;                          // bytes per block total
constexpr int kPartBuf = kMaxWakeCtas * kPartSlot;     // one buffer
struct WakeCtas {
    int rank = 0, size = 1;
    unsigned char* part = nullptr;  // 2 x kPartBuf bytes of shared memory (size > 1)
    int flip = 0;
    __device__ __forceinline__ void sync() const {
        if (size > 1) {
            asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                             : "memory");
        } else {
            __syncthreads();
        }
    }
    // this block's value v to slot `rank` of every block's current buffer,
    // then the barrier; returns the buffer (its slots in rank order)
    template <class T>
    __device__ __forceinline__ const T* exchange(T v) {
        static_assert(sizeof(T) <= kPartSlot, "scan value too large for the exchange");
        T* buf = reinterpret_cast<T*>(part + flip * kPartBuf);
        flip ^= 1;
        if ((int)threadIdx.x < size) {
            T* dst = cooperative_groups::this_cluster().map_shared_rank(buf, (int)threadIdx.x);
            *reinterpret_cast<T*>(reinterpret_cast<unsigned char*>(dst) + rank * kPartSlot) = v;
        }
        sync();
        return buf;
    }
    template <class T>
    __device__ __forceinline__ T slot(const T* buf, int r) const {
        return *reinterpret_cast<const T*>(reinterpret_cast<const unsigned char*>(buf) + r * kPartSlot);
    }
};

// exclusive scan over the wake's threads (REV: from the last thread of the
// last block down); `total` the fold over all of them
template <bool REV, class T, class Op>
__device__ __forceinline__ T wake_excl_scan(WakeCtas& C, T v, Op op, T ident, T* sbuf, T& total) {
    T bt;
    T ex = block_excl_scan<REV>(v, op, ident, sbuf, bt);
    if (C.size == 1) {
        total = bt;
        return ex;
    }
    const T* buf = C.exchange(bt);
    T pre = ident, tot = ident;
    for (int i = 0; i < C.size; ++i) {
        const int r = REV ? C.size - 1 - i : i;
        if (r == C.rank) pre = tot;
        tot = op(tot, C.slot(buf, r));
    }
    total = tot;
    return op(pre, ex);
}

// two scans over the wake's threads whose block totals travel in one
// exchange (one cluster barrier instead of two); each result as
// wake_excl_scan's
template <class T, class U>
struct TwoVals {
    T a;
    U b;
};
template <bool REV0, bool REV1, class T, class Op0, class U, class Op1>
__device__ __forceinline__ void wake_excl_scan2(WakeCtas& C, T v0, Op0 op0, T id0, T* sbuf0, T& ex0, T& tot0,
                                                U v1, Op1 op1, U id1, U* sbuf1, U& ex1, U& tot1) {
    T bt0;
    U bt1;
    ex0 = block_excl_scan<REV0>(v0, op0, id0, sbuf0, bt0);
    ex1 = block_excl_scan<REV1>(v1, op1, id1, sbuf1, bt1);
    if (C.size == 1) {
        tot0 = bt0;
        tot1 = bt1;
        return;
    }
    const TwoVals<T, U>* buf = C.exchange(TwoVals<T, U>{bt0, bt1});
    T pre0 = id0, t0 = id0;
    U pre1 = id1, t1 = id1;
    for (int i = 0; i < C.size; ++i) {
        const int r0 = REV0 ? C.size - 1 - i : i, r1 = REV1 ? C.size - 1 - i : i;
        if (r0 == C.rank) pre0 = t0;
        if (r1 == C.rank) pre1 = t1;
        t0 = op0(t0, C.slot(buf, r0).a);
        t1 = op1(t1, C.slot(buf, r1).b);
    }
    tot0 = t0;
    tot1 = t1;
    ex0 = op0(pre0, ex0);
    ex1 = op1(pre1, ex1);
}

// the forward sum of fx and the reverse (suffix) sum of ry over the wake's
// threads, exclusive; totals in tx, ty
template <class T>
__device__ __forceinline__ Pair<T> wake_excl_scan_fwd_rev(WakeCtas& C, T fx, T ry, T zero, Pair<T>* sbuf, T& tx,
                                                          T& ty) {
    T bx, by;
    Pair<T> e = block_excl_scan_fwd_rev(fx, ry, zero, sbuf, bx, by);
    if (C.size == 1) {
        tx = bx;
        ty = by;
        return e;
    }
    const Pair<T>* buf = C.exchange(Pair<T>{bx, by});
    T px = zero, ax = zero, py = zero, ay = zero;
    for (int r = 0; r < C.size; ++r) {
        if (r == C.rank) px = ax;
        ax = acc_add(ax, C.slot(buf, r).x);
    }
    for (int r = C.size - 1; r >= 0; --r) {
        if (r == C.rank) py = ay;
        ay = acc_add(ay, C.slot(buf, r).y);
    }
    tx = ax;
    ty = ay;
    return {acc_add(px, e.x), acc_add(py, e.y)};
}

// the AND (all = true) or OR (all = false) of v over the wake's threads
__device__ __forceinline__ bool wake_vote(WakeCtas& C, bool v, bool all) {
    const bool b = all ? __syncthreads_and(v) : __syncthreads_or(v);
    if (C.size == 1) return b;
    const int* buf = C.exchange((int)b);
    bool r = all;
    for (int i = 0; i < C.size; ++i) r = all ? (r && C.slot(buf, i) != 0) : (r || C.slot(buf, i) != 0);
    return r;
}

// a8: the region coefficients a_k, b_k of B_theta^(p) = a_k rho + b_k / rho
// (Eq. ai_bi with b_0 = 0, a_n = 0) for the rings at sorted positions
// [0, n) (radii sR, coefficients W.cA, W.cB, W.cC; this thread's positions
// [p0, p1)), in W.ak, W.bk [0..n].  W.cB, W.cC are overwritten with the ring
// sources gamma_p, delta_p.  Ends without a barrier after the last writes.
// With a cluster (C.size > 1) the positions span its blocks and the scans
// fold over them; the end values (R_0, D_n, a_n, b_n) are block 0's.
template <class P>
__device__ void bp_region_solve(const WakeDev<P>& W, const typename P::R* sR, int n, int p0, int p1,
                                unsigned char* sscan, WakeCtas& C) {
    using R = typename P::R;
    using A = typename P::A;
    const int tid = threadIdx.x;
    const A zeroA = acc_zero(A());
    // regular solution R_k (R_0 = (1,0)) forward, decaying solution D_k
    // (D_n = (0,1)) backward, then x_k = -G_k R_k + H_k D_k with the
    // ring sources c_p = gamma_p R_{p+1} + delta_p D_{p+1},
    // G_k = sum_{p>=k} gamma_p, H_k = sum_{p<k} delta_p.
    const Mat2<R> I2 = {1, 0, 0, 1};
    Mat2<R> Mf = I2, Mb = I2;
    for (int p = p0; p < p1; ++p) {
        R r = sR[p], hA = (R)0.5 * W.cA[p];
        Mat2<R> M = {(R)1 + hA * r, hA / r, -hA * r * r * r, (R)1 - hA * r};
        Mf = OpMatLeft()(Mf, M);
    }
    for (int p = p1 - 1; p >= p0; --p) {
        R r = sR[p], hA = (R)0.5 * W.cA[p];
        Mat2<R> Mi = {(R)1 - hA * r, -hA / r, hA * r * r * r, (R)1 + hA * r};  // inverse (det 1)
        Mb = OpMatLeft()(Mb, Mi);
    }
    Mat2<R> tf, tb;
    Mat2<R> Yf, Yb;
    wake_excl_scan2<false, true>(C, Mf, OpMatLeft(), I2, reinterpret_cast<Mat2<R>*>(sscan), Yf, tf, Mb, OpMatLeft(),
                                 I2, reinterpret_cast<Mat2<R>*>(sscan), Yb, tb);
    if (C.rank == 0 && tid == 0) {
        W.Ra[0] = 1;
        W.Rb[0] = 0;
        W.Da[n] = 0;
        W.Db[n] = 1;
    }
    for (int p = p0; p < p1; ++p) {
        R r = sR[p], hA = (R)0.5 * W.cA[p];
        Mat2<R> M = {(R)1 + hA * r, hA / r, -hA * r * r * r, (R)1 - hA * r};
        Yf = OpMatLeft()(Yf, M);
        W.Ra[p + 1] = Yf.m00;
        W.Rb[p + 1] = Yf.m10;
    }
    A gl = zeroA, dl = zeroA;
    for (int p = p1 - 1; p >= p0; --p) {
        R r = sR[p], Ac = W.cA[p], Bc = W.cB[p], Cc = W.cC[p];
        R hA = (R)0.5 * Ac;
        R d0 = Yb.m01, d1 = Yb.m11;        // D_{p+1}
        R q0 = W.Ra[p + 1], q1 = W.Rb[p + 1];  // R_{p+1}
        R s0 = (R)0.25 * ((R)2 * Bc + Ac * Cc);
        R s1 = (R)0.25 * r * ((R)4 * Cc - (R)2 * Bc * r - Ac * Cc * r);
        R wr = q0 * d1 - q1 * d0;
        R gp = (s0 * d1 - s1 * d0) / wr;
        R dp = (q0 * s1 - q1 * s0) / wr;
        W.cB[p] = gp;  // reuse: gamma_p
        W.cC[p] = dp;  // reuse: delta_p
        gl = acc_add_r(gl, gp);
        dl = acc_add_r(dl, dp);
        Mat2<R> Mi = {(R)1 - hA * r, -hA / r, hA * r * r * r, (R)1 + hA * r};
        Yb = OpMatLeft()(Yb, Mi);
        W.Da[p] = Yb.m01;
        W.Db[p] = Yb.m11;
    }
    // G_k = sum_{p >= k} gamma_p as a true suffix sum (a total minus a
    // prefix would cancel where G_k is small and R_k ~ e^rho is large)
    A g_tot, d_tot;
    Pair<A> gd = wake_excl_scan_fwd_rev(C, dl, gl, zeroA, reinterpret_cast<Pair<A>*>(sscan), d_tot, g_tot);
    // the scan's barriers order the R/D writes above before these reads (a
    // block's first R_p comes from the block before it in a cluster)
    A Gsuf = gd.y;  // sum of gamma over rings >= p1
    for (int p = p1 - 1; p >= p0; --p) {
        Gsuf = acc_add_r(Gsuf, W.cB[p]);  // sum over rings >= p
        R G = acc_to_r(Gsuf);
        W.ak[p] = -G * W.Ra[p];
        W.bk[p] = -G * W.Rb[p];
    }
    A Hex = gd.x;   // sum of delta over rings < p
    for (int p = p0; p < p1; ++p) {
        R H = acc_to_r(Hex);
        W.ak[p] += H * W.Da[p];
        W.bk[p] += H * W.Db[p];
        Hex = acc_add_r(Hex, W.cC[p]);
    }
    if (C.rank == 0 && tid == 0) {
        R H = acc_to_r(d_tot);
        W.ak[n] = H * W.Da[n];
        W.bk[n] = H * W.Db[n];
    }
}

// Bitonic sort of keys[0..n_pad) ascending, ties by vals ascending (the
// caller pads with +inf keys); every thread of the block takes part.
template <class R>
__device__ void block_bitonic_sort(R* keys, int32_t* vals, int n_pad) {
    const int T = blockDim.x, tid = threadIdx.x;
    for (int k = 2; k <= n_pad; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = tid; i < n_pad; i += T) {
                int ixj = i ^ j;
                if (ixj > i) {
                    R ki = keys[i], kj = keys[ixj];
                    int vi = vals[i], vj = vals[ixj];
                    bool gt = (ki > kj) || (ki == kj && vi > vj);
                    if (gt == ((i & k) == 0)) {
                        keys[i] = kj; keys[ixj] = ki;
                        vals[i] = vj; vals[ixj] = vi;
                    }
                }
            }
            __syncthreads();
        }
    }
}

template <class P>
__global__ void __launch_bounds__(512)
march_kernel(const WakeDev<P>* __restrict__ wakes, const int32_t* __restrict__ order,
             int32_t max_slices, int32_t mode, int32_t mb_cap) {
    using R = typename P::R;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ctl[CTL_N];
    __shared__ int s_stop;
    __shared__ __align__(16) unsigned char s_part[2 * kPartBuf];

    const uint64_t t_launch = global_ns();
    // one block per wake, or (beam-grid wakes) a thread-block cluster whose
    // blocks split the sorted rings, the grid nodes and the particles; block
    // 0 sorts and sums the node charges
    WakeCtas C;
    {
        unsigned r, c;
        asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
        asm("mov.u32 %0, %%cluster_nctarank;" : "=r"(c));
        C.rank = (int)r;
        C.size = (int)c;
        C.part = s_part;
    }
    const int wi = blockIdx.x / C.size;
    const WakeDev<P>& W = wakes[order ? order[wi] : wi];
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int gt = C.rank * T + tid;  // the thread's place in the wake
    const int GT = C.size * T;
    const int n = W.n;
    const int K = (n + GT - 1) / GT;
    const int p0 = min(n, gt * K);
    const int p1 = min(n, p0 + K);
    const bool sorter = C.rank == 0;

    unsigned char* sscan = smem;
    R* keys = reinterpret_cast<R*>(smem + kScanBytes);
    int32_t* vals = reinterpret_cast<int32_t*>(keys + W.n_pad);
    R* sR = keys;      // sorted ring radii (after the sort)
    R* sB = keys + n;  // staged beam radii of the slice

    if (tid < CTL_N) s_ctl[tid] = W.ctl[tid];
    __syncthreads();
    if (s_ctl[CTL_STATUS] != 0) return;
    int slice = s_ctl[CTL_NEXT];
    int buf = s_ctl[CTL_BUF];
    int has_prev = s_ctl[CTL_PREV];
    int status = 0, fail = -1;
    const int s_end = mode == MODE_MARCH ? min(W.n_steps, slice + max_slices) : slice + 1;

    const double dens_d = W.density, rmax_d = W.rho_max;
    const R rmax = (R)rmax_d;
    const R half_n = (R)(0.5 * dens_d), quarter_n = (R)(0.25 * dens_d);
    const A Imax = acc_from_d(0.5 * dens_d * rmax_d * rmax_d, A());
    const A c0 = acc_from_d(0.25 * dens_d * rmax_d * rmax_d - 0.5 * dens_d * rmax_d * rmax_d * log(rmax_d), A());
    const R dxi = (R)W.dxi;
    const R inv_2pi_dxi = (R)(1.0 / (6.283185307179586476925286766559 * W.dxi));
    const A zeroA = acc_zero(A());

    const int slice0 = slice;
    uint64_t t_start = 0;
    for (; slice < s_end; ++slice) {
        R* rho = W.rho[buf];
        // time budget (thread 0 decides, read after the order check's barrier)
        if (W.budget_ns > 0 && tid == 0) {
            const uint64_t now = global_ns();
            if (slice == slice0) t_start = now;
            s_stop = slice > slice0 && now - t_start >= (uint64_t)W.budget_ns;
        }
        // ---------------- a2: sort by radius (stable w.r.t. previous order)
        bool ok = true;
        for (int p = p0; p < p1; ++p)
            if (p + 1 < n && rho[p + 1] < rho[p]) ok = false;
        bool in_order = __syncthreads_and(ok);
        bool stop = W.budget_ns > 0 && s_stop;
        if (C.size > 1) {  // the cluster's blocks agree on both
            const int* v = C.exchange((int)in_order | (stop ? 2 : 0));
            in_order = true;
            stop = false;
            for (int r = 0; r < C.size; ++r) {
                const int f = C.slot(v, r);
                in_order = in_order && (f & 1) != 0;
                stop = stop || (f & 2) != 0;
            }
        }
        if (stop) break;
        if (!in_order) {
            const int nb = buf ^ 1;
            if (sorter) {
                for (int i = tid; i < W.n_pad; i += T) {
                    keys[i] = i < n ? rho[i] : (R)INFINITY;
                    vals[i] = i;
                }
                __syncthreads();
                block_bitonic_sort(keys, vals, W.n_pad);
                for (int p = tid; p < n; p += T) {
                    int src = vals[p];
                    W.rho[nb][p] = W.rho[buf][src];
                    W.ur[nb][p] = W.ur[buf][src];
                    W.frho[nb][p] = W.frho[buf][src];
                    W.fur[nb][p] = W.fur[buf][src];
                    W.rid[nb][p] = W.rid[buf][src];
                    keys[p] = W.rho_lo[src];  // the sort keys are no longer needed
                }
                __syncthreads();
                for (int p = tid; p < n; p += T) W.rho_lo[p] = keys[p];
            }
            buf = nb;
            rho = W.rho[buf];
            C.sync();
        }
        R* ur = W.ur[buf];
        R* frho = W.frho[buf];
        R* fur = W.fur[buf];
        const int32_t* rid = W.rid[buf];

        // ---------------- stage ring radii and this slice's beam radii
        const bool have_beam = W.nb > 0 && slice < W.n_steps;
        int b0 = 0, m = 0;
        R qtot = 0;
        if (have_beam) {
            b0 = W.boff[slice];
            m = W.boff[slice + 1] - b0;
            qtot = W.bTot[slice];
        }
        const bool staged = m <= mb_cap;
        for (int p = tid; p < n; p += T) sR[p] = rho[p];
        if (staged)
            for (int q = tid; q < m; q += T) sB[q] = W.br[b0 + q];
        __syncthreads();
        const R* beamR = staged ? sB : (W.br + b0);

        // ---------------- adaptive grids: B^(b) at the nodes of this slice
        const int nr = W.grid_nr;
        if (nr > 0) {
            const int nn = W.n_species * (nr + 1);
            if (sorter)
                for (int i = tid; i < nn; i += T) W.agB[i] = 0;
            C.sync();
            for (int q = gt; q < m; q += GT) {  // each particle's charge reaches the nodes above it
                const int64_t k = W.bidx[b0 + q];
                const int b = ag_species(W, k);
                const double dr = ag_extent(W, b) / nr;
                const int j = ag_cell(W.rc[k], dr, nr) + 1;
                atomicAdd(W.agB + (size_t)b * (nr + 1) + j, (R)W.qw[k]);
            }
            C.sync();
            if (sorter && tid < W.n_species) {
                R* B = W.agB + (size_t)tid * (nr + 1);
                const double dr = ag_extent(W, tid) / nr;
                double acc = 0.0;
                B[0] = 0;
                for (int j = 1; j <= nr; ++j) {
                    acc += (double)B[j];
                    B[j] = (R)(acc / (6.283185307179586476925286766559 * W.dxi * ((double)j * dr)));
                }
            }
            C.sync();
        }

        // ---------------- a3 + a4: beam field at rings, local sums
        Pair<A> loc = {zeroA, zeroA};
        for (int p = p0; p < p1; ++p) {
            R r = sR[p];
            int id = rid[p];
            A wa, wha;
            ring_weights(W.ctab, W.w, W.wh, id, wa, wha);
            R bbv = 0;
            if (nr > 0) {
                bbv = (R)ag_field(W, (double)r);
            } else if (m > 0 && r > (R)0) {
                int lb = lower_bound_dev(beamR, m, r);
                R Q = lb < m ? W.bE[b0 + lb] : qtot;
                bbv = Q * inv_2pi_dxi / r;
            }
            W.bb[p] = bbv;
            loc.x = acc_add(loc.x, wa);
            loc.y = acc_add(loc.y, acc_mul_a(ring_log(W.ctab, id, r, W.rho_lo[p]), wa));
        }
        Pair<A> tot;
        Pair<A> ex = wake_excl_scan<false>(C, loc, OpAddPair(), Pair<A>{zeroA, zeroA},
                                           reinterpret_cast<Pair<A>*>(sscan), tot);
        const A Wtot = tot.x, Ltot = tot.y;

        // ---------------- a5: psi, d_rho psi, psibar, gamma, t
        A S = ex.x, L = ex.y;
        A tl = zeroA;
        for (int p = p0; p < p1; ++p) {
            R r = sR[p];
            R u = ur[p];
            int id = rid[p];
            R w = W.w[id];
            A wa, wha;
            ring_weights(W.ctab, W.w, W.wh, id, wa, wha);
            const A X = make_radius(r, W.rho_lo[p]);
            const A lnr = ring_log(W.ctab, id, r, W.rho_lo[p]);
            A Lsuf = acc_sub(Ltot, L);
            W.regS[p] = S;
            W.regL[p] = Lsuf;
            // the ion column's terms from the radius in the accumulator type:
            // psi and d_rho psi are differences of terms ~n rho_max^2
            const A r2 = acc_mul_a(X, X);
            const A Ir = r < rmax ? acc_mul_r(r2, half_n) : Imax;
            const A psion = r <= rmax ? acc_sub(c0, acc_mul_r(r2, quarter_n)) : acc_sub(zeroA, acc_mul_a(Imax, lnr));
            A psiA = acc_add(acc_add(Lsuf, acc_mul_a(S, lnr)), psion);
            R psi = acc_to_r(psiA);
            R dprv = acc_to_r(acc_div(acc_sub(acc_add(S, wha), Ir), X));
            R pb = (R)1 + psi;
            R g = ((R)1 + u * u + pb * pb) / ((R)2 * pb);
            R t = w * u / (r * pb);
            W.psib[p] = pb;
            W.gam[p] = g;
            W.dpr[p] = dprv;
            W.tt[p] = t;
            if (mode == MODE_MARCH && W.dump_psi) {
                size_t row = (size_t)slice * n + id;
                W.dump_psi[row] = psi;
                W.dump_dpr[row] = dprv;
            }
            S = acc_add(S, wa);
            L = acc_add(L, acc_mul_a(lnr, wa));
            tl = acc_add_r(tl, t);
        }
        if (C.rank == 0 && tid == 0) {
            W.regS[n] = Wtot;
            W.regL[n] = zeroA;
            W.regT[n] = (R)0;
        }
        A Ttot;
        A Tex = wake_excl_scan<false>(C, tl, OpAdd(), zeroA, reinterpret_cast<A*>(sscan), Ttot);

        // ---------------- a6 + a7: d_zeta psi, A, B, C
        {
            A Tacc = Tex;
            for (int p = p0; p < p1; ++p) {
                R r = sR[p];
                R u = ur[p];
                int id = rid[p];
                R w = W.w[id], wh = W.wh[id];
                R t = W.tt[p];
                W.regT[p] = acc_to_r(acc_sub(Ttot, Tacc));
                Tacc = acc_add_r(Tacc, t);
                R above = acc_to_r(acc_sub(Ttot, Tacc));
                R dpz = -(above + ((R)1 - wh / w) * t);
                R pb = W.psib[p], g = W.gam[p], dprv = W.dpr[p], bbv = W.bb[p];
                R wr = w / r, pb2 = pb * pb;
                R Ac = wr / pb;
                R Bc = -wr * g * dprv / pb2 + wr * bbv / pb + (w / (r * r)) * u * u / pb2 +
                       wr * u * u * dprv / (pb2 * pb) - wr * u * dpz / pb2;
                R Cc = -wr * (g / pb - (R)1 - u * u / pb2);
                W.cA[p] = Ac;
                W.cB[p] = Bc;
                W.cC[p] = Cc;
                W.tt[p] = dpz;  // t no longer needed: keep d_zeta psi
                if (mode == MODE_MARCH && W.dump_dpz) W.dump_dpz[(size_t)slice * n + id] = dpz;
            }
        }

        // ---------------- a8: B_theta^(p) region coefficients a_k, b_k
        bp_region_solve(W, sR, n, p0, p1, sscan, C);
        C.sync();

        // ---------------- B^(p) at the rings, guard, dumps
        bool bad = false;
        for (int p = p0; p < p1; ++p) {
            R r = sR[p];
            R bpv = (R)0.5 * ((W.ak[p] + W.ak[p + 1]) * r + (W.bk[p] + W.bk[p + 1]) / r);
            W.cA[p] = bpv;  // reuse: B^(p) at the ring
            R pb = W.psib[p];
            if (!(pb > (R)0) || !real_finite(pb) || !real_finite(W.dpr[p]) || !real_finite(W.tt[p]) ||
                !real_finite(bpv) || !real_finite(W.bb[p]) || !real_finite(W.gam[p]))
                bad = true;
            if (mode == MODE_MARCH) {
                int id = rid[p];
                size_t row = (size_t)slice * n + id;
                if (W.dump_r) W.dump_r[row] = r;
                if (W.dump_ur) {
                    W.dump_ur[row] = ur[p];
                    W.dump_bp[row] = bpv;
                    W.dump_bb[row] = W.bb[p];
                }
            }
        }
        bad = wake_vote(C, bad, false);

        // ---------------- adaptive grids: the plasma fields at the nodes
        if (nr > 0 && mode == MODE_MARCH) {
            const int nn = W.n_species * (nr + 1);
            for (int i = gt; i < nn; i += GT) {
                const int b = i / (nr + 1), j = i - b * (nr + 1);
                const double dr = ag_extent(W, b) / nr;
                const R x = (R)((double)j * dr);
                R psi, dprv, dpz, bpv;
                if (x > (R)0) {
                    int k = lower_bound_dev(sR, n, x);
                    A Sk = W.regS[k];
                    psi = acc_to_r(acc_add(acc_add(W.regL[k], acc_mul_r(Sk, real_log(x))),
                                           ion_psi(x, rmax, quarter_n, Imax, c0)));
                    dprv = acc_to_r(acc_sub(Sk, ion_enclosed(x, rmax, half_n, Imax))) / x;
                    dpz = -W.regT[k];
                    bpv = W.ak[k] * x + W.bk[k] / x + (R)ag_field(W, (double)x);
                } else {
                    psi = acc_to_r(acc_add(W.regL[0], ion_psi((R)0, rmax, quarter_n, Imax, c0)));
                    dprv = 0;
                    dpz = -W.regT[0];
                    bpv = 0;
                }
                R* F = W.agF + (size_t)i * 4;
                F[0] = psi;
                F[1] = dprv;
                F[2] = dpz;
                F[3] = bpv;
            }
            C.sync();
            for (int q = gt; q < m; q += GT) {
                const int64_t kc = W.bidx[b0 + q];
                const int b = ag_species(W, kc);
                const double dr = ag_extent(W, b) / nr;
                const double x = W.rc[kc];  // the caller's FP64 radius: node membership as the oracle's
                const int j = ag_cell(x, dr, nr);
                const R t = (R)((x - (double)j * dr) / dr);
                const R* F0 = W.agF + ((size_t)b * (nr + 1) + j) * 4;
                const R* F1 = F0 + 4;
                const int64_t o = b0 + q;
                W.out_ez[o] = -(((R)1 - t) * F0[2] + t * F1[2]);
                W.out_wr[o] = -(((R)1 - t) * F0[1] + t * F1[1]);
                W.out_bt[o] = ((R)1 - t) * F0[3] + t * F1[3];
                W.out_psi[o] = ((R)1 - t) * F0[0] + t * F1[0];
            }
        }

        // ---------------- a9: fields on beam particles (or query radii)
        if (!(nr > 0 && mode == MODE_MARCH)) {
            const int64_t nq = mode == MODE_MARCH ? (int64_t)m : W.nq;
            for (int64_t q = gt; q < nq; q += GT) {
                R x;
                if (mode == MODE_MARCH) x = staged ? beamR[q] : W.br[b0 + q];
                else x = (R)W.rq[q];
                R psi, dprv, dpz, bpv, bbv;
                if (x > (R)0) {
                    int k = lower_bound_dev(sR, n, x);
                    A Sk = W.regS[k];
                    psi = acc_to_r(acc_add(acc_add(W.regL[k], acc_mul_r(Sk, real_log(x))),
                                           ion_psi(x, rmax, quarter_n, Imax, c0)));
                    dprv = acc_to_r(acc_sub(Sk, ion_enclosed(x, rmax, half_n, Imax))) / x;
                    dpz = -W.regT[k];
                    bpv = W.ak[k] * x + W.bk[k] / x;
                    if (mode == MODE_MARCH) {
                        bbv = W.bQs[b0 + q] * inv_2pi_dxi / x;
                    } else {
                        bbv = 0;
                        if (m > 0) {
                            int lb = lower_bound_dev(beamR, m, x);
                            R Q = lb < m ? W.bE[b0 + lb] : qtot;
                            bbv = Q * inv_2pi_dxi / x;
                        }
                    }
                } else {
                    psi = acc_to_r(acc_add(W.regL[0], ion_psi((R)0, rmax, quarter_n, Imax, c0)));
                    dprv = 0;
                    dpz = -W.regT[0];
                    bpv = 0;
                    bbv = 0;
                }
                if (mode == MODE_MARCH) {
                    int64_t o = b0 + q;
                    W.out_ez[o] = -dpz;
                    W.out_wr[o] = -dprv;
                    W.out_bt[o] = bpv + bbv;
                    W.out_psi[o] = psi;
                } else {
                    if (W.q_ez) W.q_ez[q] = -dpz;
                    if (W.q_wr) W.q_wr[q] = -dprv;
                    if (W.q_bt) W.q_bt[q] = bpv + bbv;
                    if (W.q_psi) W.q_psi[q] = psi;
                }
            }
        }
        if (mode != MODE_MARCH) break;
        if (bad) {
            status = 4;
            fail = slice;
            ++slice;
            break;
        }

        // ---------------- a10: AB2 push to the next slice
        for (int p = p0; p < p1; ++p) {
            R r = sR[p], u = ur[p];
            R pb = W.psib[p];
            R fr = u / pb;
            R fu = W.gam[p] * W.dpr[p] / pb - (W.cA[p] + W.bb[p]);
            R rn = r, rlo = W.rho_lo[p], un;
            if (has_prev) {
                radius_add(rn, rlo, dxi * ((R)1.5 * fr - (R)0.5 * frho[p]));
                un = u + dxi * ((R)1.5 * fu - (R)0.5 * fur[p]);
            } else {
                radius_add(rn, rlo, dxi * fr);
                un = u + dxi * fu;
            }
            if (rn < (R)0) {
                rn = -rn;
                rlo = -rlo;
                un = -un;
                fr = -fr;
                fu = -fu;
            }
            rho[p] = rn;
            W.rho_lo[p] = rlo;
            ur[p] = un;
            frho[p] = fr;
            fur[p] = fu;
        }
        has_prev = 1;
        C.sync();
    }
    C.sync();
    if (C.rank == 0 && tid == 0) {
        if (mode == MODE_MARCH) put_march_times(W.ctl, t_launch);
        W.ctl[CTL_NEXT] = mode == MODE_MARCH ? slice : s_ctl[CTL_NEXT];
        W.ctl[CTL_BUF] = buf;
        W.ctl[CTL_PREV] = has_prev;
        if (status) {
            W.ctl[CTL_STATUS] = status;
            W.ctl[CTL_FAIL] = fail;
        }
    }
}

}  // namespace gbwake
