// march_cluster.cuh -- the on-chip march of one wake by a thread-block
// cluster: CTA c of the cluster holds the sorted ring positions
// [c*T*K, (c+1)*T*K) in its shared memory (same layout as march_fast.cuh).
// The per-slice chain is that of march_fast.cuh; what crosses CTAs goes
// through distributed shared memory:
//   - block-scan totals (each CTA folds the totals of its predecessors, or
//     successors for the reverse scans, in rank order: deterministic);
//   - the sortedness vote and, when rings crossed, the sort: a local bitonic
//     sort in every CTA, then odd-even merge-split rounds between neighbour
//     CTAs (merge path over the two sorted ranges) until sorted;
//   - beam counts (atomic adds into the owning CTA), beam-particle and query
//     lookups (binary search in the owning CTA's radii), and the region
//     table entry just past each CTA's last ring.
// Every cluster barrier is reached in cluster-uniform control flow.
#pragma once

#include <cooperative_groups.h>

#include "march_fast.cuh"

namespace gbwake {

namespace cg = cooperative_groups;

template <class T>
__device__ __forceinline__ T* rmt(cg::cluster_group& cl, T* p, int rank) {
    return cl.map_shared_rank(p, rank);
}

__device__ __forceinline__ FastSmem rmt_sm(cg::cluster_group& cl, const FastSmem& s, int r) {
    FastSmem o;
    o.rh = rmt(cl, s.rh, r);
    o.rl = rmt(cl, s.rl, r);
    o.u = rmt(cl, s.u, r);
    o.fr = rmt(cl, s.fr, r);
    o.fu = rmt(cl, s.fu, r);
    o.id = rmt(cl, s.id, r);
    o.a = rmt(cl, s.a, r);
    o.b = rmt(cl, s.b, r);
    o.T = rmt(cl, s.T, r);
    o.D = rmt(cl, s.D, r);
    o.S = rmt(cl, s.S, r);
    o.psi = rmt(cl, s.psi, r);
    return o;
}

// Exchange of a block-scan total across the cluster.  Each CTA stores its
// total into every peer's receive array (remote stores need no round trip),
// one cluster barrier makes them visible, and each CTA folds locally: the
// totals of ranks < mine (forward) and of all ranks, in rank order.  recv is
// this call site's __shared__ array of 16 slots.
template <class T, class Op>
__device__ void cluster_fold_fwd(cg::cluster_group& cl, T tot, T ident, Op op, T* recv, T* s_pre, T* s_all) {
    const int rank = cl.block_rank(), size = cl.num_blocks();
    if (threadIdx.x < size) *rmt(cl, &recv[rank], threadIdx.x) = tot;
    cl.sync();
    if (threadIdx.x == 0) {
        T pre = ident, all = ident;
        for (int r = 0; r < size; ++r) {
            if (r < rank) pre = op(pre, recv[r]);
            all = op(all, recv[r]);
        }
        *s_pre = pre;
        *s_all = all;
    }
    __syncthreads();
}

// the same for a reverse scan: fold of the totals of ranks > mine, taken
// from the last rank down
template <class T, class Op>
__device__ void cluster_fold_rev(cg::cluster_group& cl, T tot, T ident, Op op, T* recv, T* s_pre, T* s_all) {
    const int rank = cl.block_rank(), size = cl.num_blocks();
    if (threadIdx.x < size) *rmt(cl, &recv[rank], threadIdx.x) = tot;
    cl.sync();
    if (threadIdx.x == 0) {
        T pre = ident, all = ident;
        for (int r = size - 1; r >= 0; --r) {
            if (r > rank) pre = op(pre, recv[r]);
            all = op(all, recv[r]);
        }
        *s_pre = pre;
        *s_all = all;
    }
    __syncthreads();
}

// cluster-wide AND of a block-uniform flag (push-style, as above)
__device__ __forceinline__ bool cluster_all(cg::cluster_group& cl, bool v, int* recv, int* s_out) {
    const int rank = cl.block_rank(), size = cl.num_blocks();
    if (threadIdx.x < size) *rmt(cl, &recv[rank], threadIdx.x) = v ? 1 : 0;
    cl.sync();
    if (threadIdx.x == 0) {
        int a = 1;
        for (int r = 0; r < size; ++r) a &= recv[r];
        *s_out = a;
    }
    __syncthreads();
    return *s_out != 0;
}

// global sorted position -> (owner rank, local slot address)
template <int K>
__device__ __forceinline__ void owner_of(int p, int TK, int* rank, int* addr) {
    *rank = p / TK;
    int l = p - *rank * TK;
    *addr = Swz<K>::at(l);
}

// number of rings in the cluster with radius < x (strict) or <= x
template <int K>
__device__ int cluster_rank(cg::cluster_group& cl, const FastSmem& sm, const float* s_first, int csize, int n,
                            int TK, float x, bool strict) {
    int c = -1;
    for (int r = 0; r < csize; ++r) {
        float f = s_first[r];
        if (strict ? (f < x) : (f <= x)) c = r;
    }
    if (c < 0) return 0;
    const int nl = min(TK, n - c * TK);
    const float* rh = rmt(cl, sm.rh, c);
    return c * TK + ring_rank<K>(rh, nl, x, strict);
}

// Odd-even merge-split round between neighbour CTAs (left = even ranks when
// parity 0, odd when 1): each CTA of a pair rebuilds its range from the merge
// of the two sorted ranges (ties: left first, which keeps the sort stable).
template <int K>
__device__ void cluster_merge_round(cg::cluster_group& cl, const FastSmem& sm, int n, int TK, int parity) {
    const int rank = cl.block_rank(), size = cl.num_blocks();
    const int tid = threadIdx.x;
    int left = -1;
    if ((rank & 1) == parity && rank + 1 < size) left = rank;
    else if (rank >= 1 && ((rank - 1) & 1) == parity) left = rank - 1;
    float g_rh[K], g_rl[K], g_u[K], g_fr[K], g_fu[K];
    int g_id[K];
    const bool active = left >= 0;
    int my_n = 0;
    if (active) {
        const int nA = min(TK, n - left * TK);
        const int nB = min(TK, n - (left + 1) * TK);
        FastSmem A = rmt_sm(cl, sm, left), B = rmt_sm(cl, sm, left + 1);
        const int off = (rank == left) ? 0 : nA;  // merged position of my local 0
        my_n = (rank == left) ? nA : nB;
        int d = off + tid * K;
        if (tid * K < my_n) {
            // merge path: i = number of A elements among the first d merged
            int lo = max(0, d - nB), hi = min(d, nA);
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (A.rh[Swz<K>::at(mid)] <= B.rh[Swz<K>::at(d - 1 - mid)]) lo = mid + 1;
                else hi = mid;
            }
            int i = lo, j = d - lo;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (tid * K + k < my_n) {
                    bool takeA = i < nA && (j >= nB || A.rh[Swz<K>::at(i)] <= B.rh[Swz<K>::at(j)]);
                    const FastSmem& S = takeA ? A : B;
                    int a = Swz<K>::at(takeA ? i : j);
                    g_rh[k] = S.rh[a]; g_rl[k] = S.rl[a]; g_u[k] = S.u[a];
                    g_fr[k] = S.fr[a]; g_fu[k] = S.fu[a]; g_id[k] = S.id[a];
                    if (takeA) ++i;
                    else ++j;
                }
            }
        }
    }
    cl.sync();  // every read of the old ranges is done
    if (active) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int l = tid * K + k;
            if (l < my_n) {
                int a = Swz<K>::at(l);
                sm.rh[a] = g_rh[k]; sm.rl[a] = g_rl[k]; sm.u[a] = g_u[k];
                sm.fr[a] = g_fr[k]; sm.fu[a] = g_fu[k]; sm.id[a] = g_id[k];
            }
        }
    }
    cl.sync();
}

template <int K>
__global__ void __launch_bounds__(512)
march_cluster_kernel(const WakeDev<PrecMixed>* __restrict__ wakes, const int32_t* __restrict__ order,
                     int32_t max_slices, int32_t mode) {
    using R = float;
    using A = ff;
    using SW = Swz<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ctl[CTL_N];
    __shared__ float s_first[16];
    __shared__ float s_edge[2];  // this CTA's first and last radius
    __shared__ float4 s_sortv[16];
    __shared__ int s_gvote[16], s_vote_out;
    __shared__ Trip<ff> x1_slot[16], x1_pre, x1_all;
    __shared__ ff x2_slot[16], x2_pre, x2_all;
    __shared__ Mat2<float> x3f_slot[16], x3f_pre, x3f_all, x3r_slot[16], x3r_pre, x3r_all;
    __shared__ ff x4f_slot[16], x4f_pre, x4f_all, x4r_slot[16], x4r_pre, x4r_all;

    cg::cluster_group cl = cg::this_cluster();
    const int crank = cl.block_rank();
    const int csize = cl.num_blocks();
    const int widx = blockIdx.x / csize;
    const WakeDev<PrecMixed>& W = wakes[order ? order[widx] : widx];
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int n = W.n;
    const int TK = T * K;
    const int base = crank * TK;            // global position of local slot 0
    const int nl = max(0, min(TK, n - base));  // rings held by this CTA
    const int p0 = tid * K;                 // local positions [p0, p0 + K)
    const int cap = TK + 8;
    const int owner_last = (n - 1) / TK;    // CTA holding the last ring (and region n)
    const float4* __restrict__ ctab = W.ctab;

    unsigned char* sscan = smem;
    FastSmem sm;
    sm.rh = reinterpret_cast<float*>(smem + kScanBytes);
    sm.rl = sm.rh + cap;
    sm.u = sm.rl + cap;
    sm.fr = sm.u + cap;
    sm.fu = sm.fr + cap;
    sm.id = reinterpret_cast<int32_t*>(sm.fu + cap);
    sm.a = reinterpret_cast<float*>(sm.id + cap);
    sm.b = sm.a + cap;
    sm.T = sm.b + cap;
    sm.D = sm.T + cap;
    sm.S = sm.D + cap;
    sm.psi = sm.S + cap;
    int32_t* t_cnt = reinterpret_cast<int32_t*>(sm.a);

    if (tid < CTL_N) s_ctl[tid] = W.ctl[tid];
    __syncthreads();
    // (status and slice are the same for every CTA of the cluster)
    if (s_ctl[CTL_STATUS] != 0) return;
    int slice = s_ctl[CTL_NEXT];
    const int buf = s_ctl[CTL_BUF];
    int has_prev = s_ctl[CTL_PREV];
    int status = 0, fail = -1;
    const int n_steps = W.n_steps;
    const int s_end = mode == MODE_MARCH ? min(n_steps, slice + max_slices) : slice + 1;

    for (int p = tid; p < nl; p += T) {
        int a = SW::at(p), g = base + p;
        sm.rh[a] = W.rho[buf][g];
        sm.rl[a] = W.rho_lo[g];
        sm.u[a] = W.ur[buf][g];
        sm.fr[a] = W.frho[buf][g];
        sm.fu[a] = W.fur[buf][g];
        sm.id[a] = W.rid[buf][g];
    }
    cl.sync();

    const double dens_d = W.density, rmax_d = W.rho_max;
    const R rmax = (R)rmax_d;
    const R half_n = (R)(0.5 * dens_d), quarter_n = (R)(0.25 * dens_d);
    const A Imax = ff_from_d(0.5 * dens_d * rmax_d * rmax_d);
    const A c0 = ff_from_d(0.25 * dens_d * rmax_d * rmax_d - 0.5 * dens_d * rmax_d * rmax_d * log(rmax_d));
    const R dxi = (R)W.dxi;
    const R inv_2pi_dxi = (R)(1.0 / (6.283185307179586476925286766559 * W.dxi));
    const A zeroA = {0.f, 0.f};
    const Mat2<R> I2 = {1, 0, 0, 1};

    R rh[K], ur[K];
    int idv[K];
    R ir[K], ipb[K];
    R pbv[K], dprv[K], bbv[K];
    R s0v[K], s1v[K], hav[K];
    R tv[K];

    for (; slice < s_end; ++slice) {
        // ---------------- a2: sort by radius if out of order (cluster-wide)
        {
            bool ok = true;
            R prev = -INFINITY;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < nl) {
                    R v = sm.rh[SW::at(p)];
                    if (v < prev) ok = false;
                    prev = v;
                }
            }
            if (p0 + K < nl && sm.rh[SW::at(p0 + K)] < prev) ok = false;
            bool blk = __syncthreads_and(ok);
            // block votes and CTA boundaries: every CTA pushes (vote, first
            // radius, last radius) into each peer's slot of its rank, one
            // cluster barrier, then every CTA checks all of them locally
            if (tid < csize)
                *rmt(cl, &s_sortv[crank], tid) =
                    make_float4(blk ? 1.f : 0.f, sm.rh[SW::at(0)], sm.rh[SW::at(nl - 1)], 0.f);
            cl.sync();
            if (tid == 0) {
                int all = 1;
                for (int r = 0; r < csize; ++r) {
                    const float4 v = s_sortv[r];
                    if (v.x == 0.f) all = 0;
                    if (r + 1 < csize && v.z > s_sortv[r + 1].y) all = 0;
                }
                s_vote_out = all;
            }
            __syncthreads();
            if (!s_vote_out) {
                // local sort of every CTA's range, then merge-split rounds
                const int nl_pad = nl < 2 ? 2 : 1 << (32 - __clz(nl - 1));
                fast_sort<K>(sm, nl, nl_pad, cap);
                for (int round = 0; round < 2 * csize + 2; ++round) {
                    if (tid == 0) {
                        s_edge[0] = sm.rh[SW::at(0)];
                        s_edge[1] = sm.rh[SW::at(nl - 1)];
                    }
                    cl.sync();
                    if (tid == 0) {
                        int all = 1;
                        for (int r = 0; r + 1 < csize; ++r)
                            if (*rmt(cl, &s_edge[1], r) > *rmt(cl, &s_edge[0], r + 1)) all = 0;
                        s_vote_out = all;
                    }
                    __syncthreads();
                    const bool sorted = s_vote_out != 0;
                    cl.sync();  // everyone has read the edges before they change
                    if (sorted) break;
                    cluster_merge_round<K>(cl, sm, n, TK, round & 1);
                }
            }
        }
        // replicated first radius of every CTA (for locating a radius)
        if (tid < csize) s_first[tid] = *rmt(cl, &sm.rh[SW::at(0)], tid);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < nl) {
                int a = SW::at(p);
                rh[k] = sm.rh[a];
                ur[k] = sm.u[a];
                idv[k] = sm.id[a];
            } else {
                ur[k] = 0.f; rh[k] = 1.f; idv[k] = 0;
            }
            ir[k] = __frcp_rn(rh[k]);
        }
        __syncthreads();

        // ---------------- a3: beam particles count into their radial place
        int b0 = 0, m = 0;
        R qtot = 0;
        if (W.nb > 0 && slice < n_steps) {
            b0 = W.boff[slice];
            m = W.boff[slice + 1] - b0;
            qtot = W.bTot[slice];
        }
        if (m > 0) {
            for (int i = tid; i < cap; i += T) t_cnt[i] = 0;
            cl.sync();
            for (int q = crank * T + tid; q < m; q += csize * T) {
                int rk = cluster_rank<K>(cl, sm, s_first, csize, n, TK, W.br[b0 + q], false);
                if (rk < n) {
                    int r2, a2;
                    owner_of<K>(rk, TK, &r2, &a2);
                    atomicAdd(rmt(cl, &t_cnt[a2], r2), 1);
                }
            }
            cl.sync();
        }

        // ---------------- a4: scan of (sum w, sum w ln rho, counts)
        A sw = zeroA, sl = zeroA;
        int64_t cnt = 0;
        R lp[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            lp[k] = 0.f;
            if (p < nl) {
                const int a = SW::at(p);
                RingConst c = ring_const(ctab, idv[k]);
                const R dl = ff_to_f(ff_acc(ff{rh[k], sm.rl[a]}, ff_neg(c.r0)));
                lp[k] = log1pf(dl * __frcp_rn(c.r0.hi));
                sw = ff_acc(sw, c.w);
                sl = ff_acc(sl, ff_acc(c.wl0, ff_two_prod(c.w.hi, lp[k])));
                if (m > 0) cnt += t_cnt[a];
            }
        }
        Trip<A> tot1;
        Trip<A> ex1 = block_excl_scan<false>(Trip<A>{sw, sl, cnt}, OpAddTrip(), Trip<A>{zeroA, zeroA, 0},
                                             reinterpret_cast<Trip<A>*>(sscan), tot1);
        cluster_fold_fwd(cl, tot1, Trip<A>{zeroA, zeroA, 0}, OpAddTrip(), x1_slot, &x1_pre, &x1_all);
        ex1 = OpAddTrip()(x1_pre, ex1);
        const A Wtot = x1_all.x, Ltot = x1_all.y;

        // ---------------- a5: psi, d_rho psi, psibar, gamma, t; beam field
        A S = ex1.x, L = ex1.y;
        A tl = zeroA;
        int lb = (int)ex1.c;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < nl) {
                const int a = SW::at(p);
                if (m > 0) lb += t_cnt[a];
                RingConst c = ring_const(ctab, idv[k]);
                R r = rh[k], u = ur[k];
                A rf = {r, sm.rl[a]};
                A r2 = ff_mul(rf, rf);
                A lnr = ff_add_f(c.ln0, lp[k]);
                A Ir = r < rmax ? ff_mul_f(r2, half_n) : Imax;
                A psion = r <= rmax ? ff_acc(c0, ff_neg(ff_mul_f(r2, quarter_n))) : ff_neg(ff_mul(Imax, lnr));
                R psi = ff_to_f(ff_acc(ff_acc(ff_acc(Ltot, ff_neg(L)), ff_mul(S, lnr)), psion));
                A Sm = ff_acc(S, ff_neg(Ir));
                R dpr = ff_to_f(ff_acc(Sm, c.wh)) * ir[k];
                R pb = 1.f + psi;
                R ip = __frcp_rn(pb);
                pbv[k] = pb;
                ipb[k] = ip;
                dprv[k] = dpr;
                tv[k] = c.w.hi * u * ir[k] * ip;
                sm.D[a] = ff_to_f(Sm);
                sm.S[a] = ff_to_f(S);
                sm.psi[a] = psi;
                R Q = 0.f;
                if (m > 0) Q = lb < m ? W.bE[b0 + lb] : qtot;
                bbv[k] = Q * inv_2pi_dxi * ir[k];
                if (mode == MODE_MARCH && W.dump_psi) {
                    size_t row = (size_t)slice * n + idv[k];
                    W.dump_psi[row] = psi;
                    W.dump_dpr[row] = dpr;
                }
                S = ff_acc(S, c.w);
                L = ff_acc(L, ff_acc(c.wl0, ff_two_prod(c.w.hi, lp[k])));
                tl = ff_add_f(tl, tv[k]);
            } else {
                pbv[k] = 1.f; ipb[k] = 1.f; dprv[k] = 0.f; tv[k] = 0.f; bbv[k] = 0.f;
            }
        }
        A Ttot_blk;
        A Tex = block_excl_scan<false>(tl, OpAdd(), zeroA, reinterpret_cast<A*>(sscan), Ttot_blk);
        cluster_fold_fwd(cl, Ttot_blk, zeroA, OpAdd(), x2_slot, &x2_pre, &x2_all);
        Tex = ff_acc(x2_pre, Tex);
        const A Ttot = x2_all;

        // ---------------- a6 + a7
        Mat2<R> Mf = I2, Mb = I2;
        {
            A Tacc = Tex;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < nl) {
                    const int a = SW::at(p);
                    const float4 cw = __ldg(ctab + 3 * idv[k] + 1);
                    const R w = cw.x, wh = cw.z;
                    R r = rh[k], u = ur[k], dpr = dprv[k], ip = ipb[k], iR = ir[k];
                    sm.T[a] = ff_to_f(ff_acc(Ttot, ff_neg(Tacc)));
                    Tacc = ff_add_f(Tacc, tv[k]);
                    R above = ff_to_f(ff_acc(Ttot, ff_neg(Tacc)));
                    R dpz = -(above + (1.f - wh * __frcp_rn(w)) * tv[k]);
                    tv[k] = dpz;
                    R pb = pbv[k];
                    R g = 0.5f * (1.f + u * u + pb * pb) * ip;
                    R wr = w * iR, ip2 = ip * ip, uu = u * u;
                    R Ac = wr * ip;
                    R Bc = wr * ip2 * (-g * dpr + bbv[k] * pb + uu * dpr * ip - u * dpz) + wr * iR * uu * ip2;
                    R Cc = -wr * (g * ip - 1.f - uu * ip2);
                    R hA = 0.5f * Ac;
                    hav[k] = hA;
                    s0v[k] = 0.25f * (2.f * Bc + Ac * Cc);
                    s1v[k] = 0.25f * r * (4.f * Cc - 2.f * Bc * r - Ac * Cc * r);
                    Mat2<R> M = {1.f + hA * r, hA * iR, -hA * r * r * r, 1.f - hA * r};
                    Mf = OpMatLeft()(Mf, M);
                    if (mode == MODE_MARCH && W.dump_dpz) W.dump_dpz[(size_t)slice * n + idv[k]] = dpz;
                } else {
                    hav[k] = 0.f; s0v[k] = 0.f; s1v[k] = 0.f;
                }
            }
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                if (p0 + k < nl) {
                    R r = rh[k], hA = hav[k];
                    Mat2<R> Mi = {1.f - hA * r, -hA * ir[k], hA * r * r * r, 1.f + hA * r};
                    Mb = OpMatLeft()(Mb, Mi);
                }
            }
        }

        // ---------------- a8: B_theta^(p)
        Mat2<R> Yf, Yb;
        block_excl_scan_mat_fwd_rev(Mf, Mb, reinterpret_cast<Pair<Mat2<R>>*>(sscan), Yf, Yb);
        {
            // this CTA's block totals: the inclusive fold of its last thread
            // (forward) and of its thread 0 (reverse), via shared memory
            Mat2<R>* tmp = reinterpret_cast<Mat2<R>*>(sscan);
            if (tid == T - 1) tmp[0] = OpMatLeft()(Yf, Mf);
            if (tid == 0) tmp[1] = OpMatLeft()(Yb, Mb);
            __syncthreads();
            Mat2<R> tf = tmp[0], tb = tmp[1];
            __syncthreads();
            cluster_fold_fwd(cl, tf, I2, OpMatLeft(), x3f_slot, &x3f_pre, &x3f_all);
            cluster_fold_rev(cl, tb, I2, OpMatLeft(), x3r_slot, &x3r_pre, &x3r_all);
            Yf = OpMatLeft()(x3f_pre, Yf);
            Yb = OpMatLeft()(x3r_pre, Yb);
        }
        R Rra[K], Rrb[K], Dda[K], Ddb[K];
        {
            Mat2<R> Y = Yf;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (p0 + k < nl) {
                    R r = rh[k], hA = hav[k];
                    Mat2<R> M = {1.f + hA * r, hA * ir[k], -hA * r * r * r, 1.f - hA * r};
                    Y = OpMatLeft()(Y, M);
                }
                Rra[k] = Y.m00;
                Rrb[k] = Y.m10;
            }
        }
        A gl = zeroA, dl = zeroA;
        R gpv[K], dpv[K];
        R Dp0a, Dp0b;
        {
            Mat2<R> Y = Yb;
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                Dda[k] = Y.m01;
                Ddb[k] = Y.m11;
                gpv[k] = 0.f;
                dpv[k] = 0.f;
                if (p0 + k < nl) {
                    R q0 = Rra[k], q1 = Rrb[k], d0 = Y.m01, d1 = Y.m11;
                    R iw = __frcp_rn(q0 * d1 - q1 * d0);
                    R gp = (s0v[k] * d1 - s1v[k] * d0) * iw;
                    R dp = (q0 * s1v[k] - q1 * s0v[k]) * iw;
                    gpv[k] = gp;
                    dpv[k] = dp;
                    gl = ff_add_f(gl, gp);
                    dl = ff_add_f(dl, dp);
                    R r = rh[k], hA = hav[k];
                    Mat2<R> Mi = {1.f - hA * r, -hA * ir[k], hA * r * r * r, 1.f + hA * r};
                    Y = OpMatLeft()(Y, Mi);
                }
            }
            Dp0a = Y.m01;
            Dp0b = Y.m11;
        }
        A g_tot, d_tot;
        Pair<A> gd = block_excl_scan_fwd_rev(dl, gl, zeroA, reinterpret_cast<Pair<A>*>(sscan), d_tot, g_tot);
        cluster_fold_fwd(cl, d_tot, zeroA, OpAdd(), x4f_slot, &x4f_pre, &x4f_all);
        cluster_fold_rev(cl, g_tot, zeroA, OpAdd(), x4r_slot, &x4r_pre, &x4r_all);
        gd.x = ff_acc(x4f_pre, gd.x);
        gd.y = ff_acc(x4r_pre, gd.y);
        {
            R Gk[K];
            A Gsuf = gd.y;
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                Gsuf = ff_add_f(Gsuf, gpv[k]);
                Gk[k] = ff_to_f(Gsuf);
            }
            A Hex = gd.x;
            R Rpa = Yf.m00, Rpb = Yf.m10;
            R Dpa = Dp0a, Dpb = Dp0b;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < nl) {
                    R G = Gk[k];
                    R H = ff_to_f(Hex);
                    int a = SW::at(p);
                    sm.a[a] = -G * Rpa + H * Dpa;
                    sm.b[a] = -G * Rpb + H * Dpb;
                    Hex = ff_add_f(Hex, dpv[k]);
                    Rpa = Rra[k];
                    Rpb = Rrb[k];
                    Dpa = Dda[k];
                    Dpb = Ddb[k];
                }
            }
            if (crank == owner_last && p0 < nl && p0 + K >= nl) {  // region n
                const int a = nl < TK ? SW::at(nl) : TK;
                sm.a[a] = 0.f;
                sm.b[a] = ff_to_f(x4f_all);
                sm.T[a] = 0.f;
                sm.D[a] = ff_to_f(ff_acc(Wtot, ff_neg(Imax)));
                sm.S[a] = ff_to_f(Wtot);
                sm.psi[a] = 0.f;
            }
        }
        cl.sync();

        // ---------------- B^(p) at the rings and the guard
        bool bad = false;
        R bpv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            bpv[k] = 0.f;
            if (p < nl) {
                const int a = SW::at(p);
                R a1v, b1v;
                if (p + 1 < nl) {
                    int a1 = SW::at(p + 1);
                    a1v = sm.a[a1];
                    b1v = sm.b[a1];
                } else if (base + p + 1 == n) {  // region n, in this CTA
                    int a1 = nl < TK ? SW::at(nl) : TK;
                    a1v = sm.a[a1];
                    b1v = sm.b[a1];
                } else {  // first region of the next CTA
                    a1v = *rmt(cl, &sm.a[SW::at(0)], crank + 1);
                    b1v = *rmt(cl, &sm.b[SW::at(0)], crank + 1);
                }
                R r = rh[k];
                bpv[k] = 0.5f * ((sm.a[a] + a1v) * r + (sm.b[a] + b1v) * ir[k]);
                R pb = pbv[k];
                if (!(pb > 0.f) || !isfinite(pb) || !isfinite(dprv[k]) || !isfinite(tv[k]) || !isfinite(bpv[k]) ||
                    !isfinite(bbv[k]))
                    bad = true;
                if (mode == MODE_MARCH) {
                    size_t row = (size_t)slice * n + idv[k];
                    if (W.dump_r) W.dump_r[row] = r;
                    if (W.dump_ur) {
                        W.dump_ur[row] = ur[k];
                        W.dump_bp[row] = bpv[k];
                        W.dump_bb[row] = bbv[k];
                    }
                }
            }
        }

        // ---------------- a9: fields on the beam particles (or query radii)
        {
            const int64_t nq = mode == MODE_MARCH ? (int64_t)m : W.nq;
            for (int64_t q = crank * T + tid; q < nq; q += (int64_t)csize * T) {
                R x = mode == MODE_MARCH ? W.br[b0 + q] : (R)W.rq[q];
                R psi, dpr, dpz, bp, bb = 0.f;
                if (x > 0.f) {
                    const int k = cluster_rank<K>(cl, sm, s_first, csize, n, TK, x, true);
                    // region k lives in the CTA holding ring k (region n: the
                    // CTA holding the last ring), at its local index
                    const int ro = k < n ? k / TK : owner_last;
                    const FastSmem so = rmt_sm(cl, sm, ro);
                    const int nl_o = min(TK, n - ro * TK);
                    fast_fields_region<K>(so, nl_o, TK, k - ro * TK, x, rmax, half_n, quarter_n, Wtot, Imax, c0,
                                          &dpr, &dpz, &bp, &psi);
                    if (mode == MODE_MARCH) {
                        bb = W.bQs[b0 + q] * inv_2pi_dxi / x;
                    } else if (m > 0) {
                        int l2 = lower_bound_dev(W.br + b0, m, x);
                        R Q = l2 < m ? W.bE[b0 + l2] : qtot;
                        bb = Q * inv_2pi_dxi / x;
                    }
                } else {
                    psi = ff_to_f(ff_add(Ltot, c0));
                    dpr = 0.f;
                    dpz = -ff_to_f(Ttot);
                    bp = 0.f;
                }
                if (mode == MODE_MARCH) {
                    int64_t o = b0 + q;
                    W.out_ez[o] = -dpz;
                    W.out_wr[o] = -dpr;
                    W.out_bt[o] = bp + bb;
                    W.out_psi[o] = psi;
                } else {
                    if (W.q_ez) W.q_ez[q] = -dpz;
                    if (W.q_wr) W.q_wr[q] = -dpr;
                    if (W.q_bt) W.q_bt[q] = bp + bb;
                    if (W.q_psi) W.q_psi[q] = psi;
                }
            }
        }
        bad = !cluster_all(cl, !__syncthreads_or(bad), s_gvote, &s_vote_out);
        if (mode != MODE_MARCH) break;
        if (bad) {
            status = 4;
            fail = slice;
            ++slice;
            break;
        }

        // ---------------- a10: AB2 push
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < nl) {
                const int a = SW::at(p);
                R u = ur[k], pb = pbv[k], ip = ipb[k];
                R g = 0.5f * (1.f + u * u + pb * pb) * ip;
                R fr = u * ip;
                R fu = g * dprv[k] * ip - (bpv[k] + bbv[k]);
                R drr, du;
                if (has_prev) {
                    drr = dxi * (1.5f * fr - 0.5f * sm.fr[a]);
                    du = dxi * (1.5f * fu - 0.5f * sm.fu[a]);
                } else {
                    drr = dxi * fr;
                    du = dxi * fu;
                }
                ff rr = ff_add_f(ff{rh[k], sm.rl[a]}, drr);
                R un = u + du;
                if (rr.hi < 0.f) {
                    rr = ff_neg(rr);
                    un = -un;
                    fr = -fr;
                    fu = -fu;
                }
                sm.rh[a] = rr.hi;
                sm.rl[a] = rr.lo;
                sm.u[a] = un;
                sm.fr[a] = fr;
                sm.fu[a] = fu;
            }
        }
        has_prev = 1;
        cl.sync();
    }

    cl.sync();
    for (int p = tid; p < nl; p += T) {
        int a = SW::at(p), g = base + p;
        W.rho[buf][g] = sm.rh[a];
        W.rho_lo[g] = sm.rl[a];
        W.ur[buf][g] = sm.u[a];
        W.frho[buf][g] = sm.fr[a];
        W.fur[buf][g] = sm.fu[a];
        W.rid[buf][g] = sm.id[a];
    }
    if (tid == 0 && crank == 0) {
        W.ctl[CTL_NEXT] = mode == MODE_MARCH ? slice : s_ctl[CTL_NEXT];
        W.ctl[CTL_PREV] = has_prev;
        if (status) {
            W.ctl[CTL_STATUS] = status;
            W.ctl[CTL_FAIL] = fail;
        }
    }
}

}  // namespace gbwake
