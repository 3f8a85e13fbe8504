// march_cluster.cuh -- the on-chip march of one wake by a thread-block
// cluster: CTA c of the cluster holds the sorted ring positions
// [c*T*K, (c+1)*T*K) in its shared memory (same layout as march_fast.cuh).
// The per-slice chain is that of march_fast.cuh; what crosses CTAs goes
// through distributed shared memory, pushed by remote stores into each
// peer's receive slots and read locally after one cluster barrier:
//   - the sortedness vote, every CTA's first and last radius and the guard
//     of the previous slice (one exchange at the top of each slice; the AB2
//     push of a slice waits in the dead region-table arrays and becomes the
//     state only if no CTA failed the guard);
//   - the four block-scan totals (each CTA folds the totals of its
//     predecessors, or successors for the reverse scans, in rank order:
//     deterministic), the two matrix scans and the two Green's-function sums
//     sharing one exchange each;
//   - the region table entry just past each CTA's last ring.
// Beam counting and the fields on beam particles stay inside each CTA: each
// CTA takes the particles (or query radii) between the previous CTA's last
// radius and its own, whose rings and regions it holds.  When rings crossed, a local
// bitonic sort in every CTA is followed by odd-even merge-split rounds
// between neighbour CTAs (merge path over the two sorted ranges).
// Every cluster barrier is reached in cluster-uniform control flow.
#pragma once

#include <cooperative_groups.h>

#include "march_fast.cuh"

namespace gbwake {

namespace cg = cooperative_groups;

template <class T>
__device__ __forceinline__ T* rmt(cg::cluster_group& cl, T* p, int rank) {
#ifdef WAKE_BOUNDS_CHECK
    rank = bounds_checked(rank, (int)cl.num_blocks());
#endif
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

// Push of one value per CTA: every CTA stores v into slot [its rank] of
// each peer's recv array (threads 0..size-1, one peer each).  The values are
// read after the next cluster barrier.
template <class T>
__device__ __forceinline__ void cluster_push(cg::cluster_group& cl, T* recv, const T& v) {
    const int rank = cl.block_rank(), size = cl.num_blocks();
    if ((int)threadIdx.x < size) *rmt(cl, &recv[rank], threadIdx.x) = v;
}

// Folds of the received totals in rank order: over ranks < mine (pre) and
// over all ranks (all).  Every thread computes them from shared memory.
template <class T, class Op>
__device__ __forceinline__ void fold_fwd(const T* recv, int rank, int size, T ident, Op op, T& pre, T& all) {
    pre = ident;
    all = ident;
    for (int r = 0; r < size; ++r) {
        if (r == rank) pre = all;
        all = op(all, recv[r]);
    }
}

// the same for a reverse scan: over ranks > mine, from the last rank down
template <class T, class Op>
__device__ __forceinline__ void fold_rev(const T* recv, int rank, int size, T ident, Op op, T& pre, T& all) {
    pre = ident;
    all = ident;
    for (int r = size - 1; r >= 0; --r) {
        if (r == rank) pre = all;
        all = op(all, recv[r]);
    }
}

// The same folds by thread 0 into shared memory, read by every thread after
// a block barrier (keeps the fold's registers out of the callers' peak).
template <class T, class Op>
__device__ __forceinline__ void fold_fwd_shared(const T* recv, int rank, int size, T ident, Op op, T* s_pre,
                                                T* s_all) {
    if (threadIdx.x == 0) {
        T pre, all;
        fold_fwd(recv, rank, size, ident, op, pre, all);
        *s_pre = pre;
        *s_all = all;
    }
    __syncthreads();
}

template <class T, class Op>
__device__ __forceinline__ void fold_rev_shared(const T* recv, int rank, int size, T ident, Op op, T* s_pre,
                                                T* s_all) {
    if (threadIdx.x == 0) {
        T pre, all;
        fold_rev(recv, rank, size, ident, op, pre, all);
        *s_pre = pre;
        *s_all = all;
    }
    __syncthreads();
}

// shared memory of the cluster march: the fast march's arrays plus one
// array of per-ring beam counts (which other CTAs add into)
__host__ __device__ inline size_t cluster_smem_bytes(int T, int K) {
    return fast_smem_bytes(T, K) + 4 * ((size_t)T * K + 8);
}

// block-uniform: are the radii rh (this CTA's rings) in order?
template <int K>
__device__ __forceinline__ bool block_sorted(const float* rh, int nl, int p0) {
    using SW = Swz<K>;
    bool ok = true;
    float prev = -INFINITY;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        int p = p0 + k;
        if (p < nl) {
            float v = rh[SW::at(p)];
            if (v < prev) ok = false;
            prev = v;
        }
    }
    if (p0 + K < nl && rh[SW::at(p0 + K)] < prev) ok = false;
    return __syncthreads_and(ok);
}

// Odd-even merge-split round between neighbour CTAs (left = even ranks when
// parity 0, odd when 1): each CTA of a pair rebuilds its range from the merge
// of the two sorted ranges (ties: left first, which keeps the sort stable).
// Each thread finds its first merged position by a merge-path search and
// records where its outputs come from; the state is then gathered into the
// dead region tables (b, T, D, S, psi; ids in registers) and written back
// once every CTA has read the old ranges.
template <int K>
// scratch: TK words of this CTA's shared memory, zero on entry and on
// return (the beam count array): the partner's radii are copied there first
// (one DSMEM load per word, in flight together), so that the merge-path
// search and the merge read them locally instead of one remote load after
// another.
__device__ void cluster_merge_round(cg::cluster_group& cl, const FastSmem& sm, int n, int TK, int parity,
                                    float* scratch) {
    using SW = Swz<K>;
    const int rank = cl.block_rank(), size = cl.num_blocks();
    const int tid = threadIdx.x;
    int left = -1;
    if ((rank & 1) == parity && rank + 1 < size) left = rank;
    else if (rank >= 1 && ((rank - 1) & 1) == parity) left = rank - 1;
    int32_t* code = reinterpret_cast<int32_t*>(sm.a);  // source: i < nA from A, else nA + j from B
    int g_id[K];
    const bool active = left >= 0;
    int my_n = 0;
    if (active) {
        const int nA = min(TK, n - left * TK);
        const int nB = min(TK, n - (left + 1) * TK);
        const float* partner = rmt(cl, sm.rh, rank == left ? left + 1 : left);
        for (int i = tid; i < TK; i += blockDim.x) scratch[i] = partner[i];
        __syncthreads();  // (active is the same for the whole CTA)
        const float* Arh = rank == left ? sm.rh : scratch;
        const float* Brh = rank == left ? scratch : sm.rh;
        const int off = (rank == left) ? 0 : nA;  // merged position of my local 0
        my_n = (rank == left) ? nA : nB;
        const int d = off + tid * K;
        if (tid * K < my_n) {
            // merge path: i = number of A elements among the first d merged
            int lo = max(0, d - nB), hi = min(d, nA);
            while (lo < hi) {
                int mid = (lo + hi) >> 1;
                if (Arh[SW::at(mid)] <= Brh[SW::at(d - 1 - mid)]) lo = mid + 1;
                else hi = mid;
            }
            int i = lo, j = d - lo;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (tid * K + k < my_n) {
                    const bool takeA = i < nA && (j >= nB || Arh[SW::at(i)] <= Brh[SW::at(j)]);
                    code[tid * K + k] = takeA ? i : nA + j;
                    if (takeA) ++i;
                    else ++j;
                }
            }
        }
        __syncthreads();
        for (int i = tid; i < TK; i += blockDim.x) scratch[i] = 0.f;  // (every search is done)
        const FastSmem A = rmt_sm(cl, sm, left), B = rmt_sm(cl, sm, left + 1);
        for (int l = tid; l < my_n; l += blockDim.x) {
            const int c = code[l];
            const FastSmem& S = c < nA ? A : B;
            const int a = SW::at(c < nA ? c : c - nA);
            sm.b[l] = S.rh[a];
            sm.T[l] = S.rl[a];
            sm.D[l] = S.u[a];
            sm.S[l] = S.fr[a];
            sm.psi[l] = S.fu[a];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = tid * K + k;
            if (l < my_n) {
                const int c = code[l];
                g_id[k] = (c < nA ? A : B).id[SW::at(c < nA ? c : c - nA)];
            }
        }
    }
    cl.sync();  // every read of the old ranges is done
    if (active) {
        for (int l = tid; l < my_n; l += blockDim.x) {
            const int a = SW::at(l);
            sm.rh[a] = sm.b[l];
            sm.rl[a] = sm.T[l];
            sm.u[a] = sm.D[l];
            sm.fr[a] = sm.S[l];
            sm.fu[a] = sm.psi[l];
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int l = tid * K + k;
            if (l < my_n) sm.id[SW::at(l)] = g_id[k];
        }
    }
    cl.sync();
}

template <int K>
__global__ void __launch_bounds__(512)
march_cluster_kernel(const WakeDev<PrecMixed>* __restrict__ wakes, const int32_t* __restrict__ order,
                     int32_t max_slices, int32_t mode, int32_t stage_particles) {
    using R = float;
    using A = ff;
    using SW = Swz<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ctl[CTL_N];
    __shared__ float4 s_xch[16];   // per rank: (in order?, first radius, last radius, failed the guard?)
    __shared__ float s_last[16];   // last radius held by every CTA, this slice
    __shared__ float s_edge[2];    // this CTA's first and last radius (merge rounds)
    __shared__ float2 s_edges[16];  // every CTA's first and last radius (merge rounds)
    __shared__ int s_stop;
    __shared__ float2 s_nab;       // (a, b) of the next CTA's first region
    __shared__ Trip<ff> x1[16], f1[2];
    __shared__ ff x2[16], f2[2];
    __shared__ Mat2<float> x3f[16], x3r[16], f3[4];
    __shared__ ff x4f[16], x4r[16], f4[4];
    __shared__ __align__(8) uint64_t s_bar[2];

    cg::cluster_group cl = cg::this_cluster();
    const int crank = cl.block_rank();
    const int csize = cl.num_blocks();
    const int widx = blockIdx.x / csize;
    const uint64_t t_launch = global_ns();
    const WakeDev<PrecMixed>& W = wakes[order ? order[widx] : widx];
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int n = W.n;
    const int TK = T * K;
    const int base = crank * TK;               // global position of local slot 0
    const int nl = max(0, min(TK, n - base));  // rings held by this CTA (>= 1)
    const int p0 = tid * K;                    // local positions [p0, p0 + K)
    const int cap = TK + 8;
    const bool last_cta = crank == csize - 1;  // holds the last ring and region n
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
    // beam particles counted at each ring position; zero between uses (other
    // CTAs add into it in the distributed count)
    int32_t* cnt_a = reinterpret_cast<int32_t*>(sm.psi + cap);
    for (int i = tid; i < cap; i += blockDim.x) cnt_a[i] = 0;

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
    __syncthreads();

    const double dens_d = W.density, rmax_d = W.rho_max;
    const R rmax = (R)rmax_d;
    const R half_n = (R)(0.5 * dens_d), quarter_n = (R)(0.25 * dens_d);
    const A Imax = ff_from_d(0.5 * dens_d * rmax_d * rmax_d);
    const A c0 = ff_from_d(0.25 * dens_d * rmax_d * rmax_d - 0.5 * dens_d * rmax_d * rmax_d * log(rmax_d));
    const R dxi = (R)W.dxi;
    const R inv_2pi_dxi = (R)(1.0 / (6.283185307179586476925286766559 * W.dxi));
    const A zeroA = {0.f, 0.f};
    const Mat2<R> I2 = {1, 0, 0, 1};

    // beam stage (march only): every CTA stages the whole slice after its
    // ring arrays and its count array
    BeamStage stg;
    stg.base = reinterpret_cast<float*>(smem + cluster_smem_bytes(T, K));
    stg.bar = s_bar;
    stg.cap = (mode == MODE_MARCH && W.nb > 0 && (W.stage & STAGE_OK)) ? stage_cap_floats(stage_particles) : 0;
    // test only: the first slice staged during the march is never copied
    bool stall_armed = (W.stage & STAGE_TEST_STALL) != 0;
    if (stg.cap > 0 && tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
    }
    uint32_t parity = 0;  // per buffer: the phase its next wait completes
    int pending = 0;      // per buffer: a staged copy not yet waited for
    __syncthreads();
    if (stg.cap > 0 && slice < n_steps &&
        stage_slice(stg, W, slice, W.boff[slice], W.boff[slice + 1] - W.boff[slice], false))
        pending |= 1 << (slice & 1);

    R rh[K], ur[K];
    int idv[K];
    R ir[K], ipb[K];
    R pbv[K], dprv[K], bbv[K];
    R s0v[K], s1v[K], hav[K];
    R tv[K];
    // at 8 rings per thread recomputed where used (the same rounding: the
    // same reciprocal of the same value), which keeps 16 registers free
    auto IR = [&](int k) -> R {
        if constexpr (K >= 8) return __frcp_rn(rh[k]);
        else return ir[k];
    };
    auto IPB = [&](int k) -> R {
        if constexpr (K >= 8) return __frcp_rn(pbv[k]);
        else return ipb[k];
    };

    const int slice0 = slice;
    uint64_t t_start = 0;
    bool pending_push = false;  // the table arrays a, b, T, D, S hold the push of slice - 1
    bool blk_bad = false;   // this CTA failed the guard at slice - 1
    int has_prev_before = has_prev;

    for (;;) {
        // the next slice's beam offsets, loaded here so that their latency
        // overlaps the exchange's cluster barrier
        int nxt0 = 0, nxt1 = 0;
        if (stg.cap > 0 && slice + 1 < s_end && slice + 1 < n_steps) {
            nxt0 = W.boff[slice + 1];
            nxt1 = W.boff[slice + 2];
        }
        // ---------------- exchange: order vote, edges, guard of the push
        {
            // time budget: thread 0 of the cluster's rank 0 decides for all
            // (flag 2 of the exchange); read after block_sorted's barrier
            if (W.budget_ns > 0 && crank == 0 && tid == 0) {
                const uint64_t now = global_ns();
                if (slice == slice0) t_start = now;
                s_stop = slice > slice0 && now - t_start >= (uint64_t)W.budget_ns;
            }
            // this slice's staged beam: wait (bounded) before the exchange,
            // so that a wait that gives up stops every CTA alike
            bool stalled = false;
            if (slice < s_end && (pending & (1 << (slice & 1)))) {
                const int bf = slice & 1;
                stalled = __syncthreads_or(!mbar_wait_bounded(&s_bar[bf], (parity >> bf) & 1u));
                parity ^= 1u << bf;
                pending &= ~(1 << bf);
            }
            const float* vr = pending_push ? sm.a : sm.rh;  // the state this slice would start from
            const bool srt = block_sorted<K>(vr, nl, p0);
            const bool stop = W.budget_ns > 0 && crank == 0 && s_stop;
            // flags: 1 failed the guard at slice - 1, 2 stop (time budget),
            // 4 this CTA's staging wait gave up
            if (tid < csize)
                *rmt(cl, &s_xch[crank], tid) = make_float4(srt ? 1.f : 0.f, vr[SW::at(0)], vr[SW::at(nl - 1)],
                                                           (blk_bad ? 1.f : 0.f) + (stop ? 2.f : 0.f) +
                                                               (stalled ? 4.f : 0.f));
        }
        cl.sync();
        bool any_bad = false, all_sorted = true, any_stalled = false;
        const bool stop_now = ((int)s_xch[0].w & 2) != 0;
        for (int r = 0; r < csize; ++r) {
            const float4 v = s_xch[r];
            const int fl = (int)v.w;
            if (fl & 1) any_bad = true;
            if (fl & 4) any_stalled = true;
            if (v.x == 0.f) all_sorted = false;
            if (r + 1 < csize && v.z > s_xch[r + 1].y) all_sorted = false;
        }
        if (any_bad) {  // slice - 1 failed the guard: its push is void
            status = 4;
            fail = slice - 1;
            has_prev = has_prev_before;
            break;
        }
        if (pending_push) {  // commit the push of slice - 1
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < nl) {
                    const int a = SW::at(p);
                    sm.rh[a] = sm.a[a];
                    sm.rl[a] = sm.b[a];
                    sm.u[a] = sm.T[a];
                    sm.fr[a] = sm.D[a];
                    sm.fu[a] = sm.S[a];
                }
            }
            pending_push = false;
            __syncthreads();
        }
        if (any_stalled) {  // the wake stops before this slice
            status = WAKE_STATUS_TIMEOUT;
            fail = slice;
            break;
        }
        if (slice >= s_end || stop_now) break;
        // prefetch the next slice's beam while this one is solved (its
        // buffer was last read by slice - 1, before the last barrier)
        if (slice + 1 < s_end && stage_slice(stg, W, slice + 1, nxt0, nxt1 - nxt0, stall_armed)) {
            pending |= 1 << ((slice + 1) & 1);
            stall_armed = false;
        }
        const int sbuf = slice & 1;

        // ---------------- a2: sort by radius if out of order (cluster-wide)
        if (!all_sorted) {
            // local sort of every CTA's range, then merge-split rounds
            const int nl_pad = nl < 2 ? 2 : 1 << (32 - __clz(nl - 1));
            resort<K>(sm, nl, nl_pad, cap);
            for (int round = 0;; ++round) {
                if (tid == 0) {
                    s_edge[0] = sm.rh[SW::at(0)];
                    s_edge[1] = sm.rh[SW::at(nl - 1)];
                }
                cl.sync();
                // every CTA's edges, one peer per thread (DSMEM loads in
                // flight together), then the vote from the local copies (the
                // same for every thread)
                if (tid < csize) {
                    const float* e = rmt(cl, s_edge, tid);
                    s_edges[tid] = make_float2(e[0], e[1]);
                }
                __syncthreads();
                bool all = true;
                for (int r = 0; r + 1 < csize; ++r)
                    if (s_edges[r].y > s_edges[r + 1].x) all = false;
                // (csize rounds sort any order; the bound is a safeguard)
                if (all || round == 2 * csize + 2) break;
                cl.sync();  // everyone has read the edges before they change
                cluster_merge_round<K>(cl, sm, n, TK, round & 1, reinterpret_cast<float*>(cnt_a));
            }
            if (tid < csize) s_last[tid] = s_edges[tid].y;
        } else if (tid < csize) {
            s_last[tid] = s_xch[tid].z;
        }
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

        // ---------------- a3: beam particles count into their radial place
        // (a particle counts at the first ring above it; the particles of
        // this CTA's rings lie between the previous CTA's last radius and
        // this CTA's last radius, a contiguous range of the sorted slice)
        int b0 = 0, m = 0;
        R qtot = 0;
        if (W.nb > 0 && slice < n_steps) {
            b0 = W.boff[slice];
            m = W.boff[slice + 1] - b0;
            qtot = W.bTot[slice];
        }
        // the slice's beam arrays: from this CTA's stage if they were staged
        SliceBeam sb = {W.br + b0, W.bQs + b0, W.bE + b0};
        const bool in_stage = stg.cap > 0 && stg.fits(m);
        if (in_stage)
            sb = {stg.arr(sbuf, 0) + (b0 & 3), stg.arr(sbuf, 1) + (b0 & 3), stg.arr(sbuf, 2) + (b0 & 3)};
        // Two ways, chosen alike by every CTA: when the slice holds at most a
        // CTA's worth of particles, each CTA counts the particles of its own
        // rings (those between the previous CTA's last radius and its own);
        // else the slice's particles are split evenly over the CTAs, which
        // add into the owning CTA's counts (a cluster barrier then orders the
        // adds before the scan).  Each thread takes a contiguous run of the
        // radius-sorted particles, along which ranks and owners only grow,
        // and adds once per run of particles at the same place.
        __syncthreads();  // (publishes s_last)
        // Usually the slice's radii fit the dead region tables: they are
        // staged there and every thread finds, for each of its rings, how
        // many particles lie strictly below it (a search for the first ring,
        // short walks for the next); cnt_a then holds that number itself.
        const bool staged = m > 0 && (in_stage || m <= kFastArrays / 2 * cap);
        const bool dist = m > T && csize > 1;
        if (staged) {
            const float* pr = sb.br;
            if (!in_stage) {  // copied into the dead tables a, b, T, D, S, psi
                float* prw = sm.a;
                for (int i0 = tid; i0 < m; i0 += kPartBatch * T) {
                    float v[kPartBatch];  // loads in flight together
#pragma unroll
                    for (int j = 0; j < kPartBatch; ++j) v[j] = i0 + j * T < m ? __ldg(W.br + b0 + i0 + j * T) : 0.f;
#pragma unroll
                    for (int j = 0; j < kPartBatch; ++j)
                        if (i0 + j * T < m) prw[i0 + j * T] = v[j];
                }
                __syncthreads();
                pr = prw;
            }
            int L = 0;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const int p = p0 + k;
                if (p < nl) {
                    L = k == 0 ? lower_bound_from(pr, m, 0, rh[k]) : lower_bound_from(pr, m, L, rh[k]);
                    cnt_a[SW::at(p)] = L;
                }
            }
            __syncthreads();  // the staged radii are overwritten from a5 on
        } else if (m > 0) {
            const float* br = sb.br;
            const int mc = dist ? (m + csize - 1) / csize : m;
            const int c0q = dist ? crank * mc : 0;
            const int c1q = dist ? min(m, c0q + mc) : m;
            const int per = (c1q - c0q + T - 1) / T;
            const int q0 = c0q + tid * per, q1 = min(c1q, q0 + per);
            int o = dist ? 0 : crank;                // owner CTA of the current run
            const float lo_own = crank > 0 ? s_last[crank - 1] : -INFINITY;
            int lo = 0, at_lo = -1, cnt = 0;
            bool past = false;
            for (int qb = q0; qb < q1 && !past; qb += kPartBatch) {
                float xb[kPartBatch];  // radii loaded together, then walked
#pragma unroll
                for (int j = 0; j < kPartBatch; ++j) xb[j] = qb + j < q1 ? br[qb + j] : INFINITY;
#pragma unroll
                for (int j = 0; j < kPartBatch; ++j) {
                    const float x = xb[j];
                    if (!dist && !(x >= lo_own)) continue;
                    // owner: the first CTA whose last radius is above x
                    int o2 = o;
                    while (o2 < csize && !(x < s_last[o2])) ++o2;
                    if (o2 >= csize || (!dist && o2 != crank)) {  // beyond (or outside this CTA)
                        past = true;
                        break;
                    }
                    if (o2 != o) {
                        if (cnt) atomicAdd(o == crank ? &cnt_a[SW::at(at_lo)] : rmt(cl, &cnt_a[SW::at(at_lo)], o), cnt);
                        o = o2;
                        lo = 0;
                        at_lo = -1;
                        cnt = 0;
                    }
                    const int nl_o = min(TK, n - o * TK);
                    const float* rh_o = o == crank ? sm.rh : rmt(cl, sm.rh, o);
                    lo = ring_rank_from<K>(rh_o, nl_o, lo, x, false);
                    if (lo != at_lo) {
                        if (cnt) atomicAdd(o == crank ? &cnt_a[SW::at(at_lo)] : rmt(cl, &cnt_a[SW::at(at_lo)], o), cnt);
                        at_lo = lo;
                        cnt = 0;
                    }
                    ++cnt;
                }
            }
            if (cnt) atomicAdd(o == crank ? &cnt_a[SW::at(at_lo)] : rmt(cl, &cnt_a[SW::at(at_lo)], o), cnt);
            if (dist) cl.sync();
            else __syncthreads();
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
                lp[k] = log1pf(dl * c.ir0);
                sw = ff_acc(sw, c.w);
                sl = ff_acc(sl, ff_acc(c.wl0, ff_two_prod(c.w.hi, lp[k])));
                if (m > 0 && !staged) cnt += cnt_a[a];
            }
        }
        Trip<A> ex1;
        A Wtot, Ltot;
        {
            Trip<A> tot1, pre1, all1;
            // (one-barrier scans: a cluster barrier separates each from the next)
            ex1 = block_excl_scan1<false>(Trip<A>{sw, sl, cnt}, OpAddTrip(), Trip<A>{zeroA, zeroA, 0},
                                          reinterpret_cast<Trip<A>*>(sscan), tot1);
            cluster_push(cl, x1, tot1);
            cl.sync();
            fold_fwd_shared(x1, crank, csize, Trip<A>{zeroA, zeroA, 0}, OpAddTrip(), &f1[0], &f1[1]);
            pre1 = f1[0];
            all1 = f1[1];
            ex1 = OpAddTrip()(pre1, ex1);
            Wtot = all1.x;
            Ltot = all1.y;
        }

        // ---------------- a5: psi, d_rho psi, psibar, gamma, t; beam field
        A S = ex1.x, L = ex1.y;
        A tl = zeroA;
        int lb = (int)ex1.c;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < nl) {
                const int a = SW::at(p);
                if (m > 0) {
                    lb = staged ? cnt_a[a] : lb + cnt_a[a];
                    cnt_a[a] = 0;  // read for the last time this slice
                }
                RingConst c = ring_const(ctab, idv[k]);
                R r = rh[k], u = ur[k];
                A rf = {r, sm.rl[a]};
                A r2 = ff_mul(rf, rf);
                A lnr = ff_add_f(c.ln0, lp[k]);
                A Ir = r < rmax ? ff_mul_f(r2, half_n) : Imax;
                A psion = r <= rmax ? ff_acc(c0, ff_neg(ff_mul_f(r2, quarter_n))) : ff_neg(ff_mul(Imax, lnr));
                R psi = ff_to_f(ff_acc(ff_acc(ff_acc(Ltot, ff_neg(L)), ff_mul(S, lnr)), psion));
                A Sm = ff_acc(S, ff_neg(Ir));
                R dpr = ff_to_f(ff_acc(Sm, c.wh)) * IR(k);
                R pb = 1.f + psi;
                R ip = __frcp_rn(pb);
                pbv[k] = pb;
                ipb[k] = ip;
                dprv[k] = dpr;
                tv[k] = c.w.hi * u * IR(k) * ip;
                sm.D[a] = ff_to_f(Sm);
                sm.S[a] = ff_to_f(S);
                sm.psi[a] = psi;
                R Q = 0.f;
                if (m > 0) Q = lb < m ? sb.be[lb] : qtot;
                bbv[k] = Q * inv_2pi_dxi * IR(k);
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
        A Tex, Ttot;
        {
            A Ttot_blk, pre2;
            Tex = block_excl_scan1<false>(tl, OpAdd(), zeroA, reinterpret_cast<A*>(sscan), Ttot_blk);
            cluster_push(cl, x2, Ttot_blk);
            cl.sync();
            fold_fwd_shared(x2, crank, csize, zeroA, OpAdd(), &f2[0], &f2[1]);
            pre2 = f2[0];
            Ttot = f2[1];
            Tex = ff_acc(pre2, Tex);
        }

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
                    R r = rh[k], u = ur[k], dpr = dprv[k], ip = IPB(k), iR = IR(k);
                    sm.T[a] = ff_to_f(ff_acc(Ttot, ff_neg(Tacc)));
                    Tacc = ff_add_f(Tacc, tv[k]);
                    R above = ff_to_f(ff_acc(Ttot, ff_neg(Tacc)));
                    R dpz = -(above + (1.f - wh * __ldg(reinterpret_cast<const float*>(ctab + 3 * idv[k] + 2) + 2)) * tv[k]);
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
                    Mat2<R> Mi = {1.f - hA * r, -hA * IR(k), hA * r * r * r, 1.f + hA * r};
                    Mb = OpMatLeft()(Mb, Mi);
                }
            }
        }

        // ---------------- a8: B_theta^(p)
        Mat2<R> Yf, Yb;
        {
            // this CTA's forward and reverse products go to every CTA
            Mat2<R> tf, tb;
            block_excl_scan_mat_fwd_rev1<true>(Mf, Mb, reinterpret_cast<Pair<Mat2<R>>*>(sscan), Yf, Yb, tf, tb);
            if (tid < csize) {
                *rmt(cl, &x3f[crank], tid) = tf;
                *rmt(cl, &x3r[crank], tid) = tb;
            }
            cl.sync();
            if (tid == 32 % T) {
                Mat2<R> pre, all;
                fold_rev(x3r, crank, csize, I2, OpMatLeft(), pre, all);
                f3[2] = pre;
            }
            fold_fwd_shared(x3f, crank, csize, I2, OpMatLeft(), &f3[0], &f3[1]);
            Yf = OpMatLeft()(f3[0], Yf);
            Yb = OpMatLeft()(f3[2], Yb);
        }
        R Rra[K], Rrb[K], Dda[K], Ddb[K];
        {
            Mat2<R> Y = Yf;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (p0 + k < nl) {
                    R r = rh[k], hA = hav[k];
                    Mat2<R> M = {1.f + hA * r, hA * IR(k), -hA * r * r * r, 1.f - hA * r};
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
                    Mat2<R> Mi = {1.f - hA * r, -hA * IR(k), hA * r * r * r, 1.f + hA * r};
                    Y = OpMatLeft()(Y, Mi);
                }
            }
            Dp0a = Y.m01;
            Dp0b = Y.m11;
        }
        A g_tot, d_tot;
        Pair<A> gd = block_excl_scan_fwd_rev1(dl, gl, zeroA, reinterpret_cast<Pair<A>*>(sscan), d_tot, g_tot);
        A all4f;
        {
            if (tid < csize) {
                *rmt(cl, &x4f[crank], tid) = d_tot;
                *rmt(cl, &x4r[crank], tid) = g_tot;
            }
            cl.sync();
            if (tid == 32 % T) {
                A pre, all;
                fold_rev(x4r, crank, csize, zeroA, OpAdd(), pre, all);
                f4[2] = pre;
            }
            fold_fwd_shared(x4f, crank, csize, zeroA, OpAdd(), &f4[0], &f4[1]);
            all4f = f4[1];
            gd.x = ff_acc(f4[0], gd.x);
            gd.y = ff_acc(f4[2], gd.y);
        }
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
            if (last_cta && p0 < nl && p0 + K >= nl) {  // region n
                const int a = nl < TK ? SW::at(nl) : TK;
                sm.a[a] = 0.f;
                sm.b[a] = ff_to_f(all4f);
                sm.T[a] = 0.f;
                sm.D[a] = ff_to_f(ff_acc(Wtot, ff_neg(Imax)));
                sm.S[a] = ff_to_f(Wtot);
                sm.psi[a] = 0.f;
            }
        }
        // the next CTA's first region, for B^(p) at this CTA's last ring
        if (tid == 0 && crank > 0) *rmt(cl, &s_nab, crank - 1) = make_float2(sm.a[SW::at(0)], sm.b[SW::at(0)]);
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
                } else if (last_cta) {  // region n
                    int a1 = nl < TK ? SW::at(nl) : TK;
                    a1v = sm.a[a1];
                    b1v = sm.b[a1];
                } else {  // first region of the next CTA
                    a1v = s_nab.x;
                    b1v = s_nab.y;
                }
                R r = rh[k];
                bpv[k] = 0.5f * ((sm.a[a] + a1v) * r + (sm.b[a] + b1v) * IR(k));
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
        // Region k (radii in (rho_{k-1}, rho_k]) lives in the CTA holding
        // ring k, region n in the last CTA: this CTA serves the radii in
        // (previous CTA's last radius, its own last radius].
        {
            const float lo_r = crank > 0 ? s_last[crank - 1] : -INFINITY;
            const float hi_r = last_cta ? INFINITY : s_last[crank];
            if (mode == MODE_MARCH) {
                // the particles split as in a3 (own range, or an even share
                // of the slice with the owner's tables read remotely);
                // region k (radii in (rho_{k-1}, rho_k]) lives in the CTA
                // holding ring k, region n in the last CTA
                const int mc = dist ? (m + csize - 1) / csize : m;
                const int c0q = dist ? crank * mc : 0;
                const int c1q = dist ? min(m, c0q + mc) : m;
                const int per = (c1q - c0q + T - 1) / T;
                const int q0 = c0q + tid * per, q1 = min(c1q, q0 + per);
                int o = crank, kr = 0;  // owner of the current run and its tables
                FastSmem so = sm;
                int nl_o = nl;
                bool past = false;
                for (int qb = q0; qb < q1 && !past; qb += kPartBatch) {
                  float xb[kPartBatch], qb_s[kPartBatch];  // loaded together, then evaluated
#pragma unroll
                  for (int j = 0; j < kPartBatch; ++j) {
                      xb[j] = qb + j < q1 ? sb.br[qb + j] : INFINITY;
                      qb_s[j] = qb + j < q1 ? sb.qs[qb + j] : 0.f;
                  }
#pragma unroll
                  for (int j = 0; j < kPartBatch; ++j) {
                    const int q = qb + j;
                    const R x = xb[j];
                    if (q >= q1) {
                        past = true;
                        break;
                    }
                    if (!dist && !(x > lo_r)) continue;
                    int o2 = dist && q == q0 ? 0 : o;  // owners only grow along the run
                    while (o2 + 1 < csize && !(x <= s_last[o2])) ++o2;
                    if (!dist && o2 != crank) {
                        past = true;
                        break;
                    }
                    if (o2 != o) {
                        o = o2;
                        so = o == crank ? sm : rmt_sm(cl, sm, o);
                        nl_o = min(TK, n - o * TK);
                        kr = 0;
                    }
                    R psi, dpr, dpz, bp, bb = 0.f;
                    if (x > 0.f) {
                        kr = ring_rank_from<K>(so.rh, nl_o, kr, x, true);
                        fast_fields_region<K>(so, nl_o, TK, kr, x, rmax, half_n, quarter_n, Wtot, Imax, c0, &dpr,
                                              &dpz, &bp, &psi);
                        bb = qb_s[j] * inv_2pi_dxi / x;
                    } else {
                        psi = ff_to_f(ff_add(Ltot, c0));
                        dpr = 0.f;
                        dpz = -ff_to_f(Ttot);
                        bp = 0.f;
                    }
                    const int64_t o_idx = b0 + q;
                    W.out_ez[o_idx] = -dpz;
                    W.out_wr[o_idx] = -dpr;
                    W.out_bt[o_idx] = bp + bb;
                    W.out_psi[o_idx] = psi;
                  }
                }
                // no CTA may overwrite its tables (the push lands there)
                // while another still reads them
                if (dist) cl.sync();
            } else {
                for (int64_t q = tid; q < W.nq; q += T) {
                    const R x = (R)W.rq[q];
                    // a radius belongs here if lo_r < x <= hi_r (CTA 0 also
                    // takes a NaN query, which no comparison places)
                    if (!(x > lo_r && x <= hi_r) && !(crank == 0 && x != x)) continue;
                    R psi, dpr, dpz, bp, bb = 0.f;
                    if (x > 0.f) {
                        const int kl = ring_rank<K>(sm.rh, nl, x, true);
                        fast_fields_region<K>(sm, nl, TK, kl, x, rmax, half_n, quarter_n, Wtot, Imax, c0, &dpr,
                                              &dpz, &bp, &psi);
                        if (m > 0) {
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
                    if (W.q_ez) W.q_ez[q] = -dpz;
                    if (W.q_wr) W.q_wr[q] = -dpr;
                    if (W.q_bt) W.q_bt[q] = bp + bb;
                    if (W.q_psi) W.q_psi[q] = psi;
                }
            }
        }
        blk_bad = __syncthreads_or(bad);  // (every read of the tables is done)
        if (mode != MODE_MARCH) break;

        // ---------------- a10: AB2 push into the table arrays (dead after
        // a9); it becomes the state at the next exchange unless some CTA
        // failed the guard
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < nl) {
                const int a = SW::at(p);
                R u = ur[k], pb = pbv[k], ip = IPB(k);
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
                sm.a[a] = rr.hi;
                sm.b[a] = rr.lo;
                sm.T[a] = un;
                sm.D[a] = fr;
                sm.S[a] = fu;
            }
        }
        has_prev_before = has_prev;
        has_prev = 1;
        pending_push = true;
        ++slice;
        __syncthreads();  // the pushed state is read across threads next
    }
    // no bulk copy may still write this CTA's shared memory when it exits:
    // wait (bounded) for any staged slice that was not consumed
    for (int bf = 0; bf < 2; ++bf)
        if ((pending & (1 << bf)) && !mbar_wait_bounded(&s_bar[bf], (parity >> bf) & 1u) && status == 0) {
            status = WAKE_STATUS_TIMEOUT;
            fail = slice;
        }
    cl.sync();  // no CTA leaves while a peer may still touch its shared memory

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
        if (mode == MODE_MARCH) put_march_times(W.ctl, t_launch);
        W.ctl[CTL_NEXT] = mode == MODE_MARCH ? slice : s_ctl[CTL_NEXT];
        W.ctl[CTL_PREV] = has_prev;
        if (status) {
            W.ctl[CTL_STATUS] = status;
            W.ctl[CTL_FAIL] = fail;
        }
    }
}

}  // namespace gbwake
