// march_fast.cuh -- the production march (mixed precision): one wake per
// thread block with the ring state resident on chip for the whole window.
//
// Thread t owns the K consecutive sorted positions [tK, tK+K) (K a
// compile-time constant) and keeps their per-slice quantities in registers.
// The ring state -- radius as a float-float pair, u_r, the AB2 history, ring
// id -- lives in shared memory in a swizzled blocked layout that makes the
// K-strided accesses bank-conflict free.
//
// Precision.  The electron sums (sum w ln rho ~ n rho_max^2 ln rho_max) and
// the ion column cancel to leave psi ~ O(1), so ln rho is split into the
// ring's constant ln rho0 (FP64-rounded float-float, from a per-ring
// constant table) plus log1p(delta/rho0) in float, delta = rho - rho0 being
// the ring's displacement from its initial cell centre; rho itself is
// integrated as a float-float pair.  Prefix sums, psi and d_rho psi are
// assembled in float-float; everything else is float.
//
// Per slice:
//   a2  sortedness check; bitonic sort of (rho, position) only if needed
//   a3  beam -> rings: each beam particle of the slice finds its radial
//       place among the rings (binary search in shared memory) and counts
//       into it; the count prefix (folded into the first block scan) gives
//       the enclosed beam charge at every ring
//   a4  block scan of (sum w, sum w ln rho, counts)
//   a5  psi, d_rho psi (self weight), psibar, gamma, t
//   a6  block scan of t -> d_zeta psi
//   a7  A, B, C and the ring sources of the B_theta^(p) system
//   a8  B_theta^(p): regular (forward) and decaying (backward) homogeneous
//       solutions from one forward+reverse 2x2 matrix-product scan, then the
//       discrete Green's function sums (one forward+reverse scan)
//   a9  fields at the slice's beam particles from per-region tables
//   a10 AB2 push (rho in float-float), axis reflection
#pragma once

#include "march.cuh"
#include "stage.cuh"

namespace gbwake {

#ifdef WAKE_BOUNDS_CHECK
// Debug build: every swizzled shared-memory position and every DSMEM peer
// rank is checked; one out of range is counted here (one counter per
// translation unit, read by the march_*_bounds_violations functions) and
// replaced by 0, which is always in range, so that the kernel goes on.
static __device__ unsigned long long g_bounds_violations;
__device__ __forceinline__ int bounds_checked(int i, int n) {
    if (i < 0 || i >= n) {
        atomicAdd(&g_bounds_violations, 1ull);
        return 0;
    }
    return i;
}
#endif

template <int K>
struct Swz {
    // position p (thread p/K, slot p%K) -> shared-memory word; XOR-swizzle of
    // the slot by the thread's group so that the K-strided accesses of a warp
    // hit 32 distinct banks
    static constexpr int kShift = (K == 2) ? 4 : (K == 4) ? 3 : (K == 8 ? 2 : (K == 16 ? 1 : 0));
    __device__ __forceinline__ static int at(int p) {
#ifdef WAKE_BOUNDS_CHECK
        p = bounds_checked(p, (int)blockDim.x * K);
#endif
        int t = p / K, j = p % K;
        return t * K + (j ^ ((t >> kShift) & (K - 1)));
    }
};

constexpr int kFastArrays = 12;  // 6 state + 6 region-table arrays

// shared-memory footprint of the fast march for blocks of T threads
__host__ __device__ inline size_t fast_smem_bytes(int T, int K) {
    size_t cap = (size_t)T * K + 8;  // ring positions (+ region n)
    return (size_t)kScanBytes + kFastArrays * 4 * cap;
}

struct RingConst {
    ff r0, ln0, w, wh, wl0;  // rho0, ln rho0, w, what, w ln rho0
    float iw, ir0;           // 1/w and 1/rho0 (of the high parts, rounded to nearest)
};
__device__ __forceinline__ RingConst ring_const(const float4* __restrict__ ctab, int id) {
    float4 a = __ldg(ctab + 3 * id), b = __ldg(ctab + 3 * id + 1), c = __ldg(ctab + 3 * id + 2);
    return {{a.x, a.y}, {a.z, a.w}, {b.x, b.y}, {b.z, b.w}, {c.x, c.y}, c.z, c.w};
}

// shared-memory arrays of the fast march
struct FastSmem {
    float *rh, *rl, *u, *fr, *fu;    // rho (hi, lo), u_r, AB2 history (sorted)
    int32_t* id;                     // ring ids
    float *a, *b, *T, *D, *S, *psi;  // region tables
};

// (key, previous position) pairs in the order of the stable sort
struct KeySrc {
    float key;
    int src;
};
__device__ __forceinline__ bool ks_less(const KeySrc& a, const KeySrc& b) {
    return a.key < b.key || (a.key == b.key && a.src < b.src);
}
__device__ __forceinline__ void ks_order(KeySrc& a, KeySrc& b) {
    if (ks_less(b, a)) {
        KeySrc t = a;
        a = b;
        b = t;
    }
}
// sorts v[0, K) ascending (K a power of two): bitonic network, static indices
template <int K>
__device__ __forceinline__ void ks_sort(KeySrc (&v)[K]) {
#pragma unroll
    for (int k2 = 2; k2 <= K; k2 <<= 1)
#pragma unroll
        for (int j = k2 >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < K; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    if ((i & k2) == 0) ks_order(v[i], v[l]);
                    else ks_order(v[l], v[i]);
                }
            }
}
// a bitonic v (after a half-cleaner) into ascending order
template <int K>
__device__ __forceinline__ void ks_bitonic_finish(KeySrc (&v)[K]) {
#pragma unroll
    for (int j = K >> 1; j > 0; j >>= 1)
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int l = i ^ j;
            if (l > i) ks_order(v[i], v[l]);
        }
}

// Re-sort of the ring state by (rho, previous position), i.e. the sort that
// is stable with respect to the previous order, after a push in which rings
// crossed.  Every thread sorts its K rings' keys in registers, then odd-even
// merge-split rounds between neighbouring threads' runs move rings up to K
// places per round, which suffices when rings crossed by few places; after
// kNearRounds rounds still out of order, a bitonic sort of the same keys.
// Either way the permutation is the stable sort's.  Keys and indices live in
// the dead region tables (a..D) and the state is gathered through S and psi,
// so that it adds few registers to the march loop.
constexpr int kNearRounds = 8;
// beam particles whose radii (and charges) one thread loads together in a3/a9
constexpr int kPartBatch = 8;
template <int K>
__device__ __forceinline__ void resort(const FastSmem& sm, int n, int n_pad, int cap) {
    using SW = Swz<K>;
    const int T = blockDim.x, tid = threadIdx.x, p0 = tid * K;
    float* key = sm.a;                                         // [n_pad] over a, b
    int32_t* idx = reinterpret_cast<int32_t*>(sm.a + 2 * cap);  // [n_pad] over T, D
    bool sorted = false;
    {
        KeySrc v[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const int p = p0 + k;
            v[k].key = p < n ? sm.rh[SW::at(p)] : INFINITY;
            v[k].src = p;
        }
        ks_sort<K>(v);
        for (int round = 0; round <= kNearRounds; ++round) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                key[p0 + k] = v[k].key;
                idx[p0 + k] = v[k].src;
            }
            __syncthreads();
            const bool ok = tid + 1 >= T || !ks_less(KeySrc{key[p0 + K], idx[p0 + K]}, v[K - 1]);
            if (__syncthreads_and(ok)) {
                sorted = true;
                break;
            }
            if (round == kNearRounds) break;
            const bool left = (tid & 1) == (round & 1);
            const int partner = left ? tid + 1 : tid - 1;
            if (partner >= 0 && partner < T) {
#pragma unroll
                for (int k = 0; k < K; ++k) {  // half-cleaner against the partner's run, reversed
                    const int q = partner * K + (K - 1 - k);
                    const KeySrc w = {key[q], idx[q]};
                    const bool lt = ks_less(v[k], w);
                    if (left ? !lt : lt) v[k] = w;
                }
                ks_bitonic_finish<K>(v);
            }
            __syncthreads();
        }
    }
    if (!sorted) {  // bitonic sort of (key, index) from the previous order, padded to n_pad
        for (int i = tid; i < n_pad; i += T) {
            key[i] = i < n ? sm.rh[SW::at(i)] : INFINITY;
            idx[i] = i;
        }
        __syncthreads();
        for (int k2 = 2; k2 <= n_pad; k2 <<= 1) {
            for (int j = k2 >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < n_pad; i += T) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const float ki = key[i], kj = key[ixj];
                        const int vi = idx[i], vj = idx[ixj];
                        const bool gt = (ki > kj) || (ki == kj && vi > vj);
                        if (gt == ((i & k2) == 0)) {
                            key[i] = kj;
                            key[ixj] = ki;
                            idx[i] = vj;
                            idx[ixj] = vi;
                        }
                    }
                }
                __syncthreads();
            }
        }
    }
    // gather the state into sorted order, two arrays per pass through S, psi
    float* g0 = sm.S;
    float* g1 = sm.psi;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
        float* x0 = pass == 0 ? sm.rh : pass == 1 ? sm.u : sm.fu;
        float* x1 = pass == 0 ? sm.rl : pass == 1 ? sm.fr : reinterpret_cast<float*>(sm.id);
        for (int i = tid; i < n; i += T) {
            const int a = SW::at(idx[i]);
            g0[i] = x0[a];
            g1[i] = x1[a];
        }
        __syncthreads();
        for (int i = tid; i < n; i += T) {
            const int a = SW::at(i);
            x0[a] = g0[i];
            x1[a] = g1[i];
        }
        __syncthreads();
    }
}

// number of sorted rings with radius < x (strict) or <= x
template <int K>
__device__ __forceinline__ int ring_rank(const float* rh, int n, float x, bool strict) {
    using SW = Swz<K>;
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        float v = rh[SW::at(mid)];
        if (strict ? (v < x) : (v <= x)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Rank of x among the sorted radii rh[0, n) (how many are < x, or <= x when
// !strict), given a rank `from` that does not exceed it: galloping from
// `from` (steps 1, 2, 4, ...), then a binary search inside the last step.
// Along a run of increasing radii successive ranks are close, so this costs
// O(log distance) instead of O(log n).
template <int K>
__device__ __forceinline__ int ring_rank_from(const float* rh, int n, int from, float x, bool strict) {
    using SW = Swz<K>;
    auto below = [&](int i) {
        const float v = rh[SW::at(i)];
        return strict ? (v < x) : (v <= x);
    };
    if (from >= n || !below(from)) return from;
    int lo = from, step = 1;  // invariant: below(lo)
    int hi = lo + 1;
    while (hi < n && below(hi)) {
        lo = hi;
        step <<= 1;
        hi = lo + step;
    }
    if (hi > n) hi = n;
    ++lo;  // the answer is in [lo, hi]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (below(mid)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// First index i >= from of the sorted a[0, n) with a[i] >= x, given that
// a[from - 1] < x (or from = 0): galloping then a binary search, as above.
__device__ __forceinline__ int lower_bound_from(const float* a, int n, int from, float x) {
    if (from >= n || !(a[from] < x)) return from;
    int lo = from, step = 1;
    int hi = lo + 1;
    while (hi < n && a[hi] < x) {
        lo = hi;
        step <<= 1;
        hi = lo + step;
    }
    if (hi > n) hi = n;
    ++lo;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Fields at radius x > 0 of the current slice from the region tables
// (Eqs. b_theta_plasma..dpsi_dzeta off the rings): d_rho psi, d_zeta psi,
// B^(p), psi.  kl = number of rings (of this table's nl) below x; kl = nl
// means beyond every ring.
template <int K>
__device__ __forceinline__ void fast_fields_region(const FastSmem& sm, int nl, int TK, int kl, float x, float rmax,
                                                   float half_n, float quarter_n, ff Wtot, ff Imax, ff c0,
                                                   float* dpr, float* dpz, float* bp, float* psi) {
    using SW = Swz<K>;
    const int a = kl < TK ? SW::at(kl) : TK;
    const float cx = fminf(x, rmax);
    if (kl < nl) {
        const float rk = sm.rh[a];
        const float ck = fminf(rk, rmax);
        // S_k - I(x): near ring k from D_k = S_k - I(rho_k) (both small in a
        // near-neutral plasma), across a wide gap from S_k directly
        float s_ix = (ck < 2.f * cx) ? sm.D[a] + half_n * (ck - cx) * (ck + cx) : sm.S[a] - half_n * cx * cx;
        *dpr = s_ix / x;
        // psi(x) = psi_k - S_k ln(rho_k/x) + (J(rho_k) - J(x)), J(r) = int_0^r I/r'
        const float lnk = log1pf((rk - x) / x);
        float dJ;
        if (rk <= rmax) dJ = quarter_n * (rk - x) * (rk + x);
        else if (x >= rmax) dJ = half_n * rmax * rmax * lnk;
        else dJ = quarter_n * (rmax - x) * (rmax + x) + half_n * rmax * rmax * logf(rk / rmax);
        *psi = sm.psi[a] - (sm.S[a] * lnk - dJ);
    } else {
        // beyond every ring: S = W_tot
        *dpr = (sm.D[a] + half_n * (rmax - cx) * (rmax + cx)) / x;
        ff lnx = {logf(x), 0.f};
        ff psion = x <= rmax ? ff_sub(c0, ff_mul_f(ff_two_prod(x, x), quarter_n)) : ff_neg(ff_mul(Imax, lnx));
        *psi = ff_to_f(ff_add(ff_mul(Wtot, lnx), psion));
    }
    *dpz = -sm.T[a];
    *bp = sm.a[a] * x + sm.b[a] / x;
}

template <int K>
__device__ __forceinline__ void fast_fields_at(const FastSmem& sm, int n, int TK, float x, float rmax, float half_n,
                                               float quarter_n, ff Wtot, ff Imax, ff c0, float* dpr, float* dpz,
                                               float* bp, float* psi) {
    const int k = ring_rank<K>(sm.rh, n, x, true);
    fast_fields_region<K>(sm, n, TK, k, x, rmax, half_n, quarter_n, Wtot, Imax, c0, dpr, dpz, bp, psi);
}

// Beam arrays of the slice being solved: staged in shared memory (TMA bulk
// copies, prefetched during the previous slice) or read from global memory
// when the slice is denser than the stage.  Particle q is at index q.
struct SliceBeam {
    const float* br;   // radius-sorted radii
    const float* qs;   // enclosed charge of each particle
    const float* be;   // exclusive charge prefix
};

// Issues the stage of slice s (particles [b0, b0 + m)) if it fits into
// buffer s & 1; every thread can tell from the offsets whether it was staged.
__device__ __forceinline__ bool stage_slice(const BeamStage& st, const WakeDev<PrecMixed>& W, int s, int b0, int m,
                                            bool skip) {
    if (st.cap == 0 || !st.fits(m)) return false;
    if (threadIdx.x == 0) stage_issue(st, s & 1, W.br, W.bQs, W.bE, b0, m, skip);
    return true;
}

// The beam offsets of slices s, s + 1 and s + 2, loaded one slice ahead so
// that their latency stays off the start of the slice, where the next
// slice's stage is issued (slices at or beyond the window hold nothing).
struct SliceOffsets {
    int o0, o1, o2;
    __device__ __forceinline__ void load(const WakeDev<PrecMixed>& W, int s, int n_steps) {
        o0 = s < n_steps ? W.boff[s] : 0;
        o1 = s + 1 <= n_steps ? W.boff[s + 1] : o0;
        o2 = s + 2 <= n_steps ? W.boff[s + 2] : o1;
    }
    // to slice s + 1
    __device__ __forceinline__ void advance(const WakeDev<PrecMixed>& W, int s, int n_steps) {
        o0 = o1;
        o1 = o2;
        o2 = s + 3 <= n_steps ? W.boff[s + 3] : o1;
    }
};

template <int K>
__global__ void __launch_bounds__(512)
march_fast_kernel(const WakeDev<PrecMixed>* __restrict__ wakes, const int32_t* __restrict__ order,
                  int32_t max_slices, int32_t mode, int32_t stage_particles) {
    using R = float;
    using A = ff;
    using SW = Swz<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ctl[CTL_N];
    __shared__ int s_stop;
    __shared__ __align__(8) uint64_t s_bar[2];

    const uint64_t t_launch = global_ns();
    const WakeDev<PrecMixed>& W = wakes[order ? order[blockIdx.x] : blockIdx.x];
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int n = W.n;
    const int p0 = tid * K;
    const int TK = T * K;
    const int cap = TK + 8;
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
    int32_t* t_cnt = reinterpret_cast<int32_t*>(sm.a);  // beam counts (reuses the a table)

    if (tid < CTL_N) s_ctl[tid] = W.ctl[tid];
    __syncthreads();
    if (s_ctl[CTL_STATUS] != 0) return;
    int slice = s_ctl[CTL_NEXT];
    const int buf = s_ctl[CTL_BUF];
    int has_prev = s_ctl[CTL_PREV];
    int status = 0, fail = -1;
    const int n_steps = W.n_steps;
    const int s_end = mode == MODE_MARCH ? min(n_steps, slice + max_slices) : slice + 1;

    // ---- load the ring state (global, sorted) into shared memory
    for (int p = tid; p < n; p += T) {
        int a = SW::at(p);
        sm.rh[a] = W.rho[buf][p];
        sm.rl[a] = W.rho_lo[p];
        sm.u[a] = W.ur[buf][p];
        sm.fr[a] = W.frho[buf][p];
        sm.fu[a] = W.fur[buf][p];
        sm.id[a] = W.rid[buf][p];
    }
    __syncthreads();

    // beam stage (march only): two buffers after the ring arrays
    BeamStage stg;
    stg.base = reinterpret_cast<float*>(smem + fast_smem_bytes(T, K));
    stg.bar = s_bar;
    stg.cap = (mode == MODE_MARCH && W.nb > 0 && (W.stage & STAGE_OK)) ? stage_cap_floats(stage_particles) : 0;
    // test only: the first slice staged during the march is never copied
    bool stall_armed = (W.stage & STAGE_TEST_STALL) != 0;
    if (stg.cap > 0 && tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        mbar_fence_init();
    }
    uint32_t parity = 0;     // per buffer: the phase its next wait completes
    int pending = 0;         // per buffer: a staged copy not yet waited for
    SliceOffsets so;
    if (W.nb > 0) so.load(W, slice, n_steps);
    else so = {0, 0, 0};
    __syncthreads();
    if (slice < n_steps && stage_slice(stg, W, slice, so.o0, so.o1 - so.o0, false)) pending |= 1 << (slice & 1);

    const double dens_d = W.density, rmax_d = W.rho_max;
    const R rmax = (R)rmax_d;
    const R half_n = (R)(0.5 * dens_d), quarter_n = (R)(0.25 * dens_d);
    const A Imax = ff_from_d(0.5 * dens_d * rmax_d * rmax_d);
    const A c0 = ff_from_d(0.25 * dens_d * rmax_d * rmax_d - 0.5 * dens_d * rmax_d * rmax_d * log(rmax_d));
    const R dxi = (R)W.dxi;
    const R inv_2pi_dxi = (R)(1.0 / (6.283185307179586476925286766559 * W.dxi));
    const A zeroA = {0.f, 0.f};

    R rh[K], ur[K];             // radius (rounded) and u_r of the thread's rings
    int idv[K];                 // their ring ids
    R ir[K], ipb[K];            // 1/rho, 1/psibar
    R pbv[K], dprv[K], bbv[K];  // psibar, d_rho psi, B^(b) at the rings
    R s0v[K], s1v[K], hav[K];   // B^(p) ring sources c_p and A_p / 2
    R tv[K];                    // t, then d_zeta psi
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
    for (; slice < s_end; ++slice) {
        // time budget (thread 0 decides, read after the order check's barrier)
        if (W.budget_ns > 0 && tid == 0) {
            const uint64_t now = global_ns();
            if (slice == slice0) t_start = now;
            s_stop = slice > slice0 && now - t_start >= (uint64_t)W.budget_ns;
        }
        // ---------------- a2: sort by radius if out of order
        {
            bool ok = true;
            R prev = -INFINITY;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < n) {
                    R v = sm.rh[SW::at(p)];
                    if (v < prev) ok = false;
                    prev = v;
                }
            }
            if (p0 + K < n && sm.rh[SW::at(p0 + K)] < prev) ok = false;
            const bool in_order = __syncthreads_and(ok);
            if (W.budget_ns > 0 && s_stop) break;
            // prefetch the next slice's beam while this one is solved (its
            // buffer was last read by slice - 1, before the barrier above)
            if (slice + 1 < s_end && stage_slice(stg, W, slice + 1, so.o1, so.o2 - so.o1, stall_armed)) {
                pending |= 1 << ((slice + 1) & 1);
                stall_armed = false;
            }
            if (!in_order) resort<K>(sm, n, W.n_pad, cap);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < n) {
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
        int b0 = 0, m = 0;
        R qtot = 0;
        if (W.nb > 0 && slice < n_steps) {
            b0 = so.o0;
            m = so.o1 - b0;
            qtot = W.bTot[slice];
        }
        SliceBeam sb = {W.br + b0, W.bQs + b0, W.bE + b0};
        if (pending & (1 << (slice & 1))) {  // staged: wait (bounded) for its copies
            const int bf = slice & 1;
            const bool got = mbar_wait_bounded(&s_bar[bf], (parity >> bf) & 1u);
            parity ^= 1u << bf;
            pending &= ~(1 << bf);
            if (__syncthreads_or(!got)) {
                status = WAKE_STATUS_TIMEOUT;
                fail = slice;
                break;
            }
            const int off = b0 & 3;
            sb = {stg.arr(bf, 0) + off, stg.arr(bf, 1) + off, stg.arr(bf, 2) + off};
        }
        if (m > 0) {
            for (int i = tid; i < cap; i += T) t_cnt[i] = 0;
            __syncthreads();
            // the first ring strictly above a particle counts it.  Each
            // thread takes a contiguous run of the slice's radius-sorted
            // particles (ranks along it only grow) and adds once per run of
            // particles at the same place.
            const int per = (m + T - 1) / T;
            const int q1 = min(m, (tid + 1) * per);
            int lo = 0, at_lo = -1, cnt = 0;
            for (int qb = tid * per; qb < q1 && lo < n; qb += kPartBatch) {
                float xb[kPartBatch];  // radii loaded together, then walked
#pragma unroll
                for (int j = 0; j < kPartBatch; ++j) xb[j] = qb + j < q1 ? sb.br[qb + j] : INFINITY;
#pragma unroll
                for (int j = 0; j < kPartBatch; ++j) {
                    lo = ring_rank_from<K>(sm.rh, n, lo, xb[j], false);
                    if (lo >= n) break;
                    if (lo != at_lo) {
                        if (cnt) atomicAdd(&t_cnt[SW::at(at_lo)], cnt);
                        at_lo = lo;
                        cnt = 0;
                    }
                    ++cnt;
                }
            }
            if (cnt) atomicAdd(&t_cnt[SW::at(at_lo)], cnt);
            __syncthreads();
        }

        // ---------------- a4: scan of (sum w, sum w ln rho, counts)
        A sw = zeroA, sl = zeroA;
        int64_t cl = 0;
        R lp[K];  // log1p(delta / rho0)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            lp[k] = 0.f;
            if (p < n) {
                const int a = SW::at(p);
                RingConst c = ring_const(ctab, idv[k]);
                const R dl = ff_to_f(ff_acc(ff{rh[k], sm.rl[a]}, ff_neg(c.r0)));  // rho - rho0
                lp[k] = log1pf(dl * c.ir0);
                sw = ff_acc(sw, c.w);
                sl = ff_acc(sl, ff_acc(c.wl0, ff_two_prod(c.w.hi, lp[k])));
                if (m > 0) cl += t_cnt[a];
            }
        }
        Trip<A> tot1;
        // (the four scans of a slice alternate the two halves of sscan: each
        // half is rewritten only after another scan's barrier)
        Trip<A> ex1 = block_excl_scan1<false>(Trip<A>{sw, sl, cl}, OpAddTrip(), Trip<A>{zeroA, zeroA, 0},
                                              reinterpret_cast<Trip<A>*>(sscan), tot1);
        const A Wtot = tot1.x, Ltot = tot1.y;

        // ---------------- a5: psi, d_rho psi, psibar, gamma, t; beam field
        A S = ex1.x, L = ex1.y;
        A tl = zeroA;
        int lb = (int)ex1.c;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < n) {
                const int a = SW::at(p);
                if (m > 0) lb += t_cnt[a];  // beam particles strictly below ring p
                RingConst c = ring_const(ctab, idv[k]);
                R r = rh[k], u = ur[k];
                A rf = {r, sm.rl[a]};  // rho in float-float
                A r2 = ff_mul(rf, rf);
                // the three large terms of psi cancel to O(1): float-float with
                // the accumulation add (error ~2^-46 of the terms, ~1e-11 here)
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
        A Ttot;
        A Tex = block_excl_scan1<false>(tl, OpAdd(), zeroA, reinterpret_cast<A*>(sscan + kScanBytes / 2), Ttot);

        // ---------------- a6 + a7: d_zeta psi, A, B, C, ring sources
        const Mat2<R> I2 = {1, 0, 0, 1};
        Mat2<R> Mf = I2, Mb = I2;
        {
            A Tacc = Tex;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < n) {
                    const int a = SW::at(p);
                    const float4 cw = __ldg(ctab + 3 * idv[k] + 1);  // w, what (hi parts)
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
                if (p0 + k < n) {
                    R r = rh[k], hA = hav[k];
                    Mat2<R> Mi = {1.f - hA * r, -hA * IR(k), hA * r * r * r, 1.f + hA * r};
                    Mb = OpMatLeft()(Mb, Mi);
                }
            }
        }

        // ---------------- a8: B_theta^(p) region coefficients
        Mat2<R> Yf, Yb;
        {
            Mat2<R> tf, tb;
            block_excl_scan_mat_fwd_rev1<false>(Mf, Mb, reinterpret_cast<Pair<Mat2<R>>*>(sscan), Yf, Yb, tf, tb);
        }
        R Rra[K], Rrb[K], Dda[K], Ddb[K];  // R_{p+1}, D_{p+1}
        {
            Mat2<R> Y = Yf;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (p0 + k < n) {
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
        R Dp0a, Dp0b;  // D at region p0 (after the backward walk)
        {
            Mat2<R> Y = Yb;
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                Dda[k] = Y.m01;
                Ddb[k] = Y.m11;
                gpv[k] = 0.f;
                dpv[k] = 0.f;
                if (p0 + k < n) {
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
        // G_k = sum_{p >= k} gamma_p must be a true suffix sum: a total minus a
        // prefix cancels where G_k is small and multiplies R_k ~ e^rho
        A g_tot, d_tot;
        Pair<A> gd = block_excl_scan_fwd_rev1(dl, gl, zeroA, reinterpret_cast<Pair<A>*>(sscan + kScanBytes / 2), d_tot,
                                              g_tot);
        {
            R Gk[K];
            A Gsuf = gd.y;  // sum over rings >= p0 + K
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                Gsuf = ff_add_f(Gsuf, gpv[k]);
                Gk[k] = ff_to_f(Gsuf);
            }
            // region p (below ring p): a_p = -G_p Ra_p + H_p Da_p, b_p likewise
            A Hex = gd.x;
            R Rpa = Yf.m00, Rpb = Yf.m10;  // R at region p0
            R Dpa = Dp0a, Dpb = Dp0b;      // D at region p0
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < n) {
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
            if (p0 < n && p0 + K >= n) {  // owner of the last ring writes region n
                const int a = n < TK ? SW::at(n) : TK;
                sm.a[a] = 0.f;             // a_n = 0 (D_n = (0, 1))
                sm.b[a] = ff_to_f(d_tot);  // b_n = H_n
                sm.T[a] = 0.f;
                sm.D[a] = ff_to_f(ff_sub(Wtot, Imax));
                sm.S[a] = ff_to_f(Wtot);
                sm.psi[a] = 0.f;
            }
        }
        __syncthreads();

        // ---------------- B^(p) at the rings and the guard
        bool bad = false;
        R bpv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            bpv[k] = 0.f;
            if (p < n) {
                const int a = SW::at(p);
                const int a1 = (p + 1 < TK) ? SW::at(p + 1) : TK;
                R r = rh[k];
                bpv[k] = 0.5f * ((sm.a[a] + sm.a[a1]) * r + (sm.b[a] + sm.b[a1]) * IR(k));
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
        if (mode == MODE_MARCH) {
            // contiguous runs of the radius-sorted particles, as in a3
            const int per = (m + T - 1) / T;
            const int q1 = min(m, (tid + 1) * per);
            int kr = 0;
            for (int qb = tid * per; qb < q1; qb += kPartBatch) {
              float xb[kPartBatch], qb_s[kPartBatch];  // loaded together, then evaluated
#pragma unroll
              for (int j = 0; j < kPartBatch; ++j) {
                  xb[j] = qb + j < q1 ? sb.br[qb + j] : 0.f;
                  qb_s[j] = qb + j < q1 ? sb.qs[qb + j] : 0.f;
              }
#pragma unroll
              for (int j = 0; j < kPartBatch; ++j) {
                const int q = qb + j;
                if (q >= q1) break;
                const R x = xb[j];
                R psi, dpr, dpz, bp, bb = 0.f;
                if (x > 0.f) {
                    kr = ring_rank_from<K>(sm.rh, n, kr, x, true);
                    fast_fields_region<K>(sm, n, TK, kr, x, rmax, half_n, quarter_n, Wtot, Imax, c0, &dpr, &dpz,
                                          &bp, &psi);
                    bb = qb_s[j] * inv_2pi_dxi / x;
                } else {
                    psi = ff_to_f(ff_add(Ltot, c0));
                    dpr = 0.f;
                    dpz = -ff_to_f(Ttot);
                    bp = 0.f;
                }
                const int64_t o = b0 + q;
                W.out_ez[o] = -dpz;
                W.out_wr[o] = -dpr;
                W.out_bt[o] = bp + bb;
                W.out_psi[o] = psi;
              }
            }
        } else {
            const int64_t nq = W.nq;
            for (int64_t q = tid; q < nq; q += T) {
                R x = (R)W.rq[q];
                R psi, dpr, dpz, bp, bb = 0.f;
                if (x > 0.f) {
                    fast_fields_at<K>(sm, n, TK, x, rmax, half_n, quarter_n, Wtot, Imax, c0, &dpr, &dpz, &bp, &psi);
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
        bad = __syncthreads_or(bad);
        if (mode != MODE_MARCH) break;
        if (bad) {
            status = 4;
            fail = slice;
            ++slice;
            break;
        }

        // ---------------- a10: AB2 push (rho in float-float)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < n) {
                const int a = SW::at(p);
                R u = ur[k], pb = pbv[k], ip = IPB(k);
                R g = 0.5f * (1.f + u * u + pb * pb) * ip;
                R fr = u * ip;
                R fu = g * dprv[k] * ip - (bpv[k] + bbv[k]);
                R dr, du;
                if (has_prev) {
                    dr = dxi * (1.5f * fr - 0.5f * sm.fr[a]);
                    du = dxi * (1.5f * fu - 0.5f * sm.fu[a]);
                } else {
                    dr = dxi * fr;
                    du = dxi * fu;
                }
                ff rr = ff_add_f(ff{rh[k], sm.rl[a]}, dr);
                R un = u + du;
                if (rr.hi < 0.f) {  // through the axis: the ring reappears at -rho
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
        if (W.nb > 0) so.advance(W, slice, n_steps);
        __syncthreads();
    }

    // ---- no bulk copy may still write this block's shared memory when it
    // exits: wait (bounded) for any staged slice that was not consumed
    for (int bf = 0; bf < 2; ++bf)
        if (pending & (1 << bf)) {
            if (!mbar_wait_bounded(&s_bar[bf], (parity >> bf) & 1u) && status == 0) {
                status = WAKE_STATUS_TIMEOUT;
                fail = slice;
            }
        }

    // ---- store the ring state back (sorted order, same buffer)
    __syncthreads();
    for (int p = tid; p < n; p += T) {
        int a = SW::at(p);
        W.rho[buf][p] = sm.rh[a];
        W.rho_lo[p] = sm.rl[a];
        W.ur[buf][p] = sm.u[a];
        W.frho[buf][p] = sm.fr[a];
        W.fur[buf][p] = sm.fu[a];
        W.rid[buf][p] = sm.id[a];
    }
    if (tid == 0) {
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
