// march_ions.cuh -- the per-slice march of a wake with mobile ions.
//
// Electrons (q = -1, m = 1) and ions (q = +Z, m = M) are both ring species
// on the same cells (Sec. II, multiple plasma species): ring ids 0..N-1 are
// electrons, N..2N-1 ions, and the sorted arrays hold the electrons at
// positions [0, N) and the ions at [N, 2N), each segment in radius order.
// Each ring carries its signed charge weight c = -q w (electrons +w, ions -w
// for neutrality), so that per species
//   psi = sum c ln max(rho, rho_j),  d_rho psi = (1/rho) sum_{rho_j<rho} c_j,
//   d_zeta psi = -sum_{rho_j>=rho} c_j u_j / (rho_j psibar_j),
// psibar = 1 - (q/m) psi.  One block owns one wake, or a thread-block
// cluster of up to 8 (for wide wakes): its blocks split each species'
// sorted positions in rank order, their scans fold over the cluster, and
// cluster barriers order the wake's global-memory arrays between them (the
// phases and their arithmetic are the same; only the fold order of the scans
// changes with the split).  Per slice:
//   a2 sort each segment (stable w.r.t. the previous order; in a cluster
//      block s sorts segment s)
//   a3 B^(b) at all rings
//   a4 per species: block scan of (c, c ln rho) -> its own psi, d_rho psi
//      at its rings (self weight in d_rho psi)
//   a5 totals at every ring: own + the other species' ring values linearly
//      interpolated at the ring's radius; psibar, gamma, t
//   a6 per species: block scan of t -> its own d_zeta psi; totals likewise
//   a7 A, B, C over the electron rings (B_theta^(p) from electrons only)
//   a8 B^(p) of the electrons (the two-sided solve of march.cuh); the ions
//      see it interpolated
//   a9 fields on beam particles (or query radii): exact sums of both species
//   a10 AB2 push of both species with their q/m, axis reflection
// Mixed precision keeps each ring radius as a float-float pair (rho, rho_lo)
// through the AB2 push and takes ln rho as ln rho0 + log1p((rho - rho0) /
// rho0) with ln rho0 float-float from the per-ring table: plain FP32 radii
// would accumulate the push's rounding over the window, which near the axis
// is a sizeable fraction of rho.
// Interpolation of a species' ring values F at radius x: between the last
// ring below x and the next; from the axis value below its first ring; to
// the exact outside value at the plasma's initial edge rho_max beyond its
// last ring; exact outside values beyond both.
#pragma once

#include "march.cuh"

namespace gbwake {

// Where radius X (hi part xh) falls among a species' n rings (hi radii rh,
// lo parts rl, increasing): case 0 between its rings k-1 and k (k = 0: the
// axis and ring 0), case 1 between its last ring and the plasma edge Xe,
// case 2 outside both (exact outside values); wgt the linear weight of the
// upper node, from radius differences taken in the accumulator type.
template <class A, class R>
struct Locate {
    int where, k;
    R wgt;   // the weight rounded to R
    A wgtA;  // the weight in the accumulator type
};
template <class A, class R>
__device__ __forceinline__ Locate<A, R> locate(const R* rh, const R* rl, int n, R edge, A Xe, A X, R xh) {
    Locate<A, R> L;
    L.k = lower_bound_dev(rh, n, xh);  // rings strictly below X
    A Xl, Xu;
    if (L.k >= n) {
        if (!(xh < edge) || !(edge > rh[n - 1])) {
            L.where = 2;
            L.wgt = 0;
            L.wgtA = acc_zero(A());
            return L;
        }
        L.where = 1;
        Xl = ring_radius(rh, rl, n - 1);
        Xu = Xe;
    } else {
        L.where = 0;
        Xl = L.k > 0 ? ring_radius(rh, rl, L.k - 1) : acc_zero(A());
        Xu = ring_radius(rh, rl, L.k);
    }
    const A den = acc_sub(Xu, Xl);
    L.wgtA = acc_to_r(den) > (R)0 ? acc_div(acc_sub(X, Xl), den) : acc_from_d(1.0, A());
    L.wgt = acc_to_r(L.wgtA);
    return L;
}
// F at the located radius from the species' ring values F (lower node F0 on
// the axis, upper node Fe at the edge), in the accumulator type
template <class A, class R>
__device__ __forceinline__ A gather_acc(const Locate<A, R>& L, const A* F, int n, A F0, A Fe) {
    A lo, up;
    if (L.where == 1) {
        lo = F[n - 1];
        up = Fe;
    } else {
        lo = L.k > 0 ? F[L.k - 1] : F0;
        up = F[L.k];
    }
    return acc_add(lo, acc_mul_a(acc_sub(up, lo), L.wgtA));
}
template <class A, class R>
__device__ __forceinline__ R gather_r(const Locate<A, R>& L, const R* F, int n, R F0, R Fe) {
    R lo, up;
    if (L.where == 1) {
        lo = F[n - 1];
        up = Fe;
    } else {
        lo = L.k > 0 ? F[L.k - 1] : F0;
        up = F[L.k];
    }
    return lo + (up - lo) * L.wgt;
}

// the per-ring values only their own thread reads (kept in shared memory
// when the launch has room): B^(b), psibar, gamma, d_rho psi, t / d_zeta psi
// and the ring's weights c, c-hat (real type), then ln rho (accumulator type)
enum { kOwnBb = 0, kOwnPsib, kOwnGam, kOwnDpr, kOwnT, kOwnW, kOwnWh, kOwnArrays };

template <class P>
__global__ void __launch_bounds__(512)
march_ions_kernel(const WakeDev<P>* __restrict__ wakes, const int32_t* __restrict__ order, int32_t max_slices,
                  int32_t mode, int32_t mb_cap) {
    using R = typename P::R;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ctl[CTL_N];
    __shared__ int s_stop;
    __shared__ __align__(16) unsigned char s_part[2 * kPartBuf];

    const uint64_t t_launch = global_ns();
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
    const int n = W.n;           // all rings
    const int N = W.n_ion;       // rings per species
    const int K = (N + GT - 1) / GT;
    const int q0 = min(N, gt * K);
    const int q1 = min(N, q0 + K);
    const bool lead = C.rank == 0 && tid == 0;  // writes the wake's single values
    const R qm[2] = {(R)-1, (R)W.ion_qm};

    unsigned char* sscan = smem;
    R* keys = reinterpret_cast<R*>(smem + kScanBytes);
    int32_t* vals = reinterpret_cast<int32_t*>(keys + W.n_pad);
    R* sR = keys;      // sorted ring radii, both segments (after the sort)
    R* sB = keys + n;  // staged beam radii of the slice
    // Per-ring values only their own thread reads (B^(b), psibar, gamma,
    // d_rho psi, t and then d_zeta psi): in shared memory after the sort and
    // staging region when the launch left room for them (the host adds it
    // when it fits), else in the wake's global arrays.
    const int TK = T * K;             // a block's positions of each species
    const int qb = min(N, C.rank * TK);
    R* own = nullptr;
    {
        unsigned dyn;
        asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
        size_t used = (size_t)(n + mb_cap) * sizeof(R);
        const size_t sort_used = (size_t)W.n_pad * (sizeof(R) + 4);
        used = kScanBytes + (used > sort_used ? used : sort_used);
        used = (used + 15) & ~(size_t)15;
        if (used + (size_t)kOwnArrays * 2 * TK * sizeof(R) + 2 * (size_t)TK * sizeof(A) <= dyn)
            own = reinterpret_cast<R*>(smem + used);
    }
    A* own_ln = own ? reinterpret_cast<A*>(own + kOwnArrays * 2 * TK) : nullptr;
    // the value `a` (kOwn*) of species s, sorted position q (this thread's)
    auto scr = [&](int a, int s, int q) -> R& {
        if (own) return own[(a * 2 + s) * TK + (q - qb)];
        R* g = a == kOwnBb ? W.bb : a == kOwnPsib ? W.psib : a == kOwnGam ? W.gam : a == kOwnDpr ? W.dpr : W.tt;
        return g[s * N + q];
    };

    if (tid < CTL_N) s_ctl[tid] = W.ctl[tid];
    __syncthreads();
    if (s_ctl[CTL_STATUS] != 0) return;
    int slice = s_ctl[CTL_NEXT];
    int buf = s_ctl[CTL_BUF];
    int has_prev = s_ctl[CTL_PREV];
    int status = 0, fail = -1;
    const int s_end = mode == MODE_MARCH ? min(W.n_steps, slice + max_slices) : slice + 1;

    const R edge = (R)W.rho_max;
    const A Xe = acc_from_d(W.rho_max, A());          // the plasma edge, accumulator precision
    const A ln_e = acc_from_d(log(W.rho_max), A());
    const A inv_e = acc_from_d(1.0 / W.rho_max, A());
    const R dxi = (R)W.dxi;
    const R inv_2pi_dxi = (R)(1.0 / (6.283185307179586476925286766559 * W.dxi));
    const A zeroA = acc_zero(A());

    const int slice0 = slice;
    uint64_t t_start = 0;
    for (; slice < s_end; ++slice) {
        // time budget (thread 0 decides, read after the order check's barrier)
        if (W.budget_ns > 0 && tid == 0) {
            const uint64_t now = global_ns();
            if (slice == slice0) t_start = now;
            s_stop = slice > slice0 && now - t_start >= (uint64_t)W.budget_ns;
        }
        // ---------------- a2: sort each segment by radius (stable)
        {
            R* rho = W.rho[buf];
            bool ok = true;
            for (int s = 0; s < 2; ++s)
                for (int q = q0; q < q1; ++q)
                    if (q + 1 < N && rho[s * N + q + 1] < rho[s * N + q]) ok = false;
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
                for (int s = 0; s < 2; ++s) {
                    if (C.size > 1 && C.rank != s) continue;
                    const int base = s * N;
                    for (int i = tid; i < W.n_pad; i += T) {
                        keys[i] = i < N ? rho[base + i] : (R)INFINITY;
                        vals[i] = i;
                    }
                    __syncthreads();
                    block_bitonic_sort(keys, vals, W.n_pad);
                    for (int i = tid; i < N; i += T) {
                        const int src = base + vals[i], dst = base + i;
                        W.rho[nb][dst] = W.rho[buf][src];
                        W.ur[nb][dst] = W.ur[buf][src];
                        W.frho[nb][dst] = W.frho[buf][src];
                        W.fur[nb][dst] = W.fur[buf][src];
                        W.rid[nb][dst] = W.rid[buf][src];
                        keys[i] = W.rho_lo[src];  // the sort keys are no longer needed
                    }
                    __syncthreads();
                    for (int i = tid; i < N; i += T) W.rho_lo[base + i] = keys[i];
                    __syncthreads();
                }
                if (C.size > 1) C.sync();
                buf = nb;
            }
        }
        R* rho = W.rho[buf];
        R* ur = W.ur[buf];
        R* frho = W.frho[buf];
        R* fur = W.fur[buf];
        const int32_t* rid = W.rid[buf];
        // the weights c, c-hat of this thread's ring (s, q)
        auto wgt = [&](int a, int s, int q) -> R {
            if (own) return own[(a * 2 + s) * TK + (q - qb)];
            return (a == kOwnW ? W.w : W.wh)[rid[s * N + q]];
        };

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

        // ---------------- a3 + a4: beam field at rings; per species own psi, d_rho psi
        A Stot[2], Ltot[2];
        Pair<A> loc[2], exs[2], tots[2];
        for (int s = 0; s < 2; ++s) {
            const int base = s * N;
            loc[s] = {zeroA, zeroA};
            for (int q = q0; q < q1; ++q) {
                const int p = base + q;
                R r = sR[p];
                const int id = rid[p];
                R c = W.w[id];
                R bbv = 0;
                if (m > 0 && r > (R)0) {
                    int lb = lower_bound_dev(beamR, m, r);
                    R Q = lb < m ? W.bE[b0 + lb] : qtot;
                    bbv = Q * inv_2pi_dxi / r;
                }
                scr(kOwnBb, s, q) = bbv;
                const A lnr = ring_log(W.ctab, id, r, W.rho_lo[p]);
                if (own) {
                    own[(kOwnW * 2 + s) * TK + (q - qb)] = c;
                    own[(kOwnWh * 2 + s) * TK + (q - qb)] = W.wh[id];
                    own_ln[s * TK + (q - qb)] = lnr;
                }
                loc[s].x = acc_add_r(loc[s].x, c);
                loc[s].y = acc_add(loc[s].y, acc_mul_r(lnr, c));
            }
        }
        // both species' scans, their block totals in one exchange
        wake_excl_scan2<false, false>(C, loc[0], OpAddPair(), Pair<A>{zeroA, zeroA},
                                      reinterpret_cast<Pair<A>*>(sscan), exs[0], tots[0], loc[1], OpAddPair(),
                                      Pair<A>{zeroA, zeroA}, reinterpret_cast<Pair<A>*>(sscan), exs[1], tots[1]);
        for (int s = 0; s < 2; ++s) {
            const int base = s * N, rb = s * (N + 1);
            const Pair<A> tot = tots[s], ex = exs[s];
            Stot[s] = tot.x;
            Ltot[s] = tot.y;
            A S = ex.x, L = ex.y;
            for (int q = q0; q < q1; ++q) {
                const int p = base + q;
                R r = sR[p];
                const R c = wgt(kOwnW, s, q), ch = wgt(kOwnWh, s, q);
                const A lnr = own ? own_ln[s * TK + (q - qb)] : ring_log(W.ctab, rid[p], r, W.rho_lo[p]);
                A Lsuf = acc_sub(tot.y, L);
                W.regS[rb + q] = S;
                W.regL[rb + q] = Lsuf;
                // own fields kept in the accumulator type: the two species'
                // values are large and cancel to the small total
                W.psio[p] = acc_add(Lsuf, acc_mul_a(S, lnr));
                W.dpro[p] = acc_div(acc_add_r(S, ch), ring_radius(sR, W.rho_lo, p));
                S = acc_add_r(S, c);
                L = acc_add(L, acc_mul_r(lnr, c));
            }
            if (lead) {
                W.regS[rb + N] = tot.x;
                W.regL[rb + N] = zeroA;
                W.regT[rb + N] = (R)0;
            }
        }
        C.sync();  // own-species fields, before the other species gathers them

        // ---------------- a5: totals of psi, d_rho psi; psibar, gamma, t
        for (int s = 0; s < 2; ++s) {
            const int base = s * N, ob = (1 - s) * N;
            const A oS = Stot[1 - s];
            const A psi_e = acc_mul_a(oS, ln_e), dpr_e = acc_mul_a(oS, inv_e);  // the other species at the edge
            for (int q = q0; q < q1; ++q) {
                const int p = base + q;
                R r = sR[p], u = ur[p];
                R c = wgt(kOwnW, s, q);
                const A X = ring_radius(sR, W.rho_lo, p);
                const auto Lc = locate(sR + ob, W.rho_lo + ob, N, edge, Xe, X, r);
                A psiA, dprA;
                if (Lc.where == 2) {
                    psiA = acc_mul_a(oS, acc_log(X, Xe, ln_e, edge));
                    dprA = acc_div(oS, X);
                } else {
                    psiA = gather_acc(Lc, W.psio + ob, N, Ltot[1 - s], psi_e);
                    dprA = gather_acc(Lc, W.dpro + ob, N, zeroA, dpr_e);
                }
                R psi = acc_to_r(acc_add(W.psio[p], psiA));
                R dprv = acc_to_r(acc_add(W.dpro[p], dprA));
                R pb = (R)1 - qm[s] * psi;
                scr(kOwnPsib, s, q) = pb;
                scr(kOwnGam, s, q) = ((R)1 + u * u + pb * pb) / ((R)2 * pb);
                scr(kOwnDpr, s, q) = dprv;
                scr(kOwnT, s, q) = c * u / (r * pb);
                if (mode == MODE_MARCH && W.dump_psi) {
                    size_t row = (size_t)slice * n + rid[p];
                    W.dump_psi[row] = psi;
                    W.dump_dpr[row] = dprv;
                }
            }
        }

        // ---------------- a6: per species own d_zeta psi, then the totals
        A Ttot[2], tl[2], Tex[2];
        for (int s = 0; s < 2; ++s) {
            tl[s] = zeroA;
            for (int q = q0; q < q1; ++q) tl[s] = acc_add_r(tl[s], scr(kOwnT, s, q));
        }
        wake_excl_scan2<false, false>(C, tl[0], OpAdd(), zeroA, reinterpret_cast<A*>(sscan), Tex[0], Ttot[0], tl[1],
                                      OpAdd(), zeroA, reinterpret_cast<A*>(sscan), Tex[1], Ttot[1]);
        for (int s = 0; s < 2; ++s) {
            const int base = s * N, rb = s * (N + 1);
            A Tacc = Tex[s];
            for (int q = q0; q < q1; ++q) {
                const int p = base + q;
                R c = wgt(kOwnW, s, q), ch = wgt(kOwnWh, s, q);
                R t = scr(kOwnT, s, q);
                W.regT[rb + q] = acc_to_r(acc_sub(Ttot[s], Tacc));
                Tacc = acc_add_r(Tacc, t);
                R above = acc_to_r(acc_sub(Ttot[s], Tacc));
                W.dpzo[p] = -(above + ((R)1 - ch / c) * t);
            }
        }
        C.sync();
        for (int s = 0; s < 2; ++s) {
            const int base = s * N, ob = (1 - s) * N;
            const R oT = acc_to_r(Ttot[1 - s]);
            for (int q = q0; q < q1; ++q) {
                const int p = base + q;
                const auto Lc = locate(sR + ob, W.rho_lo + ob, N, edge, Xe, ring_radius(sR, W.rho_lo, p), sR[p]);
                // no ring of the other species above: no d_zeta psi from it
                R dpz = W.dpzo[p] + (Lc.where == 2 ? (R)0 : gather_r(Lc, W.dpzo + ob, N, -oT, (R)0));
                scr(kOwnT, s, q) = dpz;  // t no longer needed: keep d_zeta psi
                if (mode == MODE_MARCH && W.dump_dpz) W.dump_dpz[(size_t)slice * n + rid[p]] = dpz;
            }
        }

        // ---------------- a7: A, B, C over the electron rings
        for (int q = q0; q < q1; ++q) {
            const int p = q;
            R r = sR[p], u = ur[p];
            R w = wgt(kOwnW, 0, q);
            R pb = scr(kOwnPsib, 0, q), g = scr(kOwnGam, 0, q), dprv = scr(kOwnDpr, 0, q), dpz = scr(kOwnT, 0, q),
              bbv = scr(kOwnBb, 0, q);
            R wr = w / r, pb2 = pb * pb;
            W.cA[p] = wr / pb;
            W.cB[p] = -wr * g * dprv / pb2 + wr * bbv / pb + (w / (r * r)) * u * u / pb2 +
                      wr * u * u * dprv / (pb2 * pb) - wr * u * dpz / pb2;
            W.cC[p] = -wr * (g / pb - (R)1 - u * u / pb2);
        }

        // ---------------- a8: B_theta^(p) of the electrons (regions 0..N)
        bp_region_solve(W, sR, N, q0, q1, sscan, C);
        C.sync();
        // B^(p) at the electron rings, then interpolated at the ion rings
        for (int p = q0; p < q1; ++p) {
            R r = sR[p];
            W.cA[p] = (R)0.5 * ((W.ak[p] + W.ak[p + 1]) * r + (W.bk[p] + W.bk[p + 1]) / r);
        }
        C.sync();
        {
            const R bN = W.bk[N];
            for (int q = q0; q < q1; ++q) {
                const int p = N + q;
                const R x = sR[p];
                const auto Lc = locate(sR, W.rho_lo, N, edge, Xe, ring_radius(sR, W.rho_lo, p), x);
                W.cA[p] = Lc.where == 2 ? bN / x : gather_r(Lc, W.cA, N, (R)0, bN / edge);
            }
        }

        // ---------------- guard, dumps
        bool bad = false;
        for (int s = 0; s < 2; ++s)
            for (int q = q0; q < q1; ++q) {
                const int p = s * N + q;
                R r = sR[p];
                R bpv = W.cA[p];
                R pb = scr(kOwnPsib, s, q);
                if (!(pb > (R)0) || !real_finite(pb) || !real_finite(scr(kOwnDpr, s, q)) ||
                    !real_finite(scr(kOwnT, s, q)) || !real_finite(bpv) || !real_finite(scr(kOwnBb, s, q)) ||
                    !real_finite(scr(kOwnGam, s, q)))
                    bad = true;
                if (mode == MODE_MARCH) {
                    size_t row = (size_t)slice * n + rid[p];
                    if (W.dump_r) W.dump_r[row] = r;
                    if (W.dump_ur) {
                        W.dump_ur[row] = ur[p];
                        W.dump_bp[row] = bpv;
                        W.dump_bb[row] = scr(kOwnBb, s, q);
                    }
                }
            }
        bad = wake_vote(C, bad, false);

        // ---------------- a9: fields on beam particles (or query radii)
        {
            const int64_t nq = mode == MODE_MARCH ? (int64_t)m : W.nq;
            for (int64_t q = gt; q < nq; q += GT) {
                R x;
                if (mode == MODE_MARCH) x = staged ? beamR[q] : W.br[b0 + q];
                else x = (R)W.rq[q];
                R psi = 0, dprv = 0, dpz = 0, bpv = 0, bbv = 0;
                if (x > (R)0) {
                    // the species' enclosed charges and log sums cancel: add
                    // them in the accumulator type before rounding
                    A Ssum = zeroA, Lsum = zeroA;
                    for (int s = 0; s < 2; ++s) {
                        const int rb = s * (N + 1);
                        int k = lower_bound_dev(sR + s * N, N, x);
                        Ssum = acc_add(Ssum, W.regS[rb + k]);
                        Lsum = acc_add(Lsum, W.regL[rb + k]);
                        dpz -= W.regT[rb + k];
                        if (s == 0) bpv = W.ak[k] * x + W.bk[k] / x;
                    }
                    psi = acc_to_r(acc_add(Lsum, acc_mul_r(Ssum, real_log(x))));
                    dprv = acc_to_r(Ssum) / x;
                    if (mode == MODE_MARCH) {
                        bbv = W.bQs[b0 + q] * inv_2pi_dxi / x;
                    } else if (m > 0) {
                        int lb = lower_bound_dev(beamR, m, x);
                        R Q = lb < m ? W.bE[b0 + lb] : qtot;
                        bbv = Q * inv_2pi_dxi / x;
                    }
                } else {
                    psi = acc_to_r(acc_add(W.regL[0], W.regL[N + 1]));
                    dpz = -(W.regT[0] + W.regT[N + 1]);
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

        // ---------------- a10: AB2 push of both species
        for (int s = 0; s < 2; ++s)
            for (int q = q0; q < q1; ++q) {
                const int p = s * N + q;
                R r = sR[p], u = ur[p];
                R pb = scr(kOwnPsib, s, q);
                R fr = u / pb;
                R fu = -qm[s] * (scr(kOwnGam, s, q) * scr(kOwnDpr, s, q) / pb - (W.cA[p] + scr(kOwnBb, s, q)));
                R rn = r, rlo = W.rho_lo[p], un;
                if (has_prev) {
                    radius_add(rn, rlo, dxi * ((R)1.5 * fr - (R)0.5 * frho[p]));
                    un = u + dxi * ((R)1.5 * fu - (R)0.5 * fur[p]);
                } else {
                    radius_add(rn, rlo, dxi * fr);
                    un = u + dxi * fu;
                }
                if (rn < (R)0) {  // through the axis: the ring reappears at -rho
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
    if (lead) {
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
