// march_rk4.cuh -- the per-slice march with the classical RK4 ring integrator.
//
// The ring equations (Eqs. plasma_particle_motion_1,2; xi = -zeta)
//   d rho / d xi = u / psibar,   d u / d xi = gamma d_rho psi / psibar - B_theta
// are advanced over each slice by classical fourth-order Runge-Kutta, the
// alternative to Adams-Bashforth that Sec. II names:
//   k1 = F(xi_n, y_n)                 (the slice's own fields: dumps, beam
//                                      fields, guard)
//   k2 = F(xi_n + h/2, y_n + h/2 k1)  beam source: mean of slices n, n+1
//   k3 = F(xi_n + h/2, y_n + h/2 k2)  likewise
//   k4 = F(xi_n + h, y_n + h k3)      slice n+1's source (none past the window)
//   y_{n+1} = y_n + h/6 (k1 + 2 k2 + 2 k3 + k4)
// A stage state below the axis is evaluated mirrored (rho, u -> -rho, -u) and
// its derivative mirrored back (the equations are odd in (rho, u)); each
// stage's fields are a whole slice evaluation (sort, scans, B^(p) solve) at
// the stage state.  Electrons over the immobile uniform ion column (as
// march.cuh); one block per wake, state in global memory in radius order.
// Mixed precision keeps the ring radius float-float (rho, rho_lo) for the
// state and the stage states, with ln rho from the per-ring ln rho0 table
// and the ion column's terms from the float-float radius: psi and d_rho psi
// are differences of terms ~n rho_max^2 that cancel to O(1).
#pragma once

#include "march_ions.cuh"

namespace gbwake {

// the beam source of a stage: w1 x (slice a) + w2 x (slice b, if m2 > 0)
template <class R>
struct RkSource {
    int b1, m1, b2, m2;
    R w1, w2, q1, q2;
    const R* r1;  // slice a's sorted radii (staged in shared memory, or global)
};

template <class P>
__device__ __forceinline__ typename P::R rk_beam_field(const WakeDev<P>& W, const RkSource<typename P::R>& S,
                                                       typename P::R r, typename P::R inv_2pi_dxi) {
    using R = typename P::R;
    if (!(r > (R)0)) return (R)0;
    R bb = 0;
    if (S.m1 > 0) {
        int lb = lower_bound_dev(S.r1, S.m1, r);
        bb += S.w1 * (lb < S.m1 ? W.bE[S.b1 + lb] : S.q1);
    }
    if (S.m2 > 0) {
        int lb = lower_bound_dev(W.br + S.b2, S.m2, r);
        bb += S.w2 * (lb < S.m2 ? W.bE[S.b2 + lb] : S.q2);
    }
    return bb * inv_2pi_dxi / r;
}

// Fields of one stage at a state in radius order: sorted radius i is sR[i]
// (hi; lo part rlo[perm[i]]), its u is us[perm[i]] and its ring id
// rid[perm[i]] (perm = NULL: the identity).  Writes the derivatives
// F = (d rho, d u)/d xi of sorted position i to kr[perm[i]], ku[perm[i]]
// times sg[perm[i]] (the mirror sign; sg = NULL: +1), adds them with weight
// wsum into sum_r, sum_u (wsum = 0: sets them), and with `first` the dumps.
// Returns the guard (true: a non-finite field or psibar <= 0).
template <class P>
__device__ bool rk_stage(const WakeDev<P>& W, unsigned char* sscan, const typename P::R* sR,
                         const typename P::R* rlo, const typename P::R* us, const int32_t* rid, const int32_t* perm,
                         const typename P::R* sg, const RkSource<typename P::R>& src, typename P::R* kr,
                         typename P::R* ku, typename P::R* sum_r, typename P::R* sum_u, typename P::R wsum,
                         bool first, int slice, int mode, int p0, int p1, WakeCtas& C) {
    using R = typename P::R;
    using A = typename P::A;
    const int n = W.n;
    const A zeroA = acc_zero(A());
    const double dens_d = W.density, rmax_d = W.rho_max;
    const R rmax = (R)rmax_d;
    const R half_n = (R)(0.5 * dens_d), quarter_n = (R)(0.25 * dens_d);
    const A Imax = acc_from_d(0.5 * dens_d * rmax_d * rmax_d, A());
    const A c0 = acc_from_d(0.25 * dens_d * rmax_d * rmax_d - 0.5 * dens_d * rmax_d * rmax_d * log(rmax_d), A());
    const R inv_2pi_dxi = (R)(1.0 / (6.283185307179586476925286766559 * W.dxi));
    const int tid = threadIdx.x;
    auto at = [&](int i) { return perm ? perm[i] : i; };

    // a3 + a4: beam field at the rings, prefix sums of (w, w ln rho)
    Pair<A> loc = {zeroA, zeroA};
    for (int i = p0; i < p1; ++i) {
        const int q = at(i);
        const int id = rid[q];
        A wa, wha;
        ring_weights(W.ctab, W.w, W.wh, id, wa, wha);
        W.bb[i] = rk_beam_field(W, src, sR[i], inv_2pi_dxi);
        loc.x = acc_add(loc.x, wa);
        loc.y = acc_add(loc.y, acc_mul_a(ring_log(W.ctab, id, sR[i], rlo[q]), wa));
    }
    Pair<A> tot;
    Pair<A> ex = wake_excl_scan<false>(C, loc, OpAddPair(), Pair<A>{zeroA, zeroA},
                                       reinterpret_cast<Pair<A>*>(sscan), tot);
    const A Ltot = tot.y;

    // a5: psi, d_rho psi (self weight), psibar, gamma, t
    A S = ex.x, L = ex.y;
    A tl = zeroA;
    for (int i = p0; i < p1; ++i) {
        const int q = at(i);
        const int id = rid[q];
        R r = sR[i], u = us[q];
        R w = W.w[id];
        A wa, wha;
        ring_weights(W.ctab, W.w, W.wh, id, wa, wha);
        const A Xr = make_radius(r, rlo[q]);
        const A lnr = ring_log(W.ctab, id, r, rlo[q]);
        A Lsuf = acc_sub(Ltot, L);
        W.regS[i] = S;
        W.regL[i] = Lsuf;
        const A r2 = acc_mul_a(Xr, Xr);
        const A Ir = r < rmax ? acc_mul_r(r2, half_n) : Imax;
        const A psion = r <= rmax ? acc_sub(c0, acc_mul_r(r2, quarter_n)) : acc_sub(zeroA, acc_mul_a(Imax, lnr));
        R psi = acc_to_r(acc_add(acc_add(Lsuf, acc_mul_a(S, lnr)), psion));
        R dprv = acc_to_r(acc_div(acc_sub(acc_add(S, wha), Ir), Xr));
        R pb = (R)1 + psi;
        R g = ((R)1 + u * u + pb * pb) / ((R)2 * pb);
        R t = w * u / (r * pb);
        W.psib[i] = pb;
        W.gam[i] = g;
        W.dpr[i] = dprv;
        W.tt[i] = t;
        if (first && mode == MODE_MARCH && W.dump_psi) {
            size_t row = (size_t)slice * n + id;
            W.dump_psi[row] = psi;
            W.dump_dpr[row] = dprv;
        }
        S = acc_add(S, wa);
        L = acc_add(L, acc_mul_a(lnr, wa));
        tl = acc_add_r(tl, t);
    }
    if (C.rank == 0 && tid == 0) {
        W.regS[n] = tot.x;
        W.regL[n] = zeroA;
        W.regT[n] = (R)0;
    }
    A Ttot;
    A Tex = wake_excl_scan<false>(C, tl, OpAdd(), zeroA, reinterpret_cast<A*>(sscan), Ttot);

    // a6 + a7: d_zeta psi, A, B, C
    {
        A Tacc = Tex;
        for (int i = p0; i < p1; ++i) {
            const int q = at(i);
            const int id = rid[q];
            R r = sR[i], u = us[q];
            R w = W.w[id], wh = W.wh[id];
            R t = W.tt[i];
            W.regT[i] = acc_to_r(acc_sub(Ttot, Tacc));
            Tacc = acc_add_r(Tacc, t);
            R above = acc_to_r(acc_sub(Ttot, Tacc));
            R dpz = -(above + ((R)1 - wh / w) * t);
            R pb = W.psib[i], g = W.gam[i], dprv = W.dpr[i], bbv = W.bb[i];
            R wr = w / r, pb2 = pb * pb;
            W.cA[i] = wr / pb;
            W.cB[i] = -wr * g * dprv / pb2 + wr * bbv / pb + (w / (r * r)) * u * u / pb2 +
                      wr * u * u * dprv / (pb2 * pb) - wr * u * dpz / pb2;
            W.cC[i] = -wr * (g / pb - (R)1 - u * u / pb2);
            W.tt[i] = dpz;
            if (first && mode == MODE_MARCH && W.dump_dpz) W.dump_dpz[(size_t)slice * n + id] = dpz;
        }
    }

    // a8: B_theta^(p) (the two-sided solve of march.cuh)
    bp_region_solve(W, sR, n, p0, p1, sscan, C);
    C.sync();

    // B^(p) at the rings, guard, dumps, derivatives
    bool bad = false;
    for (int i = p0; i < p1; ++i) {
        const int q = at(i);
        const int id = rid[q];
        R r = sR[i], u = us[q];
        R bpv = (R)0.5 * ((W.ak[i] + W.ak[i + 1]) * r + (W.bk[i] + W.bk[i + 1]) / r);
        R pb = W.psib[i];
        if (!(pb > (R)0) || !real_finite(pb) || !real_finite(W.dpr[i]) || !real_finite(W.tt[i]) ||
            !real_finite(bpv) || !real_finite(W.bb[i]) || !real_finite(W.gam[i]))
            bad = true;
        if (first && mode == MODE_MARCH) {
            size_t row = (size_t)slice * n + id;
            if (W.dump_r) W.dump_r[row] = r;
            if (W.dump_ur) {
                W.dump_ur[row] = u;
                W.dump_bp[row] = bpv;
                W.dump_bb[row] = W.bb[i];
            }
        }
        const R s = sg ? sg[q] : (R)1;
        const R fr = s * (u / pb);
        const R fu = s * (W.gam[i] * W.dpr[i] / pb - (bpv + W.bb[i]));
        kr[q] = fr;
        ku[q] = fu;
        if (wsum == (R)0) {
            sum_r[q] = fr;
            sum_u[q] = fu;
        } else {
            sum_r[q] += wsum * fr;
            sum_u[q] += wsum * fu;
        }
    }
    return wake_vote(C, bad, false);
}

template <class P>
__global__ void __launch_bounds__(512)
march_rk4_kernel(const WakeDev<P>* __restrict__ wakes, const int32_t* __restrict__ order, int32_t max_slices,
                 int32_t mode, int32_t mb_cap) {
    using R = typename P::R;
    using A = typename P::A;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ctl[CTL_N];
    __shared__ int s_stop;
    __shared__ __align__(16) unsigned char s_part[2 * kPartBuf];

    const uint64_t t_launch = global_ns();
    WakeCtas C;  // one block per wake, or a cluster (block 0 sorts)
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
    R* sR = keys;      // the sorted radii of the current stage
    R* sB = keys + n;  // staged beam radii of slice n

    if (tid < CTL_N) s_ctl[tid] = W.ctl[tid];
    __syncthreads();
    if (s_ctl[CTL_STATUS] != 0) return;
    int slice = s_ctl[CTL_NEXT];
    int buf = s_ctl[CTL_BUF];
    int status = 0, fail = -1;
    const int s_end = mode == MODE_MARCH ? min(W.n_steps, slice + max_slices) : slice + 1;
    const R dxi = (R)W.dxi;
    const R inv_2pi_dxi = (R)(1.0 / (6.283185307179586476925286766559 * W.dxi));

    const int slice0 = slice;
    uint64_t t_start = 0;
    for (; slice < s_end; ++slice) {
        // time budget (thread 0 decides, read after the order check's barrier)
        if (W.budget_ns > 0 && tid == 0) {
            const uint64_t now = global_ns();
            if (slice == slice0) t_start = now;
            s_stop = slice > slice0 && now - t_start >= (uint64_t)W.budget_ns;
        }
        // ---------------- a2: sort the state by radius (stable)
        {
            R* rho = W.rho[buf];
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
                        W.rid[nb][p] = W.rid[buf][src];
                        keys[p] = W.rho_lo[src];
                    }
                    __syncthreads();
                    for (int p = tid; p < n; p += T) W.rho_lo[p] = keys[p];
                }
                buf = nb;
                C.sync();
            }
        }
        R* rho = W.rho[buf];
        R* ur = W.ur[buf];
        const int32_t* rid = W.rid[buf];

        // ---------------- the slice's beam and the next slice's
        const bool have_beam = W.nb > 0 && slice < W.n_steps;
        int b0 = 0, m = 0, b1 = 0, m1 = 0;
        R qtot = 0, qtot1 = 0;
        if (have_beam) {
            b0 = W.boff[slice];
            m = W.boff[slice + 1] - b0;
            qtot = W.bTot[slice];
            if (slice + 1 < W.n_steps) {
                b1 = W.boff[slice + 1];
                m1 = W.boff[slice + 2] - b1;
                qtot1 = W.bTot[slice + 1];
            }
        }
        const bool staged = m <= mb_cap;
        for (int p = tid; p < n; p += T) sR[p] = rho[p];
        if (staged)
            for (int q = tid; q < m; q += T) sB[q] = W.br[b0 + q];
        __syncthreads();
        const R* beamR = staged ? sB : (W.br + b0);

        // ---------------- stage 1 at (xi_n, y_n): the slice's fields
        RkSource<R> s1 = {b0, m, 0, 0, (R)1, (R)0, qtot, (R)0, beamR};
        bool bad = rk_stage(W, sscan, sR, W.rho_lo, ur, rid, nullptr, nullptr, s1, W.rk_kr, W.rk_ku, W.frho[0],
                            W.fur[0], (R)0, true, slice, mode, p0, p1, C);

        // ---------------- a9: fields on beam particles (or query radii)
        {
            const double dens_d = W.density, rmax_d = W.rho_max;
            const R rmax = (R)rmax_d, half_n = (R)(0.5 * dens_d), quarter_n = (R)(0.25 * dens_d);
            const A Imax = acc_from_d(0.5 * dens_d * rmax_d * rmax_d, A());
            const A c0 = acc_from_d(0.25 * dens_d * rmax_d * rmax_d - 0.5 * dens_d * rmax_d * rmax_d * log(rmax_d), A());
            const int64_t nq = mode == MODE_MARCH ? (int64_t)m : W.nq;
            for (int64_t q = gt; q < nq; q += GT) {
                R x;
                if (mode == MODE_MARCH) x = staged ? beamR[q] : W.br[b0 + q];
                else x = (R)W.rq[q];
                R psi, dprv, dpz, bpv, bbv;
                if (x > (R)0) {
                    int k = lower_bound_dev(sR, n, x);
                    A Sk = W.regS[k];
                    const R lnx = real_log(x);
                    const A x2 = acc_sq(x);
                    const A psion = x <= rmax ? acc_sub(c0, acc_mul_r(x2, quarter_n))
                                              : acc_sub(acc_zero(A()), acc_mul_r(Imax, lnx));
                    const A Ix = x < rmax ? acc_mul_r(x2, half_n) : Imax;
                    psi = acc_to_r(acc_add(acc_add(W.regL[k], acc_mul_r(Sk, lnx)), psion));
                    dprv = acc_to_r(acc_sub(Sk, Ix)) / x;
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
                    psi = acc_to_r(acc_add(W.regL[0], c0));
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

        // ---------------- stages 2-4
        const R cst[3] = {(R)0.5, (R)0.5, (R)1};
        const R wst[3] = {(R)2, (R)2, (R)1};
        for (int stg = 0; stg < 3 && !bad; ++stg) {
            C.sync();
            // the stage state in base (sorted y_n) order, mirrored at the axis
            bool ok = true;
            for (int p = p0; p < p1; ++p) {
                R r = rho[p], rl = W.rho_lo[p];
                radius_add(r, rl, cst[stg] * dxi * W.rk_kr[p]);
                R u = ur[p] + cst[stg] * dxi * W.rk_ku[p];
                const R s = r < (R)0 ? (R)-1 : (R)1;
                W.rk_r[p] = s * r;
                W.rk_rlo[p] = s * rl;
                W.rk_u[p] = s * u;
                W.rk_sg[p] = s;
            }
            C.sync();
            for (int p = p0; p < p1; ++p)
                if (p + 1 < n && W.rk_r[p + 1] < W.rk_r[p]) ok = false;
            const int32_t* perm = nullptr;
            if (!wake_vote(C, ok, true)) {
                if (sorter) {
                    for (int i = tid; i < W.n_pad; i += T) {
                        keys[i] = i < n ? W.rk_r[i] : (R)INFINITY;
                        vals[i] = i;
                    }
                    __syncthreads();
                    block_bitonic_sort(keys, vals, W.n_pad);
                    for (int i = tid; i < n; i += T) W.rk_perm[i] = vals[i];
                }
                perm = W.rk_perm;
                C.sync();
            }
            for (int i = tid; i < n; i += T) sR[i] = W.rk_r[perm ? perm[i] : i];
            // the sort's scratch overlaps the staged beam radii: stage them again
            if (perm && staged)
                for (int q = tid; q < m; q += T) sB[q] = W.br[b0 + q];
            __syncthreads();
            RkSource<R> sst;
            if (stg < 2) sst = {b0, m, b1, m1, (R)0.5, (R)0.5, qtot, qtot1, beamR};
            else sst = {b1, m1, 0, 0, (R)1, (R)0, qtot1, (R)0, W.br + b1};
            bad = rk_stage(W, sscan, sR, W.rk_rlo, W.rk_u, rid, perm, W.rk_sg, sst, W.rk_kr, W.rk_ku, W.frho[0],
                           W.fur[0], wst[stg], false, slice, mode, p0, p1, C);
        }
        if (bad) {
            status = 4;
            fail = slice;
            ++slice;
            break;
        }

        // ---------------- y_{n+1} = y_n + h/6 (k1 + 2 k2 + 2 k3 + k4), reflection
        C.sync();
        for (int p = p0; p < p1; ++p) {
            R r = rho[p], rl = W.rho_lo[p];
            radius_add(r, rl, dxi / (R)6 * W.frho[0][p]);
            R u = ur[p] + dxi / (R)6 * W.fur[0][p];
            if (r < (R)0) {
                r = -r;
                rl = -rl;
                u = -u;
            }
            rho[p] = r;
            W.rho_lo[p] = rl;
            ur[p] = u;
        }
        C.sync();
    }
    C.sync();
    if (C.rank == 0 && tid == 0) {
        if (mode == MODE_MARCH) put_march_times(W.ctl, t_launch);
        W.ctl[CTL_NEXT] = mode == MODE_MARCH ? slice : s_ctl[CTL_NEXT];
        W.ctl[CTL_BUF] = buf;
        W.ctl[CTL_PREV] = 0;
        if (status) {
            W.ctl[CTL_STATUS] = status;
            W.ctl[CTL_FAIL] = fail;
        }
    }
}

}  // namespace gbwake
