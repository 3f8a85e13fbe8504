// march_fast.cuh -- the production march: one wake per thread block with the
// ring state resident on chip for the whole window.
//
// Thread t owns the K consecutive sorted positions [tK, tK+K) (K a
// compile-time constant), keeps their per-slice quantities in registers, and
// the ring state (rho as a float-float pair, u_r, the AB2 history, weights,
// ring id) lives in shared memory in a swizzled blocked layout that makes
// the per-thread strided accesses bank-conflict free.  Per slice:
//   a2  sortedness check; bitonic sort of (rho, position) only if needed
//   a3  beam -> rings: each beam particle of the slice finds its radial
//       place among the rings (binary search in shared memory) and counts
//       into that place; the per-ring count prefix (folded into the first
//       block scan) gives the enclosed beam charge at every ring
//   a4  block scan of (sum w, sum w ln rho, particle counts), float-float
//   a5  psi, d_rho psi (self weight), psibar, gamma, t
//   a6  block scan of t -> d_zeta psi
//   a7  A, B, C and the ring sources of the B_theta^(p) problem
//   a8  B_theta^(p): regular (forward) and decaying (backward) homogeneous
//       solutions by two 2x2 matrix-product scans, then the discrete Green's
//       function sums (one more scan) -> region coefficients a_k, b_k
//   a9  fields at the slice's beam particles from per-region tables
//   a10 AB2 push (rho accumulated in float-float), axis reflection
#pragma once

#include "march.cuh"

namespace gbwake {

template <int K>
struct Swz {
    // position p (thread p/K, slot p%K) -> shared-memory word; XOR-swizzle of
    // the slot by the thread's group so that the K-strided accesses of a warp
    // hit 32 distinct banks
    static constexpr int kShift = (K == 8) ? 2 : (K == 16 ? 1 : 0);
    __device__ __forceinline__ static int at(int p) {
        int t = p / K, j = p % K;
        return t * K + (j ^ ((t >> kShift) & (K - 1)));
    }
};

// shared-memory footprint of the fast march for blocks of T threads
__host__ __device__ inline size_t fast_smem_bytes(int T, int K) {
    size_t cap = (size_t)T * K + 8;           // ring positions (+ region n)
    return (size_t)kScanBytes + 13 * 4 * cap;  // 8 state + 5 table arrays
}

template <int K>
__global__ void __launch_bounds__(512)
march_fast_kernel(const WakeDev<PrecMixed>* __restrict__ wakes, const int32_t* __restrict__ order,
                  int32_t max_slices, int32_t mode) {
    using R = float;
    using A = ff;
    using SW = Swz<K>;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_ctl[CTL_N];

    const WakeDev<PrecMixed>& W = wakes[order ? order[blockIdx.x] : blockIdx.x];
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int n = W.n;
    const int p0 = tid * K;
    const int cap = T * K + 8;

    unsigned char* sscan = smem;
    float* s_rh = reinterpret_cast<float*>(smem + kScanBytes);  // rho (hi), sorted
    float* s_rl = s_rh + cap;                                     // rho (lo)
    float* s_u = s_rl + cap;
    float* s_fr = s_u + cap;
    float* s_fu = s_fr + cap;
    float* s_w = s_fu + cap;
    float* s_wh = s_w + cap;
    int32_t* s_id = reinterpret_cast<int32_t*>(s_wh + cap);
    float* t_a = reinterpret_cast<float*>(s_id + cap);  // region tables
    float* t_b = t_a + cap;
    float* t_T = t_b + cap;   // sum of t over rings >= k  (E_z in region k)
    float* t_D = t_T + cap;   // S_k - I(rho_k)            (for d_rho psi)
    float* t_psi = t_D + cap; // psi at ring k
    int32_t* t_cnt = reinterpret_cast<int32_t*>(t_a);  // beam counts (reuses t_a)
    float* srt_key = t_a;                               // sort scratch (reuses tables)
    int32_t* srt_idx = reinterpret_cast<int32_t*>(t_a + 2 * cap);

    if (tid < CTL_N) s_ctl[tid] = W.ctl[tid];
    __syncthreads();
    if (s_ctl[CTL_STATUS] != 0) return;
    int slice = s_ctl[CTL_NEXT];
    const int buf = s_ctl[CTL_BUF];
    int has_prev = s_ctl[CTL_PREV];
    int status = 0, fail = -1;
    const int s_end = mode == MODE_MARCH ? min(W.n_steps, slice + max_slices) : slice + 1;

    // ---- load the ring state (global, sorted) into shared memory
    for (int p = tid; p < n; p += T) {
        int a = SW::at(p);
        int id = W.rid[buf][p];
        s_rh[a] = W.rho[buf][p];
        s_rl[a] = W.rho_lo[p];
        s_u[a] = W.ur[buf][p];
        s_fr[a] = W.frho[buf][p];
        s_fu[a] = W.fur[buf][p];
        s_w[a] = W.w[id];
        s_wh[a] = W.wh[id];
        s_id[a] = id;
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

    R rh[K], ur[K], w[K], wh[K];       // ring state in registers for the slice
    R pbv[K], dprv[K], bbv[K];         // psibar, d_rho psi, B^(b) at the rings
    R s0v[K], s1v[K], hav[K];          // B^(p) sources c_p and A_p / 2

    for (; slice < s_end; ++slice) {
        // ---------------- a2: sort by radius if out of order
        {
            bool ok = true;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                rh[k] = p < n ? s_rh[SW::at(p)] : 0.f;
                if (k > 0 && p < n && rh[k] < rh[k - 1]) ok = false;
            }
            if (p0 + K < n && p0 + K - 1 < n && s_rh[SW::at(p0 + K)] < rh[K - 1]) ok = false;
            if (!__syncthreads_and(ok)) {
                const int n_pad = W.n_pad;
                for (int i = tid; i < n_pad; i += T) {
                    srt_key[i] = i < n ? s_rh[SW::at(i)] : (R)INFINITY;
                    srt_idx[i] = i;
                }
                __syncthreads();
                for (int k2 = 2; k2 <= n_pad; k2 <<= 1) {
                    for (int j = k2 >> 1; j > 0; j >>= 1) {
                        for (int i = tid; i < n_pad; i += T) {
                            int ixj = i ^ j;
                            if (ixj > i) {
                                R ki = srt_key[i], kj = srt_key[ixj];
                                int vi = srt_idx[i], vj = srt_idx[ixj];
                                bool gt = (ki > kj) || (ki == kj && vi > vj);
                                if (gt == ((i & k2) == 0)) {
                                    srt_key[i] = kj; srt_key[ixj] = ki;
                                    srt_idx[i] = vj; srt_idx[ixj] = vi;
                                }
                            }
                        }
                        __syncthreads();
                    }
                }
                // gather the new rings of this thread, then write them back in order
                R g_rh[K], g_rl[K], g_u[K], g_fr[K], g_fu[K], g_w[K], g_wh[K];
                int g_id[K];
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    int p = p0 + k;
                    if (p < n) {
                        int a = SW::at(srt_idx[p]);
                        g_rh[k] = s_rh[a]; g_rl[k] = s_rl[a]; g_u[k] = s_u[a]; g_fr[k] = s_fr[a];
                        g_fu[k] = s_fu[a]; g_w[k] = s_w[a]; g_wh[k] = s_wh[a]; g_id[k] = s_id[a];
                    }
                }
                __syncthreads();
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    int p = p0 + k;
                    if (p < n) {
                        int a = SW::at(p);
                        s_rh[a] = g_rh[k]; s_rl[a] = g_rl[k]; s_u[a] = g_u[k]; s_fr[a] = g_fr[k];
                        s_fu[a] = g_fu[k]; s_w[a] = g_w[k]; s_wh[a] = g_wh[k]; s_id[a] = g_id[k];
                        rh[k] = g_rh[k];
                    }
                }
                __syncthreads();
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < n) {
                int a = SW::at(p);
                ur[k] = s_u[a];
                w[k] = s_w[a];
                wh[k] = s_wh[a];
            } else {
                ur[k] = 0.f; w[k] = 0.f; wh[k] = 0.f; rh[k] = 1.f;
            }
        }

        // ---------------- a3: beam particles count into their radial place
        const bool have_beam = W.nb > 0 && slice < W.n_steps;
        int b0 = 0, m = 0;
        R qtot = 0;
        if (have_beam) {
            b0 = W.boff[slice];
            m = W.boff[slice + 1] - b0;
            qtot = W.bTot[slice];
        }
        if (m > 0) {
            for (int i = tid; i < cap; i += T) t_cnt[i] = 0;
            __syncthreads();
            for (int q = tid; q < m; q += T) {
                R x = W.br[b0 + q];
                // u = number of rings with rho <= x: the rings this particle is below of
                int lo = 0, hi = n;
                while (lo < hi) {
                    int mid = (lo + hi) >> 1;
                    if (s_rh[SW::at(mid)] <= x) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < n) atomicAdd(&t_cnt[SW::at(lo)], 1);
            }
            __syncthreads();
        }

        // ---------------- a4: scan of (sum w, sum w ln rho, counts)
        A sw = zeroA, sl = zeroA;
        int64_t cl = 0;
        R lnr[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            lnr[k] = logf(rh[k]);
            if (p < n) {
                sw = ff_add_f(sw, w[k]);
                sl = ff_add(sl, ff_two_prod(w[k], lnr[k]));
                if (m > 0) cl += t_cnt[SW::at(p)];
            }
        }
        Trip<A> tot1;
        Trip<A> ex1 = block_excl_scan<false>(Trip<A>{sw, sl, cl}, OpAddTrip(), Trip<A>{zeroA, zeroA, 0},
                                             reinterpret_cast<Trip<A>*>(sscan), tot1);
        const int cex = (int)ex1.c;
        const A Wtot = tot1.x, Ltot = tot1.y;

        // ---------------- a5: psi, d_rho psi, psibar, gamma, t; beam field
        A S = ex1.x, L = ex1.y;
        A tl = zeroA;
        R tv[K];
        int lb = cex;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < n && m > 0) lb += t_cnt[SW::at(p)];  // particles strictly below ring p
            if (p < n) {
                R r = rh[k], u = ur[k];
                A Lsuf = ff_sub(Ltot, L);
                A psiA = ff_add(ff_add(Lsuf, ff_mul_f(S, lnr[k])), ion_psi(r, rmax, quarter_n, Imax, c0));
                R psi = ff_to_f(psiA);
                A Sm = ff_sub(S, ion_enclosed(r, rmax, half_n, Imax));
                R dpr = ff_to_f(ff_add_f(Sm, wh[k])) / r;
                R pb = 1.f + psi;
                R g = (1.f + u * u + pb * pb) / (2.f * pb);
                (void)g;
                pbv[k] = pb;
                dprv[k] = dpr;
                tv[k] = w[k] * u / (r * pb);
                int a = SW::at(p);
                t_D[a] = ff_to_f(Sm);
                t_psi[a] = psi;
                R Q = 0.f;
                if (m > 0) Q = lb < m ? W.bE[b0 + lb] : qtot;
                bbv[k] = Q * inv_2pi_dxi / r;
                if (mode == MODE_MARCH && W.dump_psi) {
                    size_t row = (size_t)slice * n + s_id[a];
                    W.dump_psi[row] = psi;
                    W.dump_dpr[row] = dpr;
                }
                S = ff_add_f(S, w[k]);
                L = ff_add(L, ff_two_prod(w[k], lnr[k]));
                tl = ff_add_f(tl, tv[k]);
            } else {
                pbv[k] = 1.f; dprv[k] = 0.f; tv[k] = 0.f; bbv[k] = 0.f;
            }
        }
        A Ttot;
        A Tex = block_excl_scan<false>(tl, OpAdd(), zeroA, reinterpret_cast<A*>(sscan), Ttot);

        // ---------------- a6 + a7: d_zeta psi, A, B, C, ring sources
        const Mat2<R> I2 = {1, 0, 0, 1};
        Mat2<R> Mf = I2, Mb = I2;
        {
            A Tacc = Tex;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < n) {
                    R r = rh[k], u = ur[k], pb = pbv[k], dpr = dprv[k];
                    t_T[SW::at(p)] = ff_to_f(ff_sub(Ttot, Tacc));
                    Tacc = ff_add_f(Tacc, tv[k]);
                    R above = ff_to_f(ff_sub(Ttot, Tacc));
                    R dpz = -(above + (1.f - wh[k] / w[k]) * tv[k]);
                    tv[k] = dpz;
                    R g = (1.f + u * u + pb * pb) / (2.f * pb);
                    R wr = w[k] / r, pb2 = pb * pb;
                    R Ac = wr / pb;
                    R Bc = -wr * g * dpr / pb2 + wr * bbv[k] / pb + (w[k] / (r * r)) * u * u / pb2 +
                           wr * u * u * dpr / (pb2 * pb) - wr * u * dpz / pb2;
                    R Cc = -wr * (g / pb - 1.f - u * u / pb2);
                    R hA = 0.5f * Ac;
                    hav[k] = hA;
                    s0v[k] = 0.25f * (2.f * Bc + Ac * Cc);
                    s1v[k] = 0.25f * r * (4.f * Cc - 2.f * Bc * r - Ac * Cc * r);
                    Mat2<R> M = {1.f + hA * r, hA / r, -hA * r * r * r, 1.f - hA * r};
                    Mf = OpMatLeft()(Mf, M);
                    if (mode == MODE_MARCH && W.dump_dpz) W.dump_dpz[(size_t)slice * n + s_id[SW::at(p)]] = dpz;
                } else {
                    hav[k] = 0.f; s0v[k] = 0.f; s1v[k] = 0.f;
                }
            }
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                if (p0 + k < n) {
                    R r = rh[k], hA = hav[k];
                    Mat2<R> Mi = {1.f - hA * r, -hA / r, hA * r * r * r, 1.f + hA * r};
                    Mb = OpMatLeft()(Mb, Mi);
                }
            }
        }

        // ---------------- a8: B_theta^(p) region coefficients
        Mat2<R> tf, tb;
        Mat2<R> Yf = block_excl_scan<false>(Mf, OpMatLeft(), I2, reinterpret_cast<Mat2<R>*>(sscan), tf);
        Mat2<R> Yb = block_excl_scan<true>(Mb, OpMatLeft(), I2, reinterpret_cast<Mat2<R>*>(sscan), tb);
        R Rra[K], Rrb[K], Dda[K], Ddb[K];  // R_{p+1}, D_{p+1}
        {
            Mat2<R> Y = Yf;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (p0 + k < n) {
                    R r = rh[k], hA = hav[k];
                    Mat2<R> M = {1.f + hA * r, hA / r, -hA * r * r * r, 1.f - hA * r};
                    Y = OpMatLeft()(Y, M);
                }
                Rra[k] = Y.m00;
                Rrb[k] = Y.m10;
            }
        }
        A gl = zeroA, dl = zeroA;
        R gpv[K], dpv[K];
        R Dp0a = 0.f, Dp0b = 1.f;  // D at region p0 (after the walk)
        {
            Mat2<R> Y = Yb;
#pragma unroll
            for (int k = K - 1; k >= 0; --k) {
                Dda[k] = Y.m01;
                Ddb[k] = Y.m11;
                if (p0 + k < n) {
                    R q0 = Rra[k], q1 = Rrb[k], d0 = Y.m01, d1 = Y.m11;
                    R wr = q0 * d1 - q1 * d0;
                    R gp = (s0v[k] * d1 - s1v[k] * d0) / wr;
                    R dp = (q0 * s1v[k] - q1 * s0v[k]) / wr;
                    gpv[k] = gp;
                    dpv[k] = dp;
                    gl = ff_add_f(gl, gp);
                    dl = ff_add_f(dl, dp);
                    R r = rh[k], hA = hav[k];
                    Mat2<R> Mi = {1.f - hA * r, -hA / r, hA * r * r * r, 1.f + hA * r};
                    Y = OpMatLeft()(Y, Mi);
                } else {
                    gpv[k] = 0.f;
                    dpv[k] = 0.f;
                }
            }
            Dp0a = Y.m01;
            Dp0b = Y.m11;
        }
        Pair<A> gd_tot;
        Pair<A> gd = block_excl_scan<false>(Pair<A>{gl, dl}, OpAddPair(), Pair<A>{zeroA, zeroA},
                                            reinterpret_cast<Pair<A>*>(sscan), gd_tot);
        {
            // region p (k = 0..K-1) below ring p: R_p, D_p; R_p = R_{(p-1)+1}
            A Gex = gd.x, Hex = gd.y;
            R Rpa = Yf.m00, Rpb = Yf.m10;  // R at region p0
            R Dpa = Dp0a, Dpb = Dp0b;      // D at region p0
#pragma unroll
            for (int k = 0; k < K; ++k) {
                int p = p0 + k;
                if (p < n) {
                    R G = ff_to_f(ff_sub(gd_tot.x, Gex));
                    R H = ff_to_f(Hex);
                    int a = SW::at(p);
                    t_a[a] = -G * Rpa + H * Dpa;
                    t_b[a] = -G * Rpb + H * Dpb;
                    Gex = ff_add_f(Gex, gpv[k]);
                    Hex = ff_add_f(Hex, dpv[k]);
                    Rpa = Rra[k];
                    Rpb = Rrb[k];
                    // D at region p+1 was Dd[k]
                    Dpa = Dda[k];
                    Dpb = Ddb[k];
                }
            }
            if (p0 < n && p0 + K >= n) {  // owner of the last ring writes region n
                R H = ff_to_f(gd_tot.y);
                int a = n < T * K ? SW::at(n) : T * K;
                t_a[a] = 0.f;       // a_n = 0 (D_n = (0, 1))
                t_b[a] = H;         // b_n = H_n
                t_T[a] = 0.f;
                t_D[a] = ff_to_f(ff_sub(Wtot, Imax));
                t_psi[a] = 0.f;
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
                int a = SW::at(p);
                int a1 = (p + 1 < T * K) ? SW::at(p + 1) : T * K;
                if (p + 1 == n) a1 = n < T * K ? SW::at(n) : T * K;
                R r = rh[k];
                bpv[k] = 0.5f * ((t_a[a] + t_a[a1]) * r + (t_b[a] + t_b[a1]) / r);
                R pb = pbv[k];
                if (!(pb > 0.f) || !isfinite(pb) || !isfinite(dprv[k]) || !isfinite(tv[k]) || !isfinite(bpv[k]) ||
                    !isfinite(bbv[k]))
                    bad = true;
                if (mode == MODE_MARCH) {
                    size_t row = (size_t)slice * n + s_id[a];
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
            for (int64_t q = tid; q < nq; q += T) {
                R x = mode == MODE_MARCH ? W.br[b0 + q] : (R)W.rq[q];
                R psi, dpr, dpz, bp, bb;
                if (x > 0.f) {
                    int lo = 0, hi = n;  // k = number of rings with rho < x
                    while (lo < hi) {
                        int mid = (lo + hi) >> 1;
                        if (s_rh[SW::at(mid)] < x) lo = mid + 1;
                        else hi = mid;
                    }
                    const int k = lo;
                    const int a = k < T * K ? SW::at(k) : T * K;
                    const R cx = fminf(x, rmax);
                    R rk, Ik;
                    if (k < n) {
                        rk = s_rh[a];
                        R ck = fminf(rk, rmax);
                        // S_k - I(x) = D_k + (I(rho_k) - I(x))
                        dpr = (t_D[a] + half_n * (ck - cx) * (ck + cx)) / x;
                        // psi(x) = psi_k - int_x^{rho_k} d_rho psi
                        R Sk = t_D[a] + half_n * ck * ck;
                        R Jk = rk <= rmax ? quarter_n * rk * rk
                                          : quarter_n * rmax * rmax + half_n * rmax * rmax * logf(rk / rmax);
                        R Jx = x <= rmax ? quarter_n * x * x
                                         : quarter_n * rmax * rmax + half_n * rmax * rmax * logf(x / rmax);
                        psi = t_psi[a] - (Sk * logf(rk / x) - (Jk - Jx));
                        (void)Ik;
                    } else {
                        // beyond every ring: S = W_tot
                        dpr = (t_D[a] + half_n * (rmax - cx) * (rmax + cx)) / x;
                        A Sx = Wtot;
                        psi = ff_to_f(ff_add(ff_mul_f(Sx, logf(x)), ion_psi(x, rmax, quarter_n, Imax, c0)));
                    }
                    dpz = -t_T[a];
                    bp = t_a[a] * x + t_b[a] / x;
                    if (mode == MODE_MARCH) {
                        bb = W.bQs[b0 + q] * inv_2pi_dxi / x;
                    } else {
                        bb = 0.f;
                        if (m > 0) {
                            int l2 = lower_bound_dev(W.br + b0, m, x);
                            R Q = l2 < m ? W.bE[b0 + l2] : qtot;
                            bb = Q * inv_2pi_dxi / x;
                        }
                    }
                } else {
                    psi = ff_to_f(ff_add(ff_sub(Ltot, zeroA), ion_psi(0.f, rmax, quarter_n, Imax, c0)));
                    dpr = 0.f;
                    dpz = -ff_to_f(Ttot);
                    bp = 0.f;
                    bb = 0.f;
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
        bad = __syncthreads_or(bad);
        if (mode != MODE_MARCH) break;
        if (bad) {
            status = 4;
            fail = slice;
            ++slice;
            break;
        }

        // ---------------- a10: AB2 push (rho accumulated in float-float)
#pragma unroll
        for (int k = 0; k < K; ++k) {
            int p = p0 + k;
            if (p < n) {
                int a = SW::at(p);
                R u = ur[k], pb = pbv[k];
                R g = (1.f + u * u + pb * pb) / (2.f * pb);
                R fr = u / pb;
                R fu = g * dprv[k] / pb - (bpv[k] + bbv[k]);
                R dr, du;
                if (has_prev) {
                    dr = dxi * (1.5f * fr - 0.5f * s_fr[a]);
                    du = dxi * (1.5f * fu - 0.5f * s_fu[a]);
                } else {
                    dr = dxi * fr;
                    du = dxi * fu;
                }
                ff rr = ff_add_f(ff{rh[k], s_rl[a]}, dr);
                R un = u + du;
                if (rr.hi < 0.f) {
                    rr = ff_neg(rr);
                    un = -un;
                    fr = -fr;
                    fu = -fu;
                }
                s_rh[a] = rr.hi;
                s_rl[a] = rr.lo;
                s_u[a] = un;
                s_fr[a] = fr;
                s_fu[a] = fu;
            }
        }
        has_prev = 1;
        __syncthreads();
    }

    // ---- store the ring state back (sorted order, same buffer)
    __syncthreads();
    for (int p = tid; p < n; p += T) {
        int a = SW::at(p);
        W.rho[buf][p] = s_rh[a];
        W.rho_lo[p] = s_rl[a];
        W.ur[buf][p] = s_u[a];
        W.frho[buf][p] = s_fr[a];
        W.fur[buf][p] = s_fu[a];
        W.rid[buf][p] = s_id[a];
    }
    if (tid == 0) {
        W.ctl[CTL_NEXT] = mode == MODE_MARCH ? slice : s_ctl[CTL_NEXT];
        W.ctl[CTL_PREV] = has_prev;
        if (status) {
            W.ctl[CTL_STATUS] = status;
            W.ctl[CTL_FAIL] = fail;
        }
    }
}

}  // namespace gbwake
