// beam.cu -- one-time beam preparation of a wake solve and output scatter.
//
// The beam is frozen during a quasistatic wake solve (Sec. II), so its
// macroparticles are binned by nearest slice and radially sorted once:
//   1. slice s = floor(xi/dxi + 1/2) in FP64 (the beam-grid spacing equals the
//      solver step, Sec. III), histogram;
//   2. exclusive scan of the histogram -> slice offsets;
//   3. scatter of particle indices into their slices;
//   4. per slice (one block): sort by (r, caller index), exclusive prefix of
//      charge x weight in FP64, the per-particle prefix at its first tie
//      (enclosed charge strictly below r, so no self field), slice totals.
// After the march, fields computed in binned order are scattered back to the
// caller's particle order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "beam.h"
#include "common.cuh"

namespace gbwake {

__global__ void fold_charge_kernel(double* qw, const double* w, double q, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        qw[k] = q * w[k];
}

// Slice histogram.  Each block takes a contiguous chunk of particles and
// counts them in shared memory (particles of a beam crowd into the same few
// hundred slices, so global atomics per particle would serialise), then adds
// its non-zero bins to the global counts.  n_steps <= kBinSmem.
__global__ void bin_count_kernel(const double* __restrict__ xi, int64_t n, double dxi, int32_t n_steps,
                                 int32_t* __restrict__ slot, int32_t* __restrict__ cnt) {
    extern __shared__ int32_t hist[];
    for (int32_t b = threadIdx.x; b < n_steps; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = blockIdx.x * per, k1 = min(n, k0 + per);
    for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
        const double s = floor(__dadd_rn(__ddiv_rn(xi[k], dxi), 0.5));
        int32_t sl = -1;
        if (s >= 0.0 && s < (double)n_steps) {
            sl = (int32_t)s;
            atomicAdd(&hist[sl], 1);
        }
        slot[k] = sl;
    }
    __syncthreads();
    for (int32_t b = threadIdx.x; b < n_steps; b += blockDim.x)
        if (hist[b]) atomicAdd(&cnt[b], hist[b]);
}

// single block: exclusive scan of cnt[0..n) into off[0..n], off[n] = total
__global__ void excl_scan_kernel(const int32_t* __restrict__ cnt, int32_t n, int32_t* __restrict__ off,
                                 int32_t* __restrict__ max_count) {
    __shared__ int64_t sbuf[33];
    int64_t carry = 0;
    int32_t mx = 0;
    for (int32_t base = 0; base < n; base += blockDim.x) {
        int32_t i = base + threadIdx.x;
        int64_t v = i < n ? cnt[i] : 0;
        if (i < n) mx = max(mx, (int32_t)v);
        int64_t tot;
        int64_t ex = block_excl_scan<false>(v, OpAdd(), (int64_t)0, sbuf, tot);
        if (i < n) off[i] = (int32_t)(carry + ex);
        carry += tot;
    }
    __shared__ int32_t smx;
    if (threadIdx.x == 0) smx = 0;
    __syncthreads();
    atomicMax(&smx, mx);
    __syncthreads();
    if (threadIdx.x == 0) {
        off[n] = (int32_t)carry;
        *max_count = smx;
    }
}

// Particle indices into their slices.  Each block takes the same chunk as
// in the histogram, ranks its particles within each slice in shared memory,
// reserves one range per non-empty slice with a single global atomic, and
// writes every index at its slice offset + range start + local rank.
__global__ void bin_scatter_kernel(const int32_t* __restrict__ slot, int64_t n, int32_t n_steps,
                                   const int32_t* __restrict__ off, int32_t* __restrict__ fill,
                                   int32_t* __restrict__ binned_idx) {
    extern __shared__ int32_t hist[];  // [n_steps] local counts, then range starts
    for (int32_t b = threadIdx.x; b < n_steps; b += blockDim.x) hist[b] = 0;
    __syncthreads();
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t k0 = blockIdx.x * per, k1 = min(n, k0 + per);
    int32_t rank[kBinPerThread];
#pragma unroll
    for (int j = 0; j < kBinPerThread; ++j) {
        const int64_t k = k0 + threadIdx.x + (int64_t)j * blockDim.x;
        const int32_t s = k < k1 ? slot[k] : -1;
        rank[j] = s >= 0 ? atomicAdd(&hist[s], 1) : -1;
    }
    __syncthreads();
    for (int32_t b = threadIdx.x; b < n_steps; b += blockDim.x)
        if (hist[b]) hist[b] = off[b] + atomicAdd(&fill[b], hist[b]);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBinPerThread; ++j) {
        const int64_t k = k0 + threadIdx.x + (int64_t)j * blockDim.x;
        if (rank[j] >= 0) binned_idx[hist[slot[k]] + rank[j]] = (int32_t)k;
    }
}

// the slice sort's order: radius, then caller index (distinct but for the
// padding entries, which go last)
__device__ __forceinline__ bool kv_less(double ka, int32_t va, double kb, int32_t vb) {
    return ka < kb || (ka == kb && va < vb);
}

// Sorts keys/vals[0, mp) in shared memory (mp a power of two >= 4, padded
// with (+inf, INT_MAX)); keys2/vals2 are as large, scratch.  Runs of four
// entries are sorted in registers (a bitonic network), then runs of 4, 8,
// ... are merged pairwise from one buffer into the other: each group of
// four outputs finds by a merge-path search how many of its predecessors
// come from the first run and merges its four outputs sequentially; the
// block's threads take the groups in turn.  log2(mp / 4) rounds of one
// block barrier and O(mp log mp) shared-memory traffic (a bitonic network
// over the block costs O(mp log^2 mp) with a barrier per stage).  The
// order is total, so the result is the one sort.
constexpr int kRun = 4;
__device__ __forceinline__ void merge_sort_smem(double* keys, int32_t* vals, double* keys2, int32_t* vals2,
                                                int32_t mp) {
    for (int32_t p0 = (int32_t)threadIdx.x * kRun; p0 < mp; p0 += (int32_t)blockDim.x * kRun) {
        double k[kRun];
        int32_t v[kRun];
#pragma unroll
        for (int e = 0; e < kRun; ++e) {
            k[e] = keys[p0 + e];
            v[e] = vals[p0 + e];
        }
#pragma unroll
        for (int k2 = 2; k2 <= kRun; k2 <<= 1)
#pragma unroll
            for (int j = k2 >> 1; j > 0; j >>= 1)
#pragma unroll
                for (int i = 0; i < kRun; ++i) {
                    const int l = i ^ j;
                    if (l > i && kv_less(k[l], v[l], k[i], v[i]) == ((i & k2) == 0)) {
                        const double tk = k[i];
                        const int32_t tv = v[i];
                        k[i] = k[l];
                        v[i] = v[l];
                        k[l] = tk;
                        v[l] = tv;
                    }
                }
#pragma unroll
        for (int e = 0; e < kRun; ++e) {
            keys[p0 + e] = k[e];
            vals[p0 + e] = v[e];
        }
    }
    __syncthreads();
    double* sk = keys;
    int32_t* sv = vals;
    double* dk = keys2;
    int32_t* dv = vals2;
    for (int32_t L = kRun; L < mp; L <<= 1) {
        for (int32_t p0 = (int32_t)threadIdx.x * kRun; p0 < mp; p0 += (int32_t)blockDim.x * kRun) {
            const int32_t base = p0 & ~(2 * L - 1), d = p0 - base;
            const double* ak = sk + base;
            const int32_t* av = sv + base;
            const double* bk = ak + L;
            const int32_t* bv = av + L;
            int32_t lo = d > L ? d - L : 0, hi = d < L ? d : L;
            while (lo < hi) {  // outputs before d taken from the first run (it goes first on equality)
                const int32_t mid = (lo + hi) >> 1;
                if (kv_less(bk[d - 1 - mid], bv[d - 1 - mid], ak[mid], av[mid])) hi = mid;
                else lo = mid + 1;
            }
            int32_t i = lo, j = d - lo;
#pragma unroll
            for (int e = 0; e < kRun; ++e) {
                const bool take_a = j >= L || (i < L && !kv_less(bk[j], bv[j], ak[i], av[i]));
                if (take_a) {
                    dk[p0 + e] = ak[i];
                    dv[p0 + e] = av[i];
                    ++i;
                } else {
                    dk[p0 + e] = bk[j];
                    dv[p0 + e] = bv[j];
                    ++j;
                }
            }
        }
        __syncthreads();
        double* tk = sk;
        sk = dk;
        dk = tk;
        int32_t* tv = sv;
        sv = dv;
        dv = tv;
    }
    if (sk != keys) {  // an odd number of rounds: back into keys/vals
        for (int32_t i = threadIdx.x; i < mp; i += blockDim.x) {
            keys[i] = sk[i];
            vals[i] = sv[i];
        }
        __syncthreads();
    }
}

// one block per slice (grid-stride over slices) sorting the slices of
// min_m < m <= m_pad particles; m_pad a power of two, keys double, values
// caller index, prefix double.  A slice denser than m_pad is left to a later
// pass with a larger m_pad, or, in the last pass (last = 1), refuses the wake.
template <class R>
__global__ void slice_sort_kernel(const int32_t* __restrict__ off, int32_t n_steps,
                                  const double* __restrict__ r_in, const double* __restrict__ qw_in,
                                  int32_t* __restrict__ idx, R* __restrict__ br, R* __restrict__ bE,
                                  R* __restrict__ bQs, R* __restrict__ bTot, int32_t m_pad, int32_t min_m,
                                  int32_t last, int32_t* __restrict__ ctl, int32_t* __restrict__ inv) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* keys = reinterpret_cast<double*>(smem);
    double* pre = keys + m_pad;
    int32_t* vals = reinterpret_cast<int32_t*>(pre + m_pad);
    __shared__ double sbuf[33];
    for (int32_t s = blockIdx.x; s < n_steps; s += gridDim.x) {
        const int32_t b0 = off[s], m = off[s + 1] - b0;
        if (m <= min_m) continue;  // an earlier pass sorted it
        if (m > m_pad) {
            if (last && threadIdx.x == 0) {  // too dense for the shared-memory sort: refuse the wake
                ctl[CTL_STATUS] = WAKE_STATUS_INVALID;
                ctl[CTL_FAIL] = s;
                bTot[s] = 0;
            }
            continue;
        }
        int32_t mp = kRun;
        while (mp < m) mp <<= 1;
        for (int32_t i = threadIdx.x; i < mp; i += blockDim.x) {
            if (i < m) {
                int32_t k = idx[b0 + i];
                keys[i] = r_in[k];
                vals[i] = k;
            } else {
                keys[i] = INFINITY;
                vals[i] = 0x7fffffff;
            }
        }
        __syncthreads();
        merge_sort_smem(keys, vals, pre, vals + m_pad, mp);
        // exclusive prefix of charge x weight in sorted order (FP64)
        double carry = 0.0;
        for (int32_t base = 0; base < m; base += blockDim.x) {
            int32_t i = base + threadIdx.x;
            double v = i < m ? qw_in[vals[i]] : 0.0;
            double tot;
            double ex = block_excl_scan<false>(v, OpAdd(), 0.0, sbuf, tot);
            if (i < m) pre[i] = carry + ex;
            carry += tot;
        }
        __syncthreads();
        for (int32_t i = threadIdx.x; i < m; i += blockDim.x) {
            int32_t f = i;
            while (f > 0 && keys[f - 1] == keys[i]) --f;  // first of a tie group
            idx[b0 + i] = vals[i];
            if (inv) inv[vals[i]] = b0 + i;  // caller index -> sorted position
            br[b0 + i] = (R)keys[i];
            bE[b0 + i] = (R)pre[i];
            bQs[b0 + i] = (R)pre[f];
        }
        if (threadIdx.x == 0) bTot[s] = (R)carry;
        __syncthreads();
    }
}

// binned -> caller order; the binned count is read on the device (*nbin)
template <class R>
__global__ void scatter_out_kernel(const int32_t* __restrict__ idx, const int32_t* __restrict__ nbin,
                                   const R* __restrict__ src, R* __restrict__ dst) {
    const int64_t nb = *nbin;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nb; p += (int64_t)gridDim.x * blockDim.x)
        dst[idx[p]] = src[p];
}

__global__ void reset_ctl_kernel(int32_t* ctl) {
    if (threadIdx.x < CTL_N) ctl[threadIdx.x] = threadIdx.x == CTL_FAIL ? -1 : 0;
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 32) g = 152 * 32;
    return (int)g;
}

cudaError_t launch_fold_charge(double* qw, const double* w, double q, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    fold_charge_kernel<<<grid_for(n, 256), 256, 0, st>>>(qw, w, q, n);
    return cudaGetLastError();
}

// blocks of the binning kernels: chunks of kBinPerThread x 256 particles
static int bin_grid(int64_t n) {
    const int64_t chunk = (int64_t)kBinPerThread * 256;
    int64_t g = (n + chunk - 1) / chunk;
    return (int)(g < 1 ? 1 : g);
}

cudaError_t launch_bin_count(const double* xi, int64_t n, double dxi, int32_t n_steps, int32_t* slot,
                             int32_t* cnt, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n_steps > kBinSmem) return cudaErrorInvalidValue;
    bin_count_kernel<<<bin_grid(n), 256, (size_t)n_steps * sizeof(int32_t), st>>>(xi, n, dxi, n_steps, slot, cnt);
    return cudaGetLastError();
}

cudaError_t launch_excl_scan(const int32_t* cnt, int32_t n, int32_t* off, int32_t* max_count, cudaStream_t st) {
    excl_scan_kernel<<<1, 1024, 0, st>>>(cnt, n, off, max_count);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const int32_t* slot, int64_t n, int32_t n_steps, const int32_t* off, int32_t* fill,
                               int32_t* binned_idx, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (n_steps > kBinSmem) return cudaErrorInvalidValue;
    bin_scatter_kernel<<<bin_grid(n), 256, (size_t)n_steps * sizeof(int32_t), st>>>(slot, n, n_steps, off, fill,
                                                                                      binned_idx);
    return cudaGetLastError();
}

size_t slice_sort_smem(int32_t m_pad) { return (size_t)m_pad * (8 + 8 + 4 + 4); }  // keys, prefix, values, scratch

cudaError_t launch_reset_ctl(int32_t* ctl, cudaStream_t st) {
    reset_ctl_kernel<<<1, 32, 0, st>>>(ctl);
    return cudaGetLastError();
}

template <class R>
static cudaError_t slice_sort_pass(const int32_t* off, int32_t n_steps, const double* r_in, const double* qw_in,
                                   int32_t* idx, R* br, R* bE, R* bQs, R* bTot, int32_t m_pad, int32_t min_m,
                                   int32_t last, int32_t* ctl, int32_t* inv, cudaStream_t st) {
    // the attribute allows the largest slice the library accepts; a launch
    // asks only for its own m_pad
    static cudaError_t attr = cudaFuncSetAttribute(slice_sort_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)slice_sort_smem(kSliceSortMaxPad));
    if (attr != cudaSuccess) return attr;
    const size_t sm = slice_sort_smem(m_pad);
    // one block width for every pass and size: the FP64 charge prefix is
    // summed in chunks of the block's width, and its rounding must not
    // depend on how the slices were split into passes
    const int threads = 256;
    // a pass after the first (min_m > 0) sorts only the rare slices denser
    // than the first pass took, with up to 196 KB of shared memory per block
    // (one block per SM): a few blocks that walk the offsets, rather than one
    // per slice that mostly finds nothing to do
    const int cap = min_m > 0 ? 16 : 152 * 8;
    int grid = n_steps < cap ? n_steps : cap;
    if (grid < 1) grid = 1;
    slice_sort_kernel<R><<<grid, threads, sm, st>>>(off, n_steps, r_in, qw_in, idx, br, bE, bQs, bTot, m_pad, min_m,
                                                    last, ctl, inv);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_slice_sort(const int32_t* off, int32_t n_steps, const double* r_in, const double* qw_in,
                              int32_t* idx, R* br, R* bE, R* bQs, R* bTot, int32_t densest, int32_t* ctl,
                              int32_t* inv, cudaStream_t st) {
    int32_t m_pad = 64;
    if (densest >= 0) {  // known: one pass sized for it
        while (m_pad < densest && m_pad < kSliceSortMaxPad) m_pad <<= 1;
        return slice_sort_pass<R>(off, n_steps, r_in, qw_in, idx, br, bE, bQs, bTot, m_pad, -1, 1, ctl, inv, st);
    }
    // unknown (counted on the device only): the slices that fit a small
    // shared-memory sort first, then the denser ones with the largest
    cudaError_t e = slice_sort_pass<R>(off, n_steps, r_in, qw_in, idx, br, bE, bQs, bTot, kSliceSortFirstPad, -1, 0,
                                       ctl, inv, st);
    if (e != cudaSuccess) return e;
    return slice_sort_pass<R>(off, n_steps, r_in, qw_in, idx, br, bE, bQs, bTot, kSliceSortMaxPad,
                              kSliceSortFirstPad, 1, ctl, inv, st);
}

template <class R>
cudaError_t launch_scatter_out(const int32_t* idx, const int32_t* nbin, int64_t nb_max, const R* src, R* dst,
                               cudaStream_t st) {
    if (nb_max <= 0) return cudaSuccess;
    scatter_out_kernel<R><<<grid_for(nb_max, 256), 256, 0, st>>>(idx, nbin, src, dst);
    return cudaGetLastError();
}

template cudaError_t launch_slice_sort<double>(const int32_t*, int32_t, const double*, const double*, int32_t*,
                                               double*, double*, double*, double*, int32_t, int32_t*, int32_t*,
                                               cudaStream_t);
template cudaError_t launch_slice_sort<float>(const int32_t*, int32_t, const double*, const double*, int32_t*,
                                              float*, float*, float*, float*, int32_t, int32_t*, int32_t*,
                                              cudaStream_t);
template cudaError_t launch_scatter_out<double>(const int32_t*, const int32_t*, int64_t, const double*, double*,
                                                cudaStream_t);
template cudaError_t launch_scatter_out<float>(const int32_t*, const int32_t*, int64_t, const float*, float*,
                                               cudaStream_t);

// radii are >= 0, so their bit patterns order as the values do
__global__ void species_rmax_kernel(const double* __restrict__ r, SpeciesRanges sp, double* rmax) {
    const int64_t nb = sp.begin[sp.n];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nb; k += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        while (s + 1 < sp.n && k >= sp.begin[s + 1]) ++s;
        atomicMax(reinterpret_cast<unsigned long long*>(rmax + s), (unsigned long long)__double_as_longlong(r[k]));
    }
}

cudaError_t launch_species_rmax(const double* r, SpeciesRanges sp, double* rmax, cudaStream_t st) {
    const int64_t nb = sp.begin[sp.n];
    if (nb <= 0) return cudaSuccess;
    int64_t g = (nb + 255) / 256;
    if (g > 152 * 8) g = 152 * 8;
    species_rmax_kernel<<<(int)g, 256, 0, st>>>(r, sp, rmax);
    return cudaGetLastError();
}

__global__ void grid_extent_check_kernel(const double* rmax, int32_t n_species, double grid_rmax, int32_t* ctl) {
    for (int b = 0; b < n_species; ++b)
        if (!(rmax[b] < grid_rmax)) {
            ctl[CTL_STATUS] = 1;  // EINVAL
            ctl[CTL_FAIL] = -1;   // no slice ran
            return;
        }
}

cudaError_t launch_grid_extent_check(const double* rmax, int32_t n_species, double grid_rmax, int32_t* ctl,
                                     cudaStream_t st) {
    grid_extent_check_kernel<<<1, 1, 0, st>>>(rmax, n_species, grid_rmax, ctl);
    return cudaGetLastError();
}

}  // namespace gbwake
