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

__global__ void bin_count_kernel(const double* __restrict__ xi, int64_t n, double dxi, int32_t n_steps,
                                 int32_t* __restrict__ slot, int32_t* __restrict__ cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double s = floor(__dadd_rn(__ddiv_rn(xi[k], dxi), 0.5));
        int32_t sl = -1;
        if (s >= 0.0 && s < (double)n_steps) {
            sl = (int32_t)s;
            atomicAdd(&cnt[sl], 1);
        }
        slot[k] = sl;
    }
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

__global__ void bin_scatter_kernel(const int32_t* __restrict__ slot, int64_t n, const int32_t* __restrict__ off,
                                   int32_t* __restrict__ fill, int32_t* __restrict__ binned_idx) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = slot[k];
        if (s >= 0) {
            int32_t pos = off[s] + atomicAdd(&fill[s], 1);
            binned_idx[pos] = (int32_t)k;
        }
    }
}

// one block per slice (grid-stride over slices); m_pad = power of two >= the
// largest slice, keys double, values caller index, prefix double
template <class R>
__global__ void slice_sort_kernel(const int32_t* __restrict__ off, int32_t n_steps,
                                  const double* __restrict__ r_in, const double* __restrict__ qw_in,
                                  int32_t* __restrict__ idx, R* __restrict__ br, R* __restrict__ bE,
                                  R* __restrict__ bQs, R* __restrict__ bTot, int32_t m_pad,
                                  int32_t* __restrict__ ctl) {
    extern __shared__ __align__(16) unsigned char smem[];
    double* keys = reinterpret_cast<double*>(smem);
    double* pre = keys + m_pad;
    int32_t* vals = reinterpret_cast<int32_t*>(pre + m_pad);
    __shared__ double sbuf[33];
    for (int32_t s = blockIdx.x; s < n_steps; s += gridDim.x) {
        const int32_t b0 = off[s], m = off[s + 1] - b0;
        if (m > m_pad) {  // slice too dense for the shared-memory sort: refuse the wake
            if (threadIdx.x == 0) {
                ctl[1] = 1;
                ctl[2] = s;
                bTot[s] = 0;
            }
            continue;
        }
        int32_t mp = 1;
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
        for (int32_t k = 2; k <= mp; k <<= 1) {
            for (int32_t j = k >> 1; j > 0; j >>= 1) {
                for (int32_t i = threadIdx.x; i < mp; i += blockDim.x) {
                    int32_t ixj = i ^ j;
                    if (ixj > i) {
                        double ki = keys[i], kj = keys[ixj];
                        int32_t vi = vals[i], vj = vals[ixj];
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
    if (threadIdx.x < 8) ctl[threadIdx.x] = threadIdx.x == 2 ? -1 : 0;
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

cudaError_t launch_bin_count(const double* xi, int64_t n, double dxi, int32_t n_steps, int32_t* slot,
                             int32_t* cnt, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    bin_count_kernel<<<grid_for(n, 256), 256, 0, st>>>(xi, n, dxi, n_steps, slot, cnt);
    return cudaGetLastError();
}

cudaError_t launch_excl_scan(const int32_t* cnt, int32_t n, int32_t* off, int32_t* max_count, cudaStream_t st) {
    excl_scan_kernel<<<1, 1024, 0, st>>>(cnt, n, off, max_count);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const int32_t* slot, int64_t n, const int32_t* off, int32_t* fill,
                               int32_t* binned_idx, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    bin_scatter_kernel<<<grid_for(n, 256), 256, 0, st>>>(slot, n, off, fill, binned_idx);
    return cudaGetLastError();
}

size_t slice_sort_smem(int32_t m_pad) { return (size_t)m_pad * (8 + 8 + 4); }

cudaError_t launch_reset_ctl(int32_t* ctl, cudaStream_t st) {
    reset_ctl_kernel<<<1, 32, 0, st>>>(ctl);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_slice_sort(const int32_t* off, int32_t n_steps, const double* r_in, const double* qw_in,
                              int32_t* idx, R* br, R* bE, R* bQs, R* bTot, int32_t m_pad, int32_t* ctl,
                              cudaStream_t st) {
    size_t sm = slice_sort_smem(m_pad);
    cudaError_t e = cudaFuncSetAttribute(slice_sort_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int grid = n_steps < 152 * 4 ? n_steps : 152 * 4;
    if (grid < 1) grid = 1;
    slice_sort_kernel<R><<<grid, 512, sm, st>>>(off, n_steps, r_in, qw_in, idx, br, bE, bQs, bTot, m_pad, ctl);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_scatter_out(const int32_t* idx, const int32_t* nbin, int64_t nb_max, const R* src, R* dst,
                               cudaStream_t st) {
    if (nb_max <= 0) return cudaSuccess;
    scatter_out_kernel<R><<<grid_for(nb_max, 256), 256, 0, st>>>(idx, nbin, src, dst);
    return cudaGetLastError();
}

template cudaError_t launch_slice_sort<double>(const int32_t*, int32_t, const double*, const double*, int32_t*,
                                               double*, double*, double*, double*, int32_t, int32_t*,
                                               cudaStream_t);
template cudaError_t launch_slice_sort<float>(const int32_t*, int32_t, const double*, const double*, int32_t*,
                                              float*, float*, float*, float*, int32_t, int32_t*, cudaStream_t);
template cudaError_t launch_scatter_out<double>(const int32_t*, const int32_t*, int64_t, const double*, double*,
                                                cudaStream_t);
template cudaError_t launch_scatter_out<float>(const int32_t*, const int32_t*, int64_t, const float*, float*,
                                               cudaStream_t);

}  // namespace gbwake
