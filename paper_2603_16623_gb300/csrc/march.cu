// march.cu -- instantiations and launchers of the ring kernels.
#include "march.h"

namespace gbwake {

// Sec. II ring initialisation: ring j at the centre of its cell, weight
// n * centre * width (Eq. macroparticle_weight), self weight
// n * (centre * width / 2 - width^2 / 8) (the charge of the cell below the
// ring), at rest; computed in FP64 and rounded once to the state precision.
template <class R>
__global__ void ring_init_kernel(const double* __restrict__ edges, int32_t n, double density, R* w, R* wh,
                                 R* rho, R* rho_lo, R* ur, R* frho, R* fur, int32_t* rid) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        double d = edges[j + 1] - edges[j];
        double c = 0.5 * (edges[j] + edges[j + 1]);
        w[j] = (R)(density * c * d);
        wh[j] = (R)(density * (0.5 * c * d - 0.125 * d * d));
        rho[j] = (R)c;
        rho_lo[j] = (R)(c - (double)(R)c);
        ur[j] = 0;
        frho[j] = 0;
        fur[j] = 0;
        rid[j] = j;
    }
}

template <class R>
__global__ void gather_by_id_kernel(const int32_t* __restrict__ rid, const R* __restrict__ src, R* __restrict__ dst,
                                    int32_t n) {
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) dst[rid[p]] = src[p];
}

size_t march_smem(int32_t n_max, int32_t n_pad_max, size_t real_bytes, int32_t m_max, int32_t* mb_cap) {
    const int32_t kStageTarget = 8192;
    int32_t mb = m_max < kStageTarget ? m_max : kStageTarget;
    size_t sort_bytes = (size_t)n_pad_max * (real_bytes + 4);
    size_t stage_bytes = ((size_t)n_max + mb) * real_bytes;
    size_t region = sort_bytes > stage_bytes ? sort_bytes : stage_bytes;
    region = (region + 15) & ~(size_t)15;
    *mb_cap = (int32_t)(region / real_bytes) - n_max;
    return (size_t)kScanBytes + region;
}

template <class P>
cudaError_t launch_march(const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes, int32_t max_slices,
                         int32_t mode, int32_t threads, size_t smem, int32_t mb_cap, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(march_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    march_kernel<P><<<n_wakes, threads, smem, st>>>(d_wakes, d_order, max_slices, mode, mb_cap);
    return cudaGetLastError();
}

cudaError_t launch_march_fast(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                              int32_t max_slices, int32_t mode, int32_t threads, cudaStream_t st) {
    size_t smem = fast_smem_bytes(threads, kFastK);
    cudaError_t e = cudaFuncSetAttribute(march_fast_kernel<kFastK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    march_fast_kernel<kFastK><<<n_wakes, threads, smem, st>>>(d_wakes, d_order, max_slices, mode);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_ring_init(const double* edges, int32_t n, double density, R* w, R* wh, R* rho, R* rho_lo, R* ur,
                             R* frho, R* fur, int32_t* rid, cudaStream_t st) {
    int grid = (n + 255) / 256;
    ring_init_kernel<R><<<grid, 256, 0, st>>>(edges, n, density, w, wh, rho, rho_lo, ur, frho, fur, rid);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_gather_by_id(const int32_t* rid, const R* src, R* dst, int32_t n, cudaStream_t st) {
    int grid = (n + 255) / 256;
    gather_by_id_kernel<R><<<grid, 256, 0, st>>>(rid, src, dst, n);
    return cudaGetLastError();
}

template cudaError_t launch_march<PrecF64>(const WakeDev<PrecF64>*, const int32_t*, int32_t, int32_t, int32_t,
                                           int32_t, size_t, int32_t, cudaStream_t);
template cudaError_t launch_march<PrecMixed>(const WakeDev<PrecMixed>*, const int32_t*, int32_t, int32_t, int32_t,
                                             int32_t, size_t, int32_t, cudaStream_t);
template cudaError_t launch_ring_init<double>(const double*, int32_t, double, double*, double*, double*, double*,
                                              double*, double*, double*, int32_t*, cudaStream_t);
template cudaError_t launch_ring_init<float>(const double*, int32_t, double, float*, float*, float*, float*, float*,
                                             float*, float*, int32_t*, cudaStream_t);
template cudaError_t launch_gather_by_id<double>(const int32_t*, const double*, double*, int32_t, cudaStream_t);
template cudaError_t launch_gather_by_id<float>(const int32_t*, const float*, float*, int32_t, cudaStream_t);

}  // namespace gbwake
