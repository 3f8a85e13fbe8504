// march_launch.cuh -- launch templates of the on-chip marches, shared by
// the translation units that instantiate them (march.cu: 4 and 8 rings per
// thread; march_k2.cu: 2, compiled in parallel).
#pragma once
#include <algorithm>

#include "march.h"

namespace gbwake {

// Asks for a shared-memory carveout no larger than the blocks an SM holds
// need (by registers: 128 per thread), so that the rest of the SM's 256 KB
// stays L1 for the per-ring constant table gathered every slice (left to
// itself the driver may pick the largest carveout, and the table then
// misses to L2).
template <class F>
inline cudaError_t set_carveout(F kern, int32_t threads, size_t dyn_smem) {
    constexpr size_t kSmemMax = 233472, kPerBlockExtra = 3 * 1024;  // reserved + static
    int32_t blocks = 65536 / (128 * threads);
    blocks = std::max(1, std::min(blocks, 2048 / threads));
    const size_t need = (size_t)blocks * (dyn_smem + kPerBlockExtra);
    int pct = (int)((need * 100 + kSmemMax - 1) / kSmemMax);
    pct = std::max(1, std::min(pct, 100));
    return cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

template <int K>
inline cudaError_t launch_fast_k(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                 int32_t max_slices, int32_t mode, int32_t threads, int32_t stage_particles,
                                 cudaStream_t st) {
    size_t smem = fast_smem_bytes(threads, K) + stage_smem_bytes(stage_particles);
    cudaError_t e =
        cudaFuncSetAttribute(march_fast_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = set_carveout(march_fast_kernel<K>, threads, smem);
    if (e != cudaSuccess) return cudaGetLastError(), e;  // (a refused call leaves no error behind)
    march_fast_kernel<K><<<n_wakes, threads, smem, st>>>(d_wakes, d_order, max_slices, mode, stage_particles);
    return cudaGetLastError();
}

template <int K>
inline cudaError_t launch_cluster_k(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                    int32_t max_slices, int32_t mode, int32_t threads, int32_t cl,
                                    int32_t stage_particles, cudaStream_t st) {
    size_t smem = cluster_smem_bytes(threads, K) + stage_smem_bytes(stage_particles);
    auto kern = march_cluster_kernel<K>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = set_carveout(kern, threads, smem);
    if (e != cudaSuccess) return cudaGetLastError(), e;  // (a refused call leaves no error behind)
    if (cl > 8) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return cudaGetLastError(), e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_wakes * cl), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, d_wakes, d_order, max_slices, mode, stage_particles);
    if (e != cudaSuccess) return cudaGetLastError(), e;
    return cudaGetLastError();
}


// the 2-rings-per-thread instantiations (march_k2.cu)
cudaError_t launch_march_fast_k2(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                 int32_t max_slices, int32_t mode, int32_t threads, int32_t stage_particles,
                                 cudaStream_t st);
cudaError_t launch_march_cluster_k2(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                    int32_t max_slices, int32_t mode, int32_t threads, int32_t cl,
                                    int32_t stage_particles, cudaStream_t st);

}  // namespace gbwake
