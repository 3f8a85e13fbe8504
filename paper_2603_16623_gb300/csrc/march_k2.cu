// march_k2.cu -- the on-chip marches at 2 rings per thread (twice the
// warps of 4 rings per thread for the same rings: a shorter per-thread chain
// per slice), in a translation unit of their own so that they compile in
// parallel with march.cu.
#include "march_launch.cuh"

namespace gbwake {

cudaError_t launch_march_fast_k2(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                 int32_t max_slices, int32_t mode, int32_t threads, int32_t stage_particles,
                                 cudaStream_t st) {
    return launch_fast_k<2>(d_wakes, d_order, n_wakes, max_slices, mode, threads, stage_particles, st);
}

cudaError_t launch_march_cluster_k2(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                    int32_t max_slices, int32_t mode, int32_t threads, int32_t cl,
                                    int32_t stage_particles, cudaStream_t st) {
    return launch_cluster_k<2>(d_wakes, d_order, n_wakes, max_slices, mode, threads, cl, stage_particles, st);
}

int64_t march_k2_bounds_violations() {
#ifdef WAKE_BOUNDS_CHECK
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_violations, sizeof(v)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(g_bounds_violations, &z, sizeof(z)) != cudaSuccess) return -2;
    return (int64_t)v;
#else
    return -1;
#endif
}

}  // namespace gbwake
