// march.h -- host launchers of the ring kernels (march.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "march.cuh"
#include "march_cluster.cuh"
#include "march_fast.cuh"
#include "march_ions.cuh"
#include "march_rk4.cuh"

namespace gbwake {
template <class P>
cudaError_t launch_march(const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes, int32_t max_slices,
                         int32_t mode, int32_t threads, size_t smem, int32_t mb_cap, int32_t cluster_ctas,
                         cudaStream_t st);
// the on-chip march (mixed precision, k_rings = 2, 4 or 8 rings per thread,
// <= 512 threads)
constexpr int kFastMaxThreads = 512;
cudaError_t launch_march_fast(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                              int32_t max_slices, int32_t mode, int32_t threads, int32_t k_rings,
                              int32_t stage_particles, cudaStream_t st);
// particles per slice the on-chip march of `threads` x k_rings stages in
// shared memory (at most `want`, the densest slice of the launch's wakes),
// sized so that the stage never lowers the number of blocks an SM holds
// (clusters > 1: the cluster march's footprint)
int32_t march_stage_particles(int32_t threads, int32_t k_rings, int32_t cluster_ctas, int32_t want);
// the cluster march: clusters of cl CTAs of `threads` threads, k_rings = 2,
// 4 or 8 rings per thread
cudaError_t launch_march_cluster(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                 int32_t max_slices, int32_t mode, int32_t threads, int32_t k_rings, int32_t cl,
                                 int32_t stage_particles, cudaStream_t st);
// debug build (WAKE_BOUNDS_CHECK): out-of-range shared-memory positions and
// DSMEM ranks the on-chip marches met since the last call (march.cu's and
// march_k2.cu's kernels respectively); -1 in other builds, -2 on a CUDA error
int64_t march_bounds_violations();
int64_t march_k2_bounds_violations();
// gathers (next slice, status) of n wakes' control words into out[2n]
cudaError_t launch_gather_ctl(const int32_t* const* ctls, int32_t n, int32_t* out, cudaStream_t st);
// n cells; n_total = n (electrons) or 2 n (electrons, then mobile ions)
// (cell_density: NULL, or n cell densities)
template <class R>
cudaError_t launch_ring_init(const double* edges, const double* cell_density, int32_t n, int32_t n_total,
                             double density, R* w, R* wh, R* rho, R* rho_lo, R* ur, R* frho, R* fur, int32_t* rid,
                             float4* ctab, cudaStream_t st);
// the march with the RK4 ring integrator (march_rk4.cuh), one block per wake
// or a thread-block cluster of cluster_ctas (<= 8) blocks per wake
template <class P>
cudaError_t launch_march_rk4(const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                             int32_t max_slices, int32_t mode, int32_t threads, size_t smem, int32_t mb_cap,
                             int32_t cluster_ctas, cudaStream_t st);
// the march of wakes with mobile ions (march_ions.cuh), one block per wake or
// a thread-block cluster of cluster_ctas (<= 8) blocks per wake
template <class P>
cudaError_t launch_march_ions(const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                              int32_t max_slices, int32_t mode, int32_t threads, size_t smem, int32_t mb_cap,
                              int32_t cluster_ctas, cudaStream_t st);
template <class R>
cudaError_t launch_gather_by_id(const int32_t* rid, const R* src, R* dst, int32_t n, cudaStream_t st);
template <class R>
cudaError_t launch_export_state(const int32_t* rid, const R* rho, const R* rho_lo, const R* ur, const R* frho,
                                const R* fur, int32_t n, const float4* ctab, double* o_rho, double* o_ur,
                                double* o_fr, double* o_fu, cudaStream_t st);
template <class R>
cudaError_t launch_import_state(const double* i_rho, const double* i_ur, const double* i_fr, const double* i_fu,
                                int32_t n, const float4* ctab, R* rho, R* rho_lo, R* ur, R* frho, R* fur,
                                int32_t* rid, int32_t* ctl, int32_t slice, cudaStream_t st);
// shared memory of the march kernel for rings up to n_max with slices up to m_max
// staged; returns the bytes and the staging capacity mb_cap
size_t march_smem(int32_t n_max, int32_t n_pad_max, size_t real_bytes, int32_t m_max, int32_t* mb_cap);
}  // namespace gbwake
