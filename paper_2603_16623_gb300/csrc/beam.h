// beam.h -- host launchers of the beam preparation kernels (beam.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbwake {
cudaError_t launch_fold_charge(double* qw, const double* w, double q, int64_t n, cudaStream_t st);
cudaError_t launch_bin_count(const double* xi, int64_t n, double dxi, int32_t n_steps, int32_t* slot,
                             int32_t* cnt, cudaStream_t st);
cudaError_t launch_excl_scan(const int32_t* cnt, int32_t n, int32_t* off, int32_t* max_count, cudaStream_t st);
cudaError_t launch_bin_scatter(const int32_t* slot, int64_t n, int32_t n_steps, const int32_t* off, int32_t* fill,
                               int32_t* binned_idx, cudaStream_t st);
// binning: particles per thread of a block's chunk, and the most slices a
// window may have (the per-block histogram lives in shared memory)
constexpr int kBinPerThread = 16;
constexpr int32_t kBinSmem = 48 * 1024 / 4;
size_t slice_sort_smem(int32_t m_pad);
// the largest slice the per-slice shared-memory sort takes, and the first
// pass's size when the densest slice is not known on the host
constexpr int32_t kSliceSortMaxPad = 8192;
constexpr int32_t kSliceSortFirstPad = 1024;
cudaError_t launch_reset_ctl(int32_t* ctl, cudaStream_t st);
// per-slice radial sort of the binned beam; densest = the particles in the
// densest slice when the host knows them, else -1 (two passes: the slices of
// up to kSliceSortFirstPad particles, then the denser ones); a slice denser
// than kSliceSortMaxPad sets ctl's status to EINVAL
template <class R>
cudaError_t launch_slice_sort(const int32_t* off, int32_t n_steps, const double* r_in, const double* qw_in,
                              int32_t* idx, R* br, R* bE, R* bQs, R* bTot, int32_t densest, int32_t* ctl,
                              int32_t* inv, cudaStream_t st);  // inv (nullable): caller index -> sorted position
template <class R>
cudaError_t launch_scatter_out(const int32_t* idx, const int32_t* nbin, int64_t nb_max, const R* src, R* dst,
                               cudaStream_t st);
// largest radius of each beam species (caller order, species s = particles
// [begin[s], begin[s+1])) into rmax[s], which the caller has zeroed
struct SpeciesRanges {
    int32_t n;
    int64_t begin[9];
};
cudaError_t launch_species_rmax(const double* r, SpeciesRanges sp, double* rmax, cudaStream_t st);
// a fixed grid extent that some species' largest radius reaches: the wake
// stops (ctl status EINVAL, failing slice -1)
cudaError_t launch_grid_extent_check(const double* rmax, int32_t n_species, double grid_rmax, int32_t* ctl,
                                     cudaStream_t st);
}  // namespace gbwake
