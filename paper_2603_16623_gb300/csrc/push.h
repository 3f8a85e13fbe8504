// push.h -- host launchers of the beam push (push.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbwake {
// one wake of a batched push: particle arrays (caller order), the fields
// of the last march in sorted order and the caller -> sorted map (-1: the
// particle lies outside the window and sees no field)
template <class R>
struct PushWake {
    int64_t n;
    double *x, *y, *xi, *r, *ux, *uy, *uz;
    const R *ez, *wr, *bt;
    const int32_t* inv;
};
// a contiguous particle range [begin, end) of one wake and one species
// (charge q): the unit of work of one CTA of the push (ranges of at most a
// few tens of thousands of particles, so that one launch balances wakes of
// any size)
struct PushItem {
    int32_t wake;
    int32_t pad_;
    int64_t begin, end;
    double q;
};
// one Boris step of every particle of the items' wakes (one launch, one CTA
// per item); updates x, y, xi, u and r = |(x, y)| in place
template <class R>
cudaError_t launch_beam_push(const PushWake<R>* wakes, const PushItem* items, int32_t n_items, double dt,
                             cudaStream_t st);
// particles per item for a launch over `total` particles
int64_t push_item_size(int64_t total);
// r = |(x, y)|
cudaError_t launch_beam_radius(int64_t n, const double* x, const double* y, double* r, cudaStream_t st);
}  // namespace gbwake
