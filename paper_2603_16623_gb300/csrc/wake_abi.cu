// wake_abi.cu -- the C ABI of libwake.so (include/wake.h).
//
// Host side only: argument checks, device allocation owned by the handle,
// kernel launches on the handle's stream, and copies to and from caller
// buffers.  Every step of the solve itself runs in the kernels of march.cu
// and beam.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/wake.h"
#include "beam.h"
#include "march.h"
#include "push.h"

using namespace gbwake;

namespace {

thread_local std::string g_err;

wake_status fail(wake_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define WK_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return fail(WAKE_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),   \
                        __FILE__, __LINE__);                                                   \
    } while (0)

constexpr int32_t kMaxRings = 8192;           // FP64 path (one CTA per wake, sort in shared memory)
constexpr int32_t kMaxIonCells = 4096;        // mobile ions: rings per species (2 x 4096 rings per wake)
// the global-memory marches with mobile ions, RK4 or beam grids on thread-
// block clusters: the automatic cluster's positions per thread (of each
// species with ions), and a cluster's barriers per slice (per stage with
// RK4), us
constexpr int32_t kIonRingsPerThread = 2;
constexpr int32_t kRk4RingsPerThread = 2;
constexpr int32_t kGridRingsPerThread = 4;
constexpr double kGmClusterSliceUs = 20.0;
constexpr int32_t kMaxRingsMixed = 65536;     // mixed path: a 16-CTA cluster of 512 threads x 8 rings
constexpr int32_t kMaxRk4Rings = 16384;       // RK4, beam grids: the sort of one block (8 B per ring)
constexpr int32_t kMaxSliceParticles = 8192;
constexpr int32_t kDefaultThreads = 256;

int32_t next_pow2(int32_t v) {
    int32_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

struct wake_handle {
    int32_t prec = WAKE_FP64;
    int32_t n = 0, n_steps = 0, n_pad = 0, threads = kDefaultThreads, flags = 0;
    int32_t n_ion = 0;                      // > 0: mobile ions, rings per species (n = 2 n_ion)
    int32_t rk4 = 0;                        // the RK4 integrator (march_rk4.cuh)
    int32_t grid_nr = 0;                    // > 0: adaptive beam grids (march.cuh)
    double grid_rmax = 0;                   // > 0: the grids' fixed extent
    double* d_ag_rmax = nullptr;            // largest radius per beam species (grids)
    double ion_qm = 0;                      // their Z / M
    double dxi = 0, density = 1, rho_max = 0;
    cudaStream_t st = nullptr;
    int64_t nb_total = 0;  // beam particles given by the caller
    std::vector<void*> allocs;
    size_t alloc_bytes = 0;                 // device bytes held (wake_get_device_bytes)
    std::vector<int64_t> beam_n;            // particles per species
    std::vector<double> beam_q;             // charge sign per species
    double* d_density = nullptr;            // cell densities (radial profile), or NULL
    double *d_edges = nullptr, *d_xi = nullptr, *d_r = nullptr, *d_w = nullptr, *d_qw = nullptr;
    double* d_ps[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};  // beam x, y, u_x, u_y, u_z (push)
    int32_t *d_slot = nullptr, *d_cnt = nullptr, *d_fill = nullptr, *d_boff = nullptr, *d_dmax = nullptr;
    void* d_desc = nullptr;                 // device WakeDev<P>
    std::vector<unsigned char> desc_host;   // host copy of the descriptor
    int32_t* d_ctl = nullptr;
    int32_t* d_bidx = nullptr;
    int32_t* d_inv = nullptr;               // caller particle -> sorted (binned) position, -1 outside
    void* d_out[4] = {nullptr, nullptr, nullptr, nullptr};
    void* d_dump[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    void* d_rho[2] = {nullptr, nullptr};
    void* d_ur[2] = {nullptr, nullptr};
    int32_t* d_rid[2] = {nullptr, nullptr};
    int32_t fast_threads = 0;               // > 0: the on-chip march serves this wake
    int32_t fast_k = 8;                     // its rings per thread
    int32_t fast_cl = 1;                    // CTAs per wake (thread-block cluster if > 1)
    int32_t gm_cl = 1;                      // mobile ions, RK4: CTAs per wake of their march
    int32_t slice_max = kMaxSliceParticles; // particles in the densest slice (host count), or
                                            // -1: not known on the host (new beams, a push)
    size_t real_bytes() const { return prec == WAKE_FP64 ? 8 : 4; }
};

namespace {

// Device memory of the handles comes from one stream-ordered memory pool per
// device that keeps what is freed (release threshold: unlimited), so that a
// serving loop creating and destroying wakes allocates at pool speed.
cudaError_t wake_pool(cudaMemPool_t* out) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&pools[dev], &props);
        if (e != cudaSuccess) {
            pools[dev] = nullptr;
            return e;
        }
        uint64_t keep = ~0ull;
        e = cudaMemPoolSetAttribute(pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
    }
    *out = pools[dev];
    return cudaSuccess;
}

wake_status dalloc(wake_handle* h, size_t bytes, void** out) {
    void* p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaMemPool_t pool = nullptr;
    cudaError_t e = wake_pool(&pool);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&p, bytes, pool, h->st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(WAKE_ENOMEM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    h->allocs.push_back(p);
    h->alloc_bytes += bytes;
    e = cudaMemsetAsync(p, 0, bytes, h->st);
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
    *out = p;
    return WAKE_OK;
}

template <class T>
wake_status dalloc_t(wake_handle* h, size_t count, T** out) {
    void* p = nullptr;
    wake_status s = dalloc(h, count * sizeof(T), &p);
    *out = static_cast<T*>(p);
    return s;
}

// Returns the handle's memory to the pool, ordered after the work queued on
// its stream (no host synchronisation).
void free_all(wake_handle* h) {
    for (void* p : h->allocs) cudaFreeAsync(p, h->st);
    h->allocs.clear();
    h->alloc_bytes = 0;
}

#define WK_TRY(expr)                      \
    do {                                  \
        wake_status s_ = (expr);          \
        if (s_ != WAKE_OK) return s_;     \
    } while (0)

// Enqueues the a0/a1 preparation of a wake: control words, ring
// initialisation, charge folding, nearest-slice binning and per-slice radial
// sort of the (device-resident) beam, cleared outputs.  Asynchronous.
// Particles in the densest slice [0, n_steps), counted on the host with the
// kernels' nearest-slice rule (the same double division and addition).
int32_t densest_slice(const wake_beam_desc* beams, int32_t n_beams, double dxi, int32_t n_steps) {
    std::vector<int32_t> cnt((size_t)n_steps, 0);
    int32_t mx = 0;
    for (int32_t b = 0; b < n_beams; ++b)
        for (int64_t k = 0; k < beams[b].n; ++k) {
            const double s = std::floor(beams[b].xi[k] / dxi + 0.5);
            if (s >= 0.0 && s < (double)n_steps) mx = std::max(mx, ++cnt[(size_t)s]);
        }
    return mx;
}

// New beam arrays for wake_reset: same species count and sizes as at init,
// inside a fixed grid extent.
wake_status check_new_beams(const wake_handle* h, const wake_beam_desc* beams, int32_t n_beams) {
    if (!beams) return WAKE_OK;
    if (h->grid_rmax > 0.0)
        for (int32_t b = 0; b < n_beams; ++b)
            for (int64_t k = 0; k < beams[b].n && beams[b].r; ++k)
                if (!(beams[b].r[k] < h->grid_rmax))
                    return fail(WAKE_EINVAL, "wake_reset: beam %d particle %lld lies beyond grid_rmax", b,
                                (long long)k);
    if (n_beams != (int32_t)h->beam_n.size())
        return fail(WAKE_EINVAL, "wake_reset: %d species given, %zu at init", n_beams, h->beam_n.size());
    for (int32_t b = 0; b < n_beams; ++b) {
        if (beams[b].n != h->beam_n[b])
            return fail(WAKE_EINVAL, "wake_reset: species %d has %lld particles, %lld at init", b,
                        (long long)beams[b].n, (long long)h->beam_n[b]);
        if (beams[b].n > 0 && (!beams[b].xi || !beams[b].r || !beams[b].w))
            return fail(WAKE_EINVAL, "wake_reset: species %d arrays are NULL", b);
    }
    return WAKE_OK;
}

// Enqueues the host-to-device copies of checked new beam arrays on st.
wake_status upload_beams(wake_handle* h, const wake_beam_desc* beams, int32_t n_beams, cudaStream_t st,
                         bool count_on_host = true) {
    if (!beams) return WAKE_OK;
    h->slice_max = count_on_host ? densest_slice(beams, n_beams, h->dxi, h->n_steps) : -1;
    int64_t off = 0;
    for (int32_t b = 0; b < n_beams; ++b) {
        const size_t bytes = beams[b].n * sizeof(double);
        if (beams[b].n > 0) {
            WK_CUDA(cudaMemcpyAsync(h->d_xi + off, beams[b].xi, bytes, cudaMemcpyHostToDevice, st));
            WK_CUDA(cudaMemcpyAsync(h->d_r + off, beams[b].r, bytes, cudaMemcpyHostToDevice, st));
            WK_CUDA(cudaMemcpyAsync(h->d_w + off, beams[b].w, bytes, cudaMemcpyHostToDevice, st));
        }
        h->beam_q[b] = beams[b].q;
        off += beams[b].n;
    }
    return WAKE_OK;
}

template <class P>
wake_status prepare_sort(wake_handle* h, cudaStream_t st);

// The a0/a1 preparation: control words, rings, charge, slice histogram and
// offsets (whose maximum lands in d_dmax), then prepare_sort.
template <class P>
wake_status prepare_impl(wake_handle* h, cudaStream_t st) {
    using R = typename P::R;
    WakeDev<P> D;
    std::memcpy(&D, h->desc_host.data(), sizeof(D));
    const int32_t n = h->n, ns = h->n_steps;
    WK_CUDA(launch_reset_ctl(h->d_ctl, st));
    WK_CUDA(launch_ring_init<R>(h->d_edges, h->d_density, h->n_ion ? h->n_ion : n, n, h->density, const_cast<R*>(D.w),
                                const_cast<R*>(D.wh), D.rho[0],
                                D.rho_lo, D.ur[0], D.frho[0], D.fur[0], D.rid[0], const_cast<float4*>(D.ctab),
                                st));
    const size_t rb = h->real_bytes();
    WK_CUDA(cudaMemsetAsync(h->d_boff, 0, ((size_t)ns + 1) * sizeof(int32_t), st));
    WK_CUDA(cudaMemsetAsync(const_cast<R*>(D.bTot), 0, (size_t)ns * rb, st));
    if (h->nb_total > 0) {
        int64_t off = 0;
        for (size_t b = 0; b < h->beam_n.size(); ++b) {
            WK_CUDA(launch_fold_charge(h->d_qw + off, h->d_w + off, h->beam_q[b], h->beam_n[b], st));
            off += h->beam_n[b];
        }
        WK_CUDA(cudaMemsetAsync(h->d_cnt, 0, (size_t)ns * sizeof(int32_t), st));
        WK_CUDA(cudaMemsetAsync(h->d_fill, 0, (size_t)ns * sizeof(int32_t), st));
        WK_CUDA(launch_bin_count(h->d_xi, h->nb_total, h->dxi, ns, h->d_slot, h->d_cnt, st));
        if (h->grid_nr > 0) {  // the grids' extents from the beam as it is now
            SpeciesRanges sp = {};
            sp.n = (int32_t)h->beam_n.size();
            for (int32_t b = 0; b < sp.n; ++b) sp.begin[b + 1] = sp.begin[b] + h->beam_n[b];
            WK_CUDA(cudaMemsetAsync(h->d_ag_rmax, 0, (size_t)sp.n * sizeof(double), st));
            WK_CUDA(launch_species_rmax(h->d_r, sp, h->d_ag_rmax, st));
            if (h->grid_rmax > 0.0) WK_CUDA(launch_grid_extent_check(h->d_ag_rmax, sp.n, h->grid_rmax, h->d_ctl, st));
        }
        WK_CUDA(launch_excl_scan(h->d_cnt, ns, h->d_boff, h->d_dmax, st));
    }
    return prepare_sort<P>(h, st);
}

// Second part of the a1 preparation: scatter into slices and the per-slice
// radial sort (sized by h->slice_max when the host knows it, else in two
// passes sized on the device); cleared outputs and dumps.
template <class P>
wake_status prepare_sort(wake_handle* h, cudaStream_t st) {
    using R = typename P::R;
    WakeDev<P> D;
    std::memcpy(&D, h->desc_host.data(), sizeof(D));
    const int32_t n = h->n, ns = h->n_steps;
    const size_t rb = h->real_bytes();
    if (h->nb_total > 0) {
        WK_CUDA(launch_bin_scatter(h->d_slot, h->nb_total, ns, h->d_boff, h->d_fill, h->d_bidx, st));
        // (a slice beyond kMaxSliceParticles is flagged by the kernel)
        const int32_t densest = h->slice_max > kMaxSliceParticles ? kMaxSliceParticles : h->slice_max;
        WK_CUDA(cudaMemsetAsync(h->d_inv, 0xff, (size_t)h->nb_total * sizeof(int32_t), st));
        WK_CUDA(launch_slice_sort<R>(h->d_boff, ns, h->d_r, h->d_qw, h->d_bidx, const_cast<R*>(D.br),
                                     const_cast<R*>(D.bE), const_cast<R*>(D.bQs), const_cast<R*>(D.bTot),
                                     densest, h->d_ctl, h->d_inv, st));
        for (int k = 0; k < 4; ++k)
            WK_CUDA(cudaMemsetAsync(h->d_out[k], 0, (size_t)h->nb_total * rb, st));
    }
    for (int k = 0; k < 7; ++k)
        if (h->d_dump[k]) WK_CUDA(cudaMemsetAsync(h->d_dump[k], 0, (size_t)ns * n * rb, st));
    return WAKE_OK;
}

template <class P>
wake_status init_impl(wake_handle* h, const wake_config* cfg, const wake_plasma_desc* plasma,
                      const wake_beam_desc* beams, int32_t n_beams) {
    using R = typename P::R;
    using A = typename P::A;
    (void)cfg;
    const int32_t n = h->n;
    const int32_t ns = h->n_steps;
    WakeDev<P> D;
    std::memset(&D, 0, sizeof(D));
    D.n = n;
    D.n_steps = ns;
    D.n_pad = h->n_pad;
    D.dxi = h->dxi;
    D.density = h->density;
    D.rho_max = h->rho_max;
    D.n_ion = h->n_ion;
    D.ion_qm = h->ion_qm;

    // plasma column and ring state
    const int32_t n_cells = h->n_ion ? h->n_ion : n;
    WK_TRY(dalloc_t(h, (size_t)n_cells + 1, &h->d_edges));
    WK_CUDA(cudaMemcpyAsync(h->d_edges, plasma->r_edges, ((size_t)n_cells + 1) * sizeof(double),
                            cudaMemcpyHostToDevice, h->st));
    if (plasma->cell_density) {
        WK_TRY(dalloc_t(h, (size_t)n_cells, &h->d_density));
        WK_CUDA(cudaMemcpyAsync(h->d_density, plasma->cell_density, (size_t)n_cells * sizeof(double),
                                cudaMemcpyHostToDevice, h->st));
    }
    R *w, *wh;
    WK_TRY(dalloc_t(h, n, &w));
    WK_TRY(dalloc_t(h, n, &wh));
    D.w = w;
    D.wh = wh;
    for (int b = 0; b < 2; ++b) {
        WK_TRY(dalloc_t(h, n, &D.rho[b]));
        WK_TRY(dalloc_t(h, n, &D.ur[b]));
        WK_TRY(dalloc_t(h, n, &D.frho[b]));
        WK_TRY(dalloc_t(h, n, &D.fur[b]));
        WK_TRY(dalloc_t(h, n, &D.rid[b]));
        h->d_rho[b] = D.rho[b];
        h->d_ur[b] = D.ur[b];
        h->d_rid[b] = D.rid[b];
    }
    WK_TRY(dalloc_t(h, n, &D.rho_lo));
    if (h->prec == WAKE_MIXED) {  // every mixed march takes its constants from the table
        float4* ct;
        WK_TRY(dalloc_t(h, (size_t)3 * n, &ct));
        D.ctab = ct;
    }
    R** scratch[] = {&D.bb, &D.psib, &D.gam, &D.dpr, &D.tt, &D.cA, &D.cB, &D.cC};
    for (R** sp : scratch) WK_TRY(dalloc_t(h, n, sp));
    if (h->rk4) {
        R** rk[] = {&D.rk_r, &D.rk_rlo, &D.rk_u, &D.rk_sg, &D.rk_kr, &D.rk_ku};
        for (R** sp : rk) WK_TRY(dalloc_t(h, n, sp));
        WK_TRY(dalloc_t(h, n, &D.rk_perm));
    }
    if (h->n_ion) {
        WK_TRY(dalloc_t(h, n, &D.psio));
        WK_TRY(dalloc_t(h, n, &D.dpro));
        WK_TRY(dalloc_t(h, n, &D.dpzo));
    }
    // regions: n + 1 (one species), or n_ion + 1 per species
    WK_TRY(dalloc_t(h, (size_t)n + 2, &D.regS));
    WK_TRY(dalloc_t(h, (size_t)n + 2, &D.regL));
    R** regions[] = {&D.regT, &D.ak, &D.bk, &D.Ra, &D.Rb, &D.Da, &D.Db};
    for (R** sp : regions) WK_TRY(dalloc_t(h, (size_t)n + 2, sp));
    WK_TRY(dalloc_t(h, CTL_N, &D.ctl));
    h->d_ctl = D.ctl;

    // beam: device-resident raw inputs, binned arrays, outputs
    int64_t nb = 0;
    for (int32_t b = 0; b < n_beams; ++b) {
        h->beam_n.push_back(beams[b].n);
        h->beam_q.push_back(beams[b].q);
        nb += beams[b].n;
    }
    h->nb_total = nb;
    WK_TRY(dalloc_t(h, (size_t)ns + 1, &h->d_boff));
    D.boff = h->d_boff;
    R *bTot, *br, *bE, *bQs;
    WK_TRY(dalloc_t(h, (size_t)ns, &bTot));
    // 4 elements of padding: a bulk copy of a slice may read up to 3 past
    // the last particle (its span is rounded out to 16 bytes)
    WK_TRY(dalloc_t(h, (size_t)nb + 4, &br));
    WK_TRY(dalloc_t(h, (size_t)nb + 4, &bE));
    WK_TRY(dalloc_t(h, (size_t)nb + 4, &bQs));
    D.bTot = bTot;
    D.br = br;
    D.bE = bE;
    D.bQs = bQs;
    auto aligned16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    D.stage = (aligned16(br) && aligned16(bE) && aligned16(bQs) && !(h->flags & WAKE_NO_STAGE)) ? STAGE_OK : 0;
    if (h->flags & WAKE_TEST_STALL_STAGE) D.stage |= STAGE_TEST_STALL;
    if (nb > 0) {
        WK_TRY(dalloc_t(h, (size_t)nb, &h->d_xi));
        WK_TRY(dalloc_t(h, (size_t)nb, &h->d_r));
        WK_TRY(dalloc_t(h, (size_t)nb, &h->d_w));
        WK_TRY(dalloc_t(h, (size_t)nb, &h->d_qw));
        WK_TRY(dalloc_t(h, (size_t)nb, &h->d_slot));
        WK_TRY(dalloc_t(h, (size_t)nb, &h->d_bidx));
        WK_TRY(dalloc_t(h, (size_t)nb, &h->d_inv));
        WK_TRY(dalloc_t(h, (size_t)ns, &h->d_cnt));
        WK_TRY(dalloc_t(h, (size_t)ns, &h->d_fill));
        WK_TRY(dalloc_t(h, 1, &h->d_dmax));
        int64_t off = 0;
        for (int32_t b = 0; b < n_beams; ++b) {
            size_t bytes = beams[b].n * sizeof(double);
            if (beams[b].n == 0) continue;
            WK_CUDA(cudaMemcpyAsync(h->d_xi + off, beams[b].xi, bytes, cudaMemcpyHostToDevice, h->st));
            WK_CUDA(cudaMemcpyAsync(h->d_r + off, beams[b].r, bytes, cudaMemcpyHostToDevice, h->st));
            WK_CUDA(cudaMemcpyAsync(h->d_w + off, beams[b].w, bytes, cudaMemcpyHostToDevice, h->st));
            off += beams[b].n;
        }
    }
    D.nb = nb;
    for (int k = 0; k < 4; ++k) {
        R* o;
        WK_TRY(dalloc_t(h, (size_t)nb, &o));
        h->d_out[k] = o;
    }
    if (h->grid_nr > 0) {
        D.grid_nr = h->grid_nr;
        D.grid_rmax = h->grid_rmax;
        D.n_species = (int32_t)h->beam_n.size();
        int64_t off = 0;
        for (int32_t b = 0; b < D.n_species; ++b) {
            D.sp_begin[b] = off;
            off += h->beam_n[b];
        }
        D.sp_begin[D.n_species] = off;
        if (D.n_species == 0) D.n_species = 1;  // no beam: one empty grid
        D.bidx = h->d_bidx;
        D.qw = h->d_qw;
        D.rc = h->d_r;
        WK_TRY(dalloc_t(h, (size_t)D.n_species, &h->d_ag_rmax));
        D.ag_rmax = h->d_ag_rmax;
        WK_TRY(dalloc_t(h, (size_t)D.n_species * (h->grid_nr + 1), &D.agB));
        WK_TRY(dalloc_t(h, (size_t)D.n_species * (h->grid_nr + 1) * 4, &D.agF));
    }
    D.out_ez = (R*)h->d_out[0];
    D.out_wr = (R*)h->d_out[1];
    D.out_bt = (R*)h->d_out[2];
    D.out_psi = (R*)h->d_out[3];
    const size_t dump_n = (size_t)ns * n;
    if (h->flags & (WAKE_DUMP_RING_R | WAKE_DUMP_RING_FIELDS)) {
        WK_TRY(dalloc_t(h, dump_n, &D.dump_r));
        h->d_dump[0] = D.dump_r;
    }
    if (h->flags & WAKE_DUMP_RING_FIELDS) {
        R** dumps[] = {&D.dump_ur, &D.dump_psi, &D.dump_dpr, &D.dump_dpz, &D.dump_bp, &D.dump_bb};
        for (int k = 0; k < 6; ++k) {
            WK_TRY(dalloc_t(h, dump_n, dumps[k]));
            h->d_dump[k + 1] = *dumps[k];
        }
    }
    (void)sizeof(A);
    h->desc_host.resize(sizeof(D));
    std::memcpy(h->desc_host.data(), &D, sizeof(D));
    WK_TRY(dalloc(h, sizeof(D), &h->d_desc));
    WK_CUDA(cudaMemcpyAsync(h->d_desc, &D, sizeof(D), cudaMemcpyHostToDevice, h->st));
    WK_TRY(prepare_impl<P>(h, h->st));
    if (h->flags & WAKE_INIT_ASYNC) return WAKE_OK;  // a dense slice shows in wake_get_progress
    int32_t ctl[CTL_N];
    WK_CUDA(cudaMemcpyAsync(ctl, h->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->st));
    WK_CUDA(cudaStreamSynchronize(h->st));
    if (ctl[CTL_STATUS] == WAKE_EINVAL)
        return fail(WAKE_EINVAL, "slice %d holds more than %d beam particles; use a smaller dxi", ctl[CTL_FAIL],
                    kMaxSliceParticles);
    return WAKE_OK;
}

// The on-chip march (mixed precision).  Automatic shape: one CTA of up to
// 512 threads x 2 rings for wakes up to 1024 rings, of up to 512 threads x 4
// rings up to 2048 rings; up to 16,384 rings a
// thread-block cluster of ceil(n / 1024) CTAs; up to 32,768 one of
// ceil(n / 2048) CTAs (16 is the largest cluster GB300 allows); beyond, 8
// rings per thread.  A caller (or the autotuner) may instead fix the rings per thread
// (2, 4 or 8) and the CTAs per wake; the threads per CTA then follow from n.
constexpr int32_t kRingsPerCta = 4 * kFastMaxThreads;
constexpr int32_t kMaxClusterCtas = 16;

struct FastShape {
    int32_t threads = 0, k = 4, cl = 1;  // threads == 0: not served by the on-chip march
};

wake_status fast_shape_for(int32_t prec, int32_t n, int32_t want_k, int32_t want_cl, FastShape* out) {
    FastShape f;
    if (prec != WAKE_MIXED) {
        if (want_k || want_cl)
            return fail(WAKE_EINVAL, "wake_init: rings_per_thread and cluster_ctas apply to WAKE_MIXED only");
        *out = f;
        return WAKE_OK;
    }
    if (want_k != 0 && want_k != 2 && want_k != 4 && want_k != 8)
        return fail(WAKE_EINVAL, "wake_init: rings_per_thread must be 0, 2, 4 or 8");
    if (want_cl < 0 || want_cl > kMaxClusterCtas)
        return fail(WAKE_EINVAL, "wake_init: cluster_ctas must be in [0, %d]", kMaxClusterCtas);
    // automatic: one CTA up to 2048 rings; beyond, clusters of CTAs of at
    // most 1024 rings (<= 256 threads x 4, two such CTAs fit an SM's
    // registers: a shorter per-slice chain for the same SM time, measured on
    // the batched workload), then of 2048 rings, then 8 rings per thread (up
    // to 16 x 512 x 8 = 65,536 rings)
    if (want_k || want_cl) {
        f.k = want_k ? want_k : 4;
        f.cl = want_cl ? want_cl : (n + f.k * kFastMaxThreads - 1) / (f.k * kFastMaxThreads);
    } else if (n <= 2 * kFastMaxThreads) {
        // up to 1024 rings: one CTA at 2 rings per thread (measured on GB300
        // against 4 per thread: 200 rings 10.4 -> 7.3 us per slice alone, 512
        // rings 10.4 -> 7.9, 1024 rings 11.5 -> 10.1; packed at its capacity
        // 14-19 % more ring-slices/s; the 256-wake step unchanged)
        f.k = 2;
        f.cl = 1;
    } else if (n <= kRingsPerCta) {
        f.k = 4;
        f.cl = 1;
    } else if (n <= kMaxClusterCtas * kRingsPerCta / 2) {
        f.k = 4;
        f.cl = (n + kRingsPerCta / 2 - 1) / (kRingsPerCta / 2);
    } else {
        f.k = n <= kMaxClusterCtas * kRingsPerCta ? 4 : 8;
        f.cl = (n + f.k * kFastMaxThreads - 1) / (f.k * kFastMaxThreads);
    }
    if (f.cl > kMaxClusterCtas) {
        if (want_k || want_cl)
            return fail(WAKE_EINVAL, "wake_init: %d rings need more than %d CTAs of %d x %d rings", n, kMaxClusterCtas,
                        kFastMaxThreads, f.k);
        *out = FastShape{};  // automatic: beyond the on-chip march
        return WAKE_OK;
    }
    const int32_t per_cta = (n + f.cl - 1) / f.cl;
    int32_t t = (per_cta + f.k - 1) / f.k;
    t = ((t + 31) / 32) * 32;
    f.threads = t < 32 ? 32 : t;
    if (f.threads > kFastMaxThreads)
        return fail(WAKE_EINVAL, "wake_init: %d rings do not fit %d CTA(s) of %d threads x %d rings", n, f.cl,
                    kFastMaxThreads, f.k);
    if (f.cl > 1 && (int64_t)f.threads * f.k * (f.cl - 1) >= n)
        return fail(WAKE_EINVAL, "wake_init: %d rings leave the last of %d CTAs empty", n, f.cl);
    *out = f;
    return WAKE_OK;
}

// The latency shape of an automatic-shape wake: 2 rings per thread, which
// halves each thread's chain of per-ring work in every slice (measured on
// GB300, one wake alone: 8000 rings 27.8 -> 21.0 us per slice, 4000 rings
// 29.4 -> 19.2, 1000 rings 17.5 -> 15.3), at ~1.3x the SM time per slice of
// the batch shape (fast_shape_for).  Up to 1024 rings one CTA; up to 8192 a
// cluster of CTAs of at most 256 threads x 2 rings (two CTAs share an SM);
// up to 16,384 CTAs of 512 threads x 2 rings; beyond, the batch shape.
FastShape latency_shape_for(int32_t n, const FastShape& batch) {
    if (batch.threads == 0 || n > kMaxClusterCtas * 2 * kFastMaxThreads) return batch;
    FastShape f;
    f.k = 2;
    if (n <= 2 * kFastMaxThreads) f.cl = 1;
    else if (n <= kMaxClusterCtas * 512) f.cl = (n + 511) / 512;
    else f.cl = (n + 2 * kFastMaxThreads - 1) / (2 * kFastMaxThreads);
    const int32_t per_cta = (n + f.cl - 1) / f.cl;
    const int32_t t = ((per_cta + 1) / 2 + 31) / 32 * 32;
    f.threads = t < 32 ? 32 : t;
    return f;  // (2 t (cl - 1) <= 512 (cl - 1) < n, resp. 1024 (cl - 1) < n: no CTA is empty)
}

double predicted_fast_slice_us(const FastShape& f);

// Automatic-shape wakes whose predicted march time on the batch shape is at
// least this many milliseconds take their latency shape (process-wide).
// Off by default: in a full batch the latency shape's larger clusters wait
// for room in one GPC while the rest of the batch holds the SMs, and on the
// batched wakes (dense beams, rings crossing CTA boundaries) it gains less
// than alone on uniform wakes (256-wake step: 9 long wakes on it 358-366 ms
// against 273-283 ms; the longest wake alone 183 against 201 ms).
double g_latency_shape_ms = INFINITY;

// The shape wake_init gives a wake of n rings and n_steps slices: the
// caller's, else the batch shape, or the latency shape for a long wake.
wake_status wake_shape_for(int32_t prec, int32_t n, int32_t n_steps, int32_t want_k, int32_t want_cl,
                           FastShape* out) {
    WK_TRY(fast_shape_for(prec, n, want_k, want_cl, out));
    if (want_k || want_cl || out->threads == 0) return WAKE_OK;
    if ((double)n_steps * predicted_fast_slice_us(*out) * 1e-3 >= g_latency_shape_ms)
        *out = latency_shape_for(n, *out);
    return WAKE_OK;
}

// Auxiliary streams for concurrent batched launches, kStreamsPerLevel per
// priority level: level 0 gets the device's greatest priority, the last
// level its least, the levels between are spread over the range.  Level 0
// runs the preparations (short kernels that every march waits for: a
// preparation that waited behind pending march blocks would hold back its
// wake's march); levels 1.. the marches by tier, so that when the SMs are
// full the pending blocks of the longest wakes are dispatched first.  Each
// launch group of a tier needs a stream of its own: two launches on one
// stream run one after the other, so a group queued behind a long one
// would start only when that one ends (with 16 streams per level the
// 256-wake batch's 25 tier-1 groups did exactly that).
constexpr int kPrioLevels = 4, kStreamsPerLevel = 128, kAuxStreams = kPrioLevels * kStreamsPerLevel;
constexpr int kTiers = kPrioLevels - 1;
cudaError_t level_stream(int level, int i, cudaStream_t* out) {
    static cudaStream_t pool[kAuxStreams] = {nullptr};
    static int pool_dev[kAuxStreams];
    static std::mutex mu;
    const int slot = level * kStreamsPerLevel + i % kStreamsPerLevel;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(mu);
    if (pool[slot] && pool_dev[slot] != dev) {
        // created for another device: make a new one on the current device
        pool[slot] = nullptr;
    }
    if (!pool[slot]) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e != cudaSuccess) return e;
        // greatest is the numerically lowest value
        const int prio = greatest + (least - greatest) * level / (kPrioLevels - 1);
        e = cudaStreamCreateWithPriority(&pool[slot], cudaStreamNonBlocking, prio);
        if (e != cudaSuccess) {
            pool[slot] = nullptr;
            return e;
        }
        pool_dev[slot] = dev;
    }
    *out = pool[slot];
    return cudaSuccess;
}
// the preparation streams
cudaError_t aux_stream(int i, cudaStream_t* out) { return level_stream(0, i, out); }
// the march streams of a tier
cudaError_t tier_stream(int tier, int i, cudaStream_t* out) { return level_stream(1 + tier, i, out); }

// The two-species march keeps the per-ring values only their own thread
// reads (kOwnArrays in march_ions.cuh, and ln rho) in shared
// memory after its sort and staging region when the launch has room for
// them: their bytes for this wake's block, and the launch's dynamic shared
// memory with them added if that stays within a block's limit (else the
// kernel keeps them in global memory).
size_t ion_own_bytes(const wake_handle* h) {
    const int64_t per_block = (int64_t)h->threads * h->gm_cl;
    const int64_t k = (h->n_ion + per_block - 1) / per_block;
    // (and ln rho in the accumulator type: 8 bytes, a float-float or a double)
    return ((size_t)kOwnArrays * h->real_bytes() + 8) * 2 * (size_t)h->threads * (size_t)k;
}
size_t with_ion_own(size_t smem, size_t own) {
    constexpr size_t kBlockSmemMax = 227 * 1024 - 4096;  // the opt-in limit less the static shared memory
    return smem + own <= kBlockSmemMax ? smem + own : smem;
}

// Particles per slice the march should be able to stage for this wake: its
// densest slice, or the most the library accepts when that is not known.
int32_t stage_want(const wake_handle* h) { return h->slice_max < 0 ? kMaxSliceParticles : h->slice_max; }

template <class P>
wake_status launch_one(wake_handle* h, const WakeDev<P>* d_desc, int32_t max_slices, int32_t mode) {
    if constexpr (std::is_same<P, PrecMixed>::value) {
        const int32_t t = h->fast_threads, k = h->fast_k, cl = h->fast_cl;
        if (t > 0) {
            const int32_t stage = march_stage_particles(t, k, cl, stage_want(h));
            if (cl > 1) WK_CUDA(launch_march_cluster(d_desc, nullptr, 1, max_slices, mode, t, k, cl, stage, h->st));
            else WK_CUDA(launch_march_fast(d_desc, nullptr, 1, max_slices, mode, t, k, stage, h->st));
            return WAKE_OK;
        }
    }
    int32_t mb_cap = 0;
    size_t smem = march_smem(h->n, h->n_pad, h->real_bytes(), kMaxSliceParticles, &mb_cap);
    if (h->n_ion) {
        smem = with_ion_own(smem, ion_own_bytes(h));
        WK_CUDA(launch_march_ions<P>(d_desc, nullptr, 1, max_slices, mode, h->threads, smem, mb_cap, h->gm_cl,
                                     h->st));
        return WAKE_OK;
    }
    if (h->rk4) {
        WK_CUDA(launch_march_rk4<P>(d_desc, nullptr, 1, max_slices, mode, h->threads, smem, mb_cap, h->gm_cl,
                                    h->st));
        return WAKE_OK;
    }
    WK_CUDA(launch_march<P>(d_desc, nullptr, 1, max_slices, mode, h->threads, smem, mb_cap, h->gm_cl, h->st));
    return WAKE_OK;
}

wake_status check_handle(const wake_handle* h) {
    if (!h) return fail(WAKE_EINVAL, "null handle");
    return WAKE_OK;
}

// The status of a stopped wake as an error of entry point `what`.
wake_status stopped(int32_t status, const char* what) {
    if (status == WAKE_ETIMEOUT)
        return fail(WAKE_ETIMEOUT, "%s: the wake stopped: a bounded device wait for a staged beam slice gave up",
                    what);
    if (status == WAKE_EINVAL)
        return fail(WAKE_EINVAL, "%s: the wake stopped: a slice is denser than the library accepts", what);
    return fail(WAKE_ENONFINITE, "%s: the wake stopped at a non-finite slice", what);
}

template <class P>
wake_status fields_at_impl(wake_handle* h, int64_t n, const double* r, void* ez, void* wr, void* bt, void* psi,
                           int32_t device_ptrs) {
    using R = typename P::R;
    if (n == 0) return WAKE_OK;
    WakeDev<P> D;
    std::memcpy(&D, h->desc_host.data(), sizeof(D));
    void* outs_user[4] = {ez, wr, bt, psi};
    std::vector<void*> tmp;
    auto cleanup = [&]() {
        cudaStreamSynchronize(h->st);
        for (void* p : tmp) cudaFree(p);
    };
    double* d_r = nullptr;
    if (device_ptrs) {
        d_r = const_cast<double*>(r);
    } else {
        if (cudaMalloc(&d_r, n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail(WAKE_ENOMEM, "query staging allocation failed");
        }
        tmp.push_back(d_r);
        cudaMemcpyAsync(d_r, r, n * sizeof(double), cudaMemcpyHostToDevice, h->st);
    }
    R* d_out[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k) {
        if (!outs_user[k]) continue;
        if (device_ptrs) {
            d_out[k] = static_cast<R*>(outs_user[k]);
        } else {
            if (cudaMalloc(&d_out[k], n * sizeof(R)) != cudaSuccess) {
                cudaGetLastError();
                cleanup();
                return fail(WAKE_ENOMEM, "query output allocation failed");
            }
            tmp.push_back(d_out[k]);
        }
    }
    D.nq = n;
    D.rq = d_r;
    D.q_ez = d_out[0];
    D.q_wr = d_out[1];
    D.q_bt = d_out[2];
    D.q_psi = d_out[3];
    void* d_desc = nullptr;
    if (cudaMalloc(&d_desc, sizeof(D)) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(WAKE_ENOMEM, "query descriptor allocation failed");
    }
    tmp.push_back(d_desc);
    cudaMemcpyAsync(d_desc, &D, sizeof(D), cudaMemcpyHostToDevice, h->st);
    wake_status s = launch_one<P>(h, static_cast<const WakeDev<P>*>(d_desc), 1, MODE_QUERY);
    if (s == WAKE_OK && !device_ptrs) {
        for (int k = 0; k < 4; ++k)
            if (outs_user[k])
                cudaMemcpyAsync(outs_user[k], d_out[k], n * sizeof(R), cudaMemcpyDeviceToHost, h->st);
    }
    cudaError_t e = cudaStreamSynchronize(h->st);
    cleanup();
    if (s != WAKE_OK) return s;
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "wake_fields_at: %s", cudaGetErrorString(e));
    return WAKE_OK;
}

// Enqueues the fields on the beam particles, in the caller's particle order,
// into caller arrays (device, or host through a staging buffer from the
// library's pool); no synchronisation.
template <class R>
wake_status beam_fields_enqueue(wake_handle* h, void* const outs_user[4], int32_t device_ptrs) {
    const int64_t nb = h->nb_total;
    if (nb == 0) return WAKE_OK;
    R* tmp = nullptr;
    if (!device_ptrs) {
        cudaMemPool_t pool = nullptr;
        cudaError_t e = wake_pool(&pool);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&tmp), nb * sizeof(R), pool, h->st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(WAKE_ENOMEM, "beam output staging allocation failed");
        }
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 4 && e == cudaSuccess; ++k) {
        if (!outs_user[k]) continue;
        R* dst = device_ptrs ? static_cast<R*>(outs_user[k]) : tmp;
        e = cudaMemsetAsync(dst, 0, nb * sizeof(R), h->st);
        if (e == cudaSuccess)
            e = launch_scatter_out<R>(h->d_bidx, h->d_boff + h->n_steps, nb, static_cast<const R*>(h->d_out[k]),
                                      dst, h->st);
        if (e == cudaSuccess && !device_ptrs)
            e = cudaMemcpyAsync(outs_user[k], tmp, nb * sizeof(R), cudaMemcpyDeviceToHost, h->st);
    }
    if (tmp) cudaFreeAsync(tmp, h->st);
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "wake_get_beam_fields: %s", cudaGetErrorString(e));
    return WAKE_OK;
}

template <class R>
wake_status beam_fields_impl(wake_handle* h, void* const outs_user[4], int32_t device_ptrs) {
    WK_TRY(beam_fields_enqueue<R>(h, outs_user, device_ptrs));
    if (!device_ptrs) WK_CUDA(cudaStreamSynchronize(h->st));
    return WAKE_OK;
}

double predicted_ms(const wake_handle* h);

// the on-chip shape of a wake (threads 0: a one-CTA kernel)
FastShape wake_shape(const wake_handle* h) {
    FastShape f;
    f.threads = h->fast_threads;
    f.k = h->fast_k;
    f.cl = h->fast_cl;
    return f;
}

template <class P>
wake_status batch_bucket(const std::vector<wake_handle*>& hs, const FastShape& shape, cudaStream_t st,
                         int32_t max_slices, int64_t budget_ns) {
    const int32_t fast_threads = shape.threads;
    const int32_t n = (int32_t)hs.size();
    std::vector<WakeDev<P>> descs(n);
    std::vector<int32_t> order(n);
    int32_t n_max = 0, pad_max = 0;
    for (int32_t i = 0; i < n; ++i) {
        std::memcpy(&descs[i], hs[i]->desc_host.data(), sizeof(WakeDev<P>));
        descs[i].budget_ns = budget_ns;
        order[i] = i;
        n_max = std::max(n_max, hs[i]->n);
        pad_max = std::max(pad_max, hs[i]->n_pad);
    }
    // longest predicted march first: blocks are dispatched roughly in index order
    std::vector<double> t_pred(n);
    for (int32_t i = 0; i < n; ++i) t_pred[i] = predicted_ms(hs[i]);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return t_pred[a] > t_pred[b]; });
    const size_t desc_bytes = sizeof(WakeDev<P>) * (size_t)n;
    void* d_buf = nullptr;
    WK_CUDA(cudaMallocAsync(&d_buf, desc_bytes + sizeof(int32_t) * (size_t)n, st));
    WK_CUDA(cudaMemcpyAsync(d_buf, descs.data(), desc_bytes, cudaMemcpyHostToDevice, st));
    int32_t* d_order = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(d_buf) + desc_bytes);
    WK_CUDA(cudaMemcpyAsync(d_order, order.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st));
    cudaError_t e;
    if constexpr (std::is_same<P, PrecMixed>::value) {
        if (fast_threads > 0) {
            int32_t densest = 0;
            for (const wake_handle* h : hs) densest = std::max(densest, stage_want(h));
            const int32_t stage = march_stage_particles(fast_threads, shape.k, shape.cl, densest);
            if (shape.cl > 1)
                e = launch_march_cluster(static_cast<const WakeDev<P>*>(d_buf), d_order, n, max_slices, MODE_MARCH,
                                         fast_threads, shape.k, shape.cl, stage, st);
            else
                e = launch_march_fast(static_cast<const WakeDev<P>*>(d_buf), d_order, n, max_slices, MODE_MARCH,
                                      fast_threads, shape.k, stage, st);
            cudaFreeAsync(d_buf, st);
            if (e != cudaSuccess) return fail(WAKE_ECUDA, "batched march launch failed: %s", cudaGetErrorString(e));
            return WAKE_OK;
        }
    }
    int32_t mb_cap = 0;
    size_t smem = march_smem(n_max, pad_max, hs[0]->real_bytes(), kMaxSliceParticles, &mb_cap);
    if (hs[0]->n_ion) {
        size_t own = 0;
        for (const wake_handle* h : hs) own = std::max(own, ion_own_bytes(h));
        smem = with_ion_own(smem, own);
    }
    if (hs[0]->n_ion)
        e = launch_march_ions<P>(static_cast<const WakeDev<P>*>(d_buf), d_order, n, max_slices, MODE_MARCH,
                                 hs[0]->threads, smem, mb_cap, hs[0]->gm_cl, st);
    else if (hs[0]->rk4)
        e = launch_march_rk4<P>(static_cast<const WakeDev<P>*>(d_buf), d_order, n, max_slices, MODE_MARCH,
                                hs[0]->threads, smem, mb_cap, hs[0]->gm_cl, st);
    else
        e = launch_march<P>(static_cast<const WakeDev<P>*>(d_buf), d_order, n, max_slices, MODE_MARCH,
                            hs[0]->threads, smem, mb_cap, hs[0]->gm_cl, st);
    cudaFreeAsync(d_buf, st);
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "batched march launch failed: %s", cudaGetErrorString(e));
    return WAKE_OK;
}

// Predicted march time per slice, in microseconds, on GB300, of the
// on-chip march in shape f (threads > 0) or of a one-CTA kernel in blocks of
// `threads` (per_thread rings each); the batch's plan only needs it to rank
// wakes, wake_init to compare a wake with the latency-shape threshold.
// Fitted to march times measured one wake at a time (wake_get_march_times):
// at 4 rings per thread one CTA of R rings ~ 11 + 9 R/2048 us per slice and
// a cluster of cl CTAs of R rings each ~ 16.3 + 1.6 cl + 8.9 R/1024 us (its
// cluster barriers and exchanges), on the batched wakes; at 2 rings per
// thread, from uniform wakes scaled by the batched wakes' 1.2x, one CTA
// ~ 0.875 of the 4-ring time and a cluster ~ 17.8 + 0.26 cl + 6.4 R/1024 us.
// The one-CTA kernels with state in global memory grow with the rings per
// thread.
double predicted_fast_slice_us(const FastShape& f) {
    const double R = (double)f.threads * f.k;
    if (f.k == 2) return f.cl > 1 ? 17.8 + 0.26 * f.cl + 6.4 * R / 1024.0 : 0.875 * (11.0 + 9.0 * R / 2048.0);
    if (f.cl > 1) return 16.3 + 1.6 * f.cl + 8.9 * R / 1024.0;
    return 11.0 + 9.0 * R / 2048.0;
}

// Blocks per wake of the two-species and RK4 marches: a cluster once one
// block would hold more than per_thread sorted positions (of each species,
// with ions) per thread, at most kMaxWakeCtas blocks.
int32_t gm_cluster_for(int32_t positions, int32_t threads, int32_t per_thread) {
    const int32_t per_block = per_thread * threads;
    return std::max(1, std::min(kMaxWakeCtas, (positions + per_block - 1) / per_block));
}

double predicted_slice_us(const wake_handle* h) {
    if (h->fast_threads > 0) {
        FastShape f;
        f.threads = h->fast_threads;
        f.k = h->fast_k;
        f.cl = h->fast_cl;
        return predicted_fast_slice_us(f);
    }
    const double per_thread = (double)h->n / ((double)h->threads * h->gm_cl);
    const double cluster = h->gm_cl > 1 ? kGmClusterSliceUs : 0.0;
    return (h->rk4 ? 4.0 : 1.0) * (20.0 + 6.0 * per_thread + cluster);
}

double predicted_ms(const wake_handle* h) { return h->n_steps * predicted_slice_us(h) * 1e-3; }

// A batch as march launches: wakes of one kernel configuration share a
// launch, split by predicted time into three tiers (at least half of the
// longest wake's time; a fifth of it; the rest), one stream priority each, so
// that the hardware dispatches the blocks of the long wakes of every
// configuration before the short ones of any (an approximation of longest-
// processing-time-first list scheduling, whose makespan a wake started late
// lengthens by its whole march).  Groups come tier by tier, the group with
// the longest wake first within a tier.
struct LaunchGroup {
    std::vector<wake_handle*> hs;
    int tier = 0;
    double t_max = 0.0;
};

// lower bounds of the tiers' predicted times, as fractions of the longest
// (GB300 offers four stream priorities: the preparations' and three tiers';
// two levels sharing a priority measured 15-20 % slower steps)
constexpr double kTierFrac[kTiers - 1] = {0.5, 0.2};

// whole_window = false (steps bounded by a time budget, as the serving loop
// runs them): one launch per configuration, all in tier 0 -- every step ends
// at the budget anyway, and fewer launches mean less host time per step.
std::vector<LaunchGroup> plan_launches(int32_t n, wake_handle* const* hs, bool whole_window = true) {
    double t_all = 0.0;
    for (int32_t i = 0; i < n; ++i) t_all = std::max(t_all, predicted_ms(hs[i]));
    std::vector<std::pair<int64_t, int>> keys;  // (configuration and band, tier)
    std::vector<LaunchGroup> groups;
    for (int32_t i = 0; i < n; ++i) {
        int64_t key = ((int64_t)hs[i]->fast_threads * 16 + (hs[i]->fast_threads ? hs[i]->fast_k : 0)) * 32 +
                      (hs[i]->fast_threads ? hs[i]->fast_cl : 0);
        // the one-CTA kernels (plain, two-species, RK4, grids) by their block size
        if (!hs[i]->fast_threads) key = -(1 + (hs[i]->n_ion ? 1 : 0) + 2 * hs[i]->rk4 + 4 * (hs[i]->grid_nr > 0) +
                                          8 * (hs[i]->threads + 1024 * (hs[i]->gm_cl - 1)));
        const double t = predicted_ms(hs[i]);
        int tier = 0;
        while (whole_window && tier + 1 < kTiers && t < kTierFrac[tier] * t_all) ++tier;
        // bands of predicted time (each 1/1.25 of the one before) split a
        // configuration's wakes into launches, so that the launches of a tier,
        // submitted longest band first, reach the SMs longest first across
        // configurations (same-priority launches are dispatched in about the
        // order they were submitted)
        const int band = !whole_window ? 0
                       : t > 0.0 && t_all > 0.0 ? std::min(63, (int)std::floor(std::log(t_all / t) / std::log(1.25)))
                                                : 63;
        key = key * 64 + band;
        auto it = std::find(keys.begin(), keys.end(), std::make_pair(key, tier));
        if (it == keys.end()) {
            keys.emplace_back(key, tier);
            groups.emplace_back();
            groups.back().tier = tier;
            it = keys.end() - 1;
        }
        LaunchGroup& g = groups[it - keys.begin()];
        g.hs.push_back(hs[i]);
        g.t_max = std::max(g.t_max, t);
    }
    std::stable_sort(groups.begin(), groups.end(), [](const LaunchGroup& a, const LaunchGroup& b) {
        return a.tier != b.tier ? a.tier < b.tier : a.t_max > b.t_max;
    });
    return groups;
}

template <class P>
wake_status batch_impl(int32_t n, wake_handle* const* hs, int32_t max_slices, int64_t budget_ns) {
    cudaStream_t st = hs[0]->st;
    // one launch per group, each on its own stream of its tier's priority,
    // ordered after the work already queued on the handles' stream and
    // joined back into it
    std::vector<LaunchGroup> groups = plan_launches(n, hs, budget_ns <= 0);
    if (groups.size() == 1) return batch_bucket<P>(groups[0].hs, wake_shape(groups[0].hs[0]), st, max_slices, budget_ns);
    cudaEvent_t start;
    WK_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    WK_CUDA(cudaEventRecord(start, st));
    wake_status res = WAKE_OK;
    int in_tier[kTiers] = {};
    for (size_t i = 0; i < groups.size(); ++i) {
        cudaStream_t as = nullptr;
        const int tier = groups[i].tier;
        WK_CUDA(tier_stream(tier, in_tier[tier]++, &as));
        WK_CUDA(cudaStreamWaitEvent(as, start, 0));
        wake_status r = batch_bucket<P>(groups[i].hs, wake_shape(groups[i].hs[0]), as, max_slices, budget_ns);
        if (r != WAKE_OK) res = r;
        cudaEvent_t done;
        WK_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        WK_CUDA(cudaEventRecord(done, as));
        WK_CUDA(cudaStreamWaitEvent(st, done, 0));
        cudaEventDestroy(done);
    }
    cudaEventDestroy(start);
    return res;
}

// The a0/a1 preparation and the whole-window march of n wakes, pipelined:
// the preparations run on the greatest-priority streams, the longest
// groups' wakes first, and each group's march (on a stream of its tier)
// waits only for its own wakes' preparations, so that the long marches
// start while the short wakes are still being prepared.  Everything is
// ordered after the work queued on the handles' stream and joined back
// into it.
template <class P>
wake_status batch_reset_run_impl(int32_t n, wake_handle* const* hs, const wake_beam_desc* const* beams = nullptr,
                                 const int32_t* n_beams = nullptr) {
    cudaStream_t st = hs[0]->st;
    std::vector<LaunchGroup> groups = plan_launches(n, hs);
    constexpr int kPrepStreams = 16;
    cudaEvent_t start;
    WK_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    WK_CUDA(cudaEventRecord(start, st));
    for (int j = 0; j < kPrepStreams; ++j) {
        cudaStream_t ps = nullptr;
        WK_CUDA(aux_stream(j, &ps));
        WK_CUDA(cudaStreamWaitEvent(ps, start, 0));
    }
    std::vector<cudaEvent_t> events;
    auto cleanup = [&]() {
        for (cudaEvent_t e : events) cudaEventDestroy(e);
        cudaEventDestroy(start);
    };
    wake_status res = WAKE_OK;
    int next_prep = 0;
    int in_tier[kTiers] = {};
    for (size_t i = 0; i < groups.size() && res == WAKE_OK; ++i) {
        cudaStream_t ms = nullptr;
        const int tier = groups[i].tier;
        if (tier_stream(tier, in_tier[tier]++, &ms) != cudaSuccess) {
            res = fail(WAKE_ECUDA, "wake_batch_reset_run: no stream");
            break;
        }
        cudaStreamWaitEvent(ms, start, 0);
        for (wake_handle* h : groups[i].hs) {
            cudaStream_t ps = nullptr;
            aux_stream(next_prep++ % kPrepStreams, &ps);
            // the wake's new beams (its index in the caller's arrays)
            const int32_t k = (int32_t)(std::find(hs, hs + n, h) - hs);
            if (beams && beams[k]) res = upload_beams(h, beams[k], n_beams[k], ps, false);
            if (res == WAKE_OK) res = prepare_impl<P>(h, ps);
            if (res != WAKE_OK) break;
            cudaEvent_t ready;
            if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) {
                res = fail(WAKE_ECUDA, "wake_batch_reset_run: event creation failed");
                break;
            }
            events.push_back(ready);
            cudaEventRecord(ready, ps);
            cudaStreamWaitEvent(ms, ready, 0);
        }
        if (res != WAKE_OK) break;
        res = batch_bucket<P>(groups[i].hs, wake_shape(groups[i].hs[0]), ms, 1 << 30, 0);
        cudaEvent_t done;
        WK_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        events.push_back(done);
        WK_CUDA(cudaEventRecord(done, ms));
        WK_CUDA(cudaStreamWaitEvent(st, done, 0));
    }
    // the preparation streams join back too (also after an error)
    for (int j = 0; j < kPrepStreams; ++j) {
        cudaStream_t ps = nullptr;
        if (aux_stream(j, &ps) != cudaSuccess) continue;
        cudaEvent_t done;
        if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess) continue;
        events.push_back(done);
        cudaEventRecord(done, ps);
        cudaStreamWaitEvent(st, done, 0);
    }
    cleanup();
    return res;
}

template <class P>
wake_status state_io(wake_handle* h, bool export_, int32_t slice, double* rho, double* ur, double* fr, double* fu,
                     const double* irho, const double* iur, const double* ifr, const double* ifu) {
    using R = typename P::R;
    WakeDev<P> D;
    std::memcpy(&D, h->desc_host.data(), sizeof(D));
    const size_t bytes = (size_t)h->n * sizeof(double);
    double* tmp = nullptr;
    if (cudaMalloc(&tmp, 4 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(WAKE_ENOMEM, "ring state staging allocation failed");
    }
    double* t[4] = {tmp, tmp + h->n, tmp + 2 * h->n, tmp + 3 * h->n};
    cudaError_t e = cudaSuccess;
    if (export_) {
        int32_t ctl[CTL_N];
        e = cudaMemcpyAsync(ctl, h->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
        const int b = ctl[CTL_BUF];
        double* outs[4] = {rho, ur, fr, fu};
        if (e == cudaSuccess)
            e = launch_export_state<R>(D.rid[b], D.rho[b], D.rho_lo, D.ur[b], D.frho[b], D.fur[b], h->n, D.ctab,
                                       t[0], t[1], t[2], t[3], h->st);
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            if (outs[k]) e = cudaMemcpyAsync(outs[k], t[k], bytes, cudaMemcpyDeviceToHost, h->st);
    } else {
        const double* ins[4] = {irho, iur, ifr, ifu};
        for (int k = 0; k < 4 && e == cudaSuccess; ++k)
            if (ins[k]) e = cudaMemcpyAsync(t[k], ins[k], bytes, cudaMemcpyHostToDevice, h->st);
        if (e == cudaSuccess)
            e = launch_import_state<R>(t[0], t[1], ifr ? t[2] : nullptr, ifu ? t[3] : nullptr, h->n, D.ctab,
                                       D.rho[0], D.rho_lo, D.ur[0], D.frho[0], D.fur[0], D.rid[0], h->d_ctl, slice,
                                       h->st);
    }
    cudaError_t e2 = cudaStreamSynchronize(h->st);
    cudaFree(tmp);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "ring state transfer: %s", cudaGetErrorString(e));
    return WAKE_OK;
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Scratch for wake_fields_at_static, the variant of wake_fields_at that
// allocates nothing.  Its callers are the ones that cannot allocate while
// they run: a host code that has handed the device's memory to its own pool
// allocator (a cudaMalloc there fails or fragments that pool), and a
// latency-critical loop in which cudaMalloc/cudaFree would synchronise the
// device and stall the caller's other streams.  The per-call scratch that
// wake_fields_at allocates -- the query radii, the four output arrays and
// the launch descriptor -- sits in this one file-scope device array instead,
// sized for WAKE_STATIC_MAX_QUERIES queries.  There is one copy of it per
// device and process, so two calls in flight at once would race on it; a
// call made while another is in progress in this process is refused with
// WAKE_EBUSY, and each call waits for its own stream before it returns.
constexpr size_t kStaticDescBytes = 1024;  // launch descriptor, padded
constexpr size_t kStaticQueryBytes = (size_t)WAKE_STATIC_MAX_QUERIES * sizeof(double);
constexpr size_t kStaticScratchBytes = kStaticDescBytes + 5 * kStaticQueryBytes;  // r + 4 outputs
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];
static_assert(sizeof(WakeDev<PrecF64>) <= kStaticDescBytes && sizeof(WakeDev<PrecMixed>) <= kStaticDescBytes,
              "launch descriptor does not fit its static slot");

constexpr int kStaticMaxDevices = 64;
unsigned char* g_static_addr[kStaticMaxDevices] = {nullptr};  // symbol address, per device
std::atomic<int> g_static_busy{0};

// Device address of the static scratch on the current device, looked up
// with cudaGetSymbolAddress the first time for each device.
wake_status static_scratch(unsigned char** out) {
    int dev = 0;
    WK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kStaticMaxDevices)
        return fail(WAKE_EINVAL, "wake_fields_at_static: device %d is beyond the %d supported", dev,
                    kStaticMaxDevices);
    if (!g_static_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(WAKE_ECUDA, "wake_fields_at_static: cudaGetSymbolAddress of the static scratch failed: %s",
                        cudaGetErrorString(e));
        }
        g_static_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_static_addr[dev];
    return WAKE_OK;
}

template <class P>
wake_status fields_at_static_impl(wake_handle* h, int64_t n, const double* r, void* const outs_user[4],
                                  unsigned char* base) {
    using R = typename P::R;
    WakeDev<P> D;
    std::memcpy(&D, h->desc_host.data(), sizeof(D));
    double* d_r = reinterpret_cast<double*>(base + kStaticDescBytes);
    R* d_out[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int k = 0; k < 4; ++k)
        if (outs_user[k]) d_out[k] = reinterpret_cast<R*>(base + kStaticDescBytes + (1 + k) * kStaticQueryBytes);
    D.nq = n;
    D.rq = d_r;
    D.q_ez = d_out[0];
    D.q_wr = d_out[1];
    D.q_bt = d_out[2];
    D.q_psi = d_out[3];
    // every step is queued on the handle's stream; on any error the stream
    // is drained before returning so that nothing still uses the scratch
    auto drain = [&](wake_status s) {
        cudaStreamSynchronize(h->st);
        return s;
    };
    cudaError_t e = cudaMemcpyAsync(d_r, r, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base, &D, sizeof(D), cudaMemcpyHostToDevice, h->st);
    // the output slots start at zero, so no value of an earlier call can be
    // returned for a query the kernel does not write
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (d_out[k]) e = cudaMemsetAsync(d_out[k], 0, (size_t)n * sizeof(R), h->st);
    if (e != cudaSuccess)
        return drain(fail(WAKE_ECUDA, "wake_fields_at_static: staging failed: %s", cudaGetErrorString(e)));
    wake_status s = launch_one<P>(h, reinterpret_cast<const WakeDev<P>*>(base), 1, MODE_QUERY);
    if (s != WAKE_OK) return drain(s);
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (outs_user[k])
            e = cudaMemcpyAsync(outs_user[k], d_out[k], (size_t)n * sizeof(R), cudaMemcpyDeviceToHost, h->st);
    cudaError_t e2 = cudaStreamSynchronize(h->st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "wake_fields_at_static: %s", cudaGetErrorString(e));
    return WAKE_OK;
}

}  // namespace

namespace {

// One wake's push description: its particle arrays, the fields of the last
// march in sorted order, the caller -> sorted map and its species.
template <class R>
PushWake<R> push_desc(const wake_handle* h) {
    PushWake<R> d = {};
    d.n = h->nb_total;
    d.x = h->d_ps[0];
    d.y = h->d_ps[1];
    d.xi = h->d_xi;
    d.r = h->d_r;
    d.ux = h->d_ps[2];
    d.uy = h->d_ps[3];
    d.uz = h->d_ps[4];
    d.ez = static_cast<const R*>(h->d_out[0]);
    d.wr = static_cast<const R*>(h->d_out[1]);
    d.bt = static_cast<const R*>(h->d_out[2]);
    d.inv = h->d_inv;
    return d;
}

// Enqueues the push of n wakes (one launch) on stream st: each wake cut
// into particle ranges of push_item_size(total), the descriptors and ranges
// travel through one pooled device buffer.
template <class R>
wake_status push_enqueue(wake_handle* const* hs, int32_t n, double dt, cudaStream_t st) {
    std::vector<PushWake<R>> descs;
    std::vector<const wake_handle*> owner;
    int64_t total = 0;
    for (int32_t i = 0; i < n; ++i)
        if (hs[i]->nb_total > 0) {
            descs.push_back(push_desc<R>(hs[i]));
            owner.push_back(hs[i]);
            total += hs[i]->nb_total;
        }
    if (descs.empty()) return WAKE_OK;
    const int64_t chunk = push_item_size(total);
    std::vector<PushItem> items;
    for (size_t w = 0; w < descs.size(); ++w) {
        int64_t off = 0;
        for (size_t b = 0; b < owner[w]->beam_n.size(); ++b) {
            const int64_t end = off + owner[w]->beam_n[b];
            for (int64_t k = off; k < end; k += chunk)
                items.push_back(PushItem{(int32_t)w, 0, k, std::min(k + chunk, end), owner[w]->beam_q[b]});
            off = end;
        }
    }
    if (items.size() > (size_t)INT32_MAX) return fail(WAKE_EINVAL, "wake_push_beam: too many particles");
    const size_t desc_bytes = (descs.size() * sizeof(PushWake<R>) + 15) / 16 * 16;
    const size_t item_bytes = items.size() * sizeof(PushItem);
    std::vector<unsigned char> host(desc_bytes + item_bytes);
    std::memcpy(host.data(), descs.data(), descs.size() * sizeof(PushWake<R>));
    std::memcpy(host.data() + desc_bytes, items.data(), item_bytes);
    cudaMemPool_t pool = nullptr;
    WK_CUDA(wake_pool(&pool));
    void* buf = nullptr;
    WK_CUDA(cudaMallocFromPoolAsync(&buf, host.size(), pool, st));
    cudaError_t e = cudaMemcpyAsync(buf, host.data(), host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_beam_push<R>(static_cast<const PushWake<R>*>(buf),
                                reinterpret_cast<const PushItem*>(static_cast<unsigned char*>(buf) + desc_bytes),
                                (int32_t)items.size(), dt, st);
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "wake_push_beam: %s", cudaGetErrorString(e));
    // particles may have changed slices: the next binning sizes its sort
    // on the device, not from the count taken before the push
    for (int32_t i = 0; i < n; ++i) hs[i]->slice_max = -1;
    return WAKE_OK;
}

wake_status check_push(const wake_handle* h, double dt) {
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(WAKE_EINVAL, "wake_push_beam: dt must be > 0");
    if (h->nb_total > 0 && !h->d_ps[0])
        return fail(WAKE_EINVAL, "wake_push_beam: set the beam phase space first (wake_set_beam_phase_space)");
    for (double q : h->beam_q)
        if (q != 1.0 && q != -1.0)
            return fail(WAKE_EINVAL, "wake_push_beam: beam species must be electrons or positrons (q = -1 or +1)");
    return WAKE_OK;
}

}  // namespace

extern "C" {

const char* wake_last_error(void) { return g_err.c_str(); }

int64_t wake_debug_bounds_violations(void) {
    const int64_t a = march_bounds_violations(), b = march_k2_bounds_violations();
    if (a == -1 && b == -1) return -1;
    if (a < 0 || b < 0) return -2;
    return a + b;
}

int32_t wake_max_rings(int32_t precision) {
    return precision == WAKE_MIXED ? kMaxRingsMixed : kMaxRings;
}

int64_t wake_max_slice_particles(int32_t precision) {
    (void)precision;
    return kMaxSliceParticles;
}

wake_status wake_launch_shape(int32_t precision, int32_t n_rings, int32_t n_steps, int32_t rings_per_thread,
                              int32_t cluster_ctas, int32_t* threads, int32_t* rings_per_thread_out,
                              int32_t* blocks_per_wake) {
    if (precision != WAKE_FP64 && precision != WAKE_MIXED) return fail(WAKE_EINVAL, "wake_launch_shape: bad precision");
    if (n_rings < 1 || n_rings > wake_max_rings(precision))
        return fail(WAKE_EINVAL, "wake_launch_shape: n_rings must be in [1, %d]", wake_max_rings(precision));
    if (n_steps < 0) return fail(WAKE_EINVAL, "wake_launch_shape: n_steps must be >= 0");
    FastShape f;
    WK_TRY(wake_shape_for(precision, n_rings, n_steps, rings_per_thread, cluster_ctas, &f));
    if (threads) *threads = f.threads;
    if (rings_per_thread_out) *rings_per_thread_out = f.threads ? f.k : 0;
    if (blocks_per_wake) *blocks_per_wake = f.threads ? f.cl : 0;
    return WAKE_OK;
}

wake_status wake_gm_launch_shape(int32_t march, int32_t n_cells, int32_t block_threads, int32_t cluster_ctas,
                                int32_t* threads, int32_t* rings_per_thread_out, int32_t* blocks_per_wake) {
    if (march != WAKE_GM_IONS && march != WAKE_GM_RK4 && march != WAKE_GM_GRID)
        return fail(WAKE_EINVAL, "wake_gm_launch_shape: unknown march %d", march);
    const int32_t max_cells = march == WAKE_GM_IONS ? kMaxIonCells : kMaxRk4Rings;
    if (n_cells < 1 || n_cells > max_cells)
        return fail(WAKE_EINVAL, "wake_gm_launch_shape: n_cells must be in [1, %d]", max_cells);
    const bool default_threads = block_threads == 0;
    const int32_t t = default_threads ? (march == WAKE_GM_GRID ? kDefaultThreads : 512) : block_threads;
    if (t < 64 || t > 512 || t % 32)
        return fail(WAKE_EINVAL, "wake_gm_launch_shape: block_threads must be 0 or a multiple of 32 in [64, 512]");
    if (cluster_ctas < 0 || cluster_ctas > kMaxWakeCtas)
        return fail(WAKE_EINVAL, "wake_gm_launch_shape: cluster_ctas must be in [0, %d]", kMaxWakeCtas);
    const int32_t per_thread = march == WAKE_GM_IONS ? kIonRingsPerThread
                             : march == WAKE_GM_RK4  ? kRk4RingsPerThread
                                                     : kGridRingsPerThread;
    const int32_t cl = cluster_ctas ? cluster_ctas : gm_cluster_for(n_cells, t, per_thread);
    const int32_t rings = march == WAKE_GM_IONS ? 2 * n_cells : n_cells;
    if (threads) *threads = t;
    if (rings_per_thread_out) *rings_per_thread_out = (rings + t * cl - 1) / (t * cl);
    if (blocks_per_wake) *blocks_per_wake = cl;
    return WAKE_OK;
}

wake_status wake_launch_shape_latency(int32_t precision, int32_t n_rings, int32_t* threads,
                                      int32_t* rings_per_thread_out, int32_t* blocks_per_wake) {
    if (precision != WAKE_FP64 && precision != WAKE_MIXED)
        return fail(WAKE_EINVAL, "wake_launch_shape_latency: bad precision");
    if (n_rings < 1 || n_rings > wake_max_rings(precision))
        return fail(WAKE_EINVAL, "wake_launch_shape_latency: n_rings must be in [1, %d]", wake_max_rings(precision));
    FastShape f;
    WK_TRY(fast_shape_for(precision, n_rings, 0, 0, &f));
    f = latency_shape_for(n_rings, f);
    if (threads) *threads = f.threads;
    if (rings_per_thread_out) *rings_per_thread_out = f.threads ? f.k : 0;
    if (blocks_per_wake) *blocks_per_wake = f.threads ? f.cl : 0;
    return WAKE_OK;
}

wake_status wake_set_latency_shape_ms(double ms) {
    if (!(ms >= 0.0)) return fail(WAKE_EINVAL, "wake_set_latency_shape_ms: ms must be >= 0 (or infinity)");
    g_latency_shape_ms = ms;
    return WAKE_OK;
}

double wake_get_latency_shape_ms(void) { return g_latency_shape_ms; }

wake_status wake_init(const wake_config* cfg, const wake_plasma_desc* plasma, const wake_beam_desc* beams,
                      int32_t n_beams, void* cuda_stream, wake_handle** out) {
    if (!out) return fail(WAKE_EINVAL, "wake_init: out is NULL");
    *out = nullptr;
    if (!cfg || !plasma) return fail(WAKE_EINVAL, "wake_init: cfg and plasma are required");
    if (cfg->precision != WAKE_FP64 && cfg->precision != WAKE_MIXED)
        return fail(WAKE_EINVAL, "wake_init: unknown precision %d", cfg->precision);
    if (!(cfg->dxi > 0.0) || !std::isfinite(cfg->dxi)) return fail(WAKE_EINVAL, "wake_init: dxi must be > 0");
    if (cfg->n_steps < 1 || cfg->n_steps > kBinSmem)
        return fail(WAKE_EINVAL, "wake_init: n_steps must be in [1, %d]", (int)kBinSmem);
    int32_t threads = cfg->block_threads ? cfg->block_threads : kDefaultThreads;
    if (threads < 64 || threads > 512 || threads % 32)
        return fail(WAKE_EINVAL, "wake_init: block_threads must be a multiple of 32 in [64, 512]");
    const int32_t n_cells = plasma->n_rings;
    const bool ions = plasma->ion_charge != 0.0;
    if (ions && (!(plasma->ion_charge > 0.0) || !(plasma->ion_mass > 0.0) || !std::isfinite(plasma->ion_charge) ||
                 std::isnan(plasma->ion_mass)))
        return fail(WAKE_EINVAL, "wake_init: mobile ions need ion_charge > 0 and ion_mass > 0 (or +inf)");
    if (plasma->cell_density && !ions)
        return fail(WAKE_EINVAL, "wake_init: a density profile needs ion rings (ion_charge > 0)");
    if (ions && (cfg->rings_per_thread || cfg->cluster_ctas < 0 || cfg->cluster_ctas > kMaxWakeCtas))
        return fail(WAKE_EINVAL, "wake_init: with mobile ions rings_per_thread must be 0 and cluster_ctas in [0, %d]",
                    kMaxWakeCtas);
    const int32_t max_rings = ions ? kMaxIonCells : wake_max_rings(cfg->precision);
    if (n_cells < 1 || n_cells > max_rings)
        return fail(WAKE_EINVAL, "wake_init: n_rings must be in [1, %d]%s", max_rings, ions ? " with mobile ions" : "");
    const int32_t n = n_cells;
    if (cfg->integrator != WAKE_AB2 && cfg->integrator != WAKE_RK4)
        return fail(WAKE_EINVAL, "wake_init: unknown integrator %d", cfg->integrator);
    const bool rk4 = cfg->integrator == WAKE_RK4;
    if (rk4 && n_cells > kMaxRk4Rings)
        return fail(WAKE_EINVAL, "wake_init: RK4 wakes have at most %d rings (block 0 sorts the stage states in its "
                                 "shared memory)", kMaxRk4Rings);
    if (rk4 && (ions || cfg->rings_per_thread || cfg->cluster_ctas < 0 || cfg->cluster_ctas > kMaxWakeCtas))
        return fail(WAKE_EINVAL, "wake_init: RK4 runs electron-only wakes on the global-memory march (no mobile "
                                 "ions, rings_per_thread 0, cluster_ctas in [0, %d])", kMaxWakeCtas);
    if (cfg->grid_nr < 0 || cfg->grid_nr > 1024) return fail(WAKE_EINVAL, "wake_init: grid_nr must be in [0, 1024]");
    if (cfg->grid_nr > 0 && (cfg->rings_per_thread || cfg->cluster_ctas < 0 || cfg->cluster_ctas > kMaxWakeCtas))
        return fail(WAKE_EINVAL, "wake_init: beam-grid wakes take rings_per_thread 0 and cluster_ctas in [0, %d]",
                    kMaxWakeCtas);
    if (cfg->grid_nr > 0 && n_cells > kMaxRk4Rings)
        return fail(WAKE_EINVAL, "wake_init: beam-grid wakes have at most %d rings (block 0 sorts them in its "
                                 "shared memory)", kMaxRk4Rings);
    if (!(cfg->grid_rmax >= 0.0) || !std::isfinite(cfg->grid_rmax) || (cfg->grid_rmax > 0.0 && cfg->grid_nr == 0))
        return fail(WAKE_EINVAL, "wake_init: grid_rmax must be finite, >= 0, and set only with grid_nr > 0");
    if (cfg->grid_rmax > 0.0)
        for (int32_t b = 0; b < n_beams; ++b)
            for (int64_t k = 0; k < beams[b].n; ++k)
                if (!(beams[b].r[k] < cfg->grid_rmax))
                    return fail(WAKE_EINVAL, "wake_init: beam %d particle %lld lies beyond grid_rmax", b,
                                (long long)k);
    if (cfg->grid_nr > 0 && (rk4 || ions || n_beams > kMaxGridSpecies))
        return fail(WAKE_EINVAL, "wake_init: beam grids run WAKE_AB2, without mobile ions, with at most %d beam "
                                 "species", kMaxGridSpecies);
    // the two-species and RK4 marches: one CTA of 512 threads per wake
    if ((ions || rk4) && !cfg->block_threads) threads = 512;
    if (!plasma->r_edges) return fail(WAKE_EINVAL, "wake_init: r_edges is NULL");
    if (!(plasma->density > 0.0) || !std::isfinite(plasma->density))
        return fail(WAKE_EINVAL, "wake_init: density must be > 0");
    if (plasma->r_edges[0] != 0.0) return fail(WAKE_EINVAL, "wake_init: r_edges[0] must be 0");
    for (int32_t j = 0; j < n; ++j)
        if (!(plasma->r_edges[j + 1] > plasma->r_edges[j]) || !std::isfinite(plasma->r_edges[j + 1]))
            return fail(WAKE_EINVAL, "wake_init: r_edges must be finite and strictly increasing (index %d)", j + 1);
    if (plasma->cell_density)
        for (int32_t j = 0; j < n; ++j)
            if (!(plasma->cell_density[j] > 0.0) || !std::isfinite(plasma->cell_density[j]))
                return fail(WAKE_EINVAL, "wake_init: cell_density[%d] must be finite and > 0", j);
    if (n_beams < 0 || (n_beams > 0 && !beams)) return fail(WAKE_EINVAL, "wake_init: bad beams");
    int64_t nb = 0;
    for (int32_t b = 0; b < n_beams; ++b) {
        if (beams[b].n < 0) return fail(WAKE_EINVAL, "wake_init: beam %d has n < 0", b);
        if (beams[b].n > 0 && (!beams[b].xi || !beams[b].r || !beams[b].w))
            return fail(WAKE_EINVAL, "wake_init: beam %d arrays are NULL", b);
        for (int64_t k = 0; k < beams[b].n; ++k)
            if (!(beams[b].r[k] >= 0.0) || !std::isfinite(beams[b].xi[k]) || !std::isfinite(beams[b].w[k]))
                return fail(WAKE_EINVAL, "wake_init: beam %d particle %lld has r < 0 or non-finite data", b,
                            (long long)k);
        nb += beams[b].n;
    }
    if (nb > (int64_t)0x7fffffff) return fail(WAKE_EINVAL, "wake_init: more than 2^31-1 beam particles");

    wake_handle* h = new wake_handle();
    h->prec = cfg->precision;
    h->n = ions ? 2 * n : n;
    h->n_ion = ions ? n : 0;
    h->ion_qm = ions && std::isfinite(plasma->ion_mass) ? plasma->ion_charge / plasma->ion_mass : 0.0;
    h->rk4 = rk4 ? 1 : 0;
    h->grid_nr = cfg->grid_nr;
    h->grid_rmax = cfg->grid_rmax;
    h->n_steps = cfg->n_steps;
    h->n_pad = next_pow2(std::max(n, 2));  // sorts one species at a time
    h->threads = threads;
    const bool grid = cfg->grid_nr > 0;
    h->gm_cl = cfg->cluster_ctas && (ions || rk4 || grid) ? cfg->cluster_ctas
             : ions                                      ? gm_cluster_for(n, threads, kIonRingsPerThread)
             : rk4                                       ? gm_cluster_for(n, threads, kRk4RingsPerThread)
             : grid                                      ? gm_cluster_for(n, threads, kGridRingsPerThread)
                                                         : 1;
    h->flags = cfg->flags;
    h->dxi = cfg->dxi;
    h->density = plasma->density;
    h->rho_max = plasma->r_edges[n];
    h->st = static_cast<cudaStream_t>(cuda_stream);
    FastShape shape;
    {
        wake_status fs = (ions || rk4 || cfg->grid_nr > 0) ? WAKE_OK
                                       : wake_shape_for(h->prec, n, cfg->n_steps, cfg->rings_per_thread,
                                                        cfg->cluster_ctas, &shape);
        if (fs != WAKE_OK) {
            delete h;
            return fs;
        }
    }
    h->fast_threads = shape.threads;
    h->fast_k = shape.k;
    h->fast_cl = shape.cl;
    h->slice_max = densest_slice(beams, n_beams, cfg->dxi, cfg->n_steps);
    wake_status s = h->prec == WAKE_FP64 ? init_impl<PrecF64>(h, cfg, plasma, beams, n_beams)
                                         : init_impl<PrecMixed>(h, cfg, plasma, beams, n_beams);
    if (s != WAKE_OK) {
        std::string keep = g_err;
        free_all(h);
        delete h;
        g_err = keep;
        return s;
    }
    *out = h;
    return WAKE_OK;
}

wake_status wake_reset(wake_handle* h, const wake_beam_desc* beams, int32_t n_beams) {
    WK_TRY(check_handle(h));
    WK_TRY(check_new_beams(h, beams, n_beams));
    WK_TRY(upload_beams(h, beams, n_beams, h->st));
    if (h->prec == WAKE_FP64) return prepare_impl<PrecF64>(h, h->st);
    return prepare_impl<PrecMixed>(h, h->st);
}

wake_status wake_batch_reset(int32_t n, wake_handle* const* handles, const wake_beam_desc* const* beams,
                             const int32_t* n_beams) {
    if (n < 0 || (n > 0 && !handles)) return fail(WAKE_EINVAL, "wake_batch_reset: bad handle array");
    if (n == 0) return WAKE_OK;
    for (int32_t i = 0; i < n; ++i) {
        if (!handles[i]) return fail(WAKE_EINVAL, "wake_batch_reset: handle %d is NULL", i);
        if (handles[i]->st != handles[0]->st)
            return fail(WAKE_EINVAL, "wake_batch_reset: handles must share one stream");
        if (beams && beams[i]) {
            if (!n_beams) return fail(WAKE_EINVAL, "wake_batch_reset: n_beams is required with beams");
            WK_TRY(check_new_beams(handles[i], beams[i], n_beams[i]));
        }
    }
    // each wake's preparation on one of the auxiliary streams, ordered
    // after the work already queued on the handles' stream and joined back
    cudaStream_t st = handles[0]->st;
    cudaEvent_t start;
    WK_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    WK_CUDA(cudaEventRecord(start, st));
    const int32_t n_streams = n < kStreamsPerLevel ? n : kStreamsPerLevel;
    wake_status res = WAKE_OK;
    for (int32_t j = 0; j < n_streams; ++j) {
        cudaStream_t as = nullptr;
        WK_CUDA(aux_stream(j, &as));
        WK_CUDA(cudaStreamWaitEvent(as, start, 0));
    }
    // new beams are counted on the device only (the per-slice sort sizes
    // itself there): nothing here waits for the device
    for (int32_t i = 0; i < n && res == WAKE_OK; ++i) {
        wake_handle* h = handles[i];
        cudaStream_t as = nullptr;
        WK_CUDA(aux_stream(i % n_streams, &as));
        if (beams && beams[i]) res = upload_beams(h, beams[i], n_beams[i], as, false);
        if (res == WAKE_OK) res = h->prec == WAKE_FP64 ? prepare_impl<PrecF64>(h, as) : prepare_impl<PrecMixed>(h, as);
    }
    for (int32_t j = 0; j < n_streams; ++j) {
        cudaStream_t as = nullptr;
        WK_CUDA(aux_stream(j, &as));
        cudaEvent_t done;
        WK_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
        WK_CUDA(cudaEventRecord(done, as));
        WK_CUDA(cudaStreamWaitEvent(st, done, 0));
        cudaEventDestroy(done);
    }
    cudaEventDestroy(start);
    return res;
}

wake_status wake_step_slices(wake_handle* h, int32_t n_slices) {
    WK_TRY(check_handle(h));
    if (n_slices < 0) return fail(WAKE_EINVAL, "wake_step_slices: n_slices < 0");
    if (n_slices == 0) return WAKE_OK;
    if (h->prec == WAKE_FP64)
        return launch_one<PrecF64>(h, static_cast<const WakeDev<PrecF64>*>(h->d_desc), n_slices, MODE_MARCH);
    return launch_one<PrecMixed>(h, static_cast<const WakeDev<PrecMixed>*>(h->d_desc), n_slices, MODE_MARCH);
}

wake_status wake_get_progress(wake_handle* h, int32_t* next_slice, int32_t* status, int32_t* fail_slice) {
    WK_TRY(check_handle(h));
    int32_t ctl[CTL_N];
    WK_CUDA(cudaMemcpyAsync(ctl, h->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->st));
    WK_CUDA(cudaStreamSynchronize(h->st));
    if (next_slice) *next_slice = ctl[CTL_NEXT];
    if (status) *status = ctl[CTL_STATUS];
    if (fail_slice) *fail_slice = ctl[CTL_FAIL];
    return WAKE_OK;
}

wake_status wake_fields_at(wake_handle* h, int64_t n, const double* r, void* ez, void* wr, void* bt, void* psi,
                           int32_t device_ptrs) {
    WK_TRY(check_handle(h));
    if (n < 0 || (n > 0 && !r)) return fail(WAKE_EINVAL, "wake_fields_at: bad query array");
    int32_t next = 0, status = 0;
    WK_TRY(wake_get_progress(h, &next, &status, nullptr));
    if (status != 0) return stopped(status, "wake_fields_at");
    if (next >= h->n_steps)
        return fail(WAKE_EINVAL, "wake_fields_at: the window is finished (slice %d of %d)", next, h->n_steps);
    if (h->prec == WAKE_FP64) return fields_at_impl<PrecF64>(h, n, r, ez, wr, bt, psi, device_ptrs);
    return fields_at_impl<PrecMixed>(h, n, r, ez, wr, bt, psi, device_ptrs);
}

wake_status wake_get_beam_fields(wake_handle* h, void* ez, void* wr, void* bt, void* psi, int32_t device_ptrs) {
    WK_TRY(check_handle(h));
    void* outs[4] = {ez, wr, bt, psi};
    if (h->prec == WAKE_FP64) return beam_fields_impl<double>(h, outs, device_ptrs);
    return beam_fields_impl<float>(h, outs, device_ptrs);
}

wake_status wake_batch_get_beam_fields(int32_t n, wake_handle* const* handles, void* const* ez, void* const* wr,
                                       int32_t device_ptrs) {
    if (n < 0 || (n > 0 && !handles)) return fail(WAKE_EINVAL, "wake_batch_get_beam_fields: bad handle array");
    for (int32_t i = 0; i < n; ++i) {
        if (!handles[i]) return fail(WAKE_EINVAL, "wake_batch_get_beam_fields: handle %d is NULL", i);
        if (handles[i]->st != handles[0]->st)
            return fail(WAKE_EINVAL, "wake_batch_get_beam_fields: handles must share a stream");
    }
    for (int32_t i = 0; i < n; ++i) {
        void* outs[4] = {ez ? ez[i] : nullptr, wr ? wr[i] : nullptr, nullptr, nullptr};
        wake_status s = handles[i]->prec == WAKE_FP64 ? beam_fields_enqueue<double>(handles[i], outs, device_ptrs)
                                                      : beam_fields_enqueue<float>(handles[i], outs, device_ptrs);
        if (s != WAKE_OK) {
            cudaStreamSynchronize(handles[0]->st);
            return s;
        }
    }
    if (n > 0 && !device_ptrs) WK_CUDA(cudaStreamSynchronize(handles[0]->st));
    return WAKE_OK;
}

wake_status wake_run(wake_handle* h, void* beam_ez, void* beam_wr, void* ring_r) {
    WK_TRY(check_handle(h));
    WK_TRY(wake_step_slices(h, h->n_steps));
    WK_TRY(wake_get_beam_fields(h, beam_ez, beam_wr, nullptr, nullptr, 0));
    if (ring_r && h->d_dump[0])
        WK_CUDA(cudaMemcpyAsync(ring_r, h->d_dump[0], (size_t)h->n_steps * h->n * h->real_bytes(),
                                cudaMemcpyDeviceToHost, h->st));
    int32_t status = 0;
    WK_TRY(wake_get_progress(h, nullptr, &status, nullptr));
    if (status != 0) return stopped(status, "wake_run");
    return WAKE_OK;
}

wake_status wake_batch_step(int32_t n, wake_handle* const* handles, int32_t max_slices, int64_t time_budget_ns) {
    if (n < 0 || (n > 0 && !handles)) return fail(WAKE_EINVAL, "wake_batch_step: bad handle array");
    if (max_slices < 0 || time_budget_ns < 0) return fail(WAKE_EINVAL, "wake_batch_step: negative limit");
    if (n == 0 || max_slices == 0) return WAKE_OK;
    for (int32_t i = 0; i < n; ++i) {
        if (!handles[i]) return fail(WAKE_EINVAL, "wake_batch_step: handle %d is NULL", i);
        if (handles[i]->prec != handles[0]->prec || handles[i]->st != handles[0]->st)
            return fail(WAKE_EINVAL, "wake_batch_step: handles must share precision and stream");
    }
    if (handles[0]->prec == WAKE_FP64) return batch_impl<PrecF64>(n, handles, max_slices, time_budget_ns);
    return batch_impl<PrecMixed>(n, handles, max_slices, time_budget_ns);
}

wake_status wake_batch_run(int32_t n, wake_handle* const* handles) {
    return wake_batch_step(n, handles, 1 << 30, 0);
}

wake_status wake_batch_solve(int32_t n, wake_handle* const* handles, const wake_beam_desc* const* beams,
                             const int32_t* n_beams) {
    if (n < 0 || (n > 0 && !handles)) return fail(WAKE_EINVAL, "wake_batch_solve: bad handle array");
    if (n == 0) return WAKE_OK;
    for (int32_t i = 0; i < n; ++i) {
        if (!handles[i]) return fail(WAKE_EINVAL, "wake_batch_solve: handle %d is NULL", i);
        if (handles[i]->prec != handles[0]->prec || handles[i]->st != handles[0]->st)
            return fail(WAKE_EINVAL, "wake_batch_solve: handles must share precision and stream");
        if (beams && beams[i]) {
            if (!n_beams) return fail(WAKE_EINVAL, "wake_batch_solve: n_beams is required with beams");
            WK_TRY(check_new_beams(handles[i], beams[i], n_beams[i]));
        }
    }
    if (handles[0]->prec == WAKE_FP64) return batch_reset_run_impl<PrecF64>(n, handles, beams, n_beams);
    return batch_reset_run_impl<PrecMixed>(n, handles, beams, n_beams);
}

wake_status wake_batch_reset_run(int32_t n, wake_handle* const* handles) {
    return wake_batch_solve(n, handles, nullptr, nullptr);
}

wake_status wake_batch_progress(int32_t n, wake_handle* const* handles, int32_t* next_slice, int32_t* status) {
    if (n < 0 || (n > 0 && (!handles || !next_slice || !status)))
        return fail(WAKE_EINVAL, "wake_batch_progress: bad arrays");
    if (n == 0) return WAKE_OK;
    for (int32_t i = 0; i < n; ++i) {
        if (!handles[i]) return fail(WAKE_EINVAL, "wake_batch_progress: handle %d is NULL", i);
        if (handles[i]->st != handles[0]->st) return fail(WAKE_EINVAL, "wake_batch_progress: handles must share a stream");
    }
    cudaStream_t st = handles[0]->st;
    std::vector<const int32_t*> ctls(n);
    for (int32_t i = 0; i < n; ++i) ctls[i] = handles[i]->d_ctl;
    std::vector<int32_t> out(2 * (size_t)n);
    void* d = nullptr;
    const size_t pbytes = sizeof(const int32_t*) * (size_t)n, obytes = sizeof(int32_t) * 2 * (size_t)n;
    cudaMemPool_t pool = nullptr;
    WK_CUDA(wake_pool(&pool));
    WK_CUDA(cudaMallocFromPoolAsync(&d, pbytes + obytes, pool, st));
    const int32_t** d_ctls = static_cast<const int32_t**>(d);
    int32_t* d_out = reinterpret_cast<int32_t*>(static_cast<unsigned char*>(d) + pbytes);
    cudaError_t e = cudaMemcpyAsync(d_ctls, ctls.data(), pbytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_gather_ctl(d_ctls, n, d_out, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out.data(), d_out, obytes, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) return fail(WAKE_ECUDA, "wake_batch_progress: %s", cudaGetErrorString(e));
    for (int32_t i = 0; i < n; ++i) {
        next_slice[i] = out[2 * (size_t)i];
        status[i] = out[2 * (size_t)i + 1];
    }
    return WAKE_OK;
}

wake_status wake_get_march_times(wake_handle* h, int64_t* begin_ns, int64_t* end_ns) {
    WK_TRY(check_handle(h));
    int32_t ctl[CTL_N];
    WK_CUDA(cudaMemcpyAsync(ctl, h->d_ctl, sizeof(ctl), cudaMemcpyDeviceToHost, h->st));
    WK_CUDA(cudaStreamSynchronize(h->st));
    int64_t t0 = 0, t1 = 0;
    std::memcpy(&t0, ctl + CTL_T_BEGIN, sizeof(t0));
    std::memcpy(&t1, ctl + CTL_T_END, sizeof(t1));
    if (begin_ns) *begin_ns = t0;
    if (end_ns) *end_ns = t1;
    return WAKE_OK;
}

wake_status wake_get_device_bytes(wake_handle* h, int64_t* bytes) {
    WK_TRY(check_handle(h));
    if (!bytes) return fail(WAKE_EINVAL, "wake_get_device_bytes: bytes is NULL");
    *bytes = (int64_t)h->alloc_bytes;
    return WAKE_OK;
}

wake_status wake_get_ring_state(wake_handle* h, double* rho, double* ur, double* f_rho, double* f_ur) {
    WK_TRY(check_handle(h));
    if (h->prec == WAKE_FP64)
        return state_io<PrecF64>(h, true, 0, rho, ur, f_rho, f_ur, nullptr, nullptr, nullptr, nullptr);
    return state_io<PrecMixed>(h, true, 0, rho, ur, f_rho, f_ur, nullptr, nullptr, nullptr, nullptr);
}

wake_status wake_set_ring_state(wake_handle* h, int32_t slice, const double* rho, const double* ur,
                                const double* f_rho, const double* f_ur) {
    WK_TRY(check_handle(h));
    if (slice < 0 || slice > h->n_steps) return fail(WAKE_EINVAL, "wake_set_ring_state: slice out of range");
    if (!rho || !ur) return fail(WAKE_EINVAL, "wake_set_ring_state: rho and ur are required");
    if ((f_rho == nullptr) != (f_ur == nullptr))
        return fail(WAKE_EINVAL, "wake_set_ring_state: give both AB2 history arrays or neither");
    for (int32_t j = 0; j < h->n; ++j)
        if (!(rho[j] >= 0.0) || !std::isfinite(rho[j]) || !std::isfinite(ur[j]))
            return fail(WAKE_EINVAL, "wake_set_ring_state: ring %d has rho < 0 or non-finite state", j);
    if (h->prec == WAKE_FP64)
        return state_io<PrecF64>(h, false, slice, nullptr, nullptr, nullptr, nullptr, rho, ur, f_rho, f_ur);
    return state_io<PrecMixed>(h, false, slice, nullptr, nullptr, nullptr, nullptr, rho, ur, f_rho, f_ur);
}

wake_status wake_get_ring_dumps(wake_handle* h, void* r, void* ur, void* psi, void* dpsidr, void* dpsidz, void* bp,
                                void* bb) {
    WK_TRY(check_handle(h));
    void* outs[7] = {r, ur, psi, dpsidr, dpsidz, bp, bb};
    const size_t bytes = (size_t)h->n_steps * h->n * h->real_bytes();
    for (int k = 0; k < 7; ++k) {
        if (!outs[k]) continue;
        if (!h->d_dump[k]) return fail(WAKE_EINVAL, "wake_get_ring_dumps: dump %d was not requested at init", k);
        WK_CUDA(cudaMemcpyAsync(outs[k], h->d_dump[k], bytes, cudaMemcpyDeviceToHost, h->st));
    }
    WK_CUDA(cudaStreamSynchronize(h->st));
    return WAKE_OK;
}

wake_status wake_get_launch_config(wake_handle* h, int32_t* threads, int32_t* rings_per_thread,
                                   int32_t* blocks_per_wake) {
    WK_TRY(check_handle(h));
    const bool fast = h->fast_threads > 0;
    if (threads) *threads = fast ? h->fast_threads : h->threads;
    const int32_t cta_threads = h->threads * h->gm_cl;
    if (rings_per_thread) *rings_per_thread = fast ? h->fast_k : (h->n + cta_threads - 1) / cta_threads;
    if (blocks_per_wake) *blocks_per_wake = fast ? h->fast_cl : h->gm_cl;
    return WAKE_OK;
}

wake_status wake_fields_at_static(wake_handle* h, int64_t n, const double* r, void* ez, void* wr, void* bt,
                                  void* psi) {
    WK_TRY(check_handle(h));
    if (n < 0 || (n > 0 && !r)) return fail(WAKE_EINVAL, "wake_fields_at_static: bad query array");
    if (n > WAKE_STATIC_MAX_QUERIES)
        return fail(WAKE_EINVAL, "wake_fields_at_static: %lld queries exceed the static scratch limit of %d",
                    (long long)n, (int)WAKE_STATIC_MAX_QUERIES);
    int sdev = 0, cdev = 0;
    WK_CUDA(cudaStreamGetDevice(h->st, &sdev));
    WK_CUDA(cudaGetDevice(&cdev));
    if (sdev != cdev)
        return fail(WAKE_EINVAL, "wake_fields_at_static: the handle's device %d is not the current device %d", sdev,
                    cdev);
    int expected = 0;
    if (!g_static_busy.compare_exchange_strong(expected, 1))
        return fail(WAKE_EBUSY, "wake_fields_at_static: another call is using the static scratch");
    struct Release {
        ~Release() { g_static_busy.store(0); }
    } release;
    unsigned char* base = nullptr;
    WK_TRY(static_scratch(&base));
    int32_t next = 0, status = 0;
    WK_TRY(wake_get_progress(h, &next, &status, nullptr));
    if (status != 0) return stopped(status, "wake_fields_at_static");
    if (next >= h->n_steps)
        return fail(WAKE_EINVAL, "wake_fields_at_static: the window is finished (slice %d of %d)", next,
                    h->n_steps);
    if (n == 0) return WAKE_OK;
    void* outs[4] = {ez, wr, bt, psi};
    if (h->prec == WAKE_FP64) return fields_at_static_impl<PrecF64>(h, n, r, outs, base);
    return fields_at_static_impl<PrecMixed>(h, n, r, outs, base);
}

wake_status wake_set_beam_phase_space(wake_handle* h, const double* x, const double* y, const double* ux,
                                      const double* uy, const double* uz) {
    WK_TRY(check_handle(h));
    const int64_t nb = h->nb_total;
    if (nb > 0 && (!x || !y || !ux || !uy || !uz))
        return fail(WAKE_EINVAL, "wake_set_beam_phase_space: x, y, ux, uy, uz are required");
    for (int64_t k = 0; k < nb; ++k)
        if (!std::isfinite(x[k]) || !std::isfinite(y[k]) || !std::isfinite(ux[k]) || !std::isfinite(uy[k]) ||
            !std::isfinite(uz[k]))
            return fail(WAKE_EINVAL, "wake_set_beam_phase_space: particle %lld is not finite", (long long)k);
    if (nb == 0) return WAKE_OK;
    if (!h->d_ps[0])
        for (int c = 0; c < 5; ++c) WK_TRY(dalloc_t(h, (size_t)nb, &h->d_ps[c]));
    const double* src[5] = {x, y, ux, uy, uz};
    for (int c = 0; c < 5; ++c)
        WK_CUDA(cudaMemcpyAsync(h->d_ps[c], src[c], (size_t)nb * sizeof(double), cudaMemcpyHostToDevice, h->st));
    WK_CUDA(launch_beam_radius(nb, h->d_ps[0], h->d_ps[1], h->d_r, h->st));
    WK_CUDA(cudaStreamSynchronize(h->st));
    return WAKE_OK;
}

wake_status wake_get_beam_phase_space(wake_handle* h, double* x, double* y, double* xi, double* r, double* ux,
                                      double* uy, double* uz) {
    WK_TRY(check_handle(h));
    const int64_t nb = h->nb_total;
    if (nb == 0) return WAKE_OK;
    if (!h->d_ps[0] && (x || y || ux || uy || uz))
        return fail(WAKE_EINVAL, "wake_get_beam_phase_space: no phase space was set");
    double* dst[7] = {x, y, xi, r, ux, uy, uz};
    const double* src[7] = {h->d_ps[0], h->d_ps[1], h->d_xi, h->d_r, h->d_ps[2], h->d_ps[3], h->d_ps[4]};
    for (int c = 0; c < 7; ++c)
        if (dst[c]) WK_CUDA(cudaMemcpyAsync(dst[c], src[c], (size_t)nb * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    WK_CUDA(cudaStreamSynchronize(h->st));
    return WAKE_OK;
}

wake_status wake_push_beam(wake_handle* h, double dt) {
    WK_TRY(check_handle(h));
    WK_TRY(check_push(h, dt));
    if (h->prec == WAKE_FP64) return push_enqueue<double>(&h, 1, dt, h->st);
    return push_enqueue<float>(&h, 1, dt, h->st);
}

wake_status wake_batch_push_beam(int32_t n, wake_handle* const* handles, double dt) {
    if (n < 0 || (n > 0 && !handles)) return fail(WAKE_EINVAL, "wake_batch_push_beam: bad handle array");
    if (n == 0) return WAKE_OK;
    for (int32_t i = 0; i < n; ++i) {
        if (!handles[i]) return fail(WAKE_EINVAL, "wake_batch_push_beam: handle %d is NULL", i);
        if (handles[i]->st != handles[0]->st || handles[i]->prec != handles[0]->prec)
            return fail(WAKE_EINVAL, "wake_batch_push_beam: handles must share stream and precision");
        WK_TRY(check_push(handles[i], dt));
    }
    if (handles[0]->prec == WAKE_FP64) return push_enqueue<double>(handles, n, dt, handles[0]->st);
    return push_enqueue<float>(handles, n, dt, handles[0]->st);
}

void wake_destroy(wake_handle* h) {
    if (!h) return;
    free_all(h);
    delete h;
}

}  // extern "C"
