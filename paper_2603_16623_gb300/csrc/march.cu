// march.cu -- instantiations and launchers of the ring kernels.
#include <algorithm>

#include "march.h"
#include "march_launch.cuh"

namespace gbwake {

// Sec. II ring initialisation: ring j at the centre of its cell, weight
// n * centre * width (Eq. macroparticle_weight), self weight
// n * (centre * width / 2 - width^2 / 8) (the charge of the cell below the
// ring), at rest; computed in FP64 and rounded once to the state precision.
// float-float split of an FP64 value
__device__ __forceinline__ float2 split_ff(double v) {
    float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// With mobile ions (n_total = 2 n), ring n + j is the ion ring of cell j,
// with the signed charge weight -w (ions of density n / Z, charge Z).
// A radial density profile gives each cell its own density (cell_density,
// else the uniform density).
template <class R>
__global__ void ring_init_kernel(const double* __restrict__ edges, const double* __restrict__ cell_density,
                                 int32_t n, int32_t n_total, double density, R* w, R* wh, R* rho, R* rho_lo, R* ur,
                                 R* frho, R* fur, int32_t* rid, float4* ctab) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n_total; j += gridDim.x * blockDim.x) {
        const int32_t cell = j < n ? j : j - n;
        const double sign = j < n ? 1.0 : -1.0;
        const double dens = cell_density ? cell_density[cell] : density;
        double d = edges[cell + 1] - edges[cell];
        double c = 0.5 * (edges[cell] + edges[cell + 1]);
        double wj = sign * dens * c * d;
        double whj = sign * dens * (0.5 * c * d - 0.125 * d * d);
        w[j] = (R)wj;
        wh[j] = (R)whj;
        rho[j] = (R)c;
        rho_lo[j] = (R)(c - (double)(R)c);  // mixed path: rho = rho + rho_lo
        if (ctab) {     // mixed path: per-ring constants, float-float from FP64
            double l0 = log(c);
            float2 a = split_ff(c), b = split_ff(l0), e = split_ff(wj), f = split_ff(whj), g = split_ff(wj * l0);
            ctab[3 * j] = make_float4(a.x, a.y, b.x, b.y);
            ctab[3 * j + 1] = make_float4(e.x, e.y, f.x, f.y);
            // the spare slots: 1/w and 1/rho0 as the march takes them (the
            // same float reciprocals it would take of the same floats)
            ctab[3 * j + 2] = make_float4(g.x, g.y, __frcp_rn(e.x), __frcp_rn(a.x));
        }
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

// checkpoint export: sorted state -> double arrays by ring id
// (the mixed on-chip march keeps rho as rho + rho_lo)
template <class R>
__global__ void export_state_kernel(const int32_t* __restrict__ rid, const R* __restrict__ rho,
                                    const R* __restrict__ rho_lo, const R* __restrict__ ur,
                                    const R* __restrict__ frho, const R* __restrict__ fur, int32_t n,
                                    const float4* __restrict__ ctab, double* o_rho, double* o_ur, double* o_fr,
                                    double* o_fu) {
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int32_t id = rid[p];
        if (o_rho) o_rho[id] = (double)rho[p] + (ctab ? (double)rho_lo[p] : 0.0);
        if (o_ur) o_ur[id] = (double)ur[p];
        if (o_fr) o_fr[id] = (double)frho[p];
        if (o_fu) o_fu[id] = (double)fur[p];
    }
}

// checkpoint import: double arrays by ring id -> state in id order (buffer 0)
template <class R>
__global__ void import_state_kernel(const double* __restrict__ i_rho, const double* __restrict__ i_ur,
                                    const double* __restrict__ i_fr, const double* __restrict__ i_fu, int32_t n,
                                    const float4* __restrict__ ctab, R* rho, R* rho_lo, R* ur, R* frho, R* fur,
                                    int32_t* rid, int32_t* ctl, int32_t slice) {
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        R hi = (R)i_rho[j];
        rho[j] = hi;
        rho_lo[j] = (R)(i_rho[j] - (double)hi);
        ur[j] = (R)i_ur[j];
        frho[j] = i_fr ? (R)i_fr[j] : (R)0;
        fur[j] = i_fu ? (R)i_fu[j] : (R)0;
        rid[j] = j;
    }
    if (blockIdx.x == 0 && threadIdx.x < CTL_N) {
        int v = 0;
        if (threadIdx.x == CTL_NEXT) v = slice;
        if (threadIdx.x == CTL_FAIL) v = -1;
        if (threadIdx.x == CTL_PREV) v = i_fr != nullptr;
        ctl[threadIdx.x] = v;
    }
}

template <class R>
cudaError_t launch_export_state(const int32_t* rid, const R* rho, const R* rho_lo, const R* ur, const R* frho,
                                const R* fur, int32_t n, const float4* ctab, double* o_rho, double* o_ur,
                                double* o_fr, double* o_fu, cudaStream_t st) {
    export_state_kernel<R><<<(n + 255) / 256, 256, 0, st>>>(rid, rho, rho_lo, ur, frho, fur, n, ctab, o_rho, o_ur,
                                                           o_fr, o_fu);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_import_state(const double* i_rho, const double* i_ur, const double* i_fr, const double* i_fu,
                                int32_t n, const float4* ctab, R* rho, R* rho_lo, R* ur, R* frho, R* fur,
                                int32_t* rid, int32_t* ctl, int32_t slice, cudaStream_t st) {
    import_state_kernel<R><<<(n + 255) / 256, 256, 0, st>>>(i_rho, i_ur, i_fr, i_fu, n, ctab, rho, rho_lo, ur,
                                                           frho, fur, rid, ctl, slice);
    return cudaGetLastError();
}

template cudaError_t launch_export_state<double>(const int32_t*, const double*, const double*, const double*,
                                                 const double*, const double*, int32_t, const float4*, double*,
                                                 double*, double*, double*, cudaStream_t);
template cudaError_t launch_export_state<float>(const int32_t*, const float*, const float*, const float*,
                                                const float*, const float*, int32_t, const float4*, double*,
                                                double*, double*, double*, cudaStream_t);
template cudaError_t launch_import_state<double>(const double*, const double*, const double*, const double*, int32_t,
                                                 const float4*, double*, double*, double*, double*, double*,
                                                 int32_t*, int32_t*, int32_t, cudaStream_t);
template cudaError_t launch_import_state<float>(const double*, const double*, const double*, const double*, int32_t,
                                                const float4*, float*, float*, float*, float*, float*, int32_t*,
                                                int32_t*, int32_t, cudaStream_t);

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

// a global-memory march: one block per wake, or clusters of cluster_ctas
// (<= kMaxWakeCtas) blocks, one cluster per wake
template <class P>
static cudaError_t launch_gm(void (*kern)(const WakeDev<P>*, const int32_t*, int32_t, int32_t, int32_t),
                             const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                             int32_t max_slices, int32_t mode, int32_t threads, size_t smem, int32_t mb_cap,
                             int32_t cluster_ctas, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (cluster_ctas <= 1) {
        kern<<<n_wakes, threads, smem, st>>>(d_wakes, d_order, max_slices, mode, mb_cap);
        return cudaGetLastError();
    }
    if (cluster_ctas > kMaxWakeCtas) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_wakes * cluster_ctas), 1, 1);
    cfg.blockDim = dim3((unsigned)threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster_ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, d_wakes, d_order, max_slices, mode, mb_cap);
    if (e != cudaSuccess) return cudaGetLastError(), e;
    return cudaGetLastError();
}

template <class P>
cudaError_t launch_march(const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes, int32_t max_slices,
                         int32_t mode, int32_t threads, size_t smem, int32_t mb_cap, int32_t cluster_ctas,
                         cudaStream_t st) {
    return launch_gm(march_kernel<P>, d_wakes, d_order, n_wakes, max_slices, mode, threads, smem, mb_cap,
                     cluster_ctas, st);
}

int32_t march_stage_particles(int32_t threads, int32_t k_rings, int32_t cluster_ctas, int32_t want) {
    if (want <= 0) return 0;
    // Blocks an SM holds by registers (128 per thread, the kernels' budget
    // under __launch_bounds__(512)) and by threads.  The SM's 256 KB of L1
    // and shared memory must keep, as L1, room for the blocks' per-ring
    // constant tables (48 B per ring, gathered every slice; a stage that
    // pushed them out of L1 measured 8 % slower on the longest batched wake)
    // and a margin; each block also has 1 KB reserved and up to 2 KB of
    // static shared memory.  The stage gets what is left of the block's
    // share, at most the densest slice.
    constexpr int32_t kRegsPerSm = 65536, kRegsPerThread = 128, kThreadsPerSm = 2048;
    constexpr size_t kL1SmemPerSm = 256 * 1024, kMargin = 16 * 1024, kReservedAndStatic = 3 * 1024;
    constexpr size_t kMaxSmemPerBlock = 232448 - 4096, kRingConstBytes = 48;
    int32_t blocks = kRegsPerSm / (kRegsPerThread * threads);
    blocks = std::min(blocks, kThreadsPerSm / threads);
    if (blocks < 1) blocks = 1;
    const size_t ring = cluster_ctas > 1 ? cluster_smem_bytes(threads, k_rings) : fast_smem_bytes(threads, k_rings);
    const size_t l1_keep = (size_t)blocks * kRingConstBytes * threads * k_rings + kMargin;
    if (l1_keep >= kL1SmemPerSm) return 0;
    const size_t per_block = std::min((kL1SmemPerSm - l1_keep) / blocks - kReservedAndStatic, kMaxSmemPerBlock);
    if (per_block <= ring) return 0;
    int32_t fit = (int32_t)((per_block - ring) / (2 * 3 * 4)) - 9;  // stage_cap_floats slack
    if (fit < 32) return 0;
    return std::min(fit, want);
}

cudaError_t launch_march_cluster(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                                 int32_t max_slices, int32_t mode, int32_t threads, int32_t k_rings, int32_t cl,
                                 int32_t stage_particles, cudaStream_t st) {
    if (k_rings == 2)
        return launch_march_cluster_k2(d_wakes, d_order, n_wakes, max_slices, mode, threads, cl, stage_particles, st);
    if (k_rings == 4)
        return launch_cluster_k<4>(d_wakes, d_order, n_wakes, max_slices, mode, threads, cl, stage_particles, st);
    return launch_cluster_k<8>(d_wakes, d_order, n_wakes, max_slices, mode, threads, cl, stage_particles, st);
}

cudaError_t launch_march_fast(const WakeDev<PrecMixed>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                              int32_t max_slices, int32_t mode, int32_t threads, int32_t k_rings,
                              int32_t stage_particles, cudaStream_t st) {
    if (k_rings == 2)
        return launch_march_fast_k2(d_wakes, d_order, n_wakes, max_slices, mode, threads, stage_particles, st);
    if (k_rings == 4)
        return launch_fast_k<4>(d_wakes, d_order, n_wakes, max_slices, mode, threads, stage_particles, st);
    return launch_fast_k<8>(d_wakes, d_order, n_wakes, max_slices, mode, threads, stage_particles, st);
}

int64_t march_bounds_violations() {
#ifdef WAKE_BOUNDS_CHECK
    unsigned long long v = 0, z = 0;
    if (cudaMemcpyFromSymbol(&v, g_bounds_violations, sizeof(v)) != cudaSuccess) return -2;
    if (cudaMemcpyToSymbol(g_bounds_violations, &z, sizeof(z)) != cudaSuccess) return -2;
    return (int64_t)v;
#else
    return -1;
#endif
}

// (next slice, status) of n wakes into out[2n], one thread per wake
__global__ void gather_ctl_kernel(const int32_t* const* __restrict__ ctls, int32_t n, int32_t* __restrict__ out) {
    const int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        out[2 * i] = ctls[i][CTL_NEXT];
        out[2 * i + 1] = ctls[i][CTL_STATUS];
    }
}

cudaError_t launch_gather_ctl(const int32_t* const* ctls, int32_t n, int32_t* out, cudaStream_t st) {
    gather_ctl_kernel<<<(n + 127) / 128, 128, 0, st>>>(ctls, n, out);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_ring_init(const double* edges, const double* cell_density, int32_t n, int32_t n_total,
                             double density, R* w, R* wh, R* rho, R* rho_lo, R* ur, R* frho, R* fur, int32_t* rid,
                             float4* ctab, cudaStream_t st) {
    int grid = (n_total + 255) / 256;
    ring_init_kernel<R><<<grid, 256, 0, st>>>(edges, cell_density, n, n_total, density, w, wh, rho, rho_lo, ur,
                                              frho, fur, rid, ctab);
    return cudaGetLastError();
}

template <class P>
cudaError_t launch_march_ions(const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                              int32_t max_slices, int32_t mode, int32_t threads, size_t smem, int32_t mb_cap,
                              int32_t cluster_ctas, cudaStream_t st) {
    return launch_gm(march_ions_kernel<P>, d_wakes, d_order, n_wakes, max_slices, mode, threads, smem, mb_cap,
                     cluster_ctas, st);
}

template <class R>
cudaError_t launch_gather_by_id(const int32_t* rid, const R* src, R* dst, int32_t n, cudaStream_t st) {
    int grid = (n + 255) / 256;
    gather_by_id_kernel<R><<<grid, 256, 0, st>>>(rid, src, dst, n);
    return cudaGetLastError();
}

template cudaError_t launch_march<PrecF64>(const WakeDev<PrecF64>*, const int32_t*, int32_t, int32_t, int32_t,
                                           int32_t, size_t, int32_t, int32_t, cudaStream_t);
template cudaError_t launch_march<PrecMixed>(const WakeDev<PrecMixed>*, const int32_t*, int32_t, int32_t, int32_t,
                                             int32_t, size_t, int32_t, int32_t, cudaStream_t);
template cudaError_t launch_ring_init<double>(const double*, const double*, int32_t, int32_t, double, double*,
                                              double*, double*, double*, double*, double*, double*, int32_t*,
                                              float4*, cudaStream_t);
template cudaError_t launch_ring_init<float>(const double*, const double*, int32_t, int32_t, double, float*, float*,
                                             float*, float*, float*, float*, float*, int32_t*, float4*,
                                             cudaStream_t);
template <class P>
cudaError_t launch_march_rk4(const WakeDev<P>* d_wakes, const int32_t* d_order, int32_t n_wakes,
                             int32_t max_slices, int32_t mode, int32_t threads, size_t smem, int32_t mb_cap,
                             int32_t cluster_ctas, cudaStream_t st) {
    return launch_gm(march_rk4_kernel<P>, d_wakes, d_order, n_wakes, max_slices, mode, threads, smem, mb_cap,
                     cluster_ctas, st);
}

template cudaError_t launch_march_rk4<PrecF64>(const WakeDev<PrecF64>*, const int32_t*, int32_t, int32_t, int32_t,
                                               int32_t, size_t, int32_t, int32_t, cudaStream_t);
template cudaError_t launch_march_rk4<PrecMixed>(const WakeDev<PrecMixed>*, const int32_t*, int32_t, int32_t,
                                                 int32_t, int32_t, size_t, int32_t, int32_t, cudaStream_t);
template cudaError_t launch_march_ions<PrecF64>(const WakeDev<PrecF64>*, const int32_t*, int32_t, int32_t, int32_t,
                                                int32_t, size_t, int32_t, int32_t, cudaStream_t);
template cudaError_t launch_march_ions<PrecMixed>(const WakeDev<PrecMixed>*, const int32_t*, int32_t, int32_t,
                                                  int32_t, int32_t, size_t, int32_t, int32_t, cudaStream_t);
template cudaError_t launch_gather_by_id<double>(const int32_t*, const double*, double*, int32_t, cudaStream_t);
template cudaError_t launch_gather_by_id<float>(const int32_t*, const float*, float*, int32_t, cudaStream_t);

}  // namespace gbwake
