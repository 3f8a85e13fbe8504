// peaks.cu -- microbenchmarks of the on-chip rates the march kernels are
// bound by (include/wake_peaks.h): FP32 and FP64 fused multiply-add
// throughput, MUFU lg2 throughput, shared-memory load bandwidth, the latency
// of a dependent FP32 FMA, and the latency of a block barrier and of a
// thread-block-cluster barrier.  Plain user kernels timed with CUDA events
// (throughputs) or with the SM cycle counter (latencies); they change no
// setting of the GPU.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>

#include "../../include/wake_peaks.h"

namespace {

namespace cg = cooperative_groups;

constexpr int kChains = 8;  // independent dependency chains per thread

// n_iter x kChains FMAs per thread on independent accumulators; the result
// reaches memory only behind a test the inputs never pass, so nothing is
// folded away
template <class T>
__global__ void fma_kernel(T x, T y, int n_iter, T* sink) {
    T a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < n_iter; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
#pragma unroll
        for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == (T)-12345.0) sink[threadIdx.x] = s;
}

// MUFU: n_iter x kChains lg2.approx per thread (plus one add each to keep
// the chains in range: x -> lg2(x) + 3 has a fixed point near 3.3)
__global__ void lg2_kernel(int n_iter, float* sink) {
    float a[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) a[c] = 2.f + 0.01f * (threadIdx.x & 7) + c;
    for (int i = 0; i < n_iter; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            float r;
            asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a[c]));
            a[c] = r + 3.f;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += a[c];
    if (s == -12345.f) sink[threadIdx.x] = s;
}

// shared memory: every warp loads 32 consecutive float4 per step (512 bytes,
// no bank conflict), n_iter steps over a 16 KB buffer
__global__ void smem_kernel(int n_iter, float* sink) {
    __shared__ float4 buf[1024];
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) buf[i] = make_float4(i, i + 1, i + 2, i + 3);
    __syncthreads();
    float4 acc = make_float4(0, 0, 0, 0);
    int idx = threadIdx.x & 1023;
    for (int i = 0; i < n_iter; ++i) {
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float4 v = buf[(idx + u * 128) & 1023];
            acc.x += v.x;
            acc.y += v.y;
            acc.z += v.z;
            acc.w += v.w;
        }
        idx = (idx + 32) & 1023;
    }
    if (acc.x + acc.y + acc.z + acc.w == -12345.f) sink[threadIdx.x] = acc.x;
}

// one thread: n_iter dependent FMAs, cycles per FMA
__global__ void fma_latency_kernel(float x, float y, int n_iter, float* sink, long long* cycles) {
    float a = (float)threadIdx.x;
    const long long c0 = clock64();
    for (int i = 0; i < n_iter; ++i) {
        a = fmaf(a, x, y);
        a = fmaf(a, x, y);
        a = fmaf(a, x, y);
        a = fmaf(a, x, y);
    }
    const long long c1 = clock64();
    if (a == -12345.f) sink[0] = a;
    if (threadIdx.x == 0) *cycles = c1 - c0;
}

// n_iter block barriers (every thread also does one dependent add, as a
// scan step would), cycles per barrier from thread 0; and the SM clock
// from cycles over global-timer ns
__global__ void barrier_kernel(int n_iter, float* sink, long long* cycles, long long* ns) {
    float a = (float)threadIdx.x;
    __syncthreads();
    const long long c0 = clock64();
    uint64_t t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int i = 0; i < n_iter; ++i) {
        a += 1.f;
        __syncthreads();
    }
    const long long c1 = clock64();
    uint64_t t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (a == -12345.f) sink[0] = a;
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        *cycles = c1 - c0;
        *ns = (long long)(t1 - t0);
    }
}

// n_iter cluster barriers (arrive with release, wait with acquire, as the
// cluster march's exchanges use them), cycles per barrier from thread 0 of
// rank 0
__global__ void cluster_barrier_kernel(int n_iter, float* sink, long long* cycles) {
    cg::cluster_group cl = cg::this_cluster();
    float a = (float)threadIdx.x;
    cl.sync();
    const long long c0 = clock64();
    for (int i = 0; i < n_iter; ++i) {
        a += 1.f;
        cl.sync();
    }
    const long long c1 = clock64();
    if (a == -12345.f) sink[0] = a;
    if (threadIdx.x == 0 && cl.block_rank() == 0 && blockIdx.x == 0) *cycles = c1 - c0;
}

struct Scratch {
    float* sink = nullptr;
    long long* cyc = nullptr;
    ~Scratch() {
        if (sink) cudaFree(sink);
        if (cyc) cudaFree(cyc);
    }
};

// best of reps CUDA-event times of launch(), after one warm-up, in ms
template <class F>
cudaError_t time_best(F launch, int reps, float* best_ms) {
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    launch();
    e = cudaDeviceSynchronize();
    float best = 1e30f;
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        cudaEventRecord(e0);
        launch();
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *best_ms = best;
    return e;
}

}  // namespace

extern "C" int wake_measure_peaks(wake_peaks* out) {
    if (!out) return 1;
    std::memset(out, 0, sizeof(*out));
    int dev = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return 3;
    const int sms = prop.multiProcessorCount;
    Scratch s;
    if (cudaMalloc(&s.sink, 1024 * sizeof(double)) != cudaSuccess) return 2;
    if (cudaMalloc(&s.cyc, 4 * sizeof(long long)) != cudaSuccess) return 2;
    cudaError_t e;
    float ms = 0.f;
    // throughputs: 4 blocks of 256 threads per SM (every scheduler busy)
    const int blocks = 4 * sms, threads = 256;
    {
        const int it = 4096;
        e = time_best([&] { fma_kernel<float><<<blocks, threads>>>(1.0000001f, 1e-7f, it, s.sink); }, 5, &ms);
        if (e != cudaSuccess) return 3;
        out->fp32_tflops = 2.0 * 4 * kChains * (double)it * blocks * threads / (ms * 1e-3) / 1e12;
    }
    {
        const int it = 256;
        e = time_best([&] {
            fma_kernel<double><<<blocks, threads>>>(1.0000001, 1e-7, it, reinterpret_cast<double*>(s.sink));
        }, 5, &ms);
        if (e != cudaSuccess) return 3;
        out->fp64_tflops = 2.0 * 4 * kChains * (double)it * blocks * threads / (ms * 1e-3) / 1e12;
    }
    {
        const int it = 2048;
        e = time_best([&] { lg2_kernel<<<blocks, threads>>>(it, s.sink); }, 5, &ms);
        if (e != cudaSuccess) return 3;
        out->mufu_lg2_tops = (double)kChains * it * blocks * threads / (ms * 1e-3) / 1e12;
    }
    {
        const int it = 2048;
        e = time_best([&] { smem_kernel<<<blocks, threads>>>(it, s.sink); }, 5, &ms);
        if (e != cudaSuccess) return 3;
        out->smem_tbs = 8.0 * 16.0 * (double)it * blocks * threads / (ms * 1e-3) / 1e12;
    }
    long long h[2] = {0, 0};
    {
        const int it = 4096;
        fma_latency_kernel<<<1, 1>>>(1.0000001f, 1e-7f, it, s.sink, s.cyc);
        if (cudaMemcpy(h, s.cyc, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
        out->fma_latency_cycles = (double)h[0] / (4.0 * it);
    }
    {
        // one 512-thread block per SM, as the on-chip march runs
        const int it = 20000;
        barrier_kernel<<<sms, 512>>>(it, s.sink, s.cyc, s.cyc + 1);
        if (cudaMemcpy(h, s.cyc, 2 * sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
        out->syncthreads_cycles = (double)h[0] / it;
        out->sm_clock_mhz = h[1] > 0 ? (double)h[0] / (double)h[1] * 1e3 : 0.0;
        out->syncthreads_ns = out->sm_clock_mhz > 0 ? out->syncthreads_cycles / out->sm_clock_mhz * 1e3 : 0.0;
    }
    {
        // clusters of 8 CTAs of 256 threads, as the cluster march runs
        const int it = 4000;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(8 * (unsigned)(sms / 8), 1, 1);
        cfg.blockDim = dim3(256, 1, 1);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 8;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelEx(&cfg, cluster_barrier_kernel, it, s.sink, s.cyc);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return 3;
        if (cudaMemcpy(h, s.cyc, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
        out->cluster_barrier_cycles = (double)h[0] / it;
        out->cluster_barrier_ns =
            out->sm_clock_mhz > 0 ? out->cluster_barrier_cycles / out->sm_clock_mhz * 1e3 : 0.0;
    }
    out->sms = sms;
    return 0;
}
