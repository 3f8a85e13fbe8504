// stage.cuh -- staging of a slice's beam arrays into shared memory with
// bulk asynchronous copies (the Blackwell/Hopper TMA unit, cp.async.bulk)
// completed on an mbarrier, double-buffered across slices.
//
// The beam is frozen during a solve (Sec. II) and binned by slice once, so
// slice n+1's particles -- radius-sorted radii, each particle's enclosed
// charge, the charge prefix the rings gather from -- sit contiguously in
// HBM before slice n is solved.  One elected thread issues three bulk copies
// for slice n+1 while the block works on slice n; the block waits on the
// buffer's mbarrier (bounded) before its beam steps of slice n+1.  Bulk
// copies move 16-byte aligned spans: a slice's span starts at the 16-byte
// boundary at or below its first particle and is rounded up to a multiple
// of 16 bytes, so the arrays carry 4 floats of padding past their end and
// particle q of the slice sits at element (b0 & 3) + q of the stage.
#pragma once

#include <stdint.h>

#include "common.cuh"

namespace gbwake {

// a bounded wait gives up after this long (a legitimate wait on a bulk copy
// of a few tens of KB from L2 or HBM takes microseconds)
constexpr uint64_t kStageWaitLimitNs = 250ull * 1000 * 1000;

// flags of WakeDev::stage
enum {
    STAGE_OK = 1,          // the beam arrays are 16-byte aligned and padded
    STAGE_TEST_STALL = 2   // test only: the copies of the first slice staged
                           // during a march are never issued, so its bounded
                           // wait runs out
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes the initialised barriers visible to the asynchronous proxy
__device__ __forceinline__ void mbar_fence_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// orders this thread's earlier generic-proxy accesses of shared memory
// before later asynchronous-proxy writes to it
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// bytes (a multiple of 16) from global src (16-byte aligned) to shared dst
// (16-byte aligned), completing on bar
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_test_parity(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t stage_now_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits until the phase of the given parity completed; false if it did not
// within kStageWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_test_parity(bar, parity)) return true;
    const uint64_t t0 = stage_now_ns();
    for (uint32_t it = 1;; ++it) {
        if (mbar_test_parity(bar, parity)) return true;
        if ((it & 31) == 0 && stage_now_ns() - t0 > kStageWaitLimitNs) return false;
    }
}

// Stage area of a block: two buffers of three arrays (radius, enclosed
// charge, charge prefix) of cap floats each, cap a multiple of 4 that
// includes the 16-byte alignment slack.
struct BeamStage {
    float* base;      // [2][3][cap]
    uint64_t* bar;    // [2] mbarriers
    int cap;          // floats per array (0: staging off)
    __device__ __forceinline__ float* arr(int buf, int which) const { return base + (size_t)(buf * 3 + which) * cap; }
    // a slice of m particles fits if its span (at most 3 floats of slack
    // before it and 3 after) does
    __device__ __forceinline__ bool fits(int m) const { return m > 0 && m + 6 <= cap; }
};

// shared-memory bytes of a stage of `particles` particles per slice
__host__ __device__ inline int stage_cap_floats(int particles) {
    return particles <= 0 ? 0 : (int)(((size_t)particles + 6 + 3) & ~(size_t)3);
}
__host__ __device__ inline size_t stage_smem_bytes(int particles) {
    return (size_t)2 * 3 * 4 * stage_cap_floats(particles);
}

// By one thread: bulk copies of the slice [b0, b0 + m) of br, bQs, bE into
// buffer buf, completing on its mbarrier.  With skip (test only) the
// barrier expects the bytes but no copy is issued.
__device__ __forceinline__ void stage_issue(const BeamStage& st, int buf, const float* br, const float* bqs,
                                            const float* be, int b0, int m, bool skip) {
    const int s0 = b0 & ~3;
    const int len = ((b0 - s0) + m + 3) & ~3;  // floats, a multiple of 4
    const uint32_t bytes = (uint32_t)len * 4u;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(st.bar + buf, 3u * bytes);
    if (skip) return;
    bulk_copy_g2s(st.arr(buf, 0), br + s0, bytes, st.bar + buf);
    bulk_copy_g2s(st.arr(buf, 1), bqs + s0, bytes, st.bar + buf);
    bulk_copy_g2s(st.arr(buf, 2), be + s0, bytes, st.bar + buf);
}

}  // namespace gbwake
