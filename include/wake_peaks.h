/*
 * wake_peaks.h -- measured on-chip peaks of the GPU that libwake.so runs on.
 *
 * The march of a wake (Sec. III's per-slice chain: sort, prefix sums,
 * fields, B_theta^(p), push) is not a dense contraction and barely touches
 * HBM; its roofline is set by FP32 issue, the special-function unit (one
 * logarithm per ring and slice), shared-memory bandwidth, and -- for one
 * wake -- by the latency of the block and cluster barriers that separate
 * its steps.  The paper has no counterpart: this entry measures those
 * rates so that achieved work can be stated as a fraction of them.
 */
#ifndef GBWAKE_WAKE_PEAKS_H
#define GBWAKE_WAKE_PEAKS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double fp32_tflops;            /* FP32 FMA throughput, 2 flop per FMA, TFLOP/s  */
    double fp64_tflops;            /* FP64 FMA throughput, TFLOP/s                  */
    double mufu_lg2_tops;          /* lg2.approx throughput, 1e12 per second        */
    double smem_tbs;               /* shared-memory load bandwidth, TB/s (all SMs)  */
    double fma_latency_cycles;     /* one dependent FP32 FMA, SM cycles             */
    double syncthreads_cycles;     /* one __syncthreads of a 512-thread block       */
    double syncthreads_ns;
    double cluster_barrier_cycles; /* one cluster barrier of 8 CTAs x 256 threads   */
    double cluster_barrier_ns;
    double sm_clock_mhz;           /* SM clock seen by the barrier kernel           */
    int32_t sms;                   /* streaming multiprocessors                    */
} wake_peaks;

/* Runs the microbenchmarks on the current device (a few tens of ms; the
   device is synchronised) and fills *out.  Throughputs: best of 5 CUDA-event
   timed launches of 4 blocks of 256 threads per SM, each thread running 8
   independent chains.  Latencies: the SM cycle counter over 4096 dependent
   FMAs of one thread, 20,000 barriers of one 512-thread block per SM, and
   4000 barriers of 8-CTA clusters; ns from the SM clock measured by the
   same kernel against the GPU's global timer.  Allocates and frees a few
   KB of device memory.  Returns 0, 1 (NULL out), 2 (allocation failed) or
   3 (a CUDA call failed); nothing throws. */
int wake_measure_peaks(wake_peaks *out);

#ifdef __cplusplus
}
#endif
#endif /* GBWAKE_WAKE_PEAKS_H */
