/*
 * phosim_bench.h — measurement and check helpers of the phosim library (no counterpart in the paper).
 *
 * The photon path is bound by plain FP64/FP32 arithmetic, so its roofline needs the device's FMA issue
 * rate, which the vendor's published figures and the copy/GEMM peaks do not give.  The other entries
 * expose device building blocks (the random-number generator, the double-single arithmetic) to tests.
 */
#ifndef PHOSIM_BENCH_H
#define PHOSIM_BENCH_H

#include "phosim.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Sustained FMA throughput of the current device, in TFLOP/s (2 flops per FMA): every thread of a grid of
   blocks_per_sm x SM-count blocks of 256 threads runs 16 independent dependent-FMA chains of `iterations`
   steps in FP64 (fp64 != 0) or FP32.  Blocks on `stream` and synchronises it.
   Errors: INVALID_ARGUMENT (null output, iterations < 1), CUDA. */
phosim_status phosim_fma_rate(int fp64, int iterations, int blocks_per_sm, void* stream, double* tflops);

/* Sustained throughput of one double-single primitive of the PHOSIM_MIXED_DS path on the current device, in
   tera-operations per second: every thread of a grid of blocks_per_sm x SM-count blocks of 256 threads runs 8
   independent dependent chains of `iterations` operations.  op: 0 sum, 1 product, 2 fused multiply-add
   (a b + c, one normalisation), 3 quotient, 4 square root.  With the FP64-level operation mix of a workload
   (the oracle's count of its sums, products, quotients and roots), these rates give the operation rate an
   implementation doing every such operation in double-single could reach.  Blocks on `stream` and
   synchronises it.  Errors: INVALID_ARGUMENT (unknown op, null output, iterations < 1), OUT_OF_MEMORY, CUDA. */
phosim_status phosim_ds_rate(int op, int iterations, int blocks_per_sm, void* stream, double* tops);

/* Sustained rate of random 32-byte gathers from a device buffer of `bytes` bytes (a multiple of 32, at least
   32 KiB, below 128 GiB), in GB/s of gathered bytes (1e9 bytes per second): every thread of a grid of
   blocks_per_sm x SM-count blocks of 256 threads reads `gathers` aligned 32-byte blocks at hashed positions,
   four independent streams at a time, the gather shape of the atmosphere stage's screen lookups (one 2 x 2
   block of FP32 gradient pairs per lookup).  A buffer far larger than the L2 gives the HBM's random-gather
   ceiling (each 32-byte lookup fetches whole DRAM bursts); one far smaller gives the L2's.  The buffer is
   allocated, zeroed and freed inside the call.  Blocks on `stream` and synchronises it.
   Errors: INVALID_ARGUMENT (size out of range or not a multiple of 32, gathers < 1, null output),
   OUT_OF_MEMORY, CUDA. */
phosim_status phosim_gather_rate(size_t bytes, int gathers, int blocks_per_sm, void* stream, double* gbs);

/* The device Philox4x32-10 the trace kernel draws from (Salmon et al., SC'11), applied to n counters with
   one key, for known-answer checks.  ctr: host, 4 n words; key: host, 2 words; out: host, 4 n words.
   Errors: INVALID_ARGUMENT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n);

/* The double-single primitives of the PHOSIM_MIXED_DS path applied element-wise, for accuracy checks
   against FP64.  Each input double is first rounded to the nearest double-single pair; each result is
   returned as the double hi + lo.  op: 0 a + b, 1 a - b, 2 a b, 3 a / b, 4 sqrt(a), 5 1 / sqrt(a),
   6 a b + a, 7 (sin, cos) of 2 pi u with u = (a + 1/2) 2^-32 for the 32-bit integer a (2 n outputs),
   8 u itself, 9 (floor(a), a - floor(a)) (2 n outputs).  a, b: host, n values (b unused by ops 4, 5, 7-9);
   out: host, n or 2 n values.  Errors: INVALID_ARGUMENT (unknown op, null pointer, n < 1), OUT_OF_MEMORY,
   CUDA. */
phosim_status phosim_ds_eval(int op, const double* a, const double* b, double* out, int n);

/* Per-kernel timing of phosim_trace.  While on, each phosim_trace call on the scene launches its kernels
   one by one (no CUDA graph) with a CUDA event recorded on the call's stream before and after each launch.
   phosim_stage_times waits for the events of the scene's last phosim_trace call and returns the summed
   milliseconds of each kernel: ms[0] chief rays, ms[1] the one-kernel trace (PHOSIM_PLAIN_FP64,
   PHOSIM_MIXED), ms[2] the entry stage, ms[3] the optics stage and ms[4] the bundle stage (background
   bundles) of the two-kernel double-single path (PHOSIM_MIXED_DS); kernels the call did not launch read 0.
   n >= 5.  Errors: INVALID_ARGUMENT (null scene or output, n < 5), CUDA. */
phosim_status phosim_set_stage_timing(phosim_scene* scene, int on);
phosim_status phosim_stage_times(phosim_scene* scene, double* ms, int n);

#ifdef __cplusplus
}
#endif
#endif /* PHOSIM_BENCH_H */
