/*
 * phosim_bench.h — measurement helper of the phosim library (no counterpart in the paper).
 *
 * The photon path is bound by plain FP64/FP32 arithmetic, so its roofline needs the device's FMA issue
 * rate, which the vendor's published figures and the driver's copy/GEMM peaks do not give.
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

/* The device Philox4x32-10 the trace kernel draws from (Salmon et al., SC'11), applied to n counters with
   one key, for known-answer checks.  ctr: host, 4 n words; key: host, 2 words; out: host, 4 n words.
   Errors: INVALID_ARGUMENT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n);

#ifdef __cplusplus
}
#endif
#endif /* PHOSIM_BENCH_H */
