// FMA issue-rate probe: the denominator of the arithmetic roofline of the photon kernels.
#include <cuda_runtime.h>

#include "phosim_bench.h"

namespace {

template <class T>
__global__ void fma_chains(int iterations, T seed, T* sink) {
    T a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = seed + (T)(threadIdx.x + k);
    const T m = (T)0.999999, c = (T)1e-7;
    for (int i = 0; i < iterations; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) a[k] = fma(a[k], m, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += a[k];
    if (s == (T)-1.0) sink[threadIdx.x] = s;     // never true; keeps the chains alive
}

}  // namespace

extern "C" phosim_status phosim_fma_rate(int fp64, int iterations, int blocks_per_sm, void* stream, double* tflops) {
    if (!tflops || iterations < 1 || blocks_per_sm < 1) return PHOSIM_ERR_INVALID_ARGUMENT;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PHOSIM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    void* sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(double)) != cudaSuccess) return PHOSIM_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * blocks_per_sm;
    // warm-up launch, then the timed one
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        if (fp64) fma_chains<double><<<blocks, 256, 0, st>>>(iterations, 1.0, (double*)sink);
        else fma_chains<float><<<blocks, 256, 0, st>>>(iterations, 1.0f, (float*)sink);
    }
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    *tflops = 2.0 * 16.0 * (double)iterations * blocks * 256.0 / (ms * 1e-3) / 1e12;
    return PHOSIM_OK;
}
