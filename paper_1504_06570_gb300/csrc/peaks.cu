// FMA issue-rate probe (the denominator of the arithmetic roofline of the photon kernels) and the check
// entries of phosim_bench.h: the device Philox and the double-single primitives.
#include <cuda_runtime.h>

#include "phosim_bench.h"
#include "phosim_device.cuh"
#include "photon_ds.cuh"

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

namespace {

// Eight independent dependent chains of one double-single primitive per thread (op: 0 sum, 1 product, 2 fused
// multiply-add, 3 quotient, 4 square root); the constants keep every chain finite and normal.
template <int OP>
__global__ void ds_chains(int iterations, float seed, float* sink) {
    using namespace phosim;
    ds a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = ds_of(1.0 + 1e-3 * (double)(threadIdx.x + k) + (double)seed);
    const ds m = ds_of(0.99999988079071045), c = ds_of(1.000000059604645e-7), q = ds_of(1.0000001192092896);
    for (int i = 0; i < iterations; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (OP == 0) a[k] = a[k] + c;
            else if (OP == 1) a[k] = a[k] * m;
            else if (OP == 2) a[k] = dfma(a[k], m, c);
            else if (OP == 3) a[k] = a[k] / q;
            else a[k] = ds_sqrt(a[k]);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k].hi + a[k].lo;
    if (s == -1.f) sink[threadIdx.x] = s;      // never true; keeps the chains alive
}

}  // namespace

extern "C" phosim_status phosim_ds_rate(int op, int iterations, int blocks_per_sm, void* stream, double* tops) {
    if (!tops || op < 0 || op > 4 || iterations < 1 || blocks_per_sm < 1) return PHOSIM_ERR_INVALID_ARGUMENT;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PHOSIM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    float* sink = nullptr;
    if (cudaMalloc(&sink, 256 * sizeof(float)) != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_OUT_OF_MEMORY; }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int blocks = sms * blocks_per_sm;
    for (int rep = 0; rep < 2; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        switch (op) {
            case 0: ds_chains<0><<<blocks, 256, 0, st>>>(iterations, 0.f, sink); break;
            case 1: ds_chains<1><<<blocks, 256, 0, st>>>(iterations, 0.f, sink); break;
            case 2: ds_chains<2><<<blocks, 256, 0, st>>>(iterations, 0.f, sink); break;
            case 3: ds_chains<3><<<blocks, 256, 0, st>>>(iterations, 0.f, sink); break;
            default: ds_chains<4><<<blocks, 256, 0, st>>>(iterations, 0.f, sink); break;
        }
    }
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    *tops = 8.0 * (double)iterations * blocks * 256.0 / (ms * 1e-3) / 1e12;
    return PHOSIM_OK;
}

namespace {

// Random aligned 32-byte gathers: four independent index streams per thread (a multiplicative hash of a
// counter), each position the high word of hash x n_blocks (uniform over the buffer's 32-byte blocks).
__global__ void gather_chains(const float4* __restrict__ buf, uint32_t n_blocks, int gathers, float* sink) {
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t c[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) c[k] = t * 4u + (uint32_t)k;
    float acc = 0.f;
    for (int i = 0; i < gathers; i += 4) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            uint32_t h = c[k] * 0x9E3779B1u;
            h ^= h >> 15;
            h *= 0x85EBCA77u;
            h ^= h >> 13;
            const uint32_t b = __umulhi(h, n_blocks);
            const float4 x = __ldg(buf + 2 * (size_t)b), y = __ldg(buf + 2 * (size_t)b + 1);
            acc += x.x + y.w;
            c[k] += 0x01000193u;
        }
    }
    if (acc == -1.f) sink[threadIdx.x] = acc;      // never true; keeps the loads alive
}

}  // namespace

extern "C" phosim_status phosim_gather_rate(size_t bytes, int gathers, int blocks_per_sm, void* stream, double* gbs) {
    if (!gbs || gathers < 1 || blocks_per_sm < 1 || bytes % 32 || bytes < 32768 || bytes >= (128ull << 30))
        return PHOSIM_ERR_INVALID_ARGUMENT;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PHOSIM_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    void* buf = nullptr;
    float* sink = nullptr;
    if (cudaMalloc(&buf, bytes) != cudaSuccess || cudaMalloc(&sink, 256 * sizeof(float)) != cudaSuccess) {
        cudaFree(buf);
        (void)cudaGetLastError();
        return PHOSIM_ERR_OUT_OF_MEMORY;
    }
    const uint32_t n_blocks = (uint32_t)(bytes / 32);
    const int g = (gathers + 3) / 4 * 4;
    const int blocks = sms * blocks_per_sm;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaError_t e = cudaMemsetAsync(buf, 0, bytes, st);
    // warm-up launch (fills the L2 for a small buffer), then the timed one
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
        if (rep == 1) cudaEventRecord(e0, st);
        gather_chains<<<blocks, 256, 0, st>>>((const float4*)buf, n_blocks, g, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(buf);
    cudaFree(sink);
    if (e != cudaSuccess || ms <= 0.f) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    *gbs = 32.0 * (double)g * blocks * 256.0 / (ms * 1e-3) / 1e9;
    return PHOSIM_OK;
}

namespace {
__global__ void philox_kernel(const uint4* ctr, uint32_t k0, uint32_t k1, uint4* out, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = phosim::philox(ctr[i], k0, k1);
}
}  // namespace

extern "C" phosim_status phosim_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int n) {
    if (!ctr || !key || !out || n < 1) return PHOSIM_ERR_INVALID_ARGUMENT;
    void *dc = nullptr, *dout = nullptr;
    const size_t bytes = (size_t)n * sizeof(uint4);
    if (cudaMalloc(&dc, bytes) != cudaSuccess || cudaMalloc(&dout, bytes) != cudaSuccess) {
        cudaFree(dc);
        (void)cudaGetLastError();
        return PHOSIM_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaMemcpy(dc, ctr, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        philox_kernel<<<(n + 127) / 128, 128>>>((const uint4*)dc, key[0], key[1], (uint4*)dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
    cudaFree(dc);
    cudaFree(dout);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    return PHOSIM_OK;
}

namespace {
__global__ void ds_eval_kernel(int op, const double* a, const double* b, double* out, int n) {
    using namespace phosim;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ds x = ds_of(a[i]), y = ds_of(b[i]);
    ds r = ds_f(0.f);
    switch (op) {
        case 0: r = x + y; break;
        case 1: r = x - y; break;
        case 2: r = x * y; break;
        case 3: r = x / y; break;
        case 4: r = ds_sqrt(x); break;
        case 5: r = ds_rsqrt(x); break;
        case 6: r = dfma(x, y, x); break;
        case 7: {
            ds s, c;
            ds_sincos_2pi(ds_uniform((uint32_t)a[i]), s, c);
            out[2 * i] = ds_value(s);
            out[2 * i + 1] = ds_value(c);
            return;
        }
        case 8: r = ds_uniform((uint32_t)a[i]); break;
        case 9: {
            const float f = ds_floor(x);
            out[2 * i] = (double)f;
            out[2 * i + 1] = (double)ds_frac(x, f);
            return;
        }
        default: break;
    }
    out[i] = ds_value(r);
}
}  // namespace

extern "C" phosim_status phosim_ds_eval(int op, const double* a, const double* b, double* out, int n) {
    if (op < 0 || op > 9 || !a || !b || !out || n < 1) return PHOSIM_ERR_INVALID_ARGUMENT;
    const size_t in_bytes = (size_t)n * sizeof(double);
    const size_t out_bytes = (op == 7 || op == 9 ? 2 : 1) * in_bytes;
    double *da = nullptr, *db = nullptr, *dout = nullptr;
    if (cudaMalloc(&da, in_bytes) != cudaSuccess || cudaMalloc(&db, in_bytes) != cudaSuccess ||
        cudaMalloc(&dout, out_bytes) != cudaSuccess) {
        cudaFree(da);
        cudaFree(db);
        (void)cudaGetLastError();
        return PHOSIM_ERR_OUT_OF_MEMORY;
    }
    cudaError_t e = cudaMemcpy(da, a, in_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(db, b, in_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        ds_eval_kernel<<<(n + 127) / 128, 128>>>(op, da, db, dout, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, out_bytes, cudaMemcpyDeviceToHost);
    cudaFree(da);
    cudaFree(db);
    cudaFree(dout);
    if (e != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    return PHOSIM_OK;
}
