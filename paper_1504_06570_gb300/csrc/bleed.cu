// Saturation and bleeding of a finished image (Peterson et al. 2015, Sec. 2.5): charge above the full well
// moves along the row to the closest pixels with room, never across the centre implant, and is lost once
// the half-row is full.  One thread walks one half-row; the electron-by-electron alternation (left, right,
// left, ...) at each distance is applied in closed form.
#include <cstdint>

#include <cuda_runtime.h>

#include "phosim.h"

namespace {

__global__ void bleed_kernel(uint32_t* __restrict__ img, int nx, int ny, uint32_t w, unsigned long long* removed) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * ny) return;
    const int y = t >> 1, half = t & 1;
    const int lo = half ? nx / 2 : 0, hi = half ? nx : nx / 2;
    uint32_t* row = img + (size_t)y * nx;
    unsigned long long lost = 0;
    for (int x = lo; x < hi; ++x) {
        if (row[x] <= w) continue;
        unsigned long long e = row[x] - w;
        row[x] = w;
        for (int d = 1; e > 0; ++d) {
            const bool has_l = x - d >= lo, has_r = x + d < hi;
            if (!has_l && !has_r) { lost += e; break; }
            const unsigned long long cl = (has_l && row[x - d] < w) ? w - row[x - d] : 0;
            const unsigned long long cr = (has_r && row[x + d] < w) ? w - row[x + d] : 0;
            const unsigned long long m = cl < cr ? cl : cr;
            unsigned long long gl, gr;
            if (e <= 2 * m) {                     // alternating pairs, the odd one to the left
                gl = (e + 1) / 2;
                gr = e / 2;
            } else {                              // one side fills; the other takes what it can
                gl = m + (cl > m ? (e - 2 * m < cl - m ? e - 2 * m : cl - m) : 0);
                gr = m + (cr > m ? (e - 2 * m < cr - m ? e - 2 * m : cr - m) : 0);
            }
            if (has_l) row[x - d] += (uint32_t)gl;
            if (has_r) row[x + d] += (uint32_t)gr;
            e -= gl + gr;
        }
    }
    if (removed && lost) atomicAdd(removed, lost);
}

}  // namespace

extern "C" phosim_status phosim_bleed(uint32_t* image, int nx, int ny, uint32_t full_well, unsigned long long* removed,
                                      void* stream) {
    if (!image || nx < 2 || ny < 1) return PHOSIM_ERR_INVALID_ARGUMENT;
    const int threads = 128, n = 2 * ny;
    bleed_kernel<<<(n + threads - 1) / threads, threads, 0, (cudaStream_t)stream>>>(image, nx, ny, full_well, removed);
    if (cudaGetLastError() != cudaSuccess) return PHOSIM_ERR_CUDA;
    return PHOSIM_OK;
}
