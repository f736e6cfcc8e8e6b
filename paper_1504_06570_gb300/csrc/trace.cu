// Trace kernel: one persistent launch follows every photon of every source from the top of the atmosphere
// into the pixel histogram (Peterson et al. 2015, Sec. 2.2-2.5).
//
// Work is cut into tiles of consecutive photons of one source.  Each warp takes tiles from a global
// counter (persistent grid sized to the SM count), so sources of 10^2 and 10^7 photons share one launch
// without imbalance; per-source moment sums are reduced over the tile in registers before one set of
// atomics, and pixel increments are aggregated across the warp's lanes that hit the same pixel.
#include <cstdio>

#include "phosim_device.cuh"
#include "phosim_scene.hpp"
#include "photon.cuh"

namespace phosim {

__device__ __forceinline__ void kahan_add(float& sum, float& comp, float v) {
    const float y = v - comp;
    const float t = sum + y;
    comp = (t - sum) - y;
    sum = t;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <bool MIXED>
__global__ void __launch_bounds__(256) trace_kernel(const __grid_constant__ TraceParams P) {
    const int lane = threadIdx.x & 31;
    unsigned long long cnt[kNumCounters];
#pragma unroll
    for (int k = 0; k < kNumCounters; ++k) cnt[k] = 0;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(P.tile_counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= P.n_tiles) break;
        const int src = tile_source(P, t, lane);
        const DSource& s = P.sources[src];
        const uint64_t j = t - P.tile_prefix[src];
        const uint64_t off = j * P.tile_photons;
        const uint32_t count = (uint32_t)min((uint64_t)P.tile_photons, s.count - off);
        const uint64_t first = s.first + off, rec_base = s.rec_off + off;
        const double rx = s.ref_x, ry = s.ref_y;
        // moment partials: FP64 in the plain path; FP32 with Kahan compensation in the mixed path
        double m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0, m5 = 0;
        float f1 = 0, f2 = 0, f3 = 0, f4 = 0, f5 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0;
        for (uint32_t base = 0; base < count; base += 32) {
            const uint32_t k = base + lane;
            const bool valid = k < count;
            PhotonOut R;
            R.flags = 0; R.pix = -1;
            if (valid) {
                trace_photon<MIXED>(P, s, src, first + k, R);
                if (P.records) {
                    phosim_photon_record rec;
                    rec.x = R.x; rec.y = R.y; rec.xc = R.xc; rec.yc = R.yc; rec.lambda = R.lam;
                    rec.flags = R.flags; rec.pix = R.pix;
                    P.records[rec_base + k] = rec;
                }
            }
            const bool det = valid && (R.flags & PHOSIM_F_DETECTED);
            const unsigned dmask = __ballot_sync(0xffffffffu, det);
            if (det) {
                const unsigned same = __match_any_sync(dmask, R.pix);
                if (lane == __ffs(same) - 1) atomicAdd(P.image + R.pix, (unsigned)__popc(same));
                const double dx = R.x - rx, dy = R.y - ry;
                if constexpr (MIXED) {
                    const float fx = (float)dx, fy = (float)dy;
                    kahan_add(f1, c1, fx);
                    kahan_add(f2, c2, fy);
                    kahan_add(f3, c3, fx * fx);
                    kahan_add(f4, c4, fx * fy);
                    kahan_add(f5, c5, fy * fy);
                    m0 += 1.0;
                } else {
                    m0 += 1.0; m1 += dx; m2 += dy; m3 += dx * dx; m4 += dx * dy; m5 += dy * dy;
                }
            }
            const unsigned vmask = __ballot_sync(0xffffffffu, valid);
            if (lane == 0) {
                cnt[0] += __popc(vmask);
                cnt[1] += __popc(dmask);
            }
            const uint32_t reason = valid ? ((R.flags >> 8) & 0xffu) : 0u;
#pragma unroll
            for (int q = 1; q <= 7; ++q) {
                const unsigned b = __ballot_sync(0xffffffffu, reason == (uint32_t)q);
                if (lane == 0) cnt[1 + q] += __popc(b);
            }
        }
        if constexpr (MIXED) {
            m1 = (double)f1 - (double)c1; m2 = (double)f2 - (double)c2; m3 = (double)f3 - (double)c3;
            m4 = (double)f4 - (double)c4; m5 = (double)f5 - (double)c5;
        }
        if (P.moments) {
            m0 = warp_sum(m0); m1 = warp_sum(m1); m2 = warp_sum(m2);
            m3 = warp_sum(m3); m4 = warp_sum(m4); m5 = warp_sum(m5);
            if (lane == 0 && m0 > 0.0) {
                double* M = P.moments + (size_t)src * PHOSIM_MOMENT_WORDS;
                atomicAdd(M + 0, m0); atomicAdd(M + 1, m1); atomicAdd(M + 2, m2);
                atomicAdd(M + 3, m3); atomicAdd(M + 4, m4); atomicAdd(M + 5, m5);
            }
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < kNumCounters; ++k)
            if (cnt[k]) atomicAdd(P.counters + k, cnt[k]);
    }
}

// Chief ray of each source (pupil centre, source centre direction, lambda_ref, no apertures): the
// reference point of the moment sums.
__global__ void chief_ray_kernel(const __grid_constant__ TraceParams P, DSource* sources, int n_src, double* moments) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_src) return;
    DSource& S = sources[s];
    const double nx = S.xi, ny = S.eta, nz = -sqrt(1.0 - nx * nx - ny * ny);
    const double l = (P.z_ent - P.pupil_z) / (-nz);
    double X[3] = {-nx * l, -ny * l, P.z_ent}, D[3] = {nx, ny, nz};
    PhotonOut R;
    R.flags = 0; R.pix = -1; R.x = R.y = 0.0;
    const uint4 zero = make_uint4(0u, 0u, 0u, 0u);
    optics<false, false>(P, X, D, P.lam_ref, zero, zero, zero, R);
    const bool ok = (R.flags & PHOSIM_F_DETECTED) != 0;
    S.ref_x = ok ? R.x : 0.0;
    S.ref_y = ok ? R.y : 0.0;
    if (moments) {
        moments[(size_t)s * PHOSIM_MOMENT_WORDS + 6] = S.ref_x;
        moments[(size_t)s * PHOSIM_MOMENT_WORDS + 7] = S.ref_y;
    }
}

cudaError_t launch_chief_rays(const TraceParams& P, DSource* sources, int n_src, double* moments, cudaStream_t st) {
    if (n_src <= 0) return cudaSuccess;
    chief_ray_kernel<<<(n_src + 127) / 128, 128, 0, st>>>(P, sources, n_src, moments);
    return cudaGetLastError();
}

cudaError_t launch_trace(const TraceParams& P, bool mixed, int blocks, int threads, cudaStream_t st) {
    if (mixed) trace_kernel<true><<<blocks, threads, 0, st>>>(P);
    else trace_kernel<false><<<blocks, threads, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t trace_occupancy(bool mixed, int threads, int* blocks_per_sm) {
    if (mixed) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<true>, threads, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel<false>, threads, 0);
}

}  // namespace phosim
