// Trace kernel: one persistent launch follows every photon of every source from the top of the atmosphere
// into the pixel histogram (Peterson et al. 2015, Sec. 2.2-2.5).
//
// Work is cut into tiles of consecutive photons of one source.  Each warp takes tiles from a global
// counter (persistent grid sized to the SM count), so sources of 10^2 and 10^7 photons share one launch
// without imbalance; per-source moment sums are reduced over the tile in registers before one set of
// atomics, and pixel increments are aggregated across the warp's lanes that hit the same pixel.
#include <cstdio>
#include <type_traits>

#include "phosim_device.cuh"
#include "phosim_scene.hpp"
#include "photon.cuh"
#include "photon_ds.cuh"

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

// Per-lane accumulation state of one tile: the count of detected photons and the moment partials about the
// source's chief-ray position (FP64 in the plain path; FP32 with Kahan compensation in the mixed paths).
template <bool MIXED> struct TileAcc {
    uint32_t n;
    double m[5];
};
template <> struct TileAcc<true> {
    uint32_t n;
    float f[5], c[5];
};

#ifndef PHOSIM_CONSUME
#define PHOSIM_CONSUME __forceinline__
#endif
// resident blocks of 256 threads per SM the register allocation is sized for: the FP64 kernels are bound by
// the FP64 pipe, the double-single kernel by latency (more resident warps hide its dependent FP32 chains)
#ifndef PHOSIM_TRACE_MIN_BLOCKS
#define PHOSIM_TRACE_MIN_BLOCKS 2
#endif
#ifndef PHOSIM_TRACE_MIN_BLOCKS_DS
#define PHOSIM_TRACE_MIN_BLOCKS_DS 8
#endif

// Account for one batch of up to 32 photons that went through a photon path: record, image, moments and
// the detected / dropped counters (cnt: the warp's counters in shared memory, updated by lane 0).  Every
// lane of the warp calls it.  Out is PhotonOut (FP64 positions) or PhotonOutS (double-single positions);
// rx, ry are the source's chief-ray position in the same type.
template <bool MIXED, class Out, class Ref>
__device__ PHOSIM_CONSUME void consume(const TraceParams& P, const Out& R, bool valid, uint64_t rec_index,
                                        Ref rx, Ref ry, int lane, TileAcc<MIXED>& A, unsigned long long* cnt) {
    constexpr bool DS = std::is_same<Out, PhotonOutS>::value;
    if (valid && P.records) {
        phosim_photon_record rec;
        if constexpr (DS) {
            rec.x = ds_value(R.x); rec.y = ds_value(R.y); rec.xc = ds_value(R.xc); rec.yc = ds_value(R.yc);
            rec.lambda = (double)R.lam;
        } else {
            rec.x = R.x; rec.y = R.y; rec.xc = R.xc; rec.yc = R.yc; rec.lambda = R.lam;
        }
        rec.flags = R.flags; rec.pix = R.pix;
        P.records[rec_index] = rec;
    }
    const bool det = valid && (R.flags & PHOSIM_F_DETECTED);
    const unsigned dmask = __ballot_sync(0xffffffffu, det);
    if (det) {
        const unsigned same = __match_any_sync(dmask, R.pix);
        if (lane == __ffs(same) - 1) atomicAdd(P.image + R.pix, (unsigned)__popc(same));
        A.n += 1;
        if constexpr (MIXED) {
            float fx, fy;
            if constexpr (DS) {
                fx = (R.x - rx).hi;
                fy = (R.y - ry).hi;
            } else {
                fx = (float)(R.x - rx);
                fy = (float)(R.y - ry);
            }
            kahan_add(A.f[0], A.c[0], fx);
            kahan_add(A.f[1], A.c[1], fy);
            kahan_add(A.f[2], A.c[2], fx * fx);
            kahan_add(A.f[3], A.c[3], fx * fy);
            kahan_add(A.f[4], A.c[4], fy * fy);
        } else {
            const double dx = R.x - rx, dy = R.y - ry;
            A.m[0] += dx; A.m[1] += dy; A.m[2] += dx * dx; A.m[3] += dx * dy; A.m[4] += dy * dy;
        }
    }
    if (lane == 0) cnt[1] += __popc(dmask);
    const uint32_t reason = valid ? ((R.flags >> 8) & 0xffu) : 0u;
#pragma unroll
    for (int q = 1; q <= 8; ++q) {
        const unsigned b = __ballot_sync(0xffffffffu, reason == (uint32_t)q);
        if (lane == 0) cnt[1 + q] += __popc(b);
    }
}

// MODE: kPlain (every step FP64), kMixed (FP64 optics, FP32 sampling / deflections / sensor), kDS (the
// mixed path with the FP64 parts in double-single arithmetic on the FP32 pipes)
constexpr int kPlain = 0, kMixed = 1, kDS = 2;
constexpr int min_blocks(int mode) { return mode == kDS ? PHOSIM_TRACE_MIN_BLOCKS_DS : PHOSIM_TRACE_MIN_BLOCKS; }

template <int MODE>
__global__ void __launch_bounds__(256, min_blocks(MODE)) trace_kernel(const __grid_constant__ TraceParams P) {
    constexpr bool MIXED = MODE != kPlain;
    constexpr bool DS = MODE == kDS;
    using Out = typename std::conditional<DS, PhotonOutS, PhotonOut>::type;
    // With early rejection most photons stop after their wavelength is drawn.  Survivors are queued per
    // warp (photon offsets within the tile, in shared memory) and propagated 32 at a time, so the expensive
    // part runs with full warps instead of the few lanes that survived in each batch.  Lane-uniform state
    // (the launch counters, the double-single source constants) also lives in shared memory, which leaves
    // the registers to the photon path.
    __shared__ uint32_t queue_mem[kWarpsPerBlock][64];
    __shared__ unsigned long long cnt_mem[kWarpsPerBlock][kNumCounters];
    __shared__ SourceS src_mem[DS ? kWarpsPerBlock : 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* queue = queue_mem[warp];
    unsigned long long* cnt = cnt_mem[warp];
    const unsigned lanes_below = (1u << lane) - 1u;
    const bool early = (P.flags & PHOSIM_EARLY_REJECT) != 0;
    if (lane < kNumCounters) cnt[lane] = 0;
    __syncwarp();
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
        if constexpr (DS) {
            if (lane == 0) src_mem[warp] = source_s(s);
            __syncwarp();
        }
        const SourceS& ss = src_mem[DS ? warp : 0];
        TileAcc<MIXED> A = {};
        int queued = 0;
        uint32_t base = 0;
        for (;;) {
            if (base < count) {
                const uint32_t k = base + lane;
                const bool valid = k < count;
                const unsigned vmask = __ballot_sync(0xffffffffu, valid);
                if (lane == 0) cnt[0] += __popc(vmask);
                bool go_on = valid;
                if (early) {
                    // stage 1: the early coating decision alone
                    Out R;
                    int rej = -1;
                    if constexpr (DS) {
                        float lam = 0.f;
                        if (valid) rej = early_reject_certain_f(P, ss, src, ray_of(ss.bundle, first + k), lam);
                        R.x = R.y = R.xc = R.yc = ds_f(0.f);
                        R.lam = lam;
                    } else {
                        double lam = 0.0;
                        if (valid) rej = early_reject_surface<MIXED>(P, s, src, first + k, lam);
                        R.x = R.y = R.xc = R.yc = 0.0;
                        R.lam = lam;
                    }
                    go_on = valid && rej < 0;
                    R.flags = valid ? lost(PHOSIM_LOST_COATING, rej) : 0u;
                    R.pix = -1;
                    if constexpr (DS) consume<MIXED>(P, R, valid && !go_on, rec_base + k, ss.ref_x, ss.ref_y, lane, A, cnt);
                    else consume<MIXED>(P, R, valid && !go_on, rec_base + k, s.ref_x, s.ref_y, lane, A, cnt);
                }
                // queue the photons that go on
                const unsigned gmask = __ballot_sync(0xffffffffu, go_on);
                if (go_on) queue[queued + __popc(gmask & lanes_below)] = k;
                queued += __popc(gmask);
                base += 32;
                __syncwarp();
            }
            const bool drained = base >= count;
            if (queued >= 32 || (drained && queued > 0)) {
                // stage 2: propagate a warp's worth of queued photons
                const int take = queued < 32 ? queued : 32;
                queued -= take;
                const bool v = lane < take;
                const uint32_t kk = v ? queue[queued + lane] : 0u;
                __syncwarp();
                Out Q;
                Q.flags = 0; Q.pix = -1;
                if constexpr (DS) {
                    if (v) trace_photon_ds(P, ss, src, first + kk, Q);
                    consume<MIXED>(P, Q, v, rec_base + kk, ss.ref_x, ss.ref_y, lane, A, cnt);
                } else {
                    if (v) trace_photon<MIXED>(P, s, src, first + kk, Q);
                    consume<MIXED>(P, Q, v, rec_base + kk, s.ref_x, s.ref_y, lane, A, cnt);
                }
            }
            if (drained && queued == 0) break;
        }
        if (P.moments) {
            double m[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                if constexpr (MIXED) m[q] = (double)A.f[q] - (double)A.c[q];
                else m[q] = A.m[q];
                m[q] = warp_sum(m[q]);
            }
            const double m0 = warp_sum((double)A.n);
            if (lane == 0 && m0 > 0.0) {
                double* M = P.moments + (size_t)src * PHOSIM_MOMENT_WORDS;
                atomicAdd(M + 0, m0);
#pragma unroll
                for (int q = 0; q < 5; ++q) atomicAdd(M + 1 + q, m[q]);
            }
        }
        __syncwarp();
    }
    __syncwarp();
    if (lane < kNumCounters && cnt[lane]) atomicAdd(P.counters + lane, cnt[lane]);
}

// ---------------------------------------------------------------------------------------------------------
// The double-single path in two kernels.  One megakernel that samples, crosses the atmosphere and traces
// the optics keeps the whole path's code and live state at once; on this GPU its FP32 instruction stream
// outruns the instruction cache and its registers spill.  Split at the entrance plane of the telescope
// (the staging of wavefront path tracers), each half has a smaller code footprint and fewer live values:
//   ds_entry_kernel:  early rejection, sampling and the layers for the tiles of one chunk; survivors append
//                     their entrance-plane state (64 bytes) to a buffer in device memory;
//   ds_optics_kernel: the surfaces, the sensor and the accounting, one state per thread.  The warps of a
//                     block take the surfaces in step (a barrier after each surface): warps left to run
//                     freely spread over the whole surface code and the SM's instruction cache misses.
// The per-photon arithmetic and its order are those of trace_photon_ds, so both give the same results.  The
// optics and bundle stages are in trace_optics.cu, compiled with the double-single quotient and roots inline.
// ---------------------------------------------------------------------------------------------------------
#ifndef PHOSIM_DS_ENTRY_MIN_BLOCKS
#define PHOSIM_DS_ENTRY_MIN_BLOCKS 6
#endif

// Accounting of photons the entry stage stops (the dynamic transmission test): record and loss counters.
// None is detected there, so unlike consume() it carries no moment partials through the tile.
// (only_reason > 0: every lane with v was lost for that reason, one ballot counts them)
__device__ __forceinline__ void account_lost(const TraceParams& P, uint32_t flags, float lam, bool v, uint64_t rec_index,
                                             int lane, unsigned long long* cnt, int only_reason = 0) {
    if (v && P.records) {
        phosim_photon_record rec;
        rec.x = rec.y = rec.xc = rec.yc = 0.0;
        rec.lambda = (double)lam;
        rec.flags = flags; rec.pix = -1;
        P.records[rec_index] = rec;
    }
    if (only_reason > 0) {
        const unsigned b = __ballot_sync(0xffffffffu, v);
        if (lane == 0) cnt[1 + only_reason] += __popc(b);
        return;
    }
    const uint32_t reason = v ? ((flags >> 8) & 0xffu) : 0u;
#pragma unroll
    for (int q = 1; q <= 8; ++q) {
        const unsigned b = __ballot_sync(0xffffffffu, reason == (uint32_t)q);
        if (lane == 0) cnt[1 + q] += __popc(b);
    }
}

__global__ void __launch_bounds__(256, PHOSIM_DS_ENTRY_MIN_BLOCKS) ds_entry_kernel(const __grid_constant__ TraceParams P,
                                                                                   const DSStage S) {
    __shared__ uint32_t queue_mem[kWarpsPerBlock][64];
    __shared__ unsigned long long cnt_mem[kWarpsPerBlock][kNumCounters];
    __shared__ SourceS src_mem[kWarpsPerBlock];
    __shared__ float lam_lo_mem[kWarpsPerBlock * 32];   // a photon's wavelength low word, out of the registers
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* queue = queue_mem[warp];
    unsigned long long* cnt = cnt_mem[warp];
    const unsigned lanes_below = (1u << lane) - 1u;
    const bool early = (P.flags & PHOSIM_EARLY_REJECT) != 0;
    if (lane < kNumCounters) cnt[lane] = 0;
    __syncwarp();
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = S.tile_begin + atomicAdd(P.tile_counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= S.tile_end) break;
        const int src = tile_source(P, t, lane);
        const DSource& s = P.sources[src];
        const uint64_t j = t - P.tile_prefix[src];
        const uint64_t off = j * P.tile_photons;
        const uint32_t count = (uint32_t)min((uint64_t)P.tile_photons, s.ucount - off);
        const uint64_t ufirst = s.ufirst + off;
        {   // the source's constants, converted by the chief-ray kernel: one word a lane
            static_assert(sizeof(SourceS) % 4 == 0 && sizeof(SourceS) <= 128, "SourceS copy");
            const uint32_t* from = reinterpret_cast<const uint32_t*>(P.sources_s + src);
            uint32_t* to = reinterpret_cast<uint32_t*>(&src_mem[warp]);
            for (int w = lane; w < (int)(sizeof(SourceS) / 4); w += 32) to[w] = __ldg(from + w);
        }
        __syncwarp();
        const SourceS& ss = src_mem[warp];
        const uint32_t nb = ss.bundle;          // the same for the whole warp (one source per tile)
        int queued = 0;
        uint32_t base = 0;
        for (;;) {
            if (base < count) {
                const uint32_t k = base + lane;
                const bool valid = k < count;
                const uint64_t u = ufirst + k;
                if (nb <= 1) {
                    const unsigned vmask = __ballot_sync(0xffffffffu, valid);
                    if (lane == 0) cnt[0] += __popc(vmask);
                } else {
                    uint64_t lo;
                    uint32_t nm;
                    unit_members(s, nb, u, lo, nm);
                    const unsigned traced = __reduce_add_sync(0xffffffffu, valid ? nm : 0u);
                    if (lane == 0) cnt[0] += traced;
                }
                bool go_on = valid;
                if (early) {
                    // stage 1: the early coating decision alone, for every photon of the unit
                    int rej = -1;
                    float lam = 0.f;
                    if (valid) rej = early_reject_certain_f(P, ss, src, u, lam);
                    go_on = valid && rej < 0;
                    const bool dropped = valid && !go_on;
                    const uint32_t fl = dropped ? lost(PHOSIM_LOST_COATING, rej) : 0u;
                    if (nb <= 1) {
                        account_lost(P, fl, lam, dropped, s.rec_off + (u - s.first), lane, cnt, PHOSIM_LOST_COATING);
                    } else if (__any_sync(0xffffffffu, dropped)) {
                        uint64_t lo;
                        uint32_t nm;
                        unit_members(s, nb, u, lo, nm);
                        for (uint32_t m = 0; m < nb; ++m)
                            account_lost(P, fl, lam, dropped && m < nm, s.rec_off + (lo + m - s.first), lane, cnt,
                                         PHOSIM_LOST_COATING);
                    }
                }
                const unsigned gmask = __ballot_sync(0xffffffffu, go_on);
                if (go_on) queue[queued + __popc(gmask & lanes_below)] = k;
                queued += __popc(gmask);
                base += 32;
                __syncwarp();
            }
            const bool drained = base >= count;
            if (queued >= 32 || (drained && queued > 0)) {
                const int take = queued < 32 ? queued : 32;
                queued -= take;
                const bool v = lane < take;
                const uint32_t kk = v ? queue[queued + lane] : 0u;
                __syncwarp();
                PhotonOutS Q;
                Q.flags = 0; Q.pix = -1;
                ds X[3], D[3];
                float lam = 0.f;
                float& lam_lo = lam_lo_mem[threadIdx.x];
                uint4 w1, w2, w3, w4;
                const uint64_t u = ufirst + kk;
                const bool go = v && photon_entry_ds(P, ss, src, u, Q, X, D, lam, lam_lo, w1, w2, w3, w4);
                // survivors append their state, a warp at a time
                const unsigned amask = __ballot_sync(0xffffffffu, go);
                unsigned long long slot = 0;
                if (lane == 0 && amask) slot = atomicAdd(S.n_state, (unsigned long long)__popc(amask));
                slot = __shfl_sync(0xffffffffu, slot, 0) + __popc(amask & lanes_below);
                if (go) {
                    DSState e;
                    e.x = X[0]; e.y = X[1];                 // X[2] is the entrance plane's z
                    e.lam_lo = lam_lo; e.pad = 0.f;
                    e.nx = D[0]; e.ny = D[1]; e.nz = D[2];
                    e.lam = lam;
                    e.src = src;
                    e.idx = u;
                    S.state[slot] = e;
                }
                // units stopped here (by the dynamic transmission test when stage 1 is off): all their photons
                const bool dropped = v && !go;
                if (__any_sync(0xffffffffu, dropped)) {
                    uint64_t lo;
                    uint32_t nm;
                    unit_members(s, nb, u, lo, nm);
                    for (uint32_t m = 0; m < nb; ++m)
                        account_lost(P, Q.flags, Q.lam, dropped && m < nm, s.rec_off + (lo + m - s.first), lane, cnt);
                }
            }
            if (drained && queued == 0) break;
        }
        __syncwarp();
    }
    __syncwarp();
    if (lane < kNumCounters && cnt[lane]) atomicAdd(P.counters + lane, cnt[lane]);
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
    optics<false, false>(P, X, D, P.lam_ref, zero, zero, zero, zero, R);
    const bool ok = (R.flags & PHOSIM_F_DETECTED) != 0;
    S.ref_x = ok ? R.x : 0.0;
    S.ref_y = ok ? R.y : 0.0;
    const ds rx = ds_of(S.ref_x), ry = ds_of(S.ref_y);
    S.ref_s[0] = rx.hi; S.ref_s[1] = rx.lo; S.ref_s[2] = ry.hi; S.ref_s[3] = ry.lo;
    // the double-single constants of the source, converted once here instead of once per tile (the conversions
    // from double run on the FP64 pipe)
    if (P.sources_s) P.sources_s[s] = source_s(S);
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

cudaError_t launch_trace(const TraceParams& P, int mode, int blocks, int threads, cudaStream_t st) {
    if (mode == kDS) trace_kernel<kDS><<<blocks, threads, 0, st>>>(P);
    else if (mode == kMixed) trace_kernel<kMixed><<<blocks, threads, 0, st>>>(P);
    else trace_kernel<kPlain><<<blocks, threads, 0, st>>>(P);
    return cudaGetLastError();
}

const void* trace_kernel_ptr(int mode) {
    if (mode == kDS) return (const void*)trace_kernel<kDS>;
    return mode == kMixed ? (const void*)trace_kernel<kMixed> : (const void*)trace_kernel<kPlain>;
}
const void* chief_kernel_ptr() { return (const void*)chief_ray_kernel; }
size_t source_s_bytes() { return sizeof(SourceS); }
const void* ds_entry_kernel_ptr() { return (const void*)ds_entry_kernel; }
cudaError_t launch_ds_entry(const TraceParams& P, const DSStage& S, int blocks, int threads, cudaStream_t st) {
    ds_entry_kernel<<<blocks, threads, 0, st>>>(P, S);
    return cudaGetLastError();
}

cudaError_t trace_occupancy(int mode, int threads, int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel_ptr(mode), threads, 0);
}

}  // namespace phosim
