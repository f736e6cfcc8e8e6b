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

constexpr int kWarpsPerBlock = 8;

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
// The per-photon arithmetic and its order are those of trace_photon_ds, so both give the same results.
// ---------------------------------------------------------------------------------------------------------
#ifndef PHOSIM_DS_ENTRY_MIN_BLOCKS
#define PHOSIM_DS_ENTRY_MIN_BLOCKS 6
#endif
// blocks per SM the optics stage is compiled for: 3 of 80 registers (fewer spills) measured faster than 4 of 64
#ifndef PHOSIM_DS_OPTICS_MIN_BLOCKS
#define PHOSIM_DS_OPTICS_MIN_BLOCKS 3
#endif
#ifndef PHOSIM_DS_LOCKSTEP
#define PHOSIM_DS_LOCKSTEP 1
#endif
#ifndef PHOSIM_DS_DYNAMIC_BATCHES
#define PHOSIM_DS_DYNAMIC_BATCHES 1
#endif
// threads per block of the optics stage (0: the schedule's block size).  Fixed at 256: the lockstep wants
// blocks of 8 warps (128- and 64-thread blocks measured 17 % and 28 % slower), whatever the schedule chosen
// for the entry stage.
#ifndef PHOSIM_DS_OPTICS_THREADS
#define PHOSIM_DS_OPTICS_THREADS 256
#endif
constexpr int kOpticsMaxThreads = PHOSIM_DS_OPTICS_THREADS ? PHOSIM_DS_OPTICS_THREADS : 256;

// A work unit of the two-kernel path is a photon, or for a bundle of n photons per ray (Sec. 3.2) a ray:
// the ray is traced once and its photons (those in the call's range) only go through the sensor apart.
__device__ __forceinline__ void unit_members(const DSource& s, uint32_t nb, uint64_t u, uint64_t& lo, uint32_t& nm) {
    if (nb <= 1) { lo = u; nm = 1; return; }
    const uint64_t a = max(s.first, u * nb), b = min(s.first + s.count, (u + 1) * nb);
    lo = a;
    nm = b > a ? (uint32_t)(b - a) : 0u;
}

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

#ifndef PHOSIM_DS_MEMBERS_MIN_BLOCKS
#define PHOSIM_DS_MEMBERS_MIN_BLOCKS 4
#endif

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

// Account for one photon per lane of the optics or bundle stage: record, image, counters (cnt: the warp's
// counters in shared memory, lane 0) and the moment sums about the source's chief-ray position, reduced over
// the lanes of one source.  Every lane of the warp calls it.
__device__ __forceinline__ void account_ds(const TraceParams& P, const PhotonOutS& R, bool v, int src, uint64_t i,
                                           int lane, unsigned long long* cnt) {
    const DSource& s = P.sources[src];
    if (v && P.records) {
        phosim_photon_record rec;
        rec.x = ds_value(R.x); rec.y = ds_value(R.y); rec.xc = ds_value(R.xc); rec.yc = ds_value(R.yc);
        rec.lambda = (double)R.lam;
        rec.flags = R.flags; rec.pix = R.pix;
        P.records[s.rec_off + (i - s.first)] = rec;
    }
    const bool det = v && (R.flags & PHOSIM_F_DETECTED);
    const unsigned dmask = __ballot_sync(0xffffffffu, det);
    if (det) {
        const unsigned same = __match_any_sync(dmask, R.pix);
        if (lane == __ffs(same) - 1) atomicAdd(P.image + R.pix, (unsigned)__popc(same));
    }
    if (lane == 0) cnt[1] += __popc(dmask);
    const uint32_t reason = v ? ((R.flags >> 8) & 0xffu) : 0u;
#pragma unroll
    for (int q = 1; q <= 8; ++q) {
        const unsigned bq = __ballot_sync(0xffffffffu, reason == (uint32_t)q);
        if (lane == 0) cnt[1 + q] += __popc(bq);
    }
    if (P.moments && dmask) {
        // Per-source partial sums of the warp: the states arrive in runs of one source (a warp of the entry
        // stage appends its survivors together), so the lanes of a source are contiguous segments.  An
        // inclusive segmented scan in double-single (exact products of the single-precision offsets from the
        // chief ray, sums to ~2^-47) leaves each segment's sums in its last lane, which adds them to the
        // source's double-precision moments: one set of atomics per segment, not per photon, and the FP64
        // pipe (a sixty-fourth of the FP32 rate on this GPU) only converts the partials.
        ds mm[5] = {ds_f(0.f), ds_f(0.f), ds_f(0.f), ds_f(0.f), ds_f(0.f)};
        if (det) {
            const float fx = (R.x - ds{s.ref_s[0], s.ref_s[1]}).hi, fy = (R.y - ds{s.ref_s[2], s.ref_s[3]}).hi;
            mm[0] = ds_f(fx); mm[1] = ds_f(fy);
            mm[2] = two_prod(fx, fx); mm[3] = two_prod(fx, fy); mm[4] = two_prod(fy, fy);
        }
        const int prev = __shfl_up_sync(0xffffffffu, src, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != src);
        const unsigned upto = lane == 31 ? 0xffffffffu : (2u << lane) - 1u;
        const int first = 31 - __clz(heads & upto);
        // the sums in pairs (x, y), (xx, xy) and yy, the pairs added by the packed primitive (bit for bit the same)
        ds2 m01 = ds2_of(mm[0], mm[1]), m23 = ds2_of(mm[2], mm[3]);
        ds m4 = mm[4];
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const auto up = [&](float v) { return __shfl_up_sync(0xffffffffu, v, d); };
            const ds2 t01 = {make_float2(up(m01.hi.x), up(m01.hi.y)), make_float2(up(m01.lo.x), up(m01.lo.y))};
            const ds2 t23 = {make_float2(up(m23.hi.x), up(m23.hi.y)), make_float2(up(m23.lo.x), up(m23.lo.y))};
            const ds t4 = {up(m4.hi), up(m4.lo)};
            if (lane - d >= first) {
                m01 = add2(m01, t01);
                m23 = add2(m23, t23);
                m4 = m4 + t4;
            }
        }
        mm[0] = ds2_x(m01); mm[1] = ds2_y(m01); mm[2] = ds2_x(m23); mm[3] = ds2_y(m23); mm[4] = m4;
        const bool last = lane == 31 || ((heads >> (lane + 1)) & 1u);
        // the segment's detected photons, counted from the ballot
        const unsigned n_det = __popc(dmask & upto & ~((1u << first) - 1u));
        if (last && n_det > 0) {
            double* M = (P.mom_stripes ? P.mom_stripes + (size_t)(blockIdx.x % kMomStripes) * P.mom_stripe_stride
                                       : P.moments) + (size_t)src * PHOSIM_MOMENT_WORDS;
            atomicAdd(M, (double)n_det);
#pragma unroll
            for (int q = 0; q < 5; ++q) atomicAdd(M + 1 + q, ds_value(mm[q]));
        }
    }
}

__global__ void __launch_bounds__(kOpticsMaxThreads, PHOSIM_DS_OPTICS_MIN_BLOCKS)
    ds_optics_kernel(const __grid_constant__ TraceParams P, const DSStage S) {
    __shared__ unsigned long long cnt_mem[kOpticsMaxThreads / 32][kNumCounters];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lanes_below = (1u << lane) - 1u;
    unsigned long long* cnt = cnt_mem[warp];
    if (lane < kNumCounters) cnt[lane] = 0;
    __syncwarp();
    const unsigned long long n = *S.n_state;
    // any block size up to 256 threads (the schedule's)
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
#if PHOSIM_DS_LOCKSTEP
    // a block's states at a time, all its warps meeting the surfaces together (a barrier after each), so
    // that the SM's warps fetch the same stretch of code rather than as many stretches as warps; the
    // blocks claim batches as they finish (a block is as slow as its slowest ray at every surface)
#if PHOSIM_DS_DYNAMIC_BATCHES
    __shared__ unsigned long long next_batch;
    (void)stride;
    for (;;) {
        if (threadIdx.x == 0) next_batch = atomicAdd(S.batch, 1ull) * blockDim.x;
        __syncthreads();
        const unsigned long long b0 = next_batch;
        if (b0 >= n) break;
#else
    for (unsigned long long b0 = (unsigned long long)blockIdx.x * blockDim.x; b0 < n; b0 += stride) {
#endif
        const unsigned long long b = b0 + (unsigned long long)warp * 32ull;
#else
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + (unsigned long long)warp * 32ull; b < n;
         b += stride) {
#endif
        const unsigned long long e = b + lane;
        const bool v = e < n;
        PhotonOutS R;
        R.flags = 0; R.pix = -1; R.lam = 0.f;
        R.x = R.y = R.xc = R.yc = ds_f(0.f);
        int src = 0;
        uint64_t u = 0;
        DetectorHit H;
#if PHOSIM_DS_LOCKSTEP
        OpticsWalk W;
        ds lam = ds_f(0.f);
        bool go = false, bundled = false;
        if (v) {
            const DSState st = S.state[e];
            src = st.src;
            u = st.idx;
            R.lam = st.lam;
            lam = ds{st.lam, st.lam_lo};
            bundled = P.sources[src].bundle > 1;
            const ds X[3] = {st.x, st.y, P.z_ent_s}, D[3] = {st.nx, st.ny, st.nz};
            walk_start(W, X, D);
            go = true;
        }
        while (__syncthreads_or(go)) {
            if (go) go = surface_step_ds(P, W, lam, src, u, R, nullptr, bundled ? &H : nullptr);
        }
#else
        ds lam = ds_f(0.f);
        if (v) {
            const DSState st = S.state[e];
            src = st.src;
            u = st.idx;
            R.lam = st.lam;
            lam = ds{st.lam, st.lam_lo};
            const bool bundled = P.sources[src].bundle > 1;
            const ds X[3] = {st.x, st.y, P.z_ent_s}, D[3] = {st.nx, st.ny, st.nz};
            optics_ds(P, X, D, lam, src, u, R, nullptr, bundled ? &H : nullptr);
        }
#endif
        // a bundle's ray that reached the detector surface hands its hit over to the bundle stage
        const bool handed = v && R.flags == kHandedOff;
        const unsigned hmask = __ballot_sync(0xffffffffu, handed);
        if (hmask) {
            unsigned long long slot = 0;
            if (lane == 0) slot = atomicAdd(S.n_hits, (unsigned long long)__popc(hmask));
            slot = __shfl_sync(0xffffffffu, slot, 0) + __popc(hmask & lanes_below);
            if (handed) {
                DSHit h;
                h.H = H;
                h.lam = lam.hi;
                h.lam_lo = lam.lo;
                h.src = src;
                h.ray = u;
                S.hits[slot] = h;
            }
        }
        // every other unit is one photon, or a bundle's ray lost before the detector (all its photons)
        const uint32_t nb = v ? P.sources[src].bundle : 1u;
        uint64_t lo = u;
        uint32_t nm = 1;
        if (nb > 1) unit_members(P.sources[src], nb, u, lo, nm);
        const uint32_t n_loop = __reduce_max_sync(0xffffffffu, v && !handed ? nm : 0u);
        for (uint32_t m = 0; m < n_loop; ++m) account_ds(P, R, v && !handed && m < nm, src, lo + m, lane, cnt);
    }
    __syncwarp();
    if (lane < kNumCounters && cnt[lane]) atomicAdd(P.counters + lane, cnt[lane]);
}

// The photons of the bundles whose ray reached the detector surface: each its own Gaussian offset and its
// own sensor draws from the shared hit (Sec. 3.2), one hit per thread.
__global__ void __launch_bounds__(256, PHOSIM_DS_MEMBERS_MIN_BLOCKS) ds_members_kernel(const __grid_constant__ TraceParams P,
                                                                                       const DSStage S) {
    __shared__ unsigned long long cnt_mem[kWarpsPerBlock][kNumCounters];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long* cnt = cnt_mem[warp];
    if (lane < kNumCounters) cnt[lane] = 0;
    __syncwarp();
    const unsigned long long n = *S.n_hits;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long b = (unsigned long long)blockIdx.x * blockDim.x + (unsigned long long)warp * 32ull; b < n;
         b += stride) {
        const unsigned long long e = b + lane;
        const bool v = e < n;
        DSHit h;
        h.src = 0; h.ray = 0; h.lam = 0.f; h.lam_lo = 0.f;
        if (v) h = S.hits[e];
        const DSource& s = P.sources[h.src];
        const uint32_t nb = v ? s.bundle : 0u;
        uint64_t lo = 0;
        uint32_t nm = 0;
        if (v) unit_members(s, nb, h.ray, lo, nm);
        const uint32_t n_loop = __reduce_max_sync(0xffffffffu, nm);
        for (uint32_t m = 0; m < n_loop; ++m) {
            const bool vm = m < nm;
            PhotonOutS R;
            R.flags = 0; R.pix = -1; R.lam = h.lam;
            R.x = R.y = R.xc = R.yc = ds_f(0.f);
            if (vm) {
                const MemberDrawS mb = member_draw_s(P, (float)s.bsig, h.src, lo + m);
                detect_ds(P, h.H, ds{h.lam, h.lam_lo}, h.src, h.ray, R, &mb);
            }
            account_ds(P, R, vm, h.src, lo + m, lane, cnt);
        }
    }
    __syncwarp();
    if (lane < kNumCounters && cnt[lane]) atomicAdd(P.counters + lane, cnt[lane]);
}

// The striped moment accumulators of the two-kernel path added into the caller's moment sums (one thread a
// source and word)
__global__ void moment_stripes_kernel(const __grid_constant__ TraceParams P) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.n_src * 6) return;
    const size_t w = (size_t)(i / 6) * PHOSIM_MOMENT_WORDS + (size_t)(i % 6);
    double sum = 0.0;
#pragma unroll
    for (int k = 0; k < kMomStripes; ++k) sum += P.mom_stripes[(size_t)k * P.mom_stripe_stride + w];
    P.moments[w] += sum;
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
const void* ds_optics_kernel_ptr() { return (const void*)ds_optics_kernel; }
const void* moment_stripes_kernel_ptr() { return (const void*)moment_stripes_kernel; }

cudaError_t launch_moment_stripes(const TraceParams& P, cudaStream_t st) {
    if (P.n_src <= 0 || !P.moments || !P.mom_stripes) return cudaSuccess;
    moment_stripes_kernel<<<(P.n_src * 6 + 255) / 256, 256, 0, st>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_ds_entry(const TraceParams& P, const DSStage& S, int blocks, int threads, cudaStream_t st) {
    ds_entry_kernel<<<blocks, threads, 0, st>>>(P, S);
    return cudaGetLastError();
}

int ds_optics_threads(int threads) { return PHOSIM_DS_OPTICS_THREADS ? PHOSIM_DS_OPTICS_THREADS : threads; }

cudaError_t launch_ds_optics(const TraceParams& P, const DSStage& S, int blocks, int threads, cudaStream_t st) {
    ds_optics_kernel<<<blocks, ds_optics_threads(threads), 0, st>>>(P, S);
    return cudaGetLastError();
}

cudaError_t launch_ds_members(const TraceParams& P, const DSStage& S, int blocks, int threads, cudaStream_t st) {
    ds_members_kernel<<<blocks, threads, 0, st>>>(P, S);
    return cudaGetLastError();
}

const void* ds_members_kernel_ptr() { return (const void*)ds_members_kernel; }

cudaError_t ds_stage_occupancy(int threads, int* entry_per_sm, int* optics_per_sm, int* members_per_sm) {
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(entry_per_sm, ds_entry_kernel, threads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(optics_per_sm, ds_optics_kernel, ds_optics_threads(threads), 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(members_per_sm, ds_members_kernel, threads, 0);
}

cudaError_t trace_occupancy(int mode, int threads, int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, trace_kernel_ptr(mode), threads, 0);
}

}  // namespace phosim
