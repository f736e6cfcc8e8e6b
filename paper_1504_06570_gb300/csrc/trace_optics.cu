// The optics and bundle stages of the two-kernel double-single path (Peterson et al. 2015, Sec. 2.4-2.5): the
// surfaces, the sensor, the pixel counts and the per-source moment sums of the states the entry stage
// (trace.cu) leaves on the telescope's entrance plane.  This translation unit compiles the double-single
// quotient, square root and reciprocal root inline: with them inline the optics stage (80 registers) measured
// 3 % faster, and the entry stage, which keeps them out of line, 15 % slower.  The generator is inline here
// too (1 % faster; the entry stage keeps its call).
#ifndef PHOSIM_DS_HEAVY_OPTICS
#define PHOSIM_DS_HEAVY_OPTICS __forceinline__
#endif
#define PHOSIM_DS_HEAVY PHOSIM_DS_HEAVY_OPTICS
#ifndef PHOSIM_DS_PHILOX_OPTICS
#define PHOSIM_DS_PHILOX_OPTICS __forceinline__
#endif
#define PHOSIM_DS_PHILOX PHOSIM_DS_PHILOX_OPTICS

#include "phosim_device.cuh"
#include "phosim_scene.hpp"
#include "photon.cuh"
#include "photon_ds.cuh"

namespace phosim {

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

#ifndef PHOSIM_DS_MEMBERS_MIN_BLOCKS
#define PHOSIM_DS_MEMBERS_MIN_BLOCKS 4
#endif

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

const void* ds_optics_kernel_ptr() { return (const void*)ds_optics_kernel; }

const void* moment_stripes_kernel_ptr() { return (const void*)moment_stripes_kernel; }

cudaError_t launch_moment_stripes(const TraceParams& P, cudaStream_t st) {
    if (P.n_src <= 0 || !P.moments || !P.mom_stripes) return cudaSuccess;
    moment_stripes_kernel<<<(P.n_src * 6 + 255) / 256, 256, 0, st>>>(P);
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
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(entry_per_sm, ds_entry_kernel_ptr(), threads, 0);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(optics_per_sm, ds_optics_kernel, ds_optics_threads(threads), 0);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(members_per_sm, ds_members_kernel, threads, 0);
}

}  // namespace phosim
