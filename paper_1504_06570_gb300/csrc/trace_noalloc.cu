// phosim_trace_noalloc: the trace launch with its per-call scratch in a file-scope device array, for
// callers of this library that cannot allocate device memory (an application whose device memory belongs
// to an outside pool, or a latency-critical loop where an allocation would synchronise the device).
//
// The array holds the work counters, the per-source tile prefix and the source list of one call.  Its
// device address is looked up once per device (the first call on that device, with it current) and
// passed to the same kernels phosim_trace launches.  Nothing here allocates.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "phosim_device.cuh"
#include "phosim_scene.hpp"

using namespace phosim;

namespace {

constexpr size_t kCounterBytes = 256;                                   // 16 u64 words, padded
constexpr size_t kPrefixBytes = ((PHOSIM_NOALLOC_MAX_SOURCES + 1) * sizeof(unsigned long long) + 255) / 256 * 256;
constexpr size_t kSourceBytes = PHOSIM_NOALLOC_MAX_SOURCES * sizeof(DSource);
static_assert(kCounterBytes + kPrefixBytes + kSourceBytes <= PHOSIM_NOALLOC_SCRATCH_BYTES,
              "scratch layout exceeds the documented size");

// Every GPU that loads the library holds this array until the process exits.
__device__ __align__(256) unsigned char g_trace_scratch[PHOSIM_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device (host code only sees a stand-in for the symbol).
phosim_status scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    if (dev < 0 || dev >= kMaxDevices) return PHOSIM_ERR_LIMIT;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_trace_scratch);
        if (e != cudaSuccess || !p) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return PHOSIM_OK;
}

bool finite_value(double v) { return std::isfinite(v); }

}  // namespace

extern "C" phosim_status phosim_trace_noalloc(phosim_scene* sc, const phosim_source* src, int n_src,
                                              const uint64_t* n_photons, const uint64_t* first, uint32_t* image,
                                              phosim_photon_record* records, double* moments, void* stream) {
    if (!sc || n_src < 0 || (n_src > 0 && (!src || !n_photons)) || !image) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (n_src > PHOSIM_NOALLOC_MAX_SOURCES) return PHOSIM_ERR_LIMIT;
    if (!sc->optics_loaded || !sc->seds_loaded) return PHOSIM_ERR_NOT_READY;
    cudaStream_t s = (cudaStream_t)stream;
    // The source list and tile prefix below are copied from host vectors that this call frees on return, so a
    // stream being captured would record copies from freed memory: refuse before anything is enqueued.
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &capture) != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    if (capture != cudaStreamCaptureStatusNone) return PHOSIM_ERR_INVALID_ARGUMENT;
    sc->timing_used = 0;      // per-kernel timing does not cover this call
    // the scene's device must be current (the scratch address is looked up per device), and every output
    // must be device memory on it
    phosim_status st = check_scene_device(sc);
    if (st == PHOSIM_OK) st = check_device_buffer(image, sc->device);
    if (st == PHOSIM_OK) st = check_device_buffer(records, sc->device);
    if (st == PHOSIM_OK) st = check_device_buffer(moments, sc->device);
    if (st != PHOSIM_OK) return st;
    void* base = nullptr;
    st = scratch_address(&base);
    if (st != PHOSIM_OK) return st;
    const int mode = sc->precision;
    int per_sm = 0;
    if (trace_occupancy(mode, sc->threads, &per_sm) != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    per_sm = std::max(per_sm, 1);
    const int blocks = sc->sm_count * per_sm;
    const uint64_t warps = (uint64_t)blocks * (sc->threads / 32);
    uint64_t total = 0;
    for (int i = 0; i < n_src; ++i) total += n_photons[i];
    uint64_t T = sc->tile_photons;
    if (!T) {
        T = total / (warps * 8);
        T = std::min<uint64_t>(1024, std::max<uint64_t>(32, (T + 31) / 32 * 32));
    }
    // host copies of the call's source list and tile prefix (the same form phosim_trace builds)
    std::vector<DSource> hs((size_t)n_src);
    std::vector<unsigned long long> prefix((size_t)n_src + 1, 0);
    uint64_t rec = 0;
    for (int i = 0; i < n_src; ++i) {
        const phosim_source& q = src[i];
        if (q.kind < PHOSIM_POINT || q.kind > PHOSIM_GAUSS) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.sed < 0 || q.sed >= sc->n_sed) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.kind == PHOSIM_SERSIC && (q.table < 0 || q.table >= sc->sersic_tables)) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (!finite_value(q.xi) || !finite_value(q.eta) || q.xi * q.xi + q.eta * q.eta >= 1.0 || !(q.redshift > -1.0))
            return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.bundle < 0 || (q.bundle > 1 && !(q.bundle_sigma >= 0.0 && finite_value(q.bundle_sigma))))
            return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.bundle > PHOSIM_MAX_BUNDLE) return PHOSIM_ERR_LIMIT;
        DSource& d = hs[i];
        std::memset(&d, 0, sizeof(d));
        d.kind = q.kind; d.sed = q.sed; d.table = q.table;
        d.xi = q.xi; d.eta = q.eta; d.zfac = 1.0 + q.redshift; d.t0 = q.t0; d.t_exp = q.t_exp;
        d.a = q.a; d.b = q.b; d.cpa = std::cos(q.pa); d.spa = std::sin(q.pa);
        d.bundle = q.bundle > 1 ? (uint32_t)q.bundle : 1u;
        d.bsig = q.bundle > 1 ? q.bundle_sigma : 0.0;
        d.first = first ? first[i] : 0;
        d.count = n_photons[i];
        d.ufirst = d.first;
        d.ucount = d.count;
        d.rec_off = rec;
        rec += n_photons[i];
        prefix[i + 1] = prefix[i] + (n_photons[i] + T - 1) / T;
    }
    if (n_src == 0 || total == 0) return PHOSIM_OK;
    unsigned char* b = (unsigned char*)base;
    unsigned long long* d_counters = (unsigned long long*)b;
    unsigned long long* d_prefix = (unsigned long long*)(b + kCounterBytes);
    DSource* d_src = (DSource*)(b + kCounterBytes + kPrefixBytes);
    // the array keeps the previous call's contents: the counters must start at zero
    if (cudaMemsetAsync(d_counters, 0, kCounterBytes, s) != cudaSuccess ||
        cudaMemcpyAsync(d_src, hs.data(), hs.size() * sizeof(DSource), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_prefix, prefix.data(), prefix.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return PHOSIM_ERR_CUDA;
    }
    TraceParams P = sc->base;
    P.sources = d_src;
    P.tile_prefix = d_prefix;
    P.n_src = n_src;
    P.tile_photons = (uint32_t)T;
    P.n_tiles = prefix[n_src];
    P.tile_counter = d_counters;
    P.counters = d_counters + 1;
    P.image = image;
    P.moments = moments;
    P.records = records;
    if (launch_chief_rays(P, d_src, n_src, moments, s) != cudaSuccess ||
        launch_trace(P, mode, blocks, sc->threads, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return PHOSIM_ERR_CUDA;
    }
    return PHOSIM_OK;
}
