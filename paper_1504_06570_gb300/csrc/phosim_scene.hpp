// Host-side scene object behind the phosim C ABI.
#pragma once

#include <vector>

#include "phosim_device.cuh"
#include "photon_ds.cuh"

// One trace call's launch sequence as a CUDA graph: kernels ([chief rays, trace], or chief rays, then per chunk of
// the two-kernel path the entry, optics and bundle stages, then the moment-stripe sum) and the counter resets
// between chunks, one node each in launch order.  Built once for a sequence's shape and replayed with each
// call's kernel parameters and launch shapes.
struct TraceGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> func;              // per node: the kernel, or null for a memset
    std::vector<void*> memset_dst;              // per node: the memset's destination (null for a kernel)
    std::vector<size_t> memset_bytes;
    std::vector<cudaGraphNode_t> node;
};

struct phosim_scene {
    phosim::TraceParams base;       // scalars and device table pointers; per-call fields filled by a trace
    int precision = PHOSIM_PLAIN_FP64;
    int device = 0;                 // the CUDA device current at creation; every call must run with it current
    bool optics_loaded = false, seds_loaded = false;
    int sm_count = 0;
    int threads = 256;
    int tile_photons = 0;           // 0 = chosen per call from the workload
    int n_sed = 0;
    int sersic_tables = 0;
    // host copy of the loaded optics (for the adjoint)
    std::vector<phosim_surface> surfaces;
    // device memory owned by the scene
    std::vector<void*> table_mem;   // sensor tables
    std::vector<void*> optics_mem;  // coating tables
    std::vector<void*> screen_mem;  // gradient screens
    std::vector<void*> sed_mem;
    std::vector<void*> sersic_mem;
    std::vector<void*> hf_mem;      // high-frequency kick quantiles
    // per-call scratch, grown on demand
    phosim::DSource* d_src = nullptr;
    size_t cap_src = 0;
    void* d_src_s = nullptr;                    // the sources' double-single constants (phosim::SourceS, n_src)
    unsigned long long* d_prefix = nullptr;
    size_t cap_prefix = 0;
    unsigned long long* d_counters = nullptr;   // [0] tile counter, [1..9] counters
    uint32_t* d_stage = nullptr;                // staging image for host image pointers
    phosim::DSState* d_state = nullptr;         // entrance-plane states of the two-kernel double-single path
    size_t cap_state = 0;
    phosim::DSHit* d_hits = nullptr;            // detector hits of its bundle rays
    size_t cap_hits = 0;
    double* d_mom_stripes = nullptr;            // its striped per-source moment accumulators
    size_t cap_mom_stripes = 0;
    size_t cap_stage = 0;
    cudaStream_t last_stream = nullptr;
    // adjoint: Zernike monomial table (owned with the optics) and per-call scratch
    double* d_zmono = nullptr;
    double* d_grad_scratch = nullptr;           // seeds + gradient accumulators
    size_t cap_grad = 0;
    double* d_mom_scratch = nullptr;
    size_t cap_mom = 0;
    // CUDA graphs of the trace launch (PHOSIM_GRAPH), one per precision, captured on a private stream
    TraceGraph graphs[3];
    cudaStream_t capture_stream = nullptr;
    // per-kernel timing (phosim_set_stage_timing): an event pair per launch of the last call, with the
    // kernel kind (0 chief, 1 one-kernel trace, 2 entry stage, 3 optics stage)
    bool stage_timing = false;
    std::vector<cudaEvent_t> timing_events;
    std::vector<int> timing_kind;
    int timing_used = 0;
};

namespace phosim {
// mode: the scene's precision (PHOSIM_PLAIN_FP64, PHOSIM_MIXED, PHOSIM_MIXED_DS)
cudaError_t launch_trace(const TraceParams& P, int mode, int blocks, int threads, cudaStream_t st);
cudaError_t launch_chief_rays(const TraceParams& P, DSource* sources, int n_src, double* moments, cudaStream_t st);
cudaError_t trace_occupancy(int mode, int threads, int* blocks_per_sm);
const void* trace_kernel_ptr(int mode);
const void* chief_kernel_ptr();
size_t source_s_bytes();                       // sizeof(SourceS), which the host code does not see
// the two-kernel double-single path (PHOSIM_MIXED_DS in phosim_trace)
cudaError_t launch_ds_entry(const TraceParams& P, const DSStage& S, int blocks, int threads, cudaStream_t st);
cudaError_t launch_ds_optics(const TraceParams& P, const DSStage& S, int blocks, int threads, cudaStream_t st);
cudaError_t launch_ds_members(const TraceParams& P, const DSStage& S, int blocks, int threads, cudaStream_t st);
const void* ds_members_kernel_ptr();
cudaError_t ds_stage_occupancy(int threads, int* entry_per_sm, int* optics_per_sm, int* members_per_sm);
const void* ds_entry_kernel_ptr();
const void* ds_optics_kernel_ptr();
const void* moment_stripes_kernel_ptr();
cudaError_t launch_moment_stripes(const TraceParams& P, cudaStream_t st);
int ds_optics_threads(int threads);      // the optics stage's block size for a schedule's block size
void free_all(std::vector<void*>& v);
// PHOSIM_OK when the current device is the scene's, INVALID_ARGUMENT otherwise (CUDA on a failed query)
phosim_status check_scene_device(const phosim_scene* sc);
// PHOSIM_OK when p is null or device / managed memory usable on `device`; INVALID_ARGUMENT for host memory,
// unregistered pointers and another device's memory
phosim_status check_device_buffer(const void* p, int device);
// count, centroid and central second moments of n_src sources from their PHOSIM_MOMENT_WORDS additive sums
void derive_moments(const double* sums, int n_src, double* out6);
}  // namespace phosim
