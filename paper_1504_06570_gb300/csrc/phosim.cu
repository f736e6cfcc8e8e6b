// Host side of the phosim C ABI: scene construction, table preparation kernels and the trace launch.
//
// Loads copy the caller's host tables to device memory owned by the scene and prepare the forms the
// photon kernel reads: central-difference gradient screens (Sec. 2.3.2), integer thresholds of the
// photon-number cumulative SED tables (Sec. 2.2), surface frames and Zernike figures as monomials
// (Sec. 2.4.1).  phosim_trace uploads the source list and launches one persistent trace kernel.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "phosim_bench.h"
#include "phosim_device.cuh"
#include "phosim_scene.hpp"
#include "grad.hpp"

using namespace phosim;

namespace phosim {
void free_all(std::vector<void*>& v) {
    for (void* p : v) cudaFree(p);
    v.clear();
}
}  // namespace phosim

namespace {

#define CU(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            (void)cudaGetLastError();                       \
            return e_ == cudaErrorMemoryAllocation ? PHOSIM_ERR_OUT_OF_MEMORY : PHOSIM_ERR_CUDA; \
        }                                                   \
    } while (0)

template <class T>
phosim_status upload(std::vector<void*>& owner, const T* host, size_t n, T** out) {
    void* p = nullptr;
    CU(cudaMalloc(&p, std::max<size_t>(1, n) * sizeof(T)));
    owner.push_back(p);
    if (n) CU(cudaMemcpy(p, host, n * sizeof(T), cudaMemcpyHostToDevice));
    *out = (T*)p;
    return PHOSIM_OK;
}

bool is_finite(double v) { return std::isfinite(v); }

// device counter words of a scene: [0] tile counter, [1 .. kNumCounters] launch counters, then the state
// and bundle-hit counts of the two-kernel double-single path
constexpr int kStateCountWord = 1 + kNumCounters;
constexpr int kHitCountWord = kStateCountWord + 1;
constexpr int kBatchWord = kHitCountWord + 1;      // next batch of states for the optics stage's blocks
constexpr int kCounterWords = kBatchWord + 1;
// photons per chunk of the two-kernel path: its state buffer holds one chunk (64 bytes a photon, 8.6 GB)
constexpr uint64_t kStateChunk = 1ull << 27;

// ----------------------------------------------------------------------------------------- Zernike figure
// Noll index -> radial order n, |m| and whether the term is the cosine one (even j) or the sine one.
void noll(int j, int& n, int& am, bool& cosine) {
    n = (int)std::ceil((std::sqrt(8.0 * j + 1.0) - 3.0) / 2.0);
    while (n * (n + 1) / 2 >= j) --n;            // guard the floating estimate
    while ((n + 1) * (n + 2) / 2 < j) ++n;
    const int k = j - n * (n + 1) / 2 - 1;       // position within order n, 0..n
    am = (n % 2 == 0) ? 2 * ((k + 1) / 2) : 2 * (k / 2) + 1;
    cosine = (j % 2 == 0);
}

double fact(int n) { double f = 1.0; for (int i = 2; i <= n; ++i) f *= i; return f; }
double binom(int n, int k) { return fact(n) / (fact(k) * fact(n - k)); }

// coefficients P[b][a] of x^a y^b of Z_j(x, y) in coordinates normalised to the unit disk
void zernike_monomials(int j, double P[7][7]) {
    int n, am;
    bool cosine;
    noll(j, n, am, cosine);
    double A[7][7] = {}, B[7][7] = {};
    // A = sum_s c_s (x^2 + y^2)^((n - am)/2 - s): the radial polynomial divided by rho^am
    for (int s = 0; s <= (n - am) / 2; ++s) {
        const double c = ((s % 2) ? -1.0 : 1.0) * fact(n - s) /
                         (fact(s) * fact((n + am) / 2 - s) * fact((n - am) / 2 - s));
        const int q = (n - am) / 2 - s;
        for (int t = 0; t <= q; ++t) A[2 * (q - t)][2 * t] += c * binom(q, t);
    }
    // B = Re (x + i y)^am for the cosine term, Im (x + i y)^am for the sine term
    for (int t = 0; t <= am; ++t) {
        const double c = binom(am, t);
        if (t % 2 == 0 && (am == 0 || cosine)) B[t][am - t] += ((t / 2) % 2 ? -1.0 : 1.0) * c;
        if (t % 2 == 1 && am > 0 && !cosine) B[t][am - t] += (((t - 1) / 2) % 2 ? -1.0 : 1.0) * c;
    }
    const double N = am == 0 ? std::sqrt((double)n + 1.0) : std::sqrt(2.0 * (n + 1.0));
    for (int b = 0; b < 7; ++b)
        for (int a = 0; a < 7; ++a) P[b][a] = 0.0;
    for (int b1 = 0; b1 < 7; ++b1)
        for (int a1 = 0; a1 + b1 < 7; ++a1) {
            if (A[b1][a1] == 0.0) continue;
            for (int b2 = 0; b1 + b2 < 7; ++b2)
                for (int a2 = 0; a1 + a2 + b1 + b2 < 7; ++a2)
                    P[b1 + b2][a1 + a2] += N * A[b1][a1] * B[b2][a2];
        }
}

// R = Rz(tz) Ry(ty) Rx(tx) takes surface-frame directions to the telescope frame; M = R^T
void rotation(const double* pert, double M[9]) {
    const double cx = std::cos(pert[3]), sx = std::sin(pert[3]);
    const double cy = std::cos(pert[4]), sy = std::sin(pert[4]);
    const double cz = std::cos(pert[5]), sz = std::sin(pert[5]);
    const double R[3][3] = {{cz * cy, cz * sy * sx - sz * cx, cz * sy * cx + sz * sx},
                            {sz * cy, sz * sy * sx + cz * cx, sz * sy * cx - cz * sx},
                            {-sy, cy * sx, cy * cx}};
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) M[3 * i + k] = R[k][i];
}

// derivatives of M = R^T with respect to tx, ty, tz
void rotation_derivatives(const double* pert, double dM[3][9]) {
    const double cx = std::cos(pert[3]), sx = std::sin(pert[3]);
    const double cy = std::cos(pert[4]), sy = std::sin(pert[4]);
    const double cz = std::cos(pert[5]), sz = std::sin(pert[5]);
    const double Rx[3][3] = {{1, 0, 0}, {0, cx, -sx}, {0, sx, cx}}, dRx[3][3] = {{0, 0, 0}, {0, -sx, -cx}, {0, cx, -sx}};
    const double Ry[3][3] = {{cy, 0, sy}, {0, 1, 0}, {-sy, 0, cy}}, dRy[3][3] = {{-sy, 0, cy}, {0, 0, 0}, {-cy, 0, -sy}};
    const double Rz[3][3] = {{cz, -sz, 0}, {sz, cz, 0}, {0, 0, 1}}, dRz[3][3] = {{-sz, -cz, 0}, {cz, -sz, 0}, {0, 0, 0}};
    auto mul = [](const double A[3][3], const double B[3][3], double C[3][3]) {
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                C[i][j] = 0.0;
                for (int k = 0; k < 3; ++k) C[i][j] += A[i][k] * B[k][j];
            }
    };
    double T[3][3], D[3][3];
    mul(Ry, dRx, T); mul(Rz, T, D);
    for (int i = 0; i < 3; ++i) for (int k = 0; k < 3; ++k) dM[0][3 * i + k] = D[k][i];
    mul(dRy, Rx, T); mul(Rz, T, D);
    for (int i = 0; i < 3; ++i) for (int k = 0; k < 3; ++k) dM[1][3 * i + k] = D[k][i];
    mul(Ry, Rx, T); mul(dRz, T, D);
    for (int i = 0; i < 3; ++i) for (int k = 0; k < 3; ++k) dM[2][3 * i + k] = D[k][i];
}

phosim_status build_surface(const phosim_surface& s, DSurface& d) {
    std::memset(&d, 0, sizeof(d));
    d.kind = s.kind;
    d.material = s.material;
    d.coating = s.coating;
    d.coat_slot = -1;
    int flags = 0;
    if (s.R != 0.0) {
        flags |= SF_CONIC;
        d.c = 1.0 / s.R;
        d.k1c2 = (1.0 + s.kappa) / (s.R * s.R);
        d.kc = (1.0 + s.kappa) / s.R;
    }
    for (int i = 0; i < 4; ++i) {
        d.ao[i] = s.alpha[2 * i];        // alpha_3, 5, 7, 9
        d.ae[i] = s.alpha[2 * i + 1];    // alpha_4, 6, 8, 10
        if (d.ao[i] != 0.0) { flags |= SF_ODD; d.no = i + 1; }
        if (d.ae[i] != 0.0) { flags |= SF_EVEN; d.ne = i + 1; }
    }
    if (s.zern_rnorm > 0.0) d.zinv = 1.0 / s.zern_rnorm;
    if (s.n_zern > 0 && s.zern_rnorm > 0.0) {
        double P[7][7] = {}, Pj[7][7];
        bool any = false;
        for (int j = 1; j <= s.n_zern; ++j) {
            if (s.zern[j - 1] == 0.0) continue;
            any = true;
            zernike_monomials(j, Pj);
            for (int b = 0; b < 7; ++b)
                for (int a = 0; a + b < 7; ++a) P[b][a] += s.zern[j - 1] * Pj[b][a];
        }
        if (any) {
            flags |= SF_ZERN;
            int off = 0;
            for (int b = 0; b < 7; ++b)
                for (int a = 0; a + b < 7; ++a) d.zp[off++] = P[b][a];
        }
    }
    if (!(flags & (SF_CONIC | SF_EVEN | SF_ODD | SF_ZERN))) flags |= SF_FLAT_ONLY;
    if (s.pert[3] != 0.0 || s.pert[4] != 0.0 || s.pert[5] != 0.0) flags |= SF_ROTATED;
    if (s.pert[0] != 0.0 || s.pert[1] != 0.0) flags |= SF_DECENTERED;
    d.flags = flags;
    rotation(s.pert, d.M);
    d.o[0] = s.pert[0];
    d.o[1] = s.pert[1];
    d.o[2] = s.z + s.pert[2];
    d.r_in2 = s.r_in * s.r_in;
    d.r_out2 = s.r_out * s.r_out;
    return PHOSIM_OK;
}

// a double-single pair, with magnitudes beyond the single-precision range (an unlimited aperture) clamped
ds ds_clamped(double v) {
    if (v > 1e37) return ds{1e37f, 0.f};
    if (v < -1e37) return ds{-1e37f, 0.f};
    return ds_of(v);
}

// the double-single copy of a surface (DSurfaceS): asphere coefficients rescaled to rho = r / rn
void build_surface_s(const phosim_surface& s, const DSurface& d, DSurfaceS& e) {
    std::memset(&e, 0, sizeof(e));
    e.c = ds_of(d.c);
    e.k1c2 = ds_of(d.k1c2);
    e.kc = ds_of(d.kc);
    e.kmc = ds_of(d.kc - d.c);
    const double rn = (s.r_out > 0.0 && s.r_out < 1e6) ? s.r_out : 1000.0;
    for (int k = 0; k < 4; ++k) {
        const double ae = d.ae[k] * std::pow(rn, 2 * k + 4), ao = d.ao[k] * std::pow(rn, 2 * k + 3);
        e.ae[k] = ds_clamped(ae);
        e.aed[k] = ds_clamped((2 * k + 4) * ae);
        e.ao[k] = ds_clamped(ao);
        e.aod[k] = ds_clamped((2 * k + 3) * ao);
        e.ae2[k] = (float)((k + 1) * (2 * k + 4) * ae / (rn * rn * rn * rn));
        if (d.ae[k] != 0.0) e.ne = (unsigned char)(k + 1);
        if (d.ao[k] != 0.0) e.no = (unsigned char)(k + 1);
    }
    for (int i = 0; i < 9; ++i) e.M[i] = ds_of(d.M[i]);
    for (int i = 0; i < 3; ++i) e.o[i] = ds_of(d.o[i]);
    e.r_in2 = ds_clamped(d.r_in2);
    e.r_out2 = ds_clamped(d.r_out2);
    e.inv_rn = ds_of(1.0 / rn);
    e.inv_rn2 = ds_of(1.0 / (rn * rn));
    e.zinv = (float)d.zinv;
    for (int i = 0; i < kZPoly; ++i) e.zp[i] = (float)d.zp[i];
}

// integer accept thresholds of a transmission: the draw (w + 1/2) 2^-32 < T exactly when w < ceil(T 2^32 - 1/2)
unsigned long long accept_threshold(double T) {
    if (!(T > 0.0)) return 0ull;
    if (T >= 1.0) return 1ull << 32;
    return (unsigned long long)std::ceil(std::ldexp(T, 32) - 0.5);
}

// ----------------------------------------------------------------------------------------- device kernels
// central-difference gradient of a periodic phase screen, rad per mm (Sec. 2.3.2), stored per node as the
// 2 x 2 block of gradients the bilinear interpolation reads (see DScale)
__device__ __forceinline__ double2 central_gradient(const double* __restrict__ ph, int n, double two_pix, int i, int j) {
    const int ip = i + 1 == n ? 0 : i + 1, im = i == 0 ? n - 1 : i - 1;
    const int jp = j + 1 == n ? 0 : j + 1, jm = j == 0 ? n - 1 : j - 1;
    const size_t r = (size_t)j * n;
    return make_double2((ph[r + ip] - ph[r + im]) / two_pix, (ph[(size_t)jp * n + i] - ph[(size_t)jm * n + i]) / two_pix);
}

__global__ void gradient_screen_kernel(const double* __restrict__ ph, int n, double two_pix, double2* g64, float4* g32) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n) return;
    const int i1 = i + 1 == n ? 0 : i + 1, j1 = j + 1 == n ? 0 : j + 1;
    const double2 a = central_gradient(ph, n, two_pix, i, j), b = central_gradient(ph, n, two_pix, i1, j);
    const double2 c = central_gradient(ph, n, two_pix, i, j1), d = central_gradient(ph, n, two_pix, i1, j1);
    const size_t node = (size_t)j * n + i;
    g64[4 * node] = a; g64[4 * node + 1] = b; g64[4 * node + 2] = c; g64[4 * node + 3] = d;
    g32[2 * node] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    g32[2 * node + 1] = make_float4((float)c.x, (float)c.y, (float)d.x, (float)d.y);
}

// Photon-number cumulative table of each SED (flux x wavelength x bin width, summed in bin order with
// IEEE round-to-nearest operations and no contraction), turned into integer thresholds: bin k is taken by
// the draw w when ((w + 1/2) 2^-32) < cdf_k, i.e. w < ceil(cdf_k 2^32 - 1/2).
__global__ void sed_threshold_kernel(const double* __restrict__ flux, int n_sed, int n_bins, double lam0, double dlam,
                                     double* cum, unsigned long long* thr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sed) return;
    const double* f = flux + (size_t)s * n_bins;
    double* c = cum + (size_t)s * n_bins;
    double acc = 0.0;
    for (int k = 0; k < n_bins; ++k) {
        const double centre = __dadd_rn(lam0, __dmul_rn((double)k + 0.5, dlam));
        const double pk = __dmul_rn(__dmul_rn(f[k], centre), dlam);
        acc = __dadd_rn(acc, pk);
        c[k] = acc;
    }
    unsigned long long* t = thr + (size_t)s * (n_bins - 1);
    for (int k = 0; k < n_bins - 1; ++k) {
        const double ck = __ddiv_rn(c[k], acc);
        const double X = __dmul_rn(ck, 4294967296.0);
        t[k] = (unsigned long long)ceil(__dsub_rn(X, 0.5));
    }
}

// guide table of each SED's thresholds: guide[j] = the number of thresholds <= j 2^24, j = 0..kSedGuide
__global__ void sed_guide_kernel(const unsigned long long* __restrict__ thr, int n_sed, int n, int* guide) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int s = blockIdx.y;
    if (j > kSedGuide || s >= n_sed) return;
    const unsigned long long* t = thr + (size_t)s * n;
    const unsigned long long v = (unsigned long long)j << 24;
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (v < t[mid]) hi = mid;
        else lo = mid + 1;
    }
    guide[(size_t)s * (kSedGuide + 1) + j] = lo;
}

void destroy_graph(TraceGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    g = TraceGraph();
}

// Event pair number k of the scene's timing pool (grown on demand), tagged with a kernel kind.
phosim_status timing_pair(phosim_scene* sc, int kind, cudaEvent_t* a, cudaEvent_t* b) {
    const size_t k = (size_t)sc->timing_used;
    while (sc->timing_events.size() < 2 * (k + 1)) {
        cudaEvent_t e;
        CU(cudaEventCreate(&e));
        sc->timing_events.push_back(e);
    }
    if (sc->timing_kind.size() < k + 1) sc->timing_kind.resize(k + 1);
    sc->timing_kind[k] = kind;
    *a = sc->timing_events[2 * k];
    *b = sc->timing_events[2 * k + 1];
    sc->timing_used++;
    return PHOSIM_OK;
}

// one step of a trace call's launch sequence: a kernel launch (func set) or a memset to zero (func null)
struct LaunchOp {
    const void* func;
    dim3 grid, block;
    void** args;
    void* dst;
    size_t bytes;
};

// Launch a trace call's sequence as one CUDA graph: built node by node (each depending on the one before) when
// the sequence's shape (its kernels and memsets) differs from the scene's cached graph for this slot, then
// replayed on the caller's stream with this call's kernel parameters and launch shapes.
phosim_status launch_graph(phosim_scene* sc, int slot, const std::vector<LaunchOp>& ops, cudaStream_t st) {
    TraceGraph& g = sc->graphs[slot];
    const size_t n = ops.size();
    bool same = g.exec && g.func.size() == n;
    for (size_t i = 0; same && i < n; ++i)
        same = g.func[i] == ops[i].func && g.memset_dst[i] == (ops[i].func ? nullptr : ops[i].dst) &&
               g.memset_bytes[i] == (ops[i].func ? 0 : ops[i].bytes);
    if (g.exec && !same) destroy_graph(g);
    if (!g.exec) {
        if (cudaGraphCreate(&g.graph, 0) != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
        cudaGraphNode_t prev = nullptr;
        for (size_t i = 0; i < n; ++i) {
            const LaunchOp& o = ops[i];
            cudaGraphNode_t node = nullptr;
            cudaError_t e;
            if (o.func) {
                cudaKernelNodeParams kp = {};
                kp.func = (void*)o.func;
                kp.gridDim = o.grid;
                kp.blockDim = o.block;
                kp.kernelParams = o.args;
                e = cudaGraphAddKernelNode(&node, g.graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
            } else {
                cudaMemsetParams mp = {};
                mp.dst = o.dst;
                mp.value = 0;
                mp.elementSize = 4;
                mp.width = o.bytes / 4;
                mp.height = 1;
                mp.pitch = 0;
                e = cudaGraphAddMemsetNode(&node, g.graph, prev ? &prev : nullptr, prev ? 1 : 0, &mp);
            }
            if (e != cudaSuccess) { destroy_graph(g); (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
            g.func.push_back(o.func);
            g.memset_dst.push_back(o.func ? nullptr : o.dst);
            g.memset_bytes.push_back(o.func ? 0 : o.bytes);
            g.node.push_back(node);
            prev = node;
        }
        if (cudaGraphInstantiate(&g.exec, g.graph, 0) != cudaSuccess) { destroy_graph(g); (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    } else {
        for (size_t i = 0; i < n; ++i) {
            if (!ops[i].func) continue;
            cudaKernelNodeParams kp = {};
            kp.func = (void*)ops[i].func;
            kp.gridDim = ops[i].grid;
            kp.blockDim = ops[i].block;
            kp.kernelParams = ops[i].args;
            CU(cudaGraphExecKernelNodeSetParams(g.exec, g.node[i], &kp));
        }
    }
    CU(cudaGraphLaunch(g.exec, st));
    return PHOSIM_OK;
}

}  // namespace

namespace phosim {

phosim_status check_scene_device(const phosim_scene* sc) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    return dev == sc->device ? PHOSIM_OK : PHOSIM_ERR_INVALID_ARGUMENT;
}

phosim_status check_device_buffer(const void* p, int device) {
    if (!p) return PHOSIM_OK;
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) { (void)cudaGetLastError(); return PHOSIM_ERR_INVALID_ARGUMENT; }
    if (attr.type == cudaMemoryTypeManaged) return PHOSIM_OK;
    if (attr.type == cudaMemoryTypeDevice && attr.device == device) return PHOSIM_OK;
    return PHOSIM_ERR_INVALID_ARGUMENT;
}

// Sec. 3.1 (the number of detected photons of every source and their mean coordinate) and the second moments
// of the image-quality gates: the sums are about a reference point (ref_x, ref_y), so the centroid is
// ref + sum(d) / n and the central moments sum(d d') / n - mean(d) mean(d'), with d = x - ref small.
void derive_moments(const double* sums, int n_src, double* out6) {
    for (int s = 0; s < n_src; ++s) {
        const double* M = sums + (size_t)s * PHOSIM_MOMENT_WORDS;
        double* o = out6 + (size_t)s * 6;
        const double n = M[0];
        o[0] = n;
        if (n > 0) {
            const double ux = M[1] / n, uy = M[2] / n;
            o[1] = M[6] + ux; o[2] = M[7] + uy;
            o[3] = M[3] / n - ux * ux; o[4] = M[4] / n - ux * uy; o[5] = M[5] / n - uy * uy;
        } else {
            for (int k = 1; k < 6; ++k) o[k] = std::nan("");
        }
    }
}

}  // namespace phosim

// =================================================================================================
extern "C" {

const char* phosim_status_string(phosim_status s) {
    switch (s) {
        case PHOSIM_OK: return "ok";
        case PHOSIM_ERR_INVALID_ARGUMENT: return "invalid argument";
        case PHOSIM_ERR_OUT_OF_MEMORY: return "out of device memory";
        case PHOSIM_ERR_CUDA: return "CUDA error";
        case PHOSIM_ERR_UNSUPPORTED: return "unsupported";
        case PHOSIM_ERR_NOT_READY: return "scene not ready (optics or SEDs not loaded)";
        case PHOSIM_ERR_LIMIT: return "size exceeds a library maximum";
        default: return "unknown status";
    }
}

phosim_status phosim_create_scene(const phosim_scene_desc* d, phosim_scene** out) {
    if (!d || !out) return PHOSIM_ERR_INVALID_ARGUMENT;
    *out = nullptr;
    if (d->precision != PHOSIM_PLAIN_FP64 && d->precision != PHOSIM_MIXED && d->precision != PHOSIM_MIXED_DS)
        return PHOSIM_ERR_INVALID_ARGUMENT;
    if (d->nx <= 0 || d->ny <= 0 || (int64_t)d->nx * d->ny > (int64_t)1 << 31) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!(d->pixel > 0.0) || !(d->t_si > 0.0) || !(d->lambda_ref > 0.0) || !(d->ell_dlam > 0.0))
        return PHOSIM_ERR_INVALID_ARGUMENT;
    if (d->n_ell < 2 || d->n_sigma < 2 || !d->ell || !d->sigma) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!(d->pupil_r_out > d->pupil_r_in) || d->pupil_r_in < 0.0) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!(d->h_top > d->z_entrance) || !is_finite(d->h_top) || !is_finite(d->z_entrance)) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!(d->dead_layer >= 0.0) || !(d->dead_layer < d->t_si)) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!is_finite(d->t_si_gx) || !is_finite(d->t_si_gy)) return PHOSIM_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < d->n_ell; ++i) if (!(d->ell[i] > 0.0) || !is_finite(d->ell[i])) return PHOSIM_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < d->n_sigma; ++i) if (!(d->sigma[i] >= 0.0) || !is_finite(d->sigma[i])) return PHOSIM_ERR_INVALID_ARGUMENT;
    phosim_scene* sc = new (std::nothrow) phosim_scene();
    if (!sc) return PHOSIM_ERR_OUT_OF_MEMORY;
    std::memset(&sc->base, 0, sizeof(sc->base));
    TraceParams& P = sc->base;
    P.k0 = (uint32_t)d->seed;
    P.k1 = (uint32_t)(d->seed >> 32);
    P.flags = d->flags;
    P.pr_in2 = d->pupil_r_in * d->pupil_r_in;
    P.pr_dr2 = d->pupil_r_out * d->pupil_r_out - P.pr_in2;
    P.h_top = d->h_top;
    P.z_ent = d->z_entrance;
    P.lam_ref = d->lambda_ref;
    P.kick0 = d->lambda_ref * 1e-6 / (2.0 * M_PI);
    P.nx = d->nx; P.ny = d->ny;
    P.pixel = d->pixel; P.inv_pixel = 1.0 / d->pixel;
    P.xlo = d->x0 - 0.5 * d->nx * d->pixel;
    P.ylo = d->y0 - 0.5 * d->ny * d->pixel;
    P.t_si = d->t_si;
    P.ell_lam0 = d->ell_lam0; P.inv_ell_dlam = 1.0 / d->ell_dlam;
    P.n_ell = d->n_ell; P.n_sig = d->n_sigma;
    P.sig_scale = (d->n_sigma - 1) / d->t_si;
    P.dead_layer = d->dead_layer;
    // fringing: optical thickness t_si + gx (x - x0) + gy (y - y0) = fr_t0 + gx x + gy y
    P.fr_gx = d->t_si_gx; P.fr_gy = d->t_si_gy;
    P.fr_t0 = d->t_si - d->t_si_gx * d->x0 - d->t_si_gy * d->y0;
    P.fr_t0_s = ds_of(P.fr_t0); P.fr_gxf = (float)P.fr_gx; P.fr_gyf = (float)P.fr_gy;
    P.pr_in2_s = ds_of(P.pr_in2); P.pr_dr2_s = ds_of(P.pr_dr2);
    P.h_top_s = ds_of(P.h_top); P.z_ent_s = ds_of(P.z_ent);
    P.xlo_s = ds_of(P.xlo); P.ylo_s = ds_of(P.ylo); P.inv_pixel_s = ds_of(P.inv_pixel);
    P.chip_w_s = ds_of(P.nx * P.pixel); P.chip_h_s = ds_of(P.ny * P.pixel);
    P.kick0f = (float)P.kick0; P.inv_lam_ref_f = (float)(1.0 / P.lam_ref);
    P.t_sif = (float)P.t_si; P.dead_layerf = (float)P.dead_layer;
    P.ell_lam0f = (float)P.ell_lam0; P.inv_ell_dlamf = (float)P.inv_ell_dlam; P.sig_scalef = (float)P.sig_scale;
    sc->precision = d->precision;
    std::vector<float> f(d->ell, d->ell + d->n_ell), g(d->sigma, d->sigma + d->n_sigma);
    double* pd;
    float* pf;
    phosim_status st;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sc->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        delete sc;
        return PHOSIM_ERR_CUDA;
    }
    sc->device = dev;
    if ((st = upload(sc->table_mem, d->ell, (size_t)d->n_ell, &pd)) != PHOSIM_OK) goto fail;
    P.ell = pd;
    if ((st = upload(sc->table_mem, f.data(), f.size(), &pf)) != PHOSIM_OK) goto fail;
    P.ell32 = pf;
    if ((st = upload(sc->table_mem, d->sigma, (size_t)d->n_sigma, &pd)) != PHOSIM_OK) goto fail;
    P.sig = pd;
    if ((st = upload(sc->table_mem, g.data(), g.size(), &pf)) != PHOSIM_OK) goto fail;
    P.sig32 = pf;
    if (cudaMalloc(&sc->d_counters, 16 * sizeof(unsigned long long)) != cudaSuccess) {
        (void)cudaGetLastError();
        st = PHOSIM_ERR_OUT_OF_MEMORY;
        goto fail;
    }
    cudaMemset(sc->d_counters, 0, 16 * sizeof(unsigned long long));
    *out = sc;
    return PHOSIM_OK;
fail:
    phosim_destroy_scene(sc);
    return st;
}

void phosim_destroy_scene(phosim_scene* sc) {
    if (!sc) return;
    if (sc->last_stream) cudaStreamSynchronize(sc->last_stream);
    free_all(sc->table_mem);
    free_all(sc->optics_mem);
    free_all(sc->screen_mem);
    free_all(sc->sed_mem);
    free_all(sc->sersic_mem);
    free_all(sc->hf_mem);
    cudaFree(sc->d_src);
    cudaFree(sc->d_src_s);
    cudaFree(sc->d_prefix);
    cudaFree(sc->d_counters);
    cudaFree(sc->d_stage);
    cudaFree(sc->d_state);
    cudaFree(sc->d_hits);
    cudaFree(sc->d_mom_stripes);
    cudaFree(sc->d_grad_scratch);
    cudaFree(sc->d_mom_scratch);
    for (TraceGraph& g : sc->graphs) destroy_graph(g);
    for (cudaEvent_t e : sc->timing_events) cudaEventDestroy(e);
    if (sc->capture_stream) cudaStreamDestroy(sc->capture_stream);
    (void)cudaGetLastError();
    delete sc;
}

phosim_status phosim_load_optics(phosim_scene* sc, const phosim_surface* surf, int n_surf, const phosim_material* mats,
                                 int n_mat, const phosim_coating* coats, int n_coat) {
    if (!sc || !surf || n_surf < 1 || (n_mat > 0 && !mats) || (n_coat > 0 && !coats) || n_mat < 1 || n_coat < 0)
        return PHOSIM_ERR_INVALID_ARGUMENT;
    if (check_scene_device(sc) != PHOSIM_OK) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (n_surf > PHOSIM_MAX_SURFACES || n_mat > kMaxMaterials || n_coat > kMaxCoatings) return PHOSIM_ERR_LIMIT;
    for (int i = 0; i < n_surf; ++i) {
        const phosim_surface& s = surf[i];
        const bool last = i == n_surf - 1;
        if (s.kind < PHOSIM_MIRROR || s.kind > PHOSIM_DETECTOR) return PHOSIM_ERR_INVALID_ARGUMENT;
        if ((s.kind == PHOSIM_DETECTOR) != last) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (s.material < 0 || s.material >= n_mat) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (s.coating < -1 || s.coating >= n_coat) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (s.n_zern < 0 || s.n_zern > PHOSIM_MAX_ZERNIKE) return PHOSIM_ERR_LIMIT;
        if (!is_finite(s.R) || !is_finite(s.kappa) || !is_finite(s.z) || s.r_in < 0.0 || !(s.r_out >= s.r_in))
            return PHOSIM_ERR_INVALID_ARGUMENT;
    }
    for (int k = 0; k < n_mat; ++k)
        if (mats[k].kind < PHOSIM_VACUUM || mats[k].kind > PHOSIM_SILICON) return PHOSIM_ERR_INVALID_ARGUMENT;
    for (int k = 0; k < n_coat; ++k) {
        if (!coats[k].table || coats[k].n_lambda < 1 || coats[k].n_theta < 1 || !(coats[k].dlam > 0.0) ||
            !(coats[k].dtheta > 0.0))
            return PHOSIM_ERR_INVALID_ARGUMENT;
        if (coats[k].reflect)
            for (size_t i = 0; i < (size_t)coats[k].n_lambda * coats[k].n_theta; ++i)
                if (!(coats[k].reflect[i] >= 0.0) || !(coats[k].table[i] + coats[k].reflect[i] <= 1.0 + 1e-12))
                    return PHOSIM_ERR_INVALID_ARGUMENT;
    }
    TraceParams P = sc->base;
    int coated = 0;
    for (int i = 0; i < n_surf; ++i) {
        build_surface(surf[i], P.surf[i]);
        build_surface_s(surf[i], P.surf[i], P.surf_s[i]);
        if (surf[i].coating >= 0 && surf[i].kind != PHOSIM_DETECTOR) {
            if (coated >= PHOSIM_MAX_COATED) return PHOSIM_ERR_LIMIT;
            P.coated_surface[coated] = i;
            P.surf[i].coat_slot = coated++;
        }
    }
    P.pupil_surf = P.surf[0];
    P.pupil_surf.flags &= ~SF_ZERN;
    if (!(P.pupil_surf.flags & (SF_CONIC | SF_EVEN | SF_ODD))) P.pupil_surf.flags |= SF_FLAT_ONLY;
    P.pupil_z = surf[0].z;
    P.pupil_s = P.surf_s[0];
    P.pupil_z_s = ds_of(P.pupil_z);
    P.n_surf = n_surf;
    P.n_coated = coated;
    P.n_mat = n_mat;
    for (int k = 0; k < n_mat; ++k) {
        P.mat[k].kind = mats[k].kind;
        for (int q = 0; q < 3; ++q) {
            P.mat[k].B[q] = mats[k].B[q]; P.mat[k].C[q] = mats[k].C[q];
            P.mat[k].Bs[q] = ds_of(mats[k].B[q]); P.mat[k].Cs[q] = ds_of(mats[k].C[q]);
        }
    }
    std::vector<void*> mem;
    bool ghosts = false;
    for (int k = 0; k < n_coat; ++k) {
        double *d, *dmax;
        unsigned long long *dthr, *dmax_thr;
        const int nl = coats[k].n_lambda, nt = coats[k].n_theta;
        // the dynamic transmission test (early rejection) keeps a photon while it can still be transmitted or,
        // with a reflection table, reflected: its bound is the largest T + R over angles
        const double* R = coats[k].reflect;
        std::vector<double> tr((size_t)nl * nt), tmax((size_t)nl, 0.0);
        for (size_t i = 0; i < tr.size(); ++i) tr[i] = coats[k].table[i] + (R ? R[i] : 0.0);
        std::vector<unsigned long long> thr((size_t)nl * nt), tr_thr((size_t)nl * nt), tmax_thr((size_t)nl);
        for (int il = 0; il < nl; ++il)
            for (int it = 0; it < nt; ++it) tmax[il] = std::max(tmax[il], tr[(size_t)il * nt + it]);
        for (size_t i = 0; i < thr.size(); ++i) thr[i] = accept_threshold(coats[k].table[i]);
        for (size_t i = 0; i < tr.size(); ++i) tr_thr[i] = accept_threshold(tr[i]);
        for (int il = 0; il < nl; ++il) tmax_thr[il] = accept_threshold(tmax[il]);
        double* dtr = nullptr;
        unsigned long long* dtr_thr = nullptr;
        phosim_status st = upload(mem, coats[k].table, (size_t)nl * nt, &d);
        if (st == PHOSIM_OK) st = upload(mem, tmax.data(), tmax.size(), &dmax);
        if (st == PHOSIM_OK) st = upload(mem, thr.data(), thr.size(), &dthr);
        if (st == PHOSIM_OK) st = upload(mem, tmax_thr.data(), tmax_thr.size(), &dmax_thr);
        if (st == PHOSIM_OK && R) st = upload(mem, tr.data(), tr.size(), &dtr);
        if (st == PHOSIM_OK && R) st = upload(mem, tr_thr.data(), tr_thr.size(), &dtr_thr);
        if (st != PHOSIM_OK) { free_all(mem); return st; }
        if (R) ghosts = true;
        DCoating& C = P.coat[k];
        C.lam0 = coats[k].lam0; C.inv_dlam = 1.0 / coats[k].dlam;
        C.th0 = coats[k].theta0; C.inv_dth = 1.0 / coats[k].dtheta;
        C.lam0f = (float)C.lam0; C.inv_dlamf = (float)C.inv_dlam; C.th0f = (float)C.th0; C.inv_dthf = (float)C.inv_dth;
        C.lam0_s = ds_of(C.lam0); C.inv_dlam_s = ds_of(C.inv_dlam);
        C.T_thr = dthr;
        C.Tmax_thr = dmax_thr;
        C.TR = dtr;
        C.TR_thr = dtr_thr;
        C.nl = coats[k].n_lambda; C.nt = coats[k].n_theta;
        C.T = d;
        C.Tmax = dmax;
    }
    P.n_coat = n_coat;
    P.flags = ghosts ? (P.flags | kGhostFlag) : (P.flags & ~kGhostFlag);
    // the medium in front of each surface, for ghosts that refract on their way back
    {
        int m = -1;
        for (int i = 0; i < n_surf; ++i) {
            P.surf[i].mat_before = m;
            if (surf[i].kind != PHOSIM_MIRROR) m = surf[i].material;
        }
    }
    {
        std::vector<double> zm((size_t)PHOSIM_MAX_ZERNIKE * kZPoly, 0.0);
        for (int j = 1; j <= PHOSIM_MAX_ZERNIKE; ++j) {
            double Pj[7][7];
            zernike_monomials(j, Pj);
            int off = 0;
            for (int b = 0; b < 7; ++b)
                for (int a = 0; a + b < 7; ++a) zm[(size_t)(j - 1) * kZPoly + off++] = Pj[b][a];
        }
        double* dz;
        phosim_status st = upload(mem, zm.data(), zm.size(), &dz);
        if (st != PHOSIM_OK) { free_all(mem); return st; }
        sc->d_zmono = dz;
    }
    free_all(sc->optics_mem);
    sc->optics_mem = mem;
    sc->base = P;
    sc->surfaces.assign(surf, surf + n_surf);
    sc->optics_loaded = true;
    return PHOSIM_OK;
}

phosim_status phosim_load_screens(phosim_scene* sc, const phosim_layer* layers, int n_layers) {
    if (!sc || n_layers < 0 || (n_layers > 0 && !layers)) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (check_scene_device(sc) != PHOSIM_OK) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (n_layers > PHOSIM_MAX_LAYERS) return PHOSIM_ERR_LIMIT;
    for (int k = 0; k < n_layers; ++k) {
        const phosim_layer& L = layers[k];
        if (L.n_scales < 1 || L.n_scales > PHOSIM_MAX_SCALES) return PHOSIM_ERR_LIMIT;
        if (k > 0 && !(L.z < layers[k - 1].z)) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (!is_finite(L.z) || !is_finite(L.vx) || !is_finite(L.vy)) return PHOSIM_ERR_INVALID_ARGUMENT;
        for (int q = 0; q < L.n_scales; ++q)
            if (L.scales[q].n < 3 || !(L.scales[q].pixel > 0.0) || !L.scales[q].phase) return PHOSIM_ERR_INVALID_ARGUMENT;
    }
    TraceParams P = sc->base;
    std::vector<void*> mem;
    for (int k = 0; k < n_layers; ++k) {
        const phosim_layer& L = layers[k];
        DLayer& D = P.layer[k];
        D.z = L.z; D.vx = L.vx; D.vy = L.vy; D.n_scales = L.n_scales;
        D.zs = ds_of(L.z); D.vxs = ds_of(L.vx); D.vys = ds_of(L.vy);
        D.dzs = ds_of((k == 0 ? P.h_top : layers[k - 1].z) - L.z);
        for (int q = 0; q < L.n_scales; ++q) {
            const phosim_screen_scale& S = L.scales[q];
            const size_t nn = (size_t)S.n * S.n;
            double* ph = nullptr;
            void *g64 = nullptr, *g32 = nullptr;
            cudaError_t e = cudaMalloc(&ph, nn * sizeof(double));
            if (e == cudaSuccess) e = cudaMalloc(&g64, 4 * nn * sizeof(double2));
            if (e == cudaSuccess) { mem.push_back(g64); e = cudaMalloc(&g32, 2 * nn * sizeof(float4)); }
            if (e == cudaSuccess) { mem.push_back(g32); e = cudaMemcpy(ph, S.phase, nn * sizeof(double), cudaMemcpyHostToDevice); }
            if (e == cudaSuccess) {
                gradient_screen_kernel<<<dim3((S.n + 255) / 256, S.n), 256>>>(ph, S.n, 2.0 * S.pixel, (double2*)g64, (float4*)g32);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
            cudaFree(ph);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                free_all(mem);
                return e == cudaErrorMemoryAllocation ? PHOSIM_ERR_OUT_OF_MEMORY : PHOSIM_ERR_CUDA;
            }
            D.s[q].n = S.n;
            D.s[q].inv_pix = 1.0 / S.pixel;
            D.s[q].inv_pix_s = ds_of(1.0 / S.pixel);
            D.s[q].g64 = (const double2*)g64;
            D.s[q].g32 = (const float4*)g32;
        }
    }
    P.n_layers = n_layers;
    free_all(sc->screen_mem);
    sc->screen_mem = mem;
    sc->base = P;
    return PHOSIM_OK;
}

phosim_status phosim_load_seds(phosim_scene* sc, const double* flux, int n_sed, int n_bins, double lam0, double dlam) {
    if (!sc || !flux || n_sed < 1 || n_bins < 2 || !(dlam > 0.0) || !is_finite(lam0)) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (check_scene_device(sc) != PHOSIM_OK) return PHOSIM_ERR_INVALID_ARGUMENT;
    const size_t n = (size_t)n_sed * n_bins;
    double total = 0.0;
    for (int s = 0; s < n_sed; ++s) {
        double row = 0.0;
        for (int k = 0; k < n_bins; ++k) {
            const double v = flux[(size_t)s * n_bins + k];
            if (!(v >= 0.0) || !is_finite(v)) return PHOSIM_ERR_INVALID_ARGUMENT;
            row += v;
        }
        if (!(row > 0.0)) return PHOSIM_ERR_INVALID_ARGUMENT;
        total += row;
    }
    std::vector<void*> mem;
    double *d_flux = nullptr, *d_cum = nullptr;
    unsigned long long* d_thr = nullptr;
    cudaError_t e = cudaMalloc(&d_flux, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&d_cum, n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&d_thr, (size_t)n_sed * (n_bins - 1) * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(d_flux, flux, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        sed_threshold_kernel<<<(n_sed + 127) / 128, 128>>>(d_flux, n_sed, n_bins, lam0, dlam, d_cum, d_thr);
        e = cudaGetLastError();
    }
    int* d_guide = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d_guide, (size_t)n_sed * (kSedGuide + 1) * sizeof(int));
    if (e == cudaSuccess) {
        sed_guide_kernel<<<dim3((kSedGuide + 1 + 127) / 128, n_sed), 128>>>(d_thr, n_sed, n_bins - 1, d_guide);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_flux);
    cudaFree(d_cum);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(d_thr);
        cudaFree(d_guide);
        return e == cudaErrorMemoryAllocation ? PHOSIM_ERR_OUT_OF_MEMORY : PHOSIM_ERR_CUDA;
    }
    free_all(sc->sed_mem);
    sc->sed_mem.push_back(d_thr);
    sc->sed_mem.push_back(d_guide);
    sc->base.thr = d_thr;
    sc->base.sed_guide = d_guide;
    sc->base.n_bins = n_bins;
    sc->base.sed_lam0 = lam0;
    sc->base.sed_dlam = dlam;
    sc->base.sed_lam0f = (float)lam0;
    sc->base.sed_dlamf = (float)dlam;
    sc->base.sed_lam0_s = ds_of(lam0);
    sc->base.sed_dlam_s = ds_of(dlam);
    sc->n_sed = n_sed;
    sc->seds_loaded = true;
    return PHOSIM_OK;
}

phosim_status phosim_load_sersic(phosim_scene* sc, const double* table, int n_tables, int n_nodes) {
    if (!sc || !table || n_tables < 1 || n_nodes < 2) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (check_scene_device(sc) != PHOSIM_OK) return PHOSIM_ERR_INVALID_ARGUMENT;
    const size_t n = (size_t)n_tables * n_nodes;
    for (size_t i = 0; i < n; ++i) if (!(table[i] >= 0.0) || !is_finite(table[i])) return PHOSIM_ERR_INVALID_ARGUMENT;
    std::vector<float> f(table, table + n);
    std::vector<void*> mem;
    double* d;
    float* df;
    phosim_status st = upload(mem, table, n, &d);
    if (st == PHOSIM_OK) st = upload(mem, f.data(), n, &df);
    if (st != PHOSIM_OK) { free_all(mem); return st; }
    free_all(sc->sersic_mem);
    sc->sersic_mem = mem;
    sc->base.sersic = d;
    sc->base.sersic32 = df;
    sc->base.sersic_K = n_nodes;
    sc->sersic_tables = n_tables;
    return PHOSIM_OK;
}

phosim_status phosim_load_hf_kick(phosim_scene* sc, const double* q, int n) {
    if (!sc || n < 0 || (n > 0 && (!q || n < 2))) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (check_scene_device(sc) != PHOSIM_OK) return PHOSIM_ERR_INVALID_ARGUMENT;
    for (int i = 0; i < n; ++i) if (!(q[i] >= 0.0) || !is_finite(q[i]) || (i && q[i] < q[i - 1])) return PHOSIM_ERR_INVALID_ARGUMENT;
    std::vector<void*> mem;
    double* d = nullptr;
    float* df = nullptr;
    if (n > 0) {
        std::vector<float> f(q, q + n);
        phosim_status st = upload(mem, q, (size_t)n, &d);
        if (st == PHOSIM_OK) st = upload(mem, f.data(), (size_t)n, &df);
        if (st != PHOSIM_OK) { free_all(mem); return st; }
    }
    free_all(sc->hf_mem);
    sc->hf_mem = mem;
    sc->base.hf = d;
    sc->base.hf32 = df;
    sc->base.hf_K = n;
    return PHOSIM_OK;
}

phosim_status phosim_set_schedule(phosim_scene* sc, int threads, int tile) {
    if (!sc || threads < 0 || tile < 0) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (threads) {
        if (threads % 32 || threads > 256) return PHOSIM_ERR_INVALID_ARGUMENT;
        sc->threads = threads;
    }
    if (tile) {
        if (tile > (1 << 20)) return PHOSIM_ERR_LIMIT;
        sc->tile_photons = tile;
    }
    return PHOSIM_OK;
}

phosim_status phosim_get_schedule(const phosim_scene* sc, int* threads, int* tile) {
    if (!sc || !threads || !tile) return PHOSIM_ERR_INVALID_ARGUMENT;
    *threads = sc->threads;
    *tile = sc->tile_photons;
    return PHOSIM_OK;
}

phosim_status phosim_moments_derive(const double* sums, int n_src, double* out) {
    if (n_src < 0 || (n_src > 0 && (!sums || !out))) return PHOSIM_ERR_INVALID_ARGUMENT;
    derive_moments(sums, n_src, out);
    return PHOSIM_OK;
}

phosim_status phosim_autotune(phosim_scene* sc, const phosim_source* src, int n_src, const uint64_t* n_photons,
                              uint64_t sample, void* stream, int* out_threads, int* out_tile) {
    if (!sc || n_src < 1 || !src || !n_photons || sample < 1) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (check_scene_device(sc) != PHOSIM_OK) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!sc->optics_loaded || !sc->seds_loaded) return PHOSIM_ERR_NOT_READY;
    uint64_t total = 0;
    for (int s = 0; s < n_src; ++s) total += n_photons[s];
    if (total == 0) return PHOSIM_ERR_INVALID_ARGUMENT;
    std::vector<uint64_t> cnt((size_t)n_src);
    for (int s = 0; s < n_src; ++s) {
        const double f = (double)n_photons[s] * (double)sample / (double)total;
        cnt[s] = n_photons[s] ? std::max<uint64_t>(1, (uint64_t)std::llround(f)) : 0;
        cnt[s] = std::min(cnt[s], n_photons[s]);
    }
    const size_t img_bytes = (size_t)sc->base.nx * sc->base.ny * sizeof(uint32_t);
    if (sc->cap_stage < img_bytes) {
        cudaFree(sc->d_stage);
        sc->d_stage = nullptr; sc->cap_stage = 0;
        CU(cudaMalloc(&sc->d_stage, img_bytes));
        sc->cap_stage = img_bytes;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); (void)cudaGetLastError(); return PHOSIM_ERR_CUDA; }
    const int saved_threads = sc->threads, saved_tile = sc->tile_photons;
    const int threads_c[3] = {64, 128, 256};
    const int tiles_c[4] = {64, 256, 1024, 4096};
    float best = 1e30f;
    int bt = saved_threads, bk = saved_tile;
    phosim_status rs = PHOSIM_OK;
    for (int a = 0; a < 3 && rs == PHOSIM_OK; ++a)
        for (int b = 0; b < 4 && rs == PHOSIM_OK; ++b) {
            sc->threads = threads_c[a];
            sc->tile_photons = tiles_c[b];
            float ms_best = 1e30f;
            for (int rep = 0; rep < 3 && rs == PHOSIM_OK; ++rep) {
                cudaEventRecord(e0, st);
                rs = phosim_trace(sc, src, n_src, cnt.data(), nullptr, sc->d_stage, nullptr, nullptr, stream);
                cudaEventRecord(e1, st);
                if (rs == PHOSIM_OK && cudaEventSynchronize(e1) == cudaSuccess) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0) ms_best = std::min(ms_best, ms);     // the first run warms up
                }
            }
            if (ms_best < best) { best = ms_best; bt = threads_c[a]; bk = tiles_c[b]; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    (void)cudaGetLastError();
    sc->threads = rs == PHOSIM_OK ? bt : saved_threads;
    sc->tile_photons = rs == PHOSIM_OK ? bk : saved_tile;
    if (out_threads) *out_threads = sc->threads;
    if (out_tile) *out_tile = sc->tile_photons;
    return rs;
}

phosim_status phosim_set_stage_timing(phosim_scene* sc, int on) {
    if (!sc) return PHOSIM_ERR_INVALID_ARGUMENT;
    sc->stage_timing = on != 0;
    return PHOSIM_OK;
}

phosim_status phosim_stage_times(phosim_scene* sc, double* ms, int n) {
    if (!sc || !ms || n < 5) return PHOSIM_ERR_INVALID_ARGUMENT;
    for (int k = 0; k < n; ++k) ms[k] = 0.0;
    for (int k = 0; k < sc->timing_used; ++k) {
        CU(cudaEventSynchronize(sc->timing_events[2 * k + 1]));
        float t = 0.f;
        CU(cudaEventElapsedTime(&t, sc->timing_events[2 * k], sc->timing_events[2 * k + 1]));
        ms[sc->timing_kind[k]] += t;
    }
    return PHOSIM_OK;
}

phosim_status phosim_get_counters(phosim_scene* sc, uint64_t* out, int n) {
    if (!sc || !out || n < kNumCounters) return PHOSIM_ERR_INVALID_ARGUMENT;
    unsigned long long h[kNumCounters];
    CU(cudaStreamSynchronize(sc->last_stream));
    CU(cudaMemcpy(h, sc->d_counters + 1, sizeof(h), cudaMemcpyDeviceToHost));
    for (int k = 0; k < kNumCounters; ++k) out[k] = h[k];
    return PHOSIM_OK;
}

phosim_status phosim_trace(phosim_scene* sc, const phosim_source* src, int n_src, const uint64_t* n_photons,
                           const uint64_t* first, uint32_t* image, phosim_photon_record* records, double* moments,
                           void* stream) {
    if (!sc || n_src < 0 || (n_src > 0 && (!src || !n_photons)) || !image) return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!sc->optics_loaded || !sc->seds_loaded) return PHOSIM_ERR_NOT_READY;
    {   // the scene's device must be current; records and moments must be device memory on it
        phosim_status vs = check_scene_device(sc);
        if (vs == PHOSIM_OK) vs = check_device_buffer(records, sc->device);
        if (vs == PHOSIM_OK) vs = check_device_buffer(moments, sc->device);
        if (vs != PHOSIM_OK) return vs;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int mode = sc->precision;
    const bool staged = mode == PHOSIM_MIXED_DS;        // the two-kernel double-single path
    // launch shape
    int per_sm = 0, per_sm_optics = 0, per_sm_members = 0;
    if (staged) CU(ds_stage_occupancy(sc->threads, &per_sm, &per_sm_optics, &per_sm_members));
    else CU(trace_occupancy(mode, sc->threads, &per_sm));
    per_sm = std::max(per_sm, 1);
    per_sm_optics = std::max(per_sm_optics, 1);
    per_sm_members = std::max(per_sm_members, 1);
    const int blocks = sc->sm_count * per_sm, blocks_optics = sc->sm_count * per_sm_optics;
    const int blocks_members = sc->sm_count * per_sm_members;
    const uint64_t warps = (uint64_t)blocks * (sc->threads / 32);
    uint64_t total = 0;
    for (int s = 0; s < n_src; ++s) total += n_photons[s];
    uint64_t T = sc->tile_photons;
    if (!T) {
        T = total / (warps * 8);
        T = std::min<uint64_t>(1024, std::max<uint64_t>(32, (T + 31) / 32 * 32));
    }
    // sources and per-source tile prefix
    std::vector<DSource> hs((size_t)n_src);
    std::vector<unsigned long long> prefix((size_t)n_src + 1, 0);
    uint64_t rec = 0, bundled_units = 0;
    for (int s = 0; s < n_src; ++s) {
        const phosim_source& q = src[s];
        if (q.kind < PHOSIM_POINT || q.kind > PHOSIM_GAUSS) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.sed < 0 || q.sed >= sc->n_sed) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.kind == PHOSIM_SERSIC && (q.table < 0 || q.table >= sc->sersic_tables)) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (!is_finite(q.xi) || !is_finite(q.eta) || q.xi * q.xi + q.eta * q.eta >= 1.0 || !(q.redshift > -1.0))
            return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.bundle < 0 || (q.bundle > 1 && !(q.bundle_sigma >= 0.0 && is_finite(q.bundle_sigma))))
            return PHOSIM_ERR_INVALID_ARGUMENT;
        if (q.bundle > PHOSIM_MAX_BUNDLE) return PHOSIM_ERR_LIMIT;
        DSource& d = hs[s];
        std::memset(&d, 0, sizeof(d));
        d.kind = q.kind; d.sed = q.sed; d.table = q.table;
        d.xi = q.xi; d.eta = q.eta; d.zfac = 1.0 + q.redshift; d.t0 = q.t0; d.t_exp = q.t_exp;
        d.a = q.a; d.b = q.b; d.cpa = std::cos(q.pa); d.spa = std::sin(q.pa);
        d.bundle = q.bundle > 1 ? (uint32_t)q.bundle : 1u;
        d.bsig = q.bundle > 1 ? q.bundle_sigma : 0.0;
        d.first = first ? first[s] : 0;
        d.count = n_photons[s];
        d.rec_off = rec;
        rec += n_photons[s];
        // work units: photons, or in the two-kernel path the rays of a bundle that have photons in the range
        d.ufirst = d.first;
        d.ucount = d.count;
        if (staged && d.bundle > 1 && d.count > 0) {
            d.ufirst = d.first / d.bundle;
            d.ucount = (d.first + d.count + d.bundle - 1) / d.bundle - d.ufirst;
            bundled_units += d.ucount;
        }
        prefix[s + 1] = prefix[s] + (d.ucount + T - 1) / T;
    }
    if (n_src == 0 || total == 0) return PHOSIM_OK;
    if (sc->cap_src < (size_t)n_src) {
        cudaFree(sc->d_src);
        cudaFree(sc->d_src_s);
        cudaFree(sc->d_prefix);
        sc->d_src = nullptr; sc->d_src_s = nullptr; sc->d_prefix = nullptr; sc->cap_src = 0;
        CU(cudaMalloc(&sc->d_src, (size_t)n_src * sizeof(DSource)));
        CU(cudaMalloc(&sc->d_src_s, (size_t)n_src * source_s_bytes()));
        CU(cudaMalloc(&sc->d_prefix, ((size_t)n_src + 1) * sizeof(unsigned long long)));
        sc->cap_src = n_src;
    }
    // image: a pointer the device cannot use as device memory is staged through a scene buffer
    cudaPointerAttributes attr;
    bool host_image = false;
    if (cudaPointerGetAttributes(&attr, image) != cudaSuccess) {
        (void)cudaGetLastError();
        host_image = true;
    } else {
        host_image = attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged;
        if (attr.type == cudaMemoryTypeDevice && attr.device != sc->device) return PHOSIM_ERR_INVALID_ARGUMENT;
    }
    const size_t img_bytes = (size_t)sc->base.nx * sc->base.ny * sizeof(uint32_t);
    uint32_t* d_image = image;
    if (host_image) {
        if (sc->cap_stage < img_bytes) {
            cudaFree(sc->d_stage);
            sc->d_stage = nullptr; sc->cap_stage = 0;
            CU(cudaMalloc(&sc->d_stage, img_bytes));
            sc->cap_stage = img_bytes;
        }
        d_image = sc->d_stage;
        CU(cudaMemcpyAsync(d_image, image, img_bytes, cudaMemcpyHostToDevice, st));
    }
    CU(cudaMemcpyAsync(sc->d_src, hs.data(), hs.size() * sizeof(DSource), cudaMemcpyHostToDevice, st));
    CU(cudaMemcpyAsync(sc->d_prefix, prefix.data(), prefix.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    // two-kernel path: the entrance-plane states of one chunk of tiles at most (kStateChunk photons)
    const uint64_t n_tiles = prefix[n_src];
    const uint64_t chunk_tiles = staged ? std::max<uint64_t>(1, kStateChunk / T) : n_tiles;
    if (staged) {
        const size_t need = (size_t)std::min<uint64_t>(total, chunk_tiles * T);
        if (sc->cap_state < need) {
            cudaFree(sc->d_state);
            sc->d_state = nullptr; sc->cap_state = 0;
            CU(cudaMalloc(&sc->d_state, need * sizeof(DSState)));
            sc->cap_state = need;
        }
        const size_t need_hits = (size_t)std::min<uint64_t>(bundled_units, chunk_tiles * T);
        if (sc->cap_hits < need_hits) {
            cudaFree(sc->d_hits);
            sc->d_hits = nullptr; sc->cap_hits = 0;
            CU(cudaMalloc(&sc->d_hits, need_hits * sizeof(DSHit)));
            sc->cap_hits = need_hits;
        }
    }
    CU(cudaMemsetAsync(sc->d_counters, 0, kCounterWords * sizeof(unsigned long long), st));
    // the two-kernel path's striped moment accumulators, added into the caller's sums after the last stage
    const bool striped = staged && moments && n_src > 0;
    const size_t stripe_stride = (size_t)n_src * PHOSIM_MOMENT_WORDS;
    if (striped) {
        const size_t need = (size_t)kMomStripes * stripe_stride;
        if (sc->cap_mom_stripes < need) {
            cudaFree(sc->d_mom_stripes);
            sc->d_mom_stripes = nullptr; sc->cap_mom_stripes = 0;
            CU(cudaMalloc(&sc->d_mom_stripes, need * sizeof(double)));
            sc->cap_mom_stripes = need;
        }
        CU(cudaMemsetAsync(sc->d_mom_stripes, 0, need * sizeof(double), st));
    }
    TraceParams P = sc->base;
    P.mom_stripes = striped ? sc->d_mom_stripes : nullptr;
    P.mom_stripe_stride = striped ? stripe_stride : 0;
    P.sources = sc->d_src;
    P.sources_s = staged ? (SourceS*)sc->d_src_s : nullptr;
    P.tile_prefix = sc->d_prefix;
    P.n_src = n_src;
    P.tile_photons = (uint32_t)T;
    P.n_tiles = prefix[n_src];
    P.tile_counter = sc->d_counters;
    P.counters = sc->d_counters + 1;
    P.image = d_image;
    P.moments = moments;
    P.records = records;
    DSource* src_ptr = sc->d_src;
    int n_src_arg = n_src;
    double* mom_arg = moments;
    void* chief_args[4] = {&P, &src_ptr, &n_src_arg, &mom_arg};
    const dim3 chief_grid((unsigned)((n_src + 127) / 128)), chief_block(128);
    sc->timing_used = 0;
    // a launch between events of the scene's timing pool when per-kernel timing is on
    auto timed = [&](int kind, auto&& launch) -> phosim_status {
        if (!sc->stage_timing) { CU(launch()); return PHOSIM_OK; }
        cudaEvent_t a, b;
        phosim_status ts = timing_pair(sc, kind, &a, &b);
        if (ts != PHOSIM_OK) return ts;
        CU(cudaEventRecord(a, st));
        CU(launch());
        CU(cudaEventRecord(b, st));
        return PHOSIM_OK;
    };
    const bool use_graph = (P.flags & PHOSIM_GRAPH) && !sc->stage_timing;
    if (!staged) {
        void* trace_args[1] = {&P};
        if (use_graph) {
            const std::vector<LaunchOp> ops = {
                {chief_kernel_ptr(), chief_grid, chief_block, chief_args, nullptr, 0},
                {trace_kernel_ptr(mode), dim3((unsigned)blocks), dim3((unsigned)sc->threads), trace_args, nullptr, 0}};
            phosim_status gs = launch_graph(sc, mode, ops, st);
            if (gs != PHOSIM_OK) return gs;
        } else {
            phosim_status ls = timed(0, [&] { return launch_chief_rays(P, sc->d_src, n_src, moments, st); });
            if (ls == PHOSIM_OK) ls = timed(1, [&] { return launch_trace(P, mode, blocks, sc->threads, st); });
            if (ls != PHOSIM_OK) return ls;
        }
    } else {
        DSStage S;
        S.state = sc->d_state;
        S.n_state = sc->d_counters + kStateCountWord;
        S.hits = sc->d_hits;
        S.n_hits = sc->d_counters + kHitCountWord;
        S.batch = sc->d_counters + kBatchWord;
        S.tile_begin = 0;
        S.tile_end = std::min(n_tiles, chunk_tiles);
        void* stage_args[2] = {&P, &S};
        const dim3 block((unsigned)sc->threads);
        const bool bundles = bundled_units > 0;
        void* reduce_args[1] = {&P};
        const LaunchOp reduce = {moment_stripes_kernel_ptr(), dim3((unsigned)((n_src * 6 + 255) / 256)), dim3(256),
                                 reduce_args, nullptr, 0};
        if (use_graph) {
            // the whole call as one graph: chief rays; per chunk the counter resets (after the first), the entry,
            // optics and bundle stages; the moment-stripe sum
            const uint64_t n_chunks = (n_tiles + chunk_tiles - 1) / chunk_tiles;
            std::vector<DSStage> stages((size_t)n_chunks, S);
            std::vector<std::array<void*, 2>> chunk_args((size_t)n_chunks);
            std::vector<LaunchOp> ops;
            ops.reserve((size_t)n_chunks * 5 + 2);
            ops.push_back({chief_kernel_ptr(), chief_grid, chief_block, chief_args, nullptr, 0});
            for (uint64_t c = 0; c < n_chunks; ++c) {
                DSStage& Sc = stages[(size_t)c];
                Sc.tile_begin = c * chunk_tiles;
                Sc.tile_end = std::min(n_tiles, Sc.tile_begin + chunk_tiles);
                chunk_args[(size_t)c] = {&P, &Sc};
                void** a = chunk_args[(size_t)c].data();
                if (c > 0) {
                    ops.push_back({nullptr, dim3(), dim3(), nullptr, sc->d_counters, sizeof(unsigned long long)});
                    ops.push_back({nullptr, dim3(), dim3(), nullptr, sc->d_counters + kStateCountWord,
                                   3 * sizeof(unsigned long long)});
                }
                ops.push_back({ds_entry_kernel_ptr(), dim3((unsigned)blocks), block, a, nullptr, 0});
                ops.push_back({ds_optics_kernel_ptr(), dim3((unsigned)blocks_optics),
                               dim3((unsigned)ds_optics_threads(sc->threads)), a, nullptr, 0});
                if (bundles) ops.push_back({ds_members_kernel_ptr(), dim3((unsigned)blocks_members), block, a, nullptr, 0});
            }
            if (striped) ops.push_back(reduce);
            phosim_status gs = launch_graph(sc, mode, ops, st);
            if (gs != PHOSIM_OK) return gs;
        } else {
            phosim_status ls = timed(0, [&] { return launch_chief_rays(P, sc->d_src, n_src, moments, st); });
            if (ls != PHOSIM_OK) return ls;
            for (uint64_t t0 = 0; t0 < n_tiles; t0 += chunk_tiles) {
                S.tile_begin = t0;
                S.tile_end = std::min(n_tiles, t0 + chunk_tiles);
                if (t0 > 0) {
                    CU(cudaMemsetAsync(sc->d_counters, 0, sizeof(unsigned long long), st));
                    CU(cudaMemsetAsync(sc->d_counters + kStateCountWord, 0, 3 * sizeof(unsigned long long), st));
                }
                ls = timed(2, [&] { return launch_ds_entry(P, S, blocks, sc->threads, st); });
                if (ls == PHOSIM_OK) ls = timed(3, [&] { return launch_ds_optics(P, S, blocks_optics, sc->threads, st); });
                if (ls == PHOSIM_OK && bundles)
                    ls = timed(4, [&] { return launch_ds_members(P, S, blocks_members, sc->threads, st); });
                if (ls != PHOSIM_OK) return ls;
            }
            if (striped) {
                ls = timed(3, [&] { return launch_moment_stripes(P, st); });
                if (ls != PHOSIM_OK) return ls;
            }
        }
    }
    sc->last_stream = st;
    if (host_image) {
        CU(cudaMemcpyAsync(image, d_image, img_bytes, cudaMemcpyDeviceToHost, st));
        CU(cudaStreamSynchronize(st));
    }
    return PHOSIM_OK;
}

phosim_status phosim_grad(phosim_scene* sc, const phosim_source* src, int n_src, const uint64_t* n_photons,
                          const double* dL, const int32_t* ps, const int32_t* pf, int n_params, double* grad,
                          double* moments_out, void* stream) {
    if (!sc || n_src < 1 || !src || !n_photons || !dL || !ps || !pf || n_params < 1 || !grad)
        return PHOSIM_ERR_INVALID_ARGUMENT;
    if (!sc->optics_loaded || !sc->seds_loaded) return PHOSIM_ERR_NOT_READY;
    if (n_params > kMaxGradParams) return PHOSIM_ERR_LIMIT;
    if (sc->base.flags & kGhostFlag) return PHOSIM_ERR_UNSUPPORTED;   // the adjoint follows forward paths only
    {
        phosim_status vs = check_scene_device(sc);
        if (vs != PHOSIM_OK) return vs;
    }
    const TraceParams& B = sc->base;
    GradParams G;
    std::memset(&G, 0, sizeof(G));
    G.n_params = n_params;
    for (int s = 0; s < PHOSIM_MAX_SURFACES; ++s)
        for (int f = 0; f < 6; ++f) G.pert_p[s][f] = -1;
    for (int p = 0; p < n_params; ++p) {
        const int s = ps[p], f = pf[p];
        if (s < 0 || s >= B.n_surf) return PHOSIM_ERR_INVALID_ARGUMENT;
        if (f >= 0 && f < 6) {
            if (G.pert_p[s][f] >= 0) return PHOSIM_ERR_INVALID_ARGUMENT;
            G.pert_p[s][f] = p;
        } else if (f >= 100 && f < 100 + PHOSIM_MAX_ZERNIKE) {
            if (!(sc->surfaces[s].zern_rnorm > 0.0)) return PHOSIM_ERR_INVALID_ARGUMENT;
            for (int k = 0; k < G.n_zp[s]; ++k) if (G.zp_j[s][k] == f - 99) return PHOSIM_ERR_INVALID_ARGUMENT;
            G.zp_j[s][G.n_zp[s]] = f - 99;
            G.zp_p[s][G.n_zp[s]] = p;
            ++G.n_zp[s];
        } else {
            return PHOSIM_ERR_INVALID_ARGUMENT;
        }
    }
    int m = -1;
    for (int s = 0; s < B.n_surf; ++s) {
        G.mat_before[s] = m;
        if (sc->surfaces[s].kind == PHOSIM_REFRACT) m = sc->surfaces[s].material;
        rotation_derivatives(sc->surfaces[s].pert, G.dM[s]);
    }
    G.zmono = sc->d_zmono;
    cudaStream_t st = (cudaStream_t)stream;
    // forward pass in FP64: moment sums about each source's chief ray
    const size_t mom_bytes = (size_t)n_src * PHOSIM_MOMENT_WORDS * sizeof(double);
    if (sc->cap_mom < mom_bytes) {
        cudaFree(sc->d_mom_scratch);
        sc->d_mom_scratch = nullptr; sc->cap_mom = 0;
        CU(cudaMalloc(&sc->d_mom_scratch, mom_bytes));
        sc->cap_mom = mom_bytes;
    }
    const size_t img_bytes = (size_t)B.nx * B.ny * sizeof(uint32_t);
    if (sc->cap_stage < img_bytes) {
        cudaFree(sc->d_stage);
        sc->d_stage = nullptr; sc->cap_stage = 0;
        CU(cudaMalloc(&sc->d_stage, img_bytes));
        sc->cap_stage = img_bytes;
    }
    CU(cudaMemsetAsync(sc->d_mom_scratch, 0, mom_bytes, st));
    // FP64 and the dynamic transmission test (it leaves the detected photons unchanged) for both passes
    const int saved_precision = sc->precision;
    const uint32_t saved_flags = sc->base.flags;
    sc->precision = PHOSIM_PLAIN_FP64;
    sc->base.flags = (saved_flags | PHOSIM_EARLY_REJECT) & ~PHOSIM_GRAPH;
    phosim_status rs = phosim_trace(sc, src, n_src, n_photons, nullptr, sc->d_stage, nullptr, sc->d_mom_scratch, stream);
    sc->precision = saved_precision;
    sc->base.flags = saved_flags;
    if (rs != PHOSIM_OK) return rs;
    std::vector<double> mom((size_t)n_src * PHOSIM_MOMENT_WORDS);
    CU(cudaMemcpyAsync(mom.data(), sc->d_mom_scratch, mom_bytes, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    // cotangent seeds of the final positions: dL/dx_i = Ax + Bxx (x_i - mean x) + Bxy (y_i - mean y), ...
    std::vector<double> seeds((size_t)n_src * 8, 0.0);
    std::vector<double> derived((size_t)n_src * 6);
    derive_moments(mom.data(), n_src, derived.data());
    for (int s = 0; s < n_src; ++s) {
        const double* D = &derived[(size_t)s * 6];
        const double n = D[0];
        if (n > 0) {
            const double* g = dL + (size_t)s * 5;
            double* q = &seeds[(size_t)s * 8];
            q[0] = g[0] / n; q[1] = g[1] / n; q[2] = 2.0 * g[2] / n; q[3] = g[3] / n; q[4] = 2.0 * g[4] / n;
            q[5] = D[1]; q[6] = D[2];
        }
        if (moments_out) {
            double* o = moments_out + (size_t)s * 6;
            o[0] = n;
            for (int k = 1; k < 6; ++k) o[k] = n > 0 ? D[k] : 0.0;
        }
    }
    const size_t gbytes = ((size_t)n_src * 8 + (size_t)n_src * n_params) * sizeof(double);
    if (sc->cap_grad < gbytes) {
        cudaFree(sc->d_grad_scratch);
        sc->d_grad_scratch = nullptr; sc->cap_grad = 0;
        CU(cudaMalloc(&sc->d_grad_scratch, gbytes));
        sc->cap_grad = gbytes;
    }
    double* d_seeds = sc->d_grad_scratch;
    double* d_grad = d_seeds + (size_t)n_src * 8;
    CU(cudaMemcpyAsync(d_seeds, seeds.data(), seeds.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CU(cudaMemsetAsync(d_grad, 0, (size_t)n_src * n_params * sizeof(double), st));
    CU(cudaMemsetAsync(sc->d_counters, 0, sizeof(unsigned long long), st));
    G.seeds = d_seeds;
    G.grad = d_grad;
    // the trace left its source list (with chief-ray references) and tile prefix in the scene's scratch
    TraceParams P = sc->base;
    P.flags |= PHOSIM_EARLY_REJECT;
    P.sources = sc->d_src;
    P.tile_prefix = sc->d_prefix;
    P.n_src = n_src;
    uint64_t total = 0;
    for (int s = 0; s < n_src; ++s) total += n_photons[s];
    int per_sm = 0;
    CU(grad_occupancy(&per_sm));
    per_sm = std::max(per_sm, 1);
    const int blocks = sc->sm_count * per_sm;
    uint64_t T = total / ((uint64_t)blocks * 4 * 8);
    T = std::min<uint64_t>(1024, std::max<uint64_t>(32, (T + 31) / 32 * 32));
    std::vector<unsigned long long> prefix((size_t)n_src + 1, 0);
    for (int s = 0; s < n_src; ++s) prefix[s + 1] = prefix[s] + (n_photons[s] + T - 1) / T;
    CU(cudaMemcpyAsync(sc->d_prefix, prefix.data(), prefix.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice, st));
    P.tile_photons = (uint32_t)T;
    P.n_tiles = prefix[n_src];
    P.tile_counter = sc->d_counters;
    P.counters = sc->d_counters + 1;
    P.image = nullptr;
    P.moments = nullptr;
    P.records = nullptr;
    CU(launch_grad(P, G, blocks, st));
    CU(cudaMemcpyAsync(grad, d_grad, (size_t)n_src * n_params * sizeof(double), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    return PHOSIM_OK;
}

}  // extern "C"
