// Device-side data layout and per-photon physics of the GB300 photon Monte Carlo library.
//
// One thread follows one photon through Sec. 2 of Peterson et al. (2015): sampling (Sec. 2.2), the
// frozen-flow screen layers (Sec. 2.3), the surfaces (Sec. 2.4.1-2.4.2), the silicon sensor and the
// pixel (Sec. 2.4.2, 2.5).  Scene constants travel in the kernel parameter block (constant bank), so every
// per-surface read is a uniform constant-cache hit; screens and tables are read through the L1/L2 path.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "phosim.h"
#include "ds.cuh"

namespace phosim {

constexpr int kMaxMaterials = 8;
constexpr int kMaxCoatings = 8;
constexpr int kZPoly = 28;                 // monomials x^a y^b, a + b <= 6
constexpr int kSedGuide = 256;             // guide-table buckets of the wavelength-bin draw (its top 8 bits)

enum SurfFlags : int {
    SF_CONIC = 1, SF_EVEN = 2, SF_ODD = 4, SF_ZERN = 8, SF_FLAT_ONLY = 16, SF_ROTATED = 32,
    SF_DECENTERED = 64          // a vertex off the axis (the double-single transforms skip zero x, y offsets)
};

struct DSurface {
    int kind, material, coating, coat_slot;   // coat_slot: index of this surface's accept draw, -1 none
    int flags;
    int mat_before;                           // medium in front of the surface (material index, -1 vacuum)
    int ne, no;                               // terms of the even / odd polynomials up to the last nonzero one
    double c, k1c2, kc;                       // 1/R, (1 + kappa) / R^2, (1 + kappa) / R
    double ae[4];                             // alpha_4, alpha_6, alpha_8, alpha_10
    double ao[4];                             // alpha_3, alpha_5, alpha_7, alpha_9
    double M[9];                              // telescope -> surface frame rotation (row-major)
    double o[3];                              // displaced vertex in the telescope frame
    double r_in2, r_out2;
    double zinv;                              // 1 / zern_rnorm
    double zp[kZPoly];                        // sum_j c_j Z_j as monomials of (x zinv, y zinv), row b = y power
};

// The shape and placement of a surface as double-single pairs, for the FP32-pipe optics.  The asphere
// polynomials are rescaled to the normalised radius rho = r / rn (rn the clear radius), so that their
// coefficients stay far from the single-precision underflow that alpha_10 ~ 1e-30 mm^-9 would reach:
// even part  z = sum_k ae[k] u^(k+2),  u = rho^2;   (1/r) dz/dr = inv_rn2 u sum_k aed[k] u^k
// odd part   z = rho^3 sum_k ao[k] u^k;             (1/r) dz/dr = inv_rn2 rho sum_k aod[k] u^k
struct DSurfaceS {
    ds c, k1c2, kc;
    ds kmc;                                   // kc - c = kappa c: the quadric's d_z^2 term for a unit direction
    ds ae[4], aed[4], ao[4], aod[4];
    ds M[9], o[3];
    ds r_in2, r_out2;
    ds inv_rn, inv_rn2;
    float ae2[4];                             // (k + 1) aed[k] / rn^4: d^2 S / (d r^2)^2 terms of the even part, single
    float zinv;
    unsigned char ne, no, pad0, pad1;         // terms of the even / odd polynomials up to the last nonzero one
    float zp[kZPoly];
};

struct DMaterial {
    int kind, pad;
    double B[3], C[3];
    ds Bs[3], Cs[3];
};

struct DCoating {
    double lam0, inv_dlam, th0, inv_dth;
    float lam0f, inv_dlamf, th0f, inv_dthf;
    ds lam0_s, inv_dlam_s;                    // the wavelength grid as double-single pairs (its bins)
    int nl, nt, pad0, pad1;
    const double* T;                          // nl x nt
    const double* Tmax;                       // nl: the largest transmission over angles at each wavelength
    const unsigned long long* T_thr;          // the same as integer thresholds ceil(T 2^32 - 1/2) on the draw
    const unsigned long long* Tmax_thr;
    const double* TR;                         // T + R (ghosts), or null when the coating does not reflect
    const unsigned long long* TR_thr;
};

// internal scene flag: a coating reflects (ghosts)
constexpr uint32_t kGhostFlag = 1u << 24;
constexpr int kMaxGhostBounces = PHOSIM_MAX_GHOST_BOUNCES;

// A screen scale's central-difference gradient (rad / mm), stored per node (i, j) as the 2 x 2 block of
// nodes the bilinear interpolation needs, (i, j), (i+1, j), (i, j+1), (i+1, j+1) (periodic): one lookup is
// one aligned 32-byte (FP32) or 64-byte (FP64) read instead of two rows of scattered 8- or 16-byte taps.
struct DScale {
    int n, pad;
    double inv_pix;
    ds inv_pix_s;
    const double2* g64;                       // 4 double2 per node, n x n nodes
    const float4* g32;                        // 2 float4 per node: (g00, g10), (g01, g11)
};

struct DLayer {
    double z, vx, vy;
    ds zs, vxs, vys;
    ds dzs;                                   // height of the plane above (the previous layer or the top) over z
    int n_scales, pad;
    DScale s[PHOSIM_MAX_SCALES];
};

struct SourceS;                              // a source's constants as the double-single path reads them

struct DSource {
    int kind, sed, table;
    uint32_t bundle;                          // photons per ray (Sec. 3.2 background optimisation), >= 1
    double xi, eta, zfac, t0, t_exp, a, b, cpa, spa;
    double bsig;                              // sigma of the spread of a ray's photons on the detector, mm
    double ref_x, ref_y;
    float ref_s[4];                           // ref_x, ref_y as double-single pairs (hi, lo, hi, lo)
    uint64_t first, count, rec_off;           // photons [first, first + count); record index of the first
    uint64_t ufirst, ucount;                  // work units of the two-kernel path: rays of a bundle, else photons
};

// counters: [0] traced, [1] detected, [1 + r] dropped for reason r
constexpr int kNumCounters = 10;

struct TraceParams {
    // scene
    uint32_t k0, k1;                          // Philox key
    uint32_t flags;
    int n_surf, n_layers, n_coated, n_mat, n_coat;
    int coated_surface[PHOSIM_MAX_COATED];    // surface index of coated-surface draw k
    double pr_in2, pr_dr2;                    // pupil annulus
    double h_top, z_ent;
    double lam_ref, kick0;                    // kick0 = lambda_ref [mm] / 2 pi
    double pupil_z;                           // nominal vertex height of the first surface
    DSurface pupil_surf;                      // its nominal shape (no figure error, no misalignment)
    DSurface surf[PHOSIM_MAX_SURFACES];
    DMaterial mat[kMaxMaterials];
    DCoating coat[kMaxCoatings];
    DLayer layer[PHOSIM_MAX_LAYERS];
    // the same scene in double-single / single precision for the FP32-pipe path
    DSurfaceS surf_s[PHOSIM_MAX_SURFACES];
    DSurfaceS pupil_s;
    ds pr_in2_s, pr_dr2_s, h_top_s, z_ent_s, pupil_z_s, xlo_s, ylo_s, inv_pixel_s, chip_w_s, chip_h_s;
    float kick0f, inv_lam_ref_f, sed_lam0f, sed_dlamf, t_sif, dead_layerf, ell_lam0f, inv_ell_dlamf, sig_scalef;
    // sensor / detector
    int nx, ny, n_ell, n_sig;
    double pixel, inv_pixel, xlo, ylo, t_si, ell_lam0, inv_ell_dlam, sig_scale, dead_layer;
    // fringing (PHOSIM_FRINGE): the silicon's optical thickness at (x, y) of the detector surface frame is
    // fr_t0 + fr_gx x + fr_gy y
    double fr_t0, fr_gx, fr_gy;
    ds fr_t0_s;
    float fr_gxf, fr_gyf;
    const double* ell;
    const float* ell32;
    const double* sig;
    const float* sig32;
    // spectra, shapes
    int n_bins, sersic_K;
    double sed_lam0, sed_dlam;
    ds sed_lam0_s, sed_dlam_s;
    const unsigned long long* thr;            // n_sed x (n_bins - 1) integer thresholds on the bin draw
    const int* sed_guide;                     // n_sed x (kSedGuide + 1): first threshold above j 2^24
    const double* sersic;
    const float* sersic32;
    int hf_K;                                 // quantiles of the high-frequency kick (0 = none)
    const double* hf;
    const float* hf32;
    // work and outputs: tile t of the launch is tile t - tile_prefix[s] of the source s with
    // tile_prefix[s] <= t < tile_prefix[s + 1]; a tile holds tile_photons consecutive photons
    const DSource* sources;
    SourceS* sources_s;                       // the same sources converted once by the chief-ray kernel (two-kernel path)
    const unsigned long long* tile_prefix;
    int n_src;
    uint32_t tile_photons;
    uint64_t n_tiles;
    unsigned long long* tile_counter;
    unsigned long long* counters;
    uint32_t* image;
    double* moments;
    phosim_photon_record* records;
    // the two-kernel double-single path's moment accumulators: kMomStripes copies of the per-source sums
    // (PHOSIM_MOMENT_WORDS a source, mom_stripe_stride doubles a copy), a block adding to copy blockIdx %
    // kMomStripes so that a bright source's atomics spread over several cache lines; null: add to moments
    double* mom_stripes;
    unsigned long long mom_stripe_stride;
};
constexpr int kMomStripes = 16;
// warps of the entry and bundle stages' blocks (the shared-memory queues and counters are sized for it)
constexpr int kWarpsPerBlock = 8;

// ------------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds, two 32x32 multiplications per round.
// ------------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// slot map of one photon's random words: counter = (photon lo, photon hi, source, block)
//   block 0: pupil r, pupil phi, wavelength bin, wavelength blur
//   block 1: time, shape a, shape b, conversion
//   block 2: diffusion a, diffusion b, coated surface 0, coated surface 1
//   block 3: coated surfaces 2..5
//   block 4: high-frequency kick magnitude, direction, back-side reflection
//   blocks 5, 6 (photons of a bundle, counter of the photon; the ray uses blocks 0-4 of the ray's counter):
//            spread a, spread b, conversion, diffusion a; diffusion b, back-side reflection
//   blocks 7, 8, ... (ghosts): the coating decisions after the first reflection, one word each, in order
__device__ __forceinline__ double u64of(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }
// the uniform (w + 1/2) 2^-32 of a word in single precision: the whole word converts (exactly below 2^24), so
// the small values that the -log u of the conversion depth and of Box-Muller reach keep 24 significant bits
__device__ __forceinline__ float u32of(uint32_t w) {
    return __fadd_rn(__fmul_rn((float)w, 2.3283064365386963e-10f), 1.1641532182693481e-10f);
}

// ------------------------------------------------------------------------------------------------------
// surface shape (Sec. 2.4.1)
// ------------------------------------------------------------------------------------------------------
// Zernike figure as a bivariate polynomial of degree 6 in normalised coordinates (u, v).
__device__ __forceinline__ void zern_eval(const double* __restrict__ zp, double u, double v, double& z, double& zu,
                                          double& zv) {
    // rows b = 0..6 hold the x-polynomial of y^b, degree 6 - b, ascending powers of x
    double q[7], dq[7];
    int off = 0;
#pragma unroll
    for (int b = 0; b <= 6; ++b) {
        const int deg = 6 - b;
        double acc = zp[off + deg], dacc = 0.0;
#pragma unroll
        for (int a = deg - 1; a >= 0; --a) {
            dacc = fma(dacc, u, acc);
            acc = fma(acc, u, zp[off + a]);
        }
        q[b] = acc;
        dq[b] = dacc;
        off += deg + 1;
    }
    double zz = q[6], zzu = dq[6], zzv = 0.0;
#pragma unroll
    for (int b = 5; b >= 0; --b) {
        zzv = fma(zzv, v, zz);
        zz = fma(zz, v, q[b]);
        zzu = fma(zzu, v, dq[b]);
    }
    z = zz; zu = zzu; zv = zzv;
}

// sag and its partial derivatives in the surface frame; false outside the conic's domain
__device__ __forceinline__ bool sag(const DSurface& S, double x, double y, double& z, double& zx, double& zy) {
    const double r2 = x * x + y * y;
    double g = 0.0;   // (1/r) dz/dr
    z = 0.0;
    if (S.flags & SF_CONIC) {
        const double arg = 1.0 - S.k1c2 * r2;
        if (arg < 0.0) return false;
        const double rs = rsqrt(arg);
        z = S.c * r2 / fma(arg, rs, 1.0);
        g = S.c * rs;
    }
    // Horner from the last nonzero coefficient: the zero terms above it would add exact zeros
    if (S.flags & SF_EVEN) {
        int k = S.ne - 1;
        double pe = S.ae[k], pd = (2 * k + 4) * S.ae[k];
#pragma unroll 1
        while (--k >= 0) {
            pe = fma(r2, pe, S.ae[k]);
            pd = fma(r2, pd, (2 * k + 4) * S.ae[k]);
        }
        z = fma(r2 * r2, pe, z);
        g = fma(r2, pd, g);
    }
    if (S.flags & SF_ODD) {
        const double r = sqrt(r2);
        int k = S.no - 1;
        double po = S.ao[k], pd = (2 * k + 3) * S.ao[k];
#pragma unroll 1
        while (--k >= 0) {
            po = fma(r2, po, S.ao[k]);
            pd = fma(r2, pd, (2 * k + 3) * S.ao[k]);
        }
        z = fma(r2 * r, po, z);
        g = fma(r, pd, g);
    }
    zx = x * g;
    zy = y * g;
    if (S.flags & SF_ZERN) {
        double zz, zu, zv;
        zern_eval(S.zp, x * S.zinv, y * S.zinv, zz, zu, zv);
        z += zz;
        zx = fma(zu, S.zinv, zx);
        zy = fma(zv, S.zinv, zy);
    }
    return true;
}

// Intersection (Sec. 2.4.2).  The paper's first guess is the root of a quadric approximating the surface;
// here the quadric is the conic itself, c (x^2 + y^2) + (1 + kappa) c z^2 - 2 z = 0, solved exactly on the
// vertex branch (1 - (1 + kappa) c z >= 0).  A pure conic needs nothing more: its slopes follow from the
// same quadric, z_x = c x / (1 - (1 + kappa) c z).  Aspheric and Zernike terms are then added by Newton's
// method on F(l) = p_z + l d_z - S(p_x + l d_x, p_y + l d_y) until the step is below 1e-8 mm.
// On success l is the distance and (zx, zy) the slopes at the root (within 1e-8 mm of it).
__device__ __forceinline__ uint32_t intersect(const DSurface& S, const double p[3], const double d[3], double& l,
                                              double N[3]) {
    if (S.flags & SF_FLAT_ONLY) {
        if (d[2] == 0.0) return PHOSIM_LOST_MISSED;
        l = -p[2] / d[2];
        N[0] = 0.0; N[1] = 0.0; N[2] = 1.0;
        return 0;
    }
    const double A = S.c * fma(d[0], d[0], d[1] * d[1]) + S.kc * d[2] * d[2];
    const double b = S.c * fma(p[0], d[0], p[1] * d[1]) + fma(S.kc * p[2], d[2], -d[2]);
    const double C = S.c * fma(p[0], p[0], p[1] * p[1]) + fma(S.kc * p[2], p[2], -2.0 * p[2]);
    const double disc = fma(b, b, -A * C);
    if (disc < 0.0) return PHOSIM_LOST_MISSED;
    const double q = -(b + copysign(sqrt(disc), b));
    if (q == 0.0) return PHOSIM_LOST_MISSED;
    l = C / q;
    if (A != 0.0 && fma(-S.kc, fma(l, d[2], p[2]), 1.0) < 0.0) l = q / A;   // the other root is the vertex branch
    if (!(S.flags & (SF_EVEN | SF_ODD | SF_ZERN))) {
        // the quadric's gradient (-c x, -c y, 1 - (1 + kappa) c z) is along (-z_x, -z_y, 1)
        const double x = fma(l, d[0], p[0]), y = fma(l, d[1], p[1]), z = fma(l, d[2], p[2]);
        const double vx = -S.c * x, vy = -S.c * y, vz = fma(-S.kc, z, 1.0);
        const double inv = rsqrt(fma(vx, vx, fma(vy, vy, vz * vz)));
        N[0] = vx * inv; N[1] = vy * inv; N[2] = vz * inv;
        return 0;
    }
    double zx = 0.0, zy = 0.0;
#pragma unroll 1
    for (int it = 0; it < 20; ++it) {
        const double x = fma(l, d[0], p[0]), y = fma(l, d[1], p[1]);
        double zs;
        if (!sag(S, x, y, zs, zx, zy)) return PHOSIM_LOST_MISSED;
        const double F = fma(l, d[2], p[2]) - zs;
        const double dF = d[2] - zx * d[0] - zy * d[1];
        if (dF == 0.0) return PHOSIM_LOST_NEWTON;
        // a single-precision reciprocal of the slope: the iteration still contracts by ~1e-7 per step
        // (outside the single-precision range the division stays exact)
        const double adF = fabs(dF);
        const double step = (adF > 1e-30 && adF < 1e30) ? F * (double)__frcp_rn((float)dF) : F / dF;
        l -= step;
        if (fabs(step) < 1e-8) {
            const double inv = rsqrt(fma(zx, zx, fma(zy, zy, 1.0)));
            N[0] = -zx * inv; N[1] = -zy * inv; N[2] = inv;
            return 0;
        }
    }
    return PHOSIM_LOST_NEWTON;
}

__device__ __forceinline__ double sellmeier(const DMaterial& m, double lam_nm) {
    const double l2 = (lam_nm * 1e-3) * (lam_nm * 1e-3);
    double n2 = 1.0;
#pragma unroll
    for (int i = 0; i < 3; ++i) n2 += m.B[i] * l2 / (l2 - m.C[i]);
    return sqrt(n2);
}

// silicon index of Sec. 2.4.1, E in eV
__device__ __forceinline__ double silicon_index(double lam_nm) {
    const double E = 1239.841984 / lam_nm;
    return 3.36 + 0.211 * E + 2.79 * exp((E - 3.30) / 0.398);
}
__device__ __forceinline__ float silicon_index_f(float lam_nm) {
    const float E = 1239.841984f / lam_nm;
    return 3.36f + 0.211f * E + 2.79f * expf((E - 3.30f) * (1.0f / 0.398f));
}

// ------------------------------------------------------------------------------------------------------
// Fringing (Sec. 2.4.2): the back-side reflection probability from the single-layer electromagnetic
// calculation.  One layer of silicon (index n1 + i k1, thickness t) lies between the medium in front of the
// detector (real index n0) and vacuum behind it; a photon travels through it with direction cosine c1 (real,
// from its refracted direction), so its invariant is s^2 = n1^2 (1 - c1^2).  With q = N cos(theta) =
// sqrt(N^2 - s^2) in each medium, the s and p amplitude reflection coefficients of each interface, and the
// layer's round trip e = exp(i 4 pi t q1 / lambda), the layer reflects r = (r01 + r12 e) / (1 + r01 r12 e);
// the probability is (|r_s|^2 + |r_p|^2) / 2.
// ------------------------------------------------------------------------------------------------------
struct cplx {
    double re, im;
};
__device__ __forceinline__ cplx c_add(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx c_sub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx c_mul(cplx a, cplx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cplx c_div(cplx a, cplx b) {
    const double d = 1.0 / (b.re * b.re + b.im * b.im);
    return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
// principal square root, without cancellation in the smaller part
__device__ __forceinline__ cplx c_sqrt(cplx z) {
    const double m = sqrt(0.5 * (hypot(z.re, z.im) + fabs(z.re)));
    if (m == 0.0) return {0.0, 0.0};
    if (z.re >= 0.0) return {m, 0.5 * z.im / m};
    return {0.5 * fabs(z.im) / m, z.im < 0.0 ? -m : m};
}

static __device__ __noinline__ double film_reflectance(double lam_nm, double n0, double n1, double k1, double t, double c1) {
    const double s2 = n1 * n1 * fmax(0.0, 1.0 - c1 * c1);
    const cplx q0 = c_sqrt({n0 * n0 - s2, 0.0}), q2 = c_sqrt({1.0 - s2, 0.0});
    const cplx N1sq = {n1 * n1 - k1 * k1, 2.0 * n1 * k1};
    const cplx q1 = c_sqrt(c_sub(N1sq, {s2, 0.0}));
    const cplx n0sq = {n0 * n0, 0.0};
    // s and p coefficients of the front (0 -> 1) and back (1 -> vacuum) interfaces
    const cplx rs01 = c_div(c_sub(q0, q1), c_add(q0, q1)), rs12 = c_div(c_sub(q1, q2), c_add(q1, q2));
    const cplx rp01 = c_div(c_sub(c_mul(N1sq, q0), c_mul(n0sq, q1)), c_add(c_mul(N1sq, q0), c_mul(n0sq, q1)));
    const cplx rp12 = c_div(c_sub(q1, c_mul(N1sq, q2)), c_add(q1, c_mul(N1sq, q2)));
    const double w = 4.0 * M_PI * t / (lam_nm * 1e-6);
    double sn, cs;
    sincos(w * q1.re, &sn, &cs);
    const double amp = exp(-w * q1.im);
    const cplx e = {amp * cs, amp * sn};
    const cplx rs = c_div(c_add(rs01, c_mul(rs12, e)), c_add({1.0, 0.0}, c_mul(c_mul(rs01, rs12), e)));
    const cplx rp = c_div(c_add(rp01, c_mul(rp12, e)), c_add({1.0, 0.0}, c_mul(c_mul(rp01, rp12), e)));
    return 0.5 * (rs.re * rs.re + rs.im * rs.im + rp.re * rp.re + rp.im * rp.im);
}

// Snell's law in vector form (Sec. 2.4.2) with mu = n1 / n2; false on total internal reflection
__device__ __forceinline__ bool refract(double d[3], double Nx, double Ny, double Nz, double mu) {
    double cosi = -(d[0] * Nx + d[1] * Ny + d[2] * Nz);
    if (cosi < 0.0) { Nx = -Nx; Ny = -Ny; Nz = -Nz; cosi = -cosi; }
    const double k = 1.0 - mu * mu * (1.0 - cosi * cosi);
    if (k < 0.0) return false;
    const double a = mu * cosi - sqrt(k);
    d[0] = fma(mu, d[0], a * Nx);
    d[1] = fma(mu, d[1], a * Ny);
    d[2] = fma(mu, d[2], a * Nz);
    return true;
}

__device__ __forceinline__ void to_surface(const DSurface& S, const double x[3], const double d[3], double p[3],
                                           double dl[3]) {
    const double rx = x[0] - S.o[0], ry = x[1] - S.o[1], rz = x[2] - S.o[2];
    if (!(S.flags & SF_ROTATED)) {        // the identity rotation: the products below would be exact copies
        p[0] = rx; p[1] = ry; p[2] = rz;
        dl[0] = d[0]; dl[1] = d[1]; dl[2] = d[2];
        return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p[i] = fma(S.M[3 * i], rx, fma(S.M[3 * i + 1], ry, S.M[3 * i + 2] * rz));
        dl[i] = fma(S.M[3 * i], d[0], fma(S.M[3 * i + 1], d[1], S.M[3 * i + 2] * d[2]));
    }
}

__device__ __forceinline__ void from_surface(const DSurface& S, const double p[3], const double dl[3], double x[3],
                                             double d[3]) {
    if (!(S.flags & SF_ROTATED)) {
        x[0] = p[0] + S.o[0]; x[1] = p[1] + S.o[1]; x[2] = p[2] + S.o[2];
        d[0] = dl[0]; d[1] = dl[1]; d[2] = dl[2];
        return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        x[i] = fma(S.M[i], p[0], fma(S.M[3 + i], p[1], fma(S.M[6 + i], p[2], S.o[i])));
        d[i] = fma(S.M[i], dl[0], fma(S.M[3 + i], dl[1], S.M[6 + i] * dl[2]));
    }
}

}  // namespace phosim
