// Per-photon forward path shared by the trace kernel and the adjoint kernel (Peterson et al. 2015,
// Sec. 2.2-2.5): one definition, so the adjoint's recomputed forward pass takes exactly the trace's
// decisions.
#pragma once

#include "phosim_device.cuh"

namespace phosim {


struct PhotonOut {
    double x, y, xc, yc, lam;
    uint32_t flags;
    int pix;
};

__device__ __forceinline__ uint32_t lost(uint32_t reason, int surface) {
    return (reason << 8) | ((uint32_t)(surface & 0xff) << 16);
}

__device__ __forceinline__ uint32_t word(const uint4& w, int k) {
    return k == 0 ? w.x : (k == 1 ? w.y : (k == 2 ? w.z : w.w));
}

// Wavelength bin (Sec. 2.2): the first bin whose cumulative photon probability exceeds the draw, decided
// on the integer draw against thresholds precomputed from the FP64 cumulative table.  A guide table (Chen and
// Asau's indexed search) narrows the search to the thresholds between guide[j] and guide[j + 1] for the draw's
// top byte j: every threshold below guide[j] is at most j 2^24 <= w, and the one at guide[j + 1] exceeds
// (j + 1) 2^24 > w, so the answer lies in that range and is the plain search's answer.
__device__ __forceinline__ int sed_bin(const unsigned long long* __restrict__ thr, const int* __restrict__ guide, uint32_t w) {
    const int j = (int)(w >> 24);
    int lo = __ldg(guide + j), hi = __ldg(guide + j + 1);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((unsigned long long)w < __ldg(thr + mid)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

__device__ __forceinline__ int wrap_index(long long i, int n) {
    if ((n & (n - 1)) == 0) return (int)(i & (long long)(n - 1));
    long long m = i % n;
    return (int)(m < 0 ? m + n : m);
}

// Gradient of the phase at screen position (sx, sy), bilinear between central-difference nodes (Sec. 2.3.2)
template <bool MIXED>
__device__ __forceinline__ void screen_gradient(const DScale& S, double sx, double sy, double& gx, double& gy) {
    const double fx = sx * S.inv_pix, fy = sy * S.inv_pix;
    const double flx = floor(fx), fly = floor(fy);
    const int n = S.n;
    const int i0 = wrap_index((long long)flx, n), j0 = wrap_index((long long)fly, n);
    const size_t node = (size_t)j0 * n + i0;
    if constexpr (MIXED) {
        const float tx = (float)(fx - flx), ty = (float)(fy - fly);
        const float4 A = __ldg(S.g32 + 2 * node), B = __ldg(S.g32 + 2 * node + 1);
        const float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty), w01 = (1.f - tx) * ty, w11 = tx * ty;
        gx += (double)(w00 * A.x + w10 * A.z + w01 * B.x + w11 * B.z);
        gy += (double)(w00 * A.y + w10 * A.w + w01 * B.y + w11 * B.w);
    } else {
        const double tx = fx - flx, ty = fy - fly;
        const double2* q = S.g64 + 4 * node;
        const double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
        const double w00 = (1.0 - tx) * (1.0 - ty), w10 = tx * (1.0 - ty), w01 = (1.0 - tx) * ty, w11 = tx * ty;
        gx += w00 * a.x + w10 * b.x + w01 * c.x + w11 * d.x;
        gy += w00 * a.y + w10 * b.y + w01 * c.y + w11 * d.y;
    }
}

__device__ __forceinline__ double lerp_table(const double* __restrict__ t, int n, double f) {
    int k = (int)floor(f);
    k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
    double w = f - k;
    w = w < 0.0 ? 0.0 : (w > 1.0 ? 1.0 : w);
    return __ldg(t + k) * (1.0 - w) + __ldg(t + k + 1) * w;
}
__device__ __forceinline__ float lerp_table_f(const float* __restrict__ t, int n, float f) {
    int k = (int)floorf(f);
    k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
    float w = f - (float)k;
    w = w < 0.f ? 0.f : (w > 1.f ? 1.f : w);
    return __ldg(t + k) * (1.f - w) + __ldg(t + k + 1) * w;
}

// Surfaces in order (Sec. 2.4.2).  FULL = apertures, coatings and the sensor; otherwise the bare rays that
// give each source's chief-ray reference.
// Forward state kept for the adjoint sweep (RECORD): the telescope-frame position and direction entering
// each surface, and the conversion length and diffusion offset of the sensor.
struct ForwardRecord {
    double XD[PHOSIM_MAX_SURFACES][6];
    double L, ox, oy;
};

// A photon of a bundle (Sec. 3.2 background optimisation): it follows its ray (the photon index divided by
// the bundle size) to the detector surface, lands at a Gaussian offset of the source's spread sigma from the
// ray's hit and takes its own sensor draws, all from blocks 5 and 6 of its own counter.
struct MemberDraw {
    double sx, sy;
    uint32_t conv, diff_a, diff_b, back;
};

template <bool MIXED>
__device__ __forceinline__ MemberDraw member_draw(const TraceParams& P, double bsig, int src, uint64_t i) {
    const uint32_t clo = (uint32_t)i, chi = (uint32_t)(i >> 32);
    const uint4 m5 = philox(make_uint4(clo, chi, (uint32_t)src, 5u), P.k0, P.k1);
    const uint4 m6 = philox(make_uint4(clo, chi, (uint32_t)src, 6u), P.k0, P.k1);
    MemberDraw m;
    if constexpr (MIXED) {
        const float g = sqrtf(-2.f * logf(u32of(m5.x)));
        float sn, cs;
        sincospif(2.f * u32of(m5.y), &sn, &cs);
        m.sx = (double)((float)bsig * g * cs);
        m.sy = (double)((float)bsig * g * sn);
    } else {
        const double g = sqrt(-2.0 * log(u64of(m5.x)));
        double sn, cs;
        sincospi(2.0 * u64of(m5.y), &sn, &cs);
        m.sx = bsig * g * cs;
        m.sy = bsig * g * sn;
    }
    m.conv = m5.z; m.diff_a = m5.w; m.diff_b = m6.x; m.back = m6.y;
    return m;
}

// the ray a photon follows: itself, or for a bundle of n photons per ray, photon index / n
__device__ __forceinline__ uint64_t ray_of(uint32_t bundle, uint64_t i) { return bundle > 1 ? i / bundle : i; }

// Ghosts (Sec. 2.4.2): after a photon's first reflection by a coating, each coating decision draws the next
// word of blocks 7, 8, ... of the ray's counter.
__device__ __forceinline__ uint32_t ghost_word(const TraceParams& P, int src, uint64_t ray, int n) {
    return word(philox(make_uint4((uint32_t)ray, (uint32_t)(ray >> 32), (uint32_t)src, 7u + (uint32_t)n / 4u), P.k0, P.k1),
                n & 3);
}

// Surfaces in order (dir = +1); with reflecting coatings a photon reflected by a refracting surface (a ghost)
// travels back through them (dir = -1) until another reflection turns it round again.  src and ray identify
// the ghost draws.
template <bool MIXED, bool FULL, bool RECORD = false>
__device__ __forceinline__ void optics(const TraceParams& P, double X[3], double D[3], double lam, uint4 w1, uint4 w2,
                                       uint4 w3, uint4 w4, PhotonOut& R, ForwardRecord* fr = nullptr,
                                       const MemberDraw* mb = nullptr, int src = 0, uint64_t ray = 0) {
    constexpr bool GHOSTS = FULL && !RECORD;
    const bool ghosts = GHOSTS && (P.flags & kGhostFlag);
    double n_cur = 1.0;
    int glass_mat = -1;
    double glass_n = 1.0, glass_inv = 1.0;
    int si = 0, dir = 1, bounces = 0, n_ghost = 0;
#pragma unroll 1
    for (;;) {
        if (si < 0 || si >= P.n_surf) break;
        const DSurface& S = P.surf[si];
        if constexpr (RECORD) {
            fr->XD[si][0] = X[0]; fr->XD[si][1] = X[1]; fr->XD[si][2] = X[2];
            fr->XD[si][3] = D[0]; fr->XD[si][4] = D[1]; fr->XD[si][5] = D[2];
        }
        double p[3], dl[3];
        to_surface(S, X, D, p, dl);
        double l, Nv[3];
        const uint32_t why = intersect(S, p, dl, l, Nv);
        if (why) { R.flags = lost(why, si); return; }
        if (GHOSTS && bounces > 0 && !(l > 0.0)) { R.flags = lost(PHOSIM_LOST_MISSED, si); return; }
        p[0] = fma(l, dl[0], p[0]);
        p[1] = fma(l, dl[1], p[1]);
        p[2] = fma(l, dl[2], p[2]);
        const double Nx = Nv[0], Ny = Nv[1], Nz = Nv[2];
        if (S.kind == PHOSIM_DETECTOR) {
            uint32_t w_conv = w1.w, w_diff_a = w2.x, w_diff_b = w2.y, w_back = w4.z;
            if (mb) {   // a bundle's photon: its offset from the ray's hit and its own sensor draws
                p[0] += mb->sx;
                p[1] += mb->sy;
                w_conv = mb->conv; w_diff_a = mb->diff_a; w_diff_b = mb->diff_b; w_back = mb->back;
            }
            const double hx = p[0] - P.xlo, hy = p[1] - P.ylo;
            if (FULL && !(hx >= 0.0 && hy >= 0.0 && hx < P.nx * P.pixel && hy < P.ny * P.pixel)) {
                R.flags = lost(PHOSIM_LOST_OFF_CHIP, si);
                return;
            }
            double fx = p[0], fy = p[1];
            R.xc = fx; R.yc = fy;
            if (FULL && (P.flags & PHOSIM_SENSOR)) {
                // refraction into the silicon, exponential conversion length (Sec. 2.4.2)
                double L, sigma, gxd, gyd, r_back;
                if constexpr (MIXED) {
                    const float n_si = silicon_index_f((float)lam);
                    if (!refract(dl, Nx, Ny, Nz, n_cur / (double)n_si)) { R.flags = lost(PHOSIM_LOST_TIR, si); return; }
                    const float ell = lerp_table_f(P.ell32, P.n_ell, (float)((lam - P.ell_lam0) * P.inv_ell_dlam));
                    const float Lf = ell * -logf(u32of(w_conv));
                    L = (double)Lf;
                    const float rf = (n_si - 1.f) / (n_si + 1.f);
                    r_back = (double)(rf * rf);
                } else {
                    const double n_si = silicon_index(lam);
                    if (!refract(dl, Nx, Ny, Nz, n_cur / n_si)) { R.flags = lost(PHOSIM_LOST_TIR, si); return; }
                    const double ell = lerp_table(P.ell, P.n_ell, (lam - P.ell_lam0) * P.inv_ell_dlam);
                    L = ell * -log(u64of(w_conv));
                    const double rf = (n_si - 1.0) / (n_si + 1.0);
                    r_back = rf * rf;
                }
                double depth = L * fabs(dl[2]);
                if (!(depth <= P.t_si)) {
                    // back-side reflection: the photon turns round at the back and converts on its way back
                    bool back = false;
                    if (P.flags & PHOSIM_BACK_REFLECT) {
                        if (P.flags & PHOSIM_FRINGE) {
                            // fringing: the single-layer calculation in FP64 at the photon's entry point (both
                            // the plain and the mixed path: the phase spans ~10^3 cycles)
                            const double ell = lerp_table(P.ell, P.n_ell, (lam - P.ell_lam0) * P.inv_ell_dlam);
                            r_back = film_reflectance(lam, n_cur, silicon_index(lam), lam * 1e-6 / (4.0 * M_PI * ell),
                                                      P.fr_t0 + P.fr_gx * p[0] + P.fr_gy * p[1], fabs(dl[2]));
                        }
                        if (u64of(w_back) < r_back) {
                            depth = 2.0 * P.t_si - depth;
                            back = depth >= 0.0;
                        }
                    }
                    if (!back) { R.flags = lost(PHOSIM_LOST_NOT_CONVERTED, si); return; }
                }
                // field-free dead layer at the entrance: the charge is not collected
                if (depth < P.dead_layer) { R.flags = lost(PHOSIM_LOST_DEAD_LAYER, si); return; }
                fx = fma(L, dl[0], fx);
                fy = fma(L, dl[1], fy);
                R.xc = fx; R.yc = fy;
                // lateral Gaussian diffusion (Sec. 2.5)
                if constexpr (MIXED) {
                    const float sg = lerp_table_f(P.sig32, P.n_sig, (float)(depth * P.sig_scale));
                    const float g = sqrtf(-2.f * logf(u32of(w_diff_a)));
                    float sn, cs;
                    sincospif(2.f * u32of(w_diff_b), &sn, &cs);
                    sigma = 1.0; gxd = (double)(sg * g * cs); gyd = (double)(sg * g * sn);
                } else {
                    sigma = lerp_table(P.sig, P.n_sig, depth * P.sig_scale);
                    const double g = sqrt(-2.0 * log(u64of(w_diff_a)));
                    double sn, cs;
                    sincospi(2.0 * u64of(w_diff_b), &sn, &cs);
                    gxd = g * cs; gyd = g * sn;
                }
                fx = fma(sigma, gxd, fx);
                fy = fma(sigma, gyd, fy);
                if constexpr (RECORD) { fr->L = L; fr->ox = sigma * gxd; fr->oy = sigma * gyd; }
            }
            R.x = fx; R.y = fy;
            if (FULL) {
                const double ux = fx - P.xlo, uy = fy - P.ylo;
                const double px = floor(ux * P.inv_pixel), py = floor(uy * P.inv_pixel);
                if (!(px >= 0.0 && py >= 0.0 && px < (double)P.nx && py < (double)P.ny)) {
                    R.flags = lost(PHOSIM_LOST_OFF_CHIP, si);
                    return;
                }
                R.pix = (int)py * P.nx + (int)px;
            }
            R.flags = PHOSIM_F_DETECTED;
            return;
        }
        if (FULL) {
            // clear aperture
            const double r2 = p[0] * p[0] + p[1] * p[1];
            if (!(r2 <= S.r_out2 && r2 >= S.r_in2)) { R.flags = lost(PHOSIM_LOST_VIGNETTED, si); return; }
            // coating accept-reject at the incidence angle and wavelength
            if (S.coat_slot >= 0) {
                const DCoating& C = P.coat[S.coating];
                int it = 0;
                if (C.nt > 1) {
                    const double cosi = fabs(dl[0] * Nx + dl[1] * Ny + dl[2] * Nz);
                    const double th = acos(fmin(1.0, cosi));
                    it = (int)floor((th - C.th0) * C.inv_dth);
                    it = it < 0 ? 0 : (it > C.nt - 1 ? C.nt - 1 : it);
                }
                int il = (int)floor((lam - C.lam0) * C.inv_dlam);
                il = il < 0 ? 0 : (il > C.nl - 1 ? C.nl - 1 : il);
                const size_t ix = (size_t)il * C.nt + it;
                const double T = __ldg(C.T + ix);
                uint32_t w;
                if (GHOSTS && bounces > 0) {
                    w = ghost_word(P, src, ray, n_ghost++);
                } else {
                    const int k = S.coat_slot;
                    w = k < 2 ? word(w2, 2 + k) : word(w3, k - 2);
                }
                if (!(u64of(w) < T)) {
                    // reflected backwards (a ghost) with probability R, absorbed otherwise
                    if (ghosts && S.kind != PHOSIM_MIRROR && C.TR && u64of(w) < __ldg(C.TR + ix)) {
                        const double dn = dl[0] * Nx + dl[1] * Ny + dl[2] * Nz;
                        dl[0] = fma(-2.0 * dn, Nx, dl[0]);
                        dl[1] = fma(-2.0 * dn, Ny, dl[1]);
                        dl[2] = fma(-2.0 * dn, Nz, dl[2]);
                        dir = -dir;
                        if (++bounces > kMaxGhostBounces) { R.flags = lost(PHOSIM_LOST_MISSED, si); return; }
                        from_surface(S, p, dl, X, D);
                        si += dir;
                        continue;
                    }
                    R.flags = lost(PHOSIM_LOST_COATING, si);
                    return;
                }
            }
        }
        if (S.kind == PHOSIM_MIRROR) {
            const double dn = dl[0] * Nx + dl[1] * Ny + dl[2] * Nz;
            dl[0] = fma(-2.0 * dn, Nx, dl[0]);
            dl[1] = fma(-2.0 * dn, Ny, dl[1]);
            dl[2] = fma(-2.0 * dn, Nz, dl[2]);
        } else {
            // the medium beyond the surface in the direction of travel (-1: vacuum)
            const int mi = (GHOSTS && dir < 0) ? S.mat_before : S.material;
            double n_next = 1.0, inv_next = 1.0;
            if (mi >= 0) {
                const DMaterial& m = P.mat[mi];
                if (m.kind == PHOSIM_SELLMEIER) {
                    if (glass_mat != mi) {
                        glass_n = sellmeier(m, lam);
                        glass_inv = 1.0 / glass_n;
                        glass_mat = mi;
                    }
                    n_next = glass_n;
                    inv_next = glass_inv;
                } else if (m.kind == PHOSIM_SILICON) {
                    n_next = silicon_index(lam);
                    inv_next = 1.0 / n_next;
                }
            }
            if (!refract(dl, Nx, Ny, Nz, n_cur * inv_next)) { R.flags = lost(PHOSIM_LOST_TIR, si); return; }
            n_cur = n_next;
        }
        from_surface(S, p, dl, X, D);
        si += dir;
    }
    R.flags = lost(PHOSIM_LOST_MISSED, si < 0 ? 0 : P.n_surf);
}

// Wavelength (Sec. 2.2): cumulative photon-number table, blur within the bin, redshift.  FP64 in both FP64-optics
// paths: the coating decisions bin it, and a single-precision wavelength would move about one photon in 5e6
// across a band edge of a filter (a form that blurred in FP32 took as many FP64-pipe operations, in its
// conversions, as this one).
template <bool MIXED>
__device__ __forceinline__ double sample_wavelength(const TraceParams& P, const DSource& s, const uint4& w0) {
    const int bin = sed_bin(P.thr + (size_t)s.sed * (P.n_bins - 1), P.sed_guide + (size_t)s.sed * (kSedGuide + 1), w0.z);
    return fma(u64of(w0.w), P.sed_dlam, P.sed_lam0 + bin * P.sed_dlam) * s.zfac;
}

// Dynamic transmission (Sec. 3.2): the index of the first coated surface whose accept draw is not below the
// largest transmission any incidence angle allows at this wavelength (the photon is certainly rejected
// there), or -1.
__device__ __forceinline__ int early_coating_reject(const TraceParams& P, double lam, const uint4& w2, const uint4& w3) {
    // with reflecting coatings only the first coated surface's draw is certain to be used (a ghost decides
    // later surfaces with its own words)
    const int nk = (P.flags & kGhostFlag) ? min(1, P.n_coated) : P.n_coated;
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        const int si = P.coated_surface[k];
        const DCoating& C = P.coat[P.surf[si].coating];
        int il = (int)floor((lam - C.lam0) * C.inv_dlam);
        il = il < 0 ? 0 : (il > C.nl - 1 ? C.nl - 1 : il);
        const uint32_t w = k < 2 ? word(w2, 2 + k) : word(w3, k - 2);
        if (!(u64of(w) < __ldg(C.Tmax + il))) return si;
    }
    return -1;
}

// The early-rejection decision of photon i alone (no propagation): -1 if it goes on, else the surface.
template <bool MIXED>
__device__ __forceinline__ int early_reject_surface(const TraceParams& P, const DSource& s, int src, uint64_t i,
                                                    double& lam) {
    i = ray_of(s.bundle, i);
    const uint32_t clo = (uint32_t)i, chi = (uint32_t)(i >> 32);
    const uint4 w0 = philox(make_uint4(clo, chi, (uint32_t)src, 0u), P.k0, P.k1);
    lam = sample_wavelength<MIXED>(P, s, w0);
    const uint4 w2 = philox(make_uint4(clo, chi, (uint32_t)src, 2u), P.k0, P.k1);
    uint4 w3 = make_uint4(0u, 0u, 0u, 0u);
    if (P.n_coated > 2) w3 = philox(make_uint4(clo, chi, (uint32_t)src, 3u), P.k0, P.k1);
    return early_coating_reject(P, lam, w2, w3);
}

template <bool MIXED, bool RECORD = false>
__device__ __forceinline__ void trace_photon(const TraceParams& P, const DSource& s, int src, uint64_t photon,
                                             PhotonOut& R, ForwardRecord* fr = nullptr) {
    const uint64_t i = ray_of(s.bundle, photon);
    const uint32_t clo = (uint32_t)i, chi = (uint32_t)(i >> 32);
    const uint4 w0 = philox(make_uint4(clo, chi, (uint32_t)src, 0u), P.k0, P.k1);
    const uint4 w1 = philox(make_uint4(clo, chi, (uint32_t)src, 1u), P.k0, P.k1);
    R.flags = 0; R.pix = -1; R.x = R.y = R.xc = R.yc = 0.0;
    // time stamp (Sec. 2.2)
    const double t = fma(s.t_exp, u64of(w1.x), s.t0);
    const double lam = sample_wavelength<MIXED>(P, s, w0);
    R.lam = lam;
    // direction: tangent-plane components, paraxial shape offset, renormalised (Sec. 2.2, 2.2.1)
    double nx = s.xi, ny = s.eta;
    if (s.kind == PHOSIM_SERSIC) {
        if constexpr (MIXED) {
            const float r = lerp_table_f(P.sersic32 + (size_t)s.table * P.sersic_K, P.sersic_K,
                                         u32of(w1.y) * (float)P.sersic_K - 0.5f);
            float sp, cp;
            sincospif(2.f * u32of(w1.z), &sp, &cp);
            const float dx = (float)s.a * r * cp, dy = (float)s.b * r * sp;
            nx += (double)(dx * (float)s.cpa - dy * (float)s.spa);
            ny += (double)(dx * (float)s.spa + dy * (float)s.cpa);
        } else {
            const double r = lerp_table(P.sersic + (size_t)s.table * P.sersic_K, P.sersic_K,
                                        u64of(w1.y) * P.sersic_K - 0.5);
            double sp, cp;
            sincospi(2.0 * u64of(w1.z), &sp, &cp);
            const double dx = s.a * r * cp, dy = s.b * r * sp;
            nx += dx * s.cpa - dy * s.spa;
            ny += dx * s.spa + dy * s.cpa;
        }
    } else if (s.kind == PHOSIM_GAUSS) {
        if constexpr (MIXED) {
            const float g = sqrtf(-2.f * logf(u32of(w1.y)));
            float sp, cp;
            sincospif(2.f * u32of(w1.z), &sp, &cp);
            nx += (double)((float)s.a * g * cp);
            ny += (double)((float)s.a * g * sp);
        } else {
            const double g = sqrt(-2.0 * log(u64of(w1.y)));
            double sp, cp;
            sincospi(2.0 * u64of(w1.z), &sp, &cp);
            nx += s.a * g * cp;
            ny += s.a * g * sp;
        }
    }
    // 1 / |n_z| = rsqrt(1 - n_x^2 - n_y^2): layer-to-layer distances are height differences times it
    double w = fma(-nx, nx, fma(-ny, ny, 1.0));
    double rinv = rsqrt(w);
    const uint4 w2 = philox(make_uint4(clo, chi, (uint32_t)src, 2u), P.k0, P.k1);
    uint4 w3 = make_uint4(0u, 0u, 0u, 0u);
    if (P.n_coated > 2) w3 = philox(make_uint4(clo, chi, (uint32_t)src, 3u), P.k0, P.k1);
    if (P.flags & PHOSIM_EARLY_REJECT) {
        const int si = early_coating_reject(P, lam, w2, w3);
        if (si >= 0) { R.flags = lost(PHOSIM_LOST_COATING, si); return; }
    }
    // pupil point on the annulus, on the nominal first surface, moved back to the top of the atmosphere
    const double r = sqrt(fma(u64of(w0.x), P.pr_dr2, P.pr_in2));
    double sp, cp;
    sincospi(2.0 * u64of(w0.y), &sp, &cp);
    double x = r * cp, y = r * sp;
    double zs = 0.0, zx, zy;
    sag(P.pupil_surf, x, y, zs, zx, zy);
    double z = P.pupil_z + zs;
    {
        const double l = (P.h_top - z) * rinv;
        x = fma(-nx, l, x);
        y = fma(-ny, l, y);
        z = P.h_top;
    }
    uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
    if (P.hf_K > 0 || (P.flags & PHOSIM_BACK_REFLECT)) w4 = philox(make_uint4(clo, chi, (uint32_t)src, 4u), P.k0, P.k1);
    // frozen-flow layers top to bottom: propagate, refractive kick from the screen gradient (Sec. 2.3)
    if (P.flags & PHOSIM_ATMOSPHERE) {
        double kick;
        if constexpr (MIXED) {
            kick = (double)((float)P.kick0 * exp2f(-0.2f * log2f((float)(lam / P.lam_ref))));
        } else {
            // (lambda / lambda_ref)^(-1/5): single-precision seed, then two Newton steps of y -> y (1 + (1 - a y^5) / 5)
            const double a = lam / P.lam_ref;
            double y5 = (double)powf((float)a, -0.2f);
#pragma unroll
            for (int it = 0; it < 2; ++it) {
                const double y2 = y5 * y5;
                y5 = fma(y5 * 0.2, fma(-a * y2, y2 * y5, 1.0), y5);
            }
            kick = P.kick0 * y5;
        }
#pragma unroll 1
        for (int k = 0; k < P.n_layers; ++k) {
            const DLayer& L = P.layer[k];
            const double ll = (z - L.z) * rinv;
            x = fma(nx, ll, x);
            y = fma(ny, ll, y);
            z = L.z;
            const double sx = fma(-L.vx, t, x), sy = fma(-L.vy, t, y);
            double gx = 0.0, gy = 0.0;
#pragma unroll 1
            for (int q = 0; q < L.n_scales; ++q) screen_gradient<MIXED>(L.s[q], sx, sy, gx, gy);
            nx = fma(kick, gx, nx);
            ny = fma(kick, gy, ny);
            w = fma(-nx, nx, fma(-ny, ny, 1.0));
            rinv = rsqrt(w);
        }
        // second kick (Sec. 2.3.2): a draw from the long-exposure PSF of the screens above kappa_crit,
        // scaled like the refractive kick by (lambda / lambda_ref)^(-1/5)
        if (P.hf_K > 0) {
            const double scale = kick / P.kick0;
            if constexpr (MIXED) {
                const float ang = lerp_table_f(P.hf32, P.hf_K, u32of(w4.x) * (float)P.hf_K - 0.5f) * (float)scale;
                float sp, cp;
                sincospif(2.f * u32of(w4.y), &sp, &cp);
                nx += (double)(ang * cp);
                ny += (double)(ang * sp);
            } else {
                const double ang = lerp_table(P.hf, P.hf_K, u64of(w4.x) * P.hf_K - 0.5) * scale;
                double sp, cp;
                sincospi(2.0 * u64of(w4.y), &sp, &cp);
                nx = fma(ang, cp, nx);
                ny = fma(ang, sp, ny);
            }
            w = fma(-nx, nx, fma(-ny, ny, 1.0));
            rinv = rsqrt(w);
        }
    }
    const double nz = -w * rinv;
    {
        const double l = (z - P.z_ent) * rinv;
        x = fma(nx, l, x);
        y = fma(ny, l, y);
        z = P.z_ent;
    }
    double X[3] = {x, y, z}, D[3] = {nx, ny, nz};
    MemberDraw mb;
    const bool bundled = s.bundle > 1;
    if (bundled) mb = member_draw<MIXED>(P, s.bsig, src, photon);
    optics<MIXED, true, RECORD>(P, X, D, lam, w1, w2, w3, w4, R, fr, bundled ? &mb : nullptr, src, i);
}


// Which source owns launch tile t: binary search over the per-source tile prefix (lane 0, then broadcast).
__device__ __forceinline__ int tile_source(const TraceParams& P, uint64_t t, int lane) {
    int src = 0;
    if (lane == 0) {
        int lo = 0, hi = P.n_src - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (P.tile_prefix[mid] <= t) lo = mid;
            else hi = mid - 1;
        }
        src = lo;
    }
    return __shfl_sync(0xffffffffu, src, 0);
}

}  // namespace phosim
