// The photon path of Peterson et al. (2015), Sec. 2.2-2.5, with double-single arithmetic on the FP32 pipes
// (precision PHOSIM_MIXED_DS).
//
// The steps, their order and the random-number slots are those of trace_photon in photon.cuh; what
// changes is the number type.  Positions, directions, the surface transforms, the intersections and the
// final focal-plane position, which the FP64 paths keep in double precision, are double-single pairs
// (ds.cuh, about 48 significant bits); the deflections, the wavelength, the sensor draws and the moment
// partials are single precision as in the mixed path.  Accept decisions on coatings compare the integer
// random word with integer thresholds, so for a given table bin they are those of the FP64 paths exactly.
#pragma once

#include "photon.cuh"

// inlining of the larger steps (sag, intersection, refraction, Sellmeier index, pupil azimuth): inline is
// faster (no call boundaries inside the surface loop); the quotient, roots and the generator stay out of line
#ifndef PHOSIM_DS_SAG
#define PHOSIM_DS_SAG __forceinline__
#endif
#ifndef PHOSIM_DS_PHILOX
#define PHOSIM_DS_PHILOX __noinline__
#endif
#ifndef PHOSIM_DS_STEP
#define PHOSIM_DS_STEP __forceinline__
#endif

namespace phosim {

// A work unit of the two-kernel path is a photon, or for a bundle of n photons per ray (Sec. 3.2) a ray:
// the ray is traced once and its photons (those in the call's range) only go through the sensor apart.
__device__ __forceinline__ void unit_members(const DSource& s, uint32_t nb, uint64_t u, uint64_t& lo, uint32_t& nm) {
    if (nb <= 1) { lo = u; nm = 1; return; }
    const uint64_t a = max(s.first, u * nb), b = min(s.first + s.count, (u + 1) * nb);
    lo = a;
    nm = b > a ? (uint32_t)(b - a) : 0u;
}

// one out-of-line copy of the generator for the double-single path (the FP64 kernels inline it)
static __device__ PHOSIM_DS_PHILOX uint4 philox_ds(uint4 c, uint32_t k0, uint32_t k1) { return philox(c, k0, k1); }

struct PhotonOutS {
    ds x, y, xc, yc;
    float lam;
    uint32_t flags;
    int pix;
};

// A photon's state on the entrance plane of the telescope, passed from the entry stage to the optics stage
// of the two-kernel double-single path (64 bytes)
struct __align__(16) DSState {
    ds x, y;                      // on the entrance plane (z is the plane's)
    float lam_lo, pad;            // the low word of the double-single wavelength (lam + lam_lo)
    ds nx, ny, nz;
    float lam;
    int src;
    unsigned long long idx;       // photon index within its source's stream
};

// A ray on the detector surface (detector frame): hit point, direction, normal, index of the medium in front.
struct DetectorHit {
    ds px, py;
    ds dl[3], N[3];
    ds n_cur;
    int si;
};

// A bundle's ray on the detector surface, handed from the optics stage to the photons of the bundle
struct __align__(16) DSHit {
    DetectorHit H;
    float lam, lam_lo;            // the ray's double-single wavelength
    int src;
    unsigned long long ray;
};

// one chunk of the two-kernel path: tiles [tile_begin, tile_end) of the launch, their states and the
// bundle rays' detector hits, with their counts
struct DSStage {
    DSState* state;
    unsigned long long* n_state;
    DSHit* hits;
    unsigned long long* n_hits;
    unsigned long long* batch;    // the optics stage's blocks claim batches of states from this count
    uint64_t tile_begin, tile_end;
};

// the per-source constants of a tile, converted once per tile
struct SourceS {
    ds xi, eta, t0, t_exp, ref_x, ref_y;
    float zfac, a, b, cpa, spa, bsig;
    ds zfac_s;
    int kind, sed, table;
    uint32_t bundle;
};

__device__ __forceinline__ SourceS source_s(const DSource& s) {
    SourceS r;
    r.xi = ds_of(s.xi); r.eta = ds_of(s.eta); r.t0 = ds_of(s.t0); r.t_exp = ds_of(s.t_exp);
    r.ref_x = ds_of(s.ref_x); r.ref_y = ds_of(s.ref_y);
    r.zfac = (float)s.zfac; r.zfac_s = ds_of(s.zfac); r.a = (float)s.a; r.b = (float)s.b; r.cpa = (float)s.cpa; r.spa = (float)s.spa;
    r.kind = s.kind; r.sed = s.sed; r.table = s.table;
    r.bundle = s.bundle; r.bsig = (float)s.bsig;
    return r;
}

// ------------------------------------------------------------------------------------------------------
// sin and cos of 2 pi u for an exact uniform u: quadrant from v = 4u, phi = (v - k) pi / 2 in
// [-pi/4, pi/4], then the Taylor series of sin and cos in x = phi^2 to x^7 (truncation below 1e-15), the
// terms above x^4 in single precision and the rest as double-single.
// ------------------------------------------------------------------------------------------------------
static __device__ PHOSIM_DS_STEP void ds_sincos_2pi(ds u, ds& s, ds& c) {
    const ds v = {u.hi * 4.f, u.lo * 4.f};
    const float k = rintf(v.hi);
    const ds f = v - k;
    const ds phi = f * ds{1.5707963705062866f, -4.371138828673793e-08f};
    const ds x = phi * phi;
    const float xf = x.hi;
    // sin(phi) / phi
    const float ts = fmaf(xf, fmaf(xf, -7.647163609812713e-13f, 1.6059044372074283e-10f), -2.5052107943679403e-08f);
    ds ps = dfma(x, ts, ds{2.7557318844628753e-06f, 3.793571224297229e-14f});
    ps = dfma(x, ps, ds{-0.00019841270113829523f, 2.725596874933456e-12f});
    ps = dfma(x, ps, ds{0.008333333767950535f, -4.34617203337595e-10f});
    ps = dfma(x, ps, ds{-0.1666666716337204f, 4.967053879312289e-09f});
    ps = dfma(x, ps, ds_f(1.f));
    const ds sn = phi * ps;
    // cos(phi)
    const float tc = fmaf(xf, fmaf(xf, -1.147074536050896e-11f, 2.0876755879584152e-09f), -2.755731998149713e-07f);
    ds pc = dfma(x, tc, ds{2.4801587642286904e-05f, -3.40699609366682e-13f});
    pc = dfma(x, pc, ds{-0.0013888889225199819f, 3.3631094437103215e-11f});
    pc = dfma(x, pc, ds{0.0416666679084301f, -1.2417634698280722e-09f});
    pc = dfma(x, pc, ds_f(-0.5f));
    const ds cs = dfma(x, pc, ds_f(1.f));
    const int q = ((int)k) & 3;
    if (q == 0) { s = sn; c = cs; }
    else if (q == 1) { s = cs; c = -sn; }
    else if (q == 2) { s = -sn; c = -cs; }
    else { s = -cs; c = sn; }
}

// Sellmeier index (Sec. 2.4.1) of the single-precision wavelength, in double-single
static __device__ PHOSIM_DS_STEP ds sellmeier_ds(const DMaterial& m, float lam_nm) {
    const ds lu = ds_f(lam_nm) * ds{0.0010000000474974513f, -4.7497450417210985e-11f};   // micrometres
    const ds l2 = lu * lu;
    ds n2 = ds_f(1.f);
#pragma unroll
    for (int i = 0; i < 3; ++i) n2 = n2 + m.Bs[i] * l2 / (l2 - m.Cs[i]);
    return ds_sqrt(n2);
}

__device__ __forceinline__ void zern_eval_f(const float* __restrict__ zp, float u, float v, float& z, float& zu,
                                            float& zv) {
    float q[7], dq[7];
    int off = 0;
#pragma unroll
    for (int b = 0; b <= 6; ++b) {
        const int deg = 6 - b;
        float acc = zp[off + deg], dacc = 0.f;
#pragma unroll
        for (int a = deg - 1; a >= 0; --a) {
            dacc = fmaf(dacc, u, acc);
            acc = fmaf(acc, u, zp[off + a]);
        }
        q[b] = acc;
        dq[b] = dacc;
        off += deg + 1;
    }
    float zz = q[6], zzu = dq[6], zzv = 0.f;
#pragma unroll
    for (int b = 5; b >= 0; --b) {
        zzv = fmaf(zzv, v, zz);
        zz = fmaf(zz, v, q[b]);
        zzu = fmaf(zzu, v, dq[b]);
    }
    z = zz; zu = zzu; zv = zzv;
}

// Sag and slopes (Sec. 2.4.1).  The Zernike figure (tens of nanometres) is evaluated in single precision:
// its absolute error is far below the 1e-8 mm the intersection resolves.  With the slopes S_x = x g(r^2),
// S_y = y g(r^2) it returns, in single precision, g and, for the conic and even terms, g1 = dg / d(r^2), which
// give the second derivatives S_xx = g + 2 x^2 g1, S_xy = 2 x y g1, S_yy = g + 2 y^2 g1.
static __device__ PHOSIM_DS_SAG bool sag_ds(const DSurfaceS& E, int flags, ds x, ds y, ds& z, ds& zx, ds& zy,
                                            float& gf, float& g1f) {
    const ds r2 = dfma(x, x, y * y);
    ds g = ds_f(0.f);
    z = ds_f(0.f);
    g1f = 0.f;
    if (flags & SF_CONIC) {
        const ds arg = ds_f(1.f) - E.k1c2 * r2;
        if (arg.hi < 0.f) return false;
        const ds rs = ds_rsqrt(arg);
        z = E.c * r2 / dfma(arg, rs, ds_f(1.f));
        g = E.c * rs;
        // g = c (1 - k1c2 r^2)^(-1/2): dg / d(r^2) = k1c2 c rs^3 / 2
        g1f = 0.5f * E.k1c2.hi * g.hi * rs.hi * rs.hi;
    }
    // Horner from the last nonzero coefficient: the zero terms above it would add exact zeros
    if (flags & SF_EVEN) {
        const ds u = r2 * E.inv_rn2;
        int k = E.ne - 1;
        ds pe = E.ae[k], pd = E.aed[k];
#pragma unroll 1
        while (--k >= 0) {
            pe = dfma(pe, u, E.ae[k]);
            pd = dfma(pd, u, E.aed[k]);
        }
        z = dfma(u * u, pe, z);
        g = dfma(u * E.inv_rn2, pd, g);
        // the even part of g is sum_k aed[k] u^(k+1) / rn^2, so its derivative in r^2 is sum_k ae2[k] u^k
        k = E.ne - 1;
        float q = E.ae2[k];
#pragma unroll 1
        while (--k >= 0) q = fmaf(q, u.hi, E.ae2[k]);
        g1f += q;
    }
    if (flags & SF_ODD) {
        const ds rho = ds_sqrt(r2) * E.inv_rn;
        const ds u = rho * rho;
        int k = E.no - 1;
        ds po = E.ao[k], pd = E.aod[k];
#pragma unroll 1
        while (--k >= 0) {
            po = dfma(po, u, E.ao[k]);
            pd = dfma(pd, u, E.aod[k]);
        }
        z = dfma(u * rho, po, z);
        g = dfma(rho * E.inv_rn2, pd, g);
    }
    {
        const ds2 q = mul2(ds2_of(x, y), g);
        zx = ds2_x(q);
        zy = ds2_y(q);
    }
    gf = g.hi;
    if (flags & SF_ZERN) {
        float zz, zu, zv;
        zern_eval_f(E.zp, x.hi * E.zinv, y.hi * E.zinv, zz, zu, zv);
        z = z + zz;
        zx = zx + zu * E.zinv;
        zy = zy + zv * E.zinv;
    }
    return true;
}

// the unit normal (-S_x, -S_y, 1) / |.| from the slopes
__device__ __forceinline__ void slope_normal_ds(ds zx, ds zy, ds N[3]) {
    const ds inv = ds_rsqrt(dfma(zx, zx, dfma(zy, zy, ds_f(1.f))));
    const ds2 nxy = mul2(ds2_of(zx, zy), inv);
    N[0] = -ds2_x(nxy); N[1] = -ds2_y(nxy); N[2] = inv;
}

// Newton's method in double-single on F(l) = p_z + l d_z - S(p_x + l d_x, p_y + l d_y) from l until the step
// is below 1e-8 mm (the Newton slope F'(l) only scales the step, so it is taken in single precision); the
// normal from the slopes at the last point.  Newton's error after a step s is about F'' s^2 / (2 F'), with
// F'' = -d^T H d (H the sag's second derivatives, d the direction's x, y part): where that bound is below
// 1e-10 mm the root is taken after this step, with the slopes carried to the new point by H (their change
// over the step, tens of nanoradians, in single precision), instead of a further evaluation of the sag.
// The single-precision second derivatives cover the conic and even terms, so surfaces with odd or Zernike
// terms iterate until the step itself is below 1e-8 mm.
// The hit point is the last point of the iteration moved by the last step along the ray.
__device__ __forceinline__ uint32_t newton_ds(const DSurfaceS& E, int flags, const ds p[3], const ds d[3], ds& l,
                                              ds N[3], ds hit[3]) {
    ds zx = ds_f(0.f), zy = ds_f(0.f);
#pragma unroll 1
    for (int it = 0; it < 20; ++it) {
        const ds2 xy = dfma2(l, ds2_of(d[0], d[1]), ds2_of(p[0], p[1]));
        const ds x = ds2_x(xy), y = ds2_y(xy);
        ds zs;
        float gf, g1f;
        if (!sag_ds(E, flags, x, y, zs, zx, zy, gf, g1f)) return PHOSIM_LOST_MISSED;
        const ds zr = dfma(l, d[2], p[2]);
        const ds F = zr - zs;
        const float dF = d[2].hi - zx.hi * d[0].hi - zy.hi * d[1].hi;
        if (dF == 0.f) return PHOSIM_LOST_NEWTON;
        const float step = F.hi * __fdividef(1.f, dF);
        l = l - step;
        const auto moved = [&] {
            const ds2 h = dfma2(ds2_of(d[0], d[1]), -step, xy);
            hit[0] = ds2_x(h); hit[1] = ds2_y(h);
            hit[2] = dfma(d[2], -step, zr);
        };
        if (fabsf(step) < 1e-8f) {
            slope_normal_ds(zx, zy, N);
            moved();
            return 0;
        }
        if (!(flags & (SF_ODD | SF_ZERN))) {
            const float xf = x.hi, yf = y.hi, dx = d[0].hi, dy = d[1].hi;
            const float hxy = 2.f * xf * yf * g1f;
            const float hdx = fmaf(fmaf(2.f * xf * xf, g1f, gf), dx, hxy * dy);
            const float hdy = fmaf(hxy, dx, fmaf(2.f * yf * yf, g1f, gf) * dy);
            const float fpp = fmaf(dx, hdx, dy * hdy);
            if (fabsf(fpp) * (step * step) < 2e-10f * fabsf(dF)) {
                // the point moved by -step (dx, dy): the slopes by -step H (dx, dy)
                const ds2 zn = add2(ds2_of(zx, zy), make_float2(-step * hdx, -step * hdy));
                slope_normal_ds(ds2_x(zn), ds2_y(zn), N);
                moved();
                return 0;
            }
        }
    }
    return PHOSIM_LOST_NEWTON;
}

// Sag and slopes in single precision (the hi parts of the surface's constants), for the first Newton steps
__device__ __forceinline__ bool sag_f(const DSurfaceS& E, int flags, float x, float y, float& z, float& zx, float& zy) {
    const float r2 = fmaf(x, x, y * y);
    float g = 0.f;
    z = 0.f;
    if (flags & SF_CONIC) {
        const float arg = fmaf(-E.k1c2.hi, r2, 1.f);
        if (arg < 0.f) return false;
        const float rs = rsqrtf(arg);
        z = E.c.hi * r2 / fmaf(arg, rs, 1.f);
        g = E.c.hi * rs;
    }
    if (flags & SF_EVEN) {
        const float u = r2 * E.inv_rn2.hi;
        int k = E.ne - 1;
        float pe = E.ae[k].hi, pd = E.aed[k].hi;
#pragma unroll 1
        while (--k >= 0) {
            pe = fmaf(pe, u, E.ae[k].hi);
            pd = fmaf(pd, u, E.aed[k].hi);
        }
        z = fmaf(u * u, pe, z);
        g = fmaf(u * E.inv_rn2.hi, pd, g);
    }
    if (flags & SF_ODD) {
        const float rho = sqrtf(r2) * E.inv_rn.hi;
        const float u = rho * rho;
        int k = E.no - 1;
        float po = E.ao[k].hi, pd = E.aod[k].hi;
#pragma unroll 1
        while (--k >= 0) {
            po = fmaf(po, u, E.ao[k].hi);
            pd = fmaf(pd, u, E.aod[k].hi);
        }
        z = fmaf(u * rho, po, z);
        g = fmaf(rho * E.inv_rn2.hi, pd, g);
    }
    zx = x * g;
    zy = y * g;
    if (flags & SF_ZERN) {
        float zz, zu, zv;
        zern_eval_f(E.zp, x * E.zinv, y * E.zinv, zz, zu, zv);
        z += zz;
        zx = fmaf(zu, E.zinv, zx);
        zy = fmaf(zv, E.zinv, zy);
    }
    return true;
}

// The unit normal of a conic at a point (x, y, z) on it: (-c x, -c y, 1 - kc z) normalised.  For a sphere
// (kappa = 0, kc = c) that vector's squared length is 1 + c Q with Q = c (x^2 + y^2) + c z^2 - 2 z the quadric,
// which vanishes at the intersection: it is already a unit vector (to the root's 1e-14) and needs no root.
__device__ __forceinline__ void conic_normal_ds(const DSurfaceS& E, ds x, ds y, ds z, ds N[3]) {
    const ds2 cxy = mul2(E.c, ds2_of(x, y));
    const ds vx = -ds2_x(cxy), vy = -ds2_y(cxy), vz = ds_f(1.f) - E.kc * z;
    if (E.kmc.hi == 0.f) {
        N[0] = vx; N[1] = vy; N[2] = vz;
        return;
    }
    const ds inv = ds_rsqrt(dfma(vx, vx, dfma(vy, vy, vz * vz)));
    const ds2 nxy = mul2(ds2_of(vx, vy), inv);
    N[0] = ds2_x(nxy); N[1] = ds2_y(nxy);
    N[2] = vz * inv;
}

// the point p + l d of a ray (x and y as a packed pair)
__device__ __forceinline__ void ray_point_ds(ds l, const ds p[3], const ds d[3], ds out[3]) {
    const ds2 q = dfma2(l, ds2_of(d[0], d[1]), ds2_of(p[0], p[1]));
    out[0] = ds2_x(q);
    out[1] = ds2_y(q);
    out[2] = dfma(l, d[2], p[2]);
}

// Intersection (Sec. 2.4.2), the steps of intersect() in phosim_device.cuh: the conic's exact root on the
// vertex branch, then Newton's method for the aspheric and Zernike terms until the step is below 1e-8 mm.
// Newton converges to the same root from any start close enough to it, so the start is computed in single
// precision: the conic's root, then for the aspheric and Zernike surfaces Newton steps while they exceed 10 um
// (the asphere moves the root by up to millimetres).  For those, the double-single Newton steps take it from
// there to the final 1e-8 mm; for a plain conic one double-single Newton step on the quadric Q = c (x^2 + y^2) +
// kc z^2 - 2 z along the ray does: from a single-precision root (error below 1e-3 mm for the paths here) it
// leaves an error of about (Q'' / 2 Q') e^2 ~ c e^2, below 1e-10 mm (Q', which only scales the step, in single
// precision).  A ray whose single-precision discriminant is not clearly positive (grazing or missing the
// conic) takes the double-single root.
static __device__ PHOSIM_DS_STEP uint32_t intersect_ds(const DSurfaceS& E, int flags, const ds p[3], const ds d[3], ds& l,
                                                 ds N[3], ds hit[3]) {
    if (flags & SF_FLAT_ONLY) {
        if (d[2].hi == 0.f) return PHOSIM_LOST_MISSED;
        l = -(p[2] / d[2]);
        N[0] = ds_f(0.f); N[1] = ds_f(0.f); N[2] = ds_f(1.f);
        ray_point_ds(l, p, d, hit);
        return 0;
    }
    const bool newton = (flags & (SF_EVEN | SF_ODD | SF_ZERN)) != 0;
    if (newton) {
        const float c = E.c.hi, kc = E.kc.hi;
        const float Af = fmaf(E.kmc.hi * d[2].hi, d[2].hi, c);
        const float bf = fmaf(kc * p[2].hi, d[2].hi, c * fmaf(p[0].hi, d[0].hi, p[1].hi * d[1].hi)) - d[2].hi;
        const float Cf = fmaf(kc * p[2].hi, p[2].hi, c * fmaf(p[0].hi, p[0].hi, p[1].hi * p[1].hi)) - 2.f * p[2].hi;
        const float disc = fmaf(bf, bf, -(Af * Cf));
        if (disc > 1e-6f * bf * bf) {
            const float sq = sqrtf(disc);
            const float qf = bf >= 0.f ? -(bf + sq) : sq - bf;
            float lf = Cf / qf;
            if (Af != 0.f && fmaf(-kc, fmaf(lf, d[2].hi, p[2].hi), 1.f) < 0.f) lf = qf / Af;
#pragma unroll 1
            for (int it = 0; it < 4; ++it) {
                const float x = fmaf(lf, d[0].hi, p[0].hi), y = fmaf(lf, d[1].hi, p[1].hi);
                float zs, zxf, zyf;
                if (!sag_f(E, flags, x, y, zs, zxf, zyf)) break;
                const float dF = d[2].hi - zxf * d[0].hi - zyf * d[1].hi;
                const float step = (fmaf(lf, d[2].hi, p[2].hi) - zs) / dF;
                if (!(fabsf(step) < 1e30f)) break;
                lf -= step;
                if (fabsf(step) < 1e-2f) break;
            }
            if (fabsf(lf) < 1e30f) {
                l = ds_f(lf);
                return newton_ds(E, flags, p, d, l, N, hit);
            }
        }
    } else {
        const float c = E.c.hi, kc = E.kc.hi;
        const float Af = fmaf(E.kmc.hi * d[2].hi, d[2].hi, c);
        const float bf = fmaf(kc * p[2].hi, d[2].hi, c * fmaf(p[0].hi, d[0].hi, p[1].hi * d[1].hi)) - d[2].hi;
        const float Cf = fmaf(kc * p[2].hi, p[2].hi, c * fmaf(p[0].hi, p[0].hi, p[1].hi * p[1].hi)) - 2.f * p[2].hi;
        const float disc = fmaf(bf, bf, -(Af * Cf));
        if (disc > 1e-6f * bf * bf) {
            const float sq = sqrtf(disc);
            const float qf = bf >= 0.f ? -(bf + sq) : sq - bf;
            float lf = Cf / qf;
            if (Af != 0.f && fmaf(-kc, fmaf(lf, d[2].hi, p[2].hi), 1.f) < 0.f) lf = qf / Af;
            if (fabsf(lf) < 1e30f) {
                l = ds_f(lf);
                ds q0[3];
                ray_point_ds(l, p, d, q0);
                const ds x = q0[0], y = q0[1], z = q0[2];
                const ds Q = dfma(E.c, dfma(x, x, y * y), dfma(E.kc * z, z, z * -2.f));
                const float dQ = 2.f * (fmaf(c, fmaf(x.hi, d[0].hi, y.hi * d[1].hi), kc * z.hi * d[2].hi) - d[2].hi);
                if (dQ != 0.f) {
                    l = l - Q.hi / dQ;
                    ray_point_ds(l, p, d, hit);
                    conic_normal_ds(E, hit[0], hit[1], hit[2], N);
                    return 0;
                }
            }
        }
    }
    // the quadric's l^2 coefficient c (d_x^2 + d_y^2) + kc d_z^2, which for the unit direction is c + (kc - c) d_z^2
    const ds A = dfma(E.kmc * d[2], d[2], E.c);
    const ds b = dfma(E.kc * p[2], d[2], E.c * dfma(p[0], d[0], p[1] * d[1])) - d[2];
    const ds C = dfma(E.kc * p[2], p[2], E.c * dfma(p[0], p[0], p[1] * p[1])) - p[2] * 2.f;
    const ds disc = dfma(b, b, -(A * C));
    if (disc.hi < 0.f) return PHOSIM_LOST_MISSED;
    const ds sq = ds_sqrt(disc);
    const ds q = b.hi >= 0.f ? -(b + sq) : sq - b;
    if (q.hi == 0.f) return PHOSIM_LOST_MISSED;
    l = C / q;
    if (A.hi != 0.f && (ds_f(1.f) - E.kc * dfma(l, d[2], p[2])).hi < 0.f) l = q / A;
    if (newton) return newton_ds(E, flags, p, d, l, N, hit);
    ray_point_ds(l, p, d, hit);
    conic_normal_ds(E, hit[0], hit[1], hit[2], N);
    return 0;
}

__device__ __forceinline__ ds dot3(const ds a[3], const ds b[3]) { return dfma(a[0], b[0], dfma(a[1], b[1], a[2] * b[2])); }

// Snell's law in vector form (Sec. 2.4.2), mu = n1 / n2; false on total internal reflection
static __device__ PHOSIM_DS_STEP bool refract_ds(ds d[3], ds N[3], ds mu) {
    ds cosi = -dot3(d, N);
    ds n0 = N[0], n1 = N[1], n2 = N[2];
    if (cosi.hi < 0.f) { n0 = -n0; n1 = -n1; n2 = -n2; cosi = -cosi; }
    const ds k = ds_f(1.f) - mu * mu * (ds_f(1.f) - cosi * cosi);
    if (k.hi < 0.f) return false;
    const ds a = mu * cosi - ds_sqrt(k);
    {
        const ds2 q = dfma2(mu, ds2_of(d[0], d[1]), mul2(a, ds2_of(n0, n1)));
        d[0] = ds2_x(q);
        d[1] = ds2_y(q);
    }
    d[2] = dfma(mu, d[2], a * n2);
    return true;
}

__device__ __forceinline__ void to_surface_ds(const DSurfaceS& E, int flags, const ds x[3], const ds d[3], ds p[3],
                                              ds dl[3]) {
    if (!(flags & (SF_ROTATED | SF_DECENTERED))) {     // a vertex on the axis: x - 0 is x
        p[0] = x[0]; p[1] = x[1]; p[2] = x[2] - E.o[2];
        dl[0] = d[0]; dl[1] = d[1]; dl[2] = d[2];
        return;
    }
    const ds rx = x[0] - E.o[0], ry = x[1] - E.o[1], rz = x[2] - E.o[2];
    if (!(flags & SF_ROTATED)) {
        p[0] = rx; p[1] = ry; p[2] = rz;
        dl[0] = d[0]; dl[1] = d[1]; dl[2] = d[2];
        return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        p[i] = dfma(E.M[3 * i], rx, dfma(E.M[3 * i + 1], ry, E.M[3 * i + 2] * rz));
        dl[i] = dfma(E.M[3 * i], d[0], dfma(E.M[3 * i + 1], d[1], E.M[3 * i + 2] * d[2]));
    }
}

__device__ __forceinline__ void from_surface_ds(const DSurfaceS& E, int flags, const ds p[3], const ds dl[3], ds x[3],
                                                ds d[3]) {
    if (!(flags & SF_ROTATED)) {
        if (flags & SF_DECENTERED) {
            x[0] = p[0] + E.o[0]; x[1] = p[1] + E.o[1];
        } else {
            x[0] = p[0]; x[1] = p[1];
        }
        x[2] = p[2] + E.o[2];
        d[0] = dl[0]; d[1] = dl[1]; d[2] = dl[2];
        return;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        x[i] = dfma(E.M[i], p[0], dfma(E.M[3 + i], p[1], dfma(E.M[6 + i], p[2], E.o[i])));
        d[i] = dfma(E.M[i], dl[0], dfma(E.M[3 + i], dl[1], E.M[6 + i] * dl[2]));
    }
}

// the coating accept-reject: the draw (w + 1/2) 2^-32 < T exactly when w < ceil(T 2^32 - 1/2)
// The coating's wavelength bin of a photon, from its double-single wavelength: the FP64 paths' bin except within
// ~1e-14 of an edge (a single-precision wavelength would move about one photon in 5e6 across a band edge of
// the filter, and with it the photon's fate and its star's moments)
__device__ __forceinline__ int coat_lambda_bin(const DCoating& C, ds lam) {
    const int il = (int)ds_floor((lam - C.lam0_s) * C.inv_dlam_s);
    return il < 0 ? 0 : (il > C.nl - 1 ? C.nl - 1 : il);
}
// The wavelength of a photon (Sec. 2.2): (bin + u) dlam + lam0, redshifted, with the bin from the SED's
// thresholds and u = (w + 1/2) 2^-32 exact from word w of block 0, as a double-single pair (the FP64 paths'
// value to ~1e-14); its high word is the single-precision wavelength of the FP32 steps.
__device__ __forceinline__ int sed_bin_of(const TraceParams& P, int sed, const uint4& w0) {
    return sed_bin(P.thr + (size_t)sed * (P.n_bins - 1), P.sed_guide + (size_t)sed * (kSedGuide + 1), w0.z);
}
__device__ __forceinline__ ds sample_wavelength_ds(const TraceParams& P, const SourceS& s, const uint4& w0) {
    const ds lo = P.sed_lam0_s + P.sed_dlam_s * (float)sed_bin_of(P, s.sed, w0);
    return dfma(ds_uniform(w0.w), P.sed_dlam_s, lo) * s.zfac_s;
}
// dynamic transmission (Sec. 3.2) on the single-precision wavelength, as early_coating_reject
__device__ __forceinline__ int early_coating_reject_f(const TraceParams& P, ds lam, const uint4& w2, const uint4& w3) {
    const int nk = (P.flags & kGhostFlag) ? min(1, P.n_coated) : P.n_coated;   // see early_coating_reject
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        const int si = P.coated_surface[k];
        const DCoating& C = P.coat[P.surf[si].coating];
        const uint32_t w = k < 2 ? word(w2, 2 + k) : word(w3, k - 2);
        if (!((unsigned long long)w < __ldg(C.Tmax_thr + coat_lambda_bin(C, lam)))) return si;
    }
    return -1;
}

// The first stage of the dynamic transmission test (Sec. 3.2) of the double-single path, for every photon:
// the wavelength, and the coated surfaces whose worst-case transmission there is 0 (lost whatever its draw)
// or 1 (passed whatever its draw).  Returns the surface that certainly loses the photon, or -1: the photon
// goes on to the full test (early_coating_reject_f, with its draws) at the start of its propagation, which
// decides the photons a draw decides exactly as a one-stage test would, so fates, records and counts do not
// change; the coating words (a generator call) are drawn only for the photons that get that far.
// i is the photon, or for a bundle the ray.
__device__ __forceinline__ int early_reject_certain_f(const TraceParams& P, const SourceS& s, int src, uint64_t i,
                                                     float& lam) {
    const uint4 w0 = philox_ds(make_uint4((uint32_t)i, (uint32_t)(i >> 32), (uint32_t)src, 0u), P.k0, P.k1);
    // the wavelength in single precision, within ~2.5e-7 of the double-single value (relative): a bin taken
    // from it is the exact bin unless it lies that close to a bin edge, and such a photon is left to the full
    // test, which bins the double-single wavelength
    const float bin = (float)sed_bin_of(P, s.sed, w0);
    lam = fmaf(u32of(w0.w), P.sed_dlamf, fmaf(bin, P.sed_dlamf, P.sed_lam0f)) * s.zfac;
    const int nk = (P.flags & kGhostFlag) ? min(1, P.n_coated) : P.n_coated;   // see early_coating_reject
#pragma unroll 1
    for (int k = 0; k < nk; ++k) {
        const int si = P.coated_surface[k];
        const DCoating& C = P.coat[P.surf[si].coating];
        const float t = (lam - C.lam0f) * C.inv_dlamf, f = floorf(t), margin = 1e-6f * fabsf(lam) * C.inv_dlamf + 1e-6f;
        if (!(t - f > margin && t - f < 1.f - margin)) return -1;
        int il = (int)f;
        il = il < 0 ? 0 : (il > C.nl - 1 ? C.nl - 1 : il);
        const unsigned long long thr = __ldg(C.Tmax_thr + il);
        if (thr == 0ull) return si;               // no draw passes: lost here whatever the draw
        if (thr < (1ull << 32)) return -1;        // a draw decides: the full test with the photon's words
    }
    return -1;
}

// A bundle's photon (member_draw in photon.cuh) with a single-precision spread
struct MemberDrawS {
    float sx, sy;
    uint32_t conv, diff_a, diff_b, back;
};

__device__ __forceinline__ MemberDrawS member_draw_s(const TraceParams& P, float bsig, int src, uint64_t i) {
    const uint32_t clo = (uint32_t)i, chi = (uint32_t)(i >> 32);
    const uint4 m5 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 5u), P.k0, P.k1);
    const uint4 m6 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 6u), P.k0, P.k1);
    MemberDrawS m;
    const float g = sqrtf(-2.f * logf(u32of(m5.x)));
    float sn, cs;
    sincospif(2.f * u32of(m5.y), &sn, &cs);
    m.sx = bsig * g * cs;
    m.sy = bsig * g * sn;
    m.conv = m5.z; m.diff_a = m5.w; m.diff_b = m6.x; m.back = m6.y;
    return m;
}

// The random words of the surfaces and the sensor, drawn where they are used (keeping the 16 words of blocks
// 1-4 live through the whole surface loop would cost registers): the accept draw of coated surface k, and the
// sensor's conversion, diffusion and back-side reflection words (blocks 1, 2 and 4 of the ray's counter).
__device__ __forceinline__ uint32_t coat_word(const TraceParams& P, int src, uint64_t ray, int k) {
    const uint4 w = philox_ds(make_uint4((uint32_t)ray, (uint32_t)(ray >> 32), (uint32_t)src, k < 2 ? 2u : 3u), P.k0, P.k1);
    return k < 2 ? word(w, 2 + k) : word(w, k - 2);
}

// the ghost draws (ghost_word in photon.cuh), through the out-of-line generator
__device__ __forceinline__ uint32_t ghost_word_ds(const TraceParams& P, int src, uint64_t ray, int n) {
    return word(philox_ds(make_uint4((uint32_t)ray, (uint32_t)(ray >> 32), (uint32_t)src, 7u + (uint32_t)n / 4u), P.k0,
                          P.k1),
                n & 3);
}

struct SensorWords {
    uint32_t conv, diff_a, diff_b, back;
};

__device__ __forceinline__ SensorWords sensor_words(const TraceParams& P, int src, uint64_t ray) {
    const uint32_t clo = (uint32_t)ray, chi = (uint32_t)(ray >> 32);
    const uint4 w1 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 1u), P.k0, P.k1);
    const uint4 w2 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 2u), P.k0, P.k1);
    SensorWords sw;
    sw.conv = w1.w; sw.diff_a = w2.x; sw.diff_b = w2.y; sw.back = 0u;
    if (P.flags & PHOSIM_BACK_REFLECT) sw.back = philox_ds(make_uint4(clo, chi, (uint32_t)src, 4u), P.k0, P.k1).z;
    return sw;
}

// Fringing (Sec. 2.4.2) in the double-single path: the single-layer calculation of film_reflectance
// (phosim_device.cuh) with the layer's round-trip phase, about 10^3 cycles, in double-single (the wavelength,
// the silicon index's large terms, the thickness and the direction cosine c1), and the rest in single
// precision.  With q1 = N1 cos(theta1) = sqrt((n1 + i k1)^2 - s^2), s^2 = n1^2 (1 - c1^2): Re q1 = n1 c1 +
// k1^2 (1 / c1^2 - 1) / (2 n1 c1) and Im q1 = k1 / c1 to second order in k1 / n1 (k1 < 1e-2 here).
struct cfl {
    float re, im;
};
__device__ __forceinline__ cfl cf_add(cfl a, cfl b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cfl cf_sub(cfl a, cfl b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cfl cf_mul(cfl a, cfl b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cfl cf_div(cfl a, cfl b) {
    const float d = 1.f / (b.re * b.re + b.im * b.im);
    return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
__device__ __forceinline__ cfl cf_sqrt_real(float v) {     // principal root of a real number
    return v >= 0.f ? cfl{sqrtf(v), 0.f} : cfl{0.f, sqrtf(-v)};
}

static __device__ __noinline__ float film_reflectance_ds(const TraceParams& P, ds lam, float n0, ds c1, ds x, ds y,
                                                          float ell) {
    const ds E = ds_of(1239.841984) / lam;                             // photon energy, eV
    const ds n1 = dfma(ds_of(0.211), E, ds_of(3.36)) + 2.79f * expf((E.hi - 3.30f) * (1.0f / 0.398f));
    const ds lam_mm = lam * ds_of(1e-6);
    const float c1f = c1.hi, n1f = n1.hi;
    const float k1 = lam_mm.hi / (4.f * (float)M_PI * ell);
    const ds q1r = n1 * c1 + k1 * k1 * (1.f / (c1f * c1f) - 1.f) / (2.f * n1f * c1f);
    const float q1i = k1 / c1f;
    const ds t = P.fr_t0_s + x * P.fr_gxf + y * P.fr_gyf;
    const ds cycles = (t * q1r) * 2.f / lam_mm;                        // round trip: 2 t Re(q1) / lambda
    const float f = ds_frac(cycles, ds_floor(cycles));
    float sn, cs;
    sincospif(2.f * f, &sn, &cs);
    const float amp = expf(-4.f * (float)M_PI * t.hi * q1i / lam_mm.hi);
    const cfl e = {amp * cs, amp * sn};
    const float s2 = n1f * n1f * fmaxf(0.f, 1.f - c1f * c1f);
    const cfl q0 = cf_sqrt_real(n0 * n0 - s2), q2 = cf_sqrt_real(1.f - s2), q1 = {q1r.hi, q1i};
    const cfl N1sq = {n1f * n1f - k1 * k1, 2.f * n1f * k1}, n0sq = {n0 * n0, 0.f}, one = {1.f, 0.f};
    const cfl rs01 = cf_div(cf_sub(q0, q1), cf_add(q0, q1)), rs12 = cf_div(cf_sub(q1, q2), cf_add(q1, q2));
    const cfl rp01 = cf_div(cf_sub(cf_mul(N1sq, q0), cf_mul(n0sq, q1)), cf_add(cf_mul(N1sq, q0), cf_mul(n0sq, q1)));
    const cfl rp12 = cf_div(cf_sub(q1, cf_mul(N1sq, q2)), cf_add(q1, cf_mul(N1sq, q2)));
    const cfl rs = cf_div(cf_add(rs01, cf_mul(rs12, e)), cf_add(one, cf_mul(cf_mul(rs01, rs12), e)));
    const cfl rp = cf_div(cf_add(rp01, cf_mul(rp12, e)), cf_add(one, cf_mul(cf_mul(rp01, rp12), e)));
    return 0.5f * (rs.re * rs.re + rs.im * rs.im + rp.re * rp.re + rp.im * rp.im);
}

// The sensor and the pixel for a ray's hit on the detector surface (Sec. 2.4.2, 2.5): the detector steps of
// optics<MIXED = true, FULL = true>, with a bundle photon's offset and draws when mb is given.
__device__ __forceinline__ void detect_ds(const TraceParams& P, const DetectorHit& H, ds lamd, int src, uint64_t ray,
                                          PhotonOutS& R, const MemberDrawS* mb = nullptr) {
    const float lam = lamd.hi;
    const int si = H.si;
    ds p0 = H.px, p1 = H.py;
    ds dl[3] = {H.dl[0], H.dl[1], H.dl[2]}, Nv[3] = {H.N[0], H.N[1], H.N[2]};
    uint32_t w_conv, w_diff_a, w_diff_b, w_back;
    if (mb) {   // a bundle's photon: its offset from the ray's hit and its own sensor draws
        p0 = p0 + mb->sx;
        p1 = p1 + mb->sy;
        w_conv = mb->conv; w_diff_a = mb->diff_a; w_diff_b = mb->diff_b; w_back = mb->back;
    } else {
        const SensorWords sw = sensor_words(P, src, ray);
        w_conv = sw.conv; w_diff_a = sw.diff_a; w_diff_b = sw.diff_b; w_back = sw.back;
    }
    const ds hx = p0 - P.xlo_s, hy = p1 - P.ylo_s;
    if (!(hx.hi >= 0.f && hy.hi >= 0.f && ds_lt(hx, P.chip_w_s) && ds_lt(hy, P.chip_h_s))) {
        R.flags = lost(PHOSIM_LOST_OFF_CHIP, si);
        return;
    }
    ds fx = p0, fy = p1;
    R.xc = fx; R.yc = fy;
    if (P.flags & PHOSIM_SENSOR) {
        // refraction into the silicon, exponential conversion length (Sec. 2.4.2)
        const float n_si = silicon_index_f(lam);
        if (!refract_ds(dl, Nv, H.n_cur / ds_f(n_si))) { R.flags = lost(PHOSIM_LOST_TIR, si); return; }
        const float ell = lerp_table_f(P.ell32, P.n_ell, (lam - P.ell_lam0f) * P.inv_ell_dlamf);
        const float L = ell * -logf(u32of(w_conv));
        const float rf = (n_si - 1.f) / (n_si + 1.f);
        float depth = L * fabsf(dl[2].hi);
        if (!(depth <= P.t_sif)) {
            // back-side reflection: the photon turns round at the back and converts on its way back
            bool back = false;
            if (P.flags & PHOSIM_BACK_REFLECT) {
                const float r_back = (P.flags & PHOSIM_FRINGE) ? film_reflectance_ds(P, lamd, H.n_cur.hi, ds_abs(dl[2]),
                                                                                    p0, p1, ell)
                                                                : rf * rf;
                if (u32of(w_back) < r_back) {
                    depth = 2.f * P.t_sif - depth;
                    back = depth >= 0.f;
                }
            }
            if (!back) { R.flags = lost(PHOSIM_LOST_NOT_CONVERTED, si); return; }
        }
        if (depth < P.dead_layerf) { R.flags = lost(PHOSIM_LOST_DEAD_LAYER, si); return; }
        ds2 f = dfma2(ds2_of(dl[0], dl[1]), L, ds2_of(fx, fy));
        R.xc = ds2_x(f); R.yc = ds2_y(f);
        // lateral Gaussian diffusion (Sec. 2.5)
        const float sg = lerp_table_f(P.sig32, P.n_sig, depth * P.sig_scalef);
        const float g = sqrtf(-2.f * logf(u32of(w_diff_a)));
        float sn, cs;
        sincospif(2.f * u32of(w_diff_b), &sn, &cs);
        f = add2(f, make_float2(sg * g * cs, sg * g * sn));
        fx = ds2_x(f); fy = ds2_y(f);
    }
    R.x = fx; R.y = fy;
    const ds2 u = mul2(add2(ds2_of(fx, fy), neg2(ds2_of(P.xlo_s, P.ylo_s))), P.inv_pixel_s);
    const float px = ds_floor(ds2_x(u)), py = ds_floor(ds2_y(u));
    if (!(px >= 0.f && py >= 0.f && px < (float)P.nx && py < (float)P.ny)) {
        R.flags = lost(PHOSIM_LOST_OFF_CHIP, si);
        return;
    }
    R.pix = (int)py * P.nx + (int)px;
    R.flags = PHOSIM_F_DETECTED;
}

// Surfaces in order (Sec. 2.4.2) and at the detector surface the sensor (detect_ds): the steps of
// optics<MIXED = true, FULL = true> in photon.cuh, one surface per call of surface_step_ds.  For a bundle's ray
// (hand_off given) the hit on the detector surface is handed over for its photons instead, and
// R.flags = kHandedOff.
constexpr uint32_t kHandedOff = 0x80000000u;

// where a ray is in its walk through the surfaces: position and direction in the telescope frame, the surface
// it meets next and the way it travels (backwards after a ghost reflection), the index of the medium it is in
// and the last glass index computed
struct OpticsWalk {
    ds X[3], D[3];
    ds n_cur, glass_n, glass_inv;
    int glass_mat, si, dir, bounces, n_ghost;
};

__device__ __forceinline__ void walk_start(OpticsWalk& W, const ds X[3], const ds D[3]) {
#pragma unroll
    for (int k = 0; k < 3; ++k) { W.X[k] = X[k]; W.D[k] = D[k]; }
    W.n_cur = ds_f(1.f);
    W.glass_n = ds_f(1.f);
    W.glass_inv = ds_f(1.f);
    W.glass_mat = -1;
    W.si = 0; W.dir = 1; W.bounces = 0; W.n_ghost = 0;
}

// The next surface of the walk; false once the ray has left it (R.flags then says lost, detected or handed off).
__device__ __forceinline__ bool surface_step_ds(const TraceParams& P, OpticsWalk& W, ds lam, int src, uint64_t ray,
                                                PhotonOutS& R, const MemberDrawS* mb = nullptr,
                                                DetectorHit* hand_off = nullptr) {
    const int si = W.si;
    if (si < 0 || si >= P.n_surf) {
        R.flags = lost(PHOSIM_LOST_MISSED, si < 0 ? 0 : P.n_surf);
        return false;
    }
    const DSurface& S = P.surf[si];
    const DSurfaceS& E = P.surf_s[si];
    const int flags = S.flags;
    ds p[3], dl[3];
    to_surface_ds(E, flags, W.X, W.D, p, dl);
    ds l, Nv[3], hit[3];
    const uint32_t why = intersect_ds(E, flags, p, dl, l, Nv, hit);
    if (why) { R.flags = lost(why, si); return false; }
    if (W.bounces > 0 && !(l.hi > 0.f)) { R.flags = lost(PHOSIM_LOST_MISSED, si); return false; }
    p[0] = hit[0]; p[1] = hit[1]; p[2] = hit[2];
    if (S.kind == PHOSIM_DETECTOR) {
        // the hit on the detector surface, its direction and the medium in front of it
        DetectorHit H;
        H.px = p[0]; H.py = p[1];
        H.dl[0] = dl[0]; H.dl[1] = dl[1]; H.dl[2] = dl[2];
        H.N[0] = Nv[0]; H.N[1] = Nv[1]; H.N[2] = Nv[2];
        H.n_cur = W.n_cur;
        H.si = si;
        if (hand_off) {
            *hand_off = H;
            R.flags = kHandedOff;
            return false;
        }
        detect_ds(P, H, lam, src, ray, R, mb);
        return false;
    }
    // clear aperture
    {   // decided in single precision unless the radius is within 1e-5 (relative) of a bound
        const float r2f = fmaf(p[0].hi, p[0].hi, p[1].hi * p[1].hi);
        const float ro = E.r_out2.hi, ri = E.r_in2.hi;
        if (fabsf(r2f - ro) > 1e-5f * ro && fabsf(r2f - ri) > 1e-5f * ri) {
            if (!(r2f <= ro && r2f >= ri)) { R.flags = lost(PHOSIM_LOST_VIGNETTED, si); return false; }
        } else {
            const ds r2 = dfma(p[0], p[0], p[1] * p[1]);
            if (!(ds_le(r2, E.r_out2) && ds_le(E.r_in2, r2))) { R.flags = lost(PHOSIM_LOST_VIGNETTED, si); return false; }
        }
    }
    // coating accept-reject at the incidence angle and wavelength
    if (S.coat_slot >= 0) {
        const DCoating& C = P.coat[S.coating];
        int it = 0;
        if (C.nt > 1) {
            const float cosi = fabsf(dl[0].hi * Nv[0].hi + dl[1].hi * Nv[1].hi + dl[2].hi * Nv[2].hi);
            const float th = acosf(fminf(1.f, cosi));
            it = (int)floorf((th - C.th0f) * C.inv_dthf);
            it = it < 0 ? 0 : (it > C.nt - 1 ? C.nt - 1 : it);
        }
        const size_t ix = (size_t)coat_lambda_bin(C, lam) * C.nt + it;
        const uint32_t w = W.bounces > 0 ? ghost_word_ds(P, src, ray, W.n_ghost++) : coat_word(P, src, ray, S.coat_slot);
        if (!((unsigned long long)w < __ldg(C.T_thr + ix))) {
            // reflected backwards (a ghost) with probability R, absorbed otherwise
            if ((P.flags & kGhostFlag) && S.kind != PHOSIM_MIRROR && C.TR_thr &&
                (unsigned long long)w < __ldg(C.TR_thr + ix)) {
                const ds dn2 = dot3(dl, Nv) * -2.f;
                {
                    const ds2 q = dfma2(dn2, ds2_of(Nv[0], Nv[1]), ds2_of(dl[0], dl[1]));
                    dl[0] = ds2_x(q);
                    dl[1] = ds2_y(q);
                }
                dl[2] = dfma(dn2, Nv[2], dl[2]);
                W.dir = -W.dir;
                if (++W.bounces > kMaxGhostBounces) { R.flags = lost(PHOSIM_LOST_MISSED, si); return false; }
                from_surface_ds(E, flags, p, dl, W.X, W.D);
                W.si = si + W.dir;
                return true;
            }
            R.flags = lost(PHOSIM_LOST_COATING, si);
            return false;
        }
    }
    if (S.kind == PHOSIM_MIRROR) {
        const ds dn2 = dot3(dl, Nv) * -2.f;
        {
            const ds2 q = dfma2(dn2, ds2_of(Nv[0], Nv[1]), ds2_of(dl[0], dl[1]));
            dl[0] = ds2_x(q);
            dl[1] = ds2_y(q);
        }
        dl[2] = dfma(dn2, Nv[2], dl[2]);
    } else {
        // the medium beyond the surface in the direction of travel (-1: vacuum)
        const int mi = W.dir < 0 ? S.mat_before : S.material;
        ds n_next = ds_f(1.f), inv_next = ds_f(1.f);
        if (mi >= 0) {
            const DMaterial& m = P.mat[mi];
            if (m.kind == PHOSIM_SELLMEIER) {
                if (W.glass_mat != mi) {
                    W.glass_n = sellmeier_ds(m, lam.hi);
                    W.glass_inv = ds_rcp(W.glass_n);
                    W.glass_mat = mi;
                }
                n_next = W.glass_n;
                inv_next = W.glass_inv;
            } else if (m.kind == PHOSIM_SILICON) {
                n_next = ds_f(silicon_index_f(lam.hi));
                inv_next = ds_rcp(n_next);
            }
        }
        if (!refract_ds(dl, Nv, W.n_cur * inv_next)) { R.flags = lost(PHOSIM_LOST_TIR, si); return false; }
        W.n_cur = n_next;
    }
    from_surface_ds(E, flags, p, dl, W.X, W.D);
    W.si = si + W.dir;
    return true;
}

// the whole walk of one ray
__device__ __forceinline__ void optics_ds(const TraceParams& P, const ds X[3], const ds D[3], ds lam, int src,
                                          uint64_t ray, PhotonOutS& R, const MemberDrawS* mb = nullptr,
                                          DetectorHit* hand_off = nullptr) {
    OpticsWalk W;
    walk_start(W, X, D);
#pragma unroll 1
    while (surface_step_ds(P, W, lam, src, ray, R, mb, hand_off)) {
    }
}

// Bilinear screen gradient (Sec. 2.3.2) at a double-single screen position; single-precision weights
__device__ __forceinline__ void screen_gradient_ds(const DScale& S, ds sx, ds sy, float& gx, float& gy) {
    const ds fx = sx * S.inv_pix_s, fy = sy * S.inv_pix_s;
    const float flx = ds_floor(fx), fly = ds_floor(fy);
    const int n = S.n;
    const int ix = (int)flx, iy = (int)fly;
    int i0, j0;
    if ((n & (n - 1)) == 0) {
        i0 = ix & (n - 1);
        j0 = iy & (n - 1);
    } else {
        i0 = ix % n; i0 += i0 < 0 ? n : 0;
        j0 = iy % n; j0 += j0 < 0 ? n : 0;
    }
    const size_t node = (size_t)j0 * n + i0;
    const float tx = ds_frac(fx, flx), ty = ds_frac(fy, fly);
    const float4 A = __ldg(S.g32 + 2 * node), B = __ldg(S.g32 + 2 * node + 1);
    const float w00 = (1.f - tx) * (1.f - ty), w10 = tx * (1.f - ty), w01 = (1.f - tx) * ty, w11 = tx * ty;
    gx += w00 * A.x + w10 * A.z + w01 * B.x + w11 * B.z;
    gy += w00 * A.y + w10 * A.w + w01 * B.y + w11 * B.w;
}

// Ray i from the top of the atmosphere to the entrance plane of the telescope (Sec. 2.2, 2.3): the sampling
// and layer steps of trace_photon<MIXED = true> (i is the photon, or for a bundle the ray).  False when the
// dynamic transmission test drops it (R.flags says where); otherwise X, D are its position and direction on
// the entrance plane.
__device__ __forceinline__ bool photon_entry_ds(const TraceParams& P, const SourceS& s, int src, uint64_t i,
                                                PhotonOutS& R, ds X[3], ds D[3], float& lam_out, float& lam_lo, uint4& w1,
                                                uint4& w2, uint4& w3, uint4& w4) {
    const uint32_t clo = (uint32_t)i, chi = (uint32_t)(i >> 32);
    const uint4 w0 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 0u), P.k0, P.k1);
    w1 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 1u), P.k0, P.k1);
    R.flags = 0; R.pix = -1;
    R.x = R.y = R.xc = R.yc = ds_f(0.f);
    // time stamp, wavelength (Sec. 2.2)
    const ds t = dfma(s.t_exp, ds_uniform(w1.x), s.t0);
    const ds lamd = sample_wavelength_ds(P, s, w0);
    const float lam = lamd.hi;
    lam_lo = lamd.lo;           // stored at once: the caller may keep it out of the registers of the layer loop
    R.lam = lam;
    // direction with the paraxial shape offset (Sec. 2.2, 2.2.1)
    ds nx = s.xi, ny = s.eta;
    if (s.kind == PHOSIM_SERSIC) {
        const float r = lerp_table_f(P.sersic32 + (size_t)s.table * P.sersic_K, P.sersic_K,
                                     u32of(w1.y) * (float)P.sersic_K - 0.5f);
        float sp, cp;
        sincospif(2.f * u32of(w1.z), &sp, &cp);
        const float dx = s.a * r * cp, dy = s.b * r * sp;
        nx = nx + (dx * s.cpa - dy * s.spa);
        ny = ny + (dx * s.spa + dy * s.cpa);
    } else if (s.kind == PHOSIM_GAUSS) {
        const float g = sqrtf(-2.f * logf(u32of(w1.y)));
        float sp, cp;
        sincospif(2.f * u32of(w1.z), &sp, &cp);
        nx = nx + s.a * g * cp;
        ny = ny + s.a * g * sp;
    }
    ds w = ds_f(1.f) - dfma(nx, nx, ny * ny);
    ds rinv = ds_rsqrt(w);
    w2 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 2u), P.k0, P.k1);
    w3 = make_uint4(0u, 0u, 0u, 0u);
    if (P.n_coated > 2) w3 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 3u), P.k0, P.k1);
    if (P.flags & PHOSIM_EARLY_REJECT) {
        const int si = early_coating_reject_f(P, lamd, w2, w3);
        if (si >= 0) { R.flags = lost(PHOSIM_LOST_COATING, si); return false; }
    }
    // pupil point on the annulus, on the nominal first surface, moved back to the top of the atmosphere
    const ds r = ds_sqrt(dfma(ds_uniform(w0.x), P.pr_dr2_s, P.pr_in2_s));
    ds sp, cp;
    ds_sincos_2pi(ds_uniform(w0.y), sp, cp);
    ds x = r * cp, y = r * sp;
    ds zs = ds_f(0.f), zx, zy;
    float gf, g1f;
    sag_ds(P.pupil_s, P.pupil_surf.flags, x, y, zs, zx, zy, gf, g1f);
    ds z = P.pupil_z_s + zs;
    {
        const ds l = (P.h_top_s - z) * rinv;
        x = x - nx * l;
        y = y - ny * l;
        z = P.h_top_s;
    }
    w4 = make_uint4(0u, 0u, 0u, 0u);
    if (P.hf_K > 0 || (P.flags & PHOSIM_BACK_REFLECT)) w4 = philox_ds(make_uint4(clo, chi, (uint32_t)src, 4u), P.k0, P.k1);
    // frozen-flow layers top to bottom (Sec. 2.3)
    if (P.flags & PHOSIM_ATMOSPHERE) {
        const float kick = P.kick0f * exp2f(-0.2f * log2f(lam * P.inv_lam_ref_f));
#pragma unroll 1
        for (int k = 0; k < P.n_layers; ++k) {
            const DLayer& L = P.layer[k];
            const ds ll = L.dzs * rinv;           // the drop from the plane above, z_above - z_k
            x = dfma(nx, ll, x);
            y = dfma(ny, ll, y);
            z = L.zs;
            const ds sx = x - L.vxs * t, sy = y - L.vys * t;
            float gx = 0.f, gy = 0.f;
#pragma unroll 1
            for (int q = 0; q < L.n_scales; ++q) screen_gradient_ds(L.s[q], sx, sy, gx, gy);
            nx = nx + kick * gx;
            ny = ny + kick * gy;
            w = ds_f(1.f) - dfma(nx, nx, ny * ny);
            rinv = ds_rsqrt(w);
        }
        // second kick (Sec. 2.3.2) from the long-exposure PSF of the screens above kappa_crit
        if (P.hf_K > 0) {
            const float ang = lerp_table_f(P.hf32, P.hf_K, u32of(w4.x) * (float)P.hf_K - 0.5f) * (kick / P.kick0f);
            float sa, ca;
            sincospif(2.f * u32of(w4.y), &sa, &ca);
            nx = nx + ang * ca;
            ny = ny + ang * sa;
            w = ds_f(1.f) - dfma(nx, nx, ny * ny);
            rinv = ds_rsqrt(w);
        }
    }
    const ds nz = -(w * rinv);
    {
        const ds l = (z - P.z_ent_s) * rinv;
        x = dfma(nx, l, x);
        y = dfma(ny, l, y);
        z = P.z_ent_s;
    }
    X[0] = x; X[1] = y; X[2] = z;
    D[0] = nx; D[1] = ny; D[2] = nz;
    lam_out = lam;
    return true;
}

// One photon from the top of the atmosphere to the pixel: the steps of trace_photon<MIXED = true>.
__device__ __forceinline__ void trace_photon_ds(const TraceParams& P, const SourceS& s, int src, uint64_t i,
                                                PhotonOutS& R) {
    ds X[3], D[3];
    float lam, lam_lo;
    uint4 w1, w2, w3, w4;
    const uint64_t ray = ray_of(s.bundle, i);
    if (!photon_entry_ds(P, s, src, ray, R, X, D, lam, lam_lo, w1, w2, w3, w4)) return;
    MemberDrawS mb;
    const bool bundled = s.bundle > 1;
    if (bundled) mb = member_draw_s(P, s.bsig, src, i);
    optics_ds(P, X, D, ds{lam, lam_lo}, src, ray, R, bundled ? &mb : nullptr);
}

}  // namespace phosim
