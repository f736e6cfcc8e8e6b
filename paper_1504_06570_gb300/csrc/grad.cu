// Adjoint raytrace: pathwise gradients of per-source PSF moments with respect to surface misalignments and
// Zernike figure coefficients (the optics of Peterson et al. 2015, Sec. 2.4.1-2.4.2, differentiated).
//
// Per photon the forward path is recomputed with the trace's own code (same random numbers, same accept
// decisions), keeping only the telescope-frame state entering each surface.  The reverse sweep then walks
// the surfaces backwards; at each one it recomputes that surface's local quantities from the kept state
// and applies the hand-derived vector-Jacobian products of: the frame transform, the implicit intersection
// (dl = -F_theta / F_l at the root), the normal from the sag slopes, and reflection or Snell refraction.
// Parameter adjoints accumulate per lane over a tile of one source and reduce once per warp.
#include "phosim_device.cuh"
#include "phosim_scene.hpp"
#include "photon.cuh"
#include "grad.hpp"

namespace phosim {

// sag, slopes and second derivatives (surface frame)
__device__ __forceinline__ bool sag_d2(const DSurface& S, const double* __restrict__ zmono_unused, double x, double y,
                                       double& z, double& zx, double& zy, double& zxx, double& zxy, double& zyy) {
    (void)zmono_unused;
    const double r2 = x * x + y * y;
    double g = 0.0, G2 = 0.0;          // (1/r) dz/dr and (1/r) dg/dr
    z = 0.0;
    if (S.flags & SF_CONIC) {
        const double A = 1.0 - S.k1c2 * r2;
        if (A < 0.0) return false;
        const double s = sqrt(A);
        z = S.c * r2 / (1.0 + s);
        g = S.c / s;
        G2 = S.c * S.k1c2 / (A * s);
    }
    if (S.flags & SF_EVEN) {
        const double pe = fma(r2, fma(r2, fma(r2, S.ae[3], S.ae[2]), S.ae[1]), S.ae[0]);
        z = fma(r2 * r2, pe, z);
        g = fma(r2, fma(r2, fma(r2, fma(r2, 10.0 * S.ae[3], 8.0 * S.ae[2]), 6.0 * S.ae[1]), 4.0 * S.ae[0]), 0.0) + g;
        G2 += 2.0 * fma(r2, fma(r2, fma(r2, 40.0 * S.ae[3], 24.0 * S.ae[2]), 12.0 * S.ae[1]), 4.0 * S.ae[0]);
    }
    if (S.flags & SF_ODD) {
        const double r = sqrt(r2);
        const double po = fma(r2, fma(r2, fma(r2, S.ao[3], S.ao[2]), S.ao[1]), S.ao[0]);
        z = fma(r2 * r, po, z);
        g = fma(r, fma(r2, fma(r2, fma(r2, 9.0 * S.ao[3], 7.0 * S.ao[2]), 5.0 * S.ao[1]), 3.0 * S.ao[0]), g);
        if (r > 0.0)
            G2 += fma(r2, fma(r2, fma(r2, 63.0 * S.ao[3], 35.0 * S.ao[2]), 15.0 * S.ao[1]), 3.0 * S.ao[0]) / r;
    }
    zx = x * g;
    zy = y * g;
    zxx = fma(x * x, G2, g);
    zxy = x * y * G2;
    zyy = fma(y * y, G2, g);
    if (S.flags & SF_ZERN) {
        const double u = x * S.zinv, v = y * S.zinv;
        double pu[7], pv[7];
        pu[0] = 1.0; pv[0] = 1.0;
#pragma unroll
        for (int k = 1; k < 7; ++k) { pu[k] = pu[k - 1] * u; pv[k] = pv[k - 1] * v; }
        double Z = 0, Zu = 0, Zv = 0, Zuu = 0, Zuv = 0, Zvv = 0;
        int off = 0;
#pragma unroll
        for (int b = 0; b <= 6; ++b) {
#pragma unroll
            for (int a = 0; a + b <= 6; ++a) {
                const double c = S.zp[off++];
                Z = fma(c, pu[a] * pv[b], Z);
                if (a >= 1) Zu = fma(c * a, pu[a - 1] * pv[b], Zu);
                if (b >= 1) Zv = fma(c * b, pu[a] * pv[b - 1], Zv);
                if (a >= 2) Zuu = fma(c * a * (a - 1), pu[a - 2] * pv[b], Zuu);
                if (a >= 1 && b >= 1) Zuv = fma(c * a * b, pu[a - 1] * pv[b - 1], Zuv);
                if (b >= 2) Zvv = fma(c * b * (b - 1), pu[a] * pv[b - 2], Zvv);
            }
        }
        const double k = S.zinv, k2 = S.zinv * S.zinv;
        z += Z; zx = fma(Zu, k, zx); zy = fma(Zv, k, zy);
        zxx = fma(Zuu, k2, zxx); zxy = fma(Zuv, k2, zxy); zyy = fma(Zvv, k2, zyy);
    }
    return true;
}

// one Zernike term (unit coefficient) and its slopes at the surface-frame point (x, y)
__device__ __forceinline__ void zern_term(const double* __restrict__ mono, double zinv, double x, double y, double& Z,
                                          double& Zx, double& Zy) {
    double zu, zv;
    zern_eval(mono, x * zinv, y * zinv, Z, zu, zv);
    Zx = zu * zinv;
    Zy = zv * zinv;
}

__device__ __forceinline__ double material_index(const TraceParams& P, int m, double lam) {
    if (m < 0) return 1.0;
    const DMaterial& M = P.mat[m];
    if (M.kind == PHOSIM_SELLMEIER) return sellmeier(M, lam);
    if (M.kind == PHOSIM_SILICON) return silicon_index(lam);
    return 1.0;
}

// Snell refraction forward (out) and its adjoint: given ob = d(L)/d(out), add to db and Nb.
__device__ __forceinline__ void refract_adjoint(const double d[3], const double Nin[3], double n1, double n2,
                                                const double ob[3], double db[3], double Nb[3]) {
    double s = 1.0;
    double cosi = -(d[0] * Nin[0] + d[1] * Nin[1] + d[2] * Nin[2]);
    if (cosi < 0.0) { s = -1.0; cosi = -cosi; }
    const double N[3] = {s * Nin[0], s * Nin[1], s * Nin[2]};
    const double mu = n1 / n2;
    const double k = 1.0 - mu * mu * (1.0 - cosi * cosi);
    const double sk = sqrt(k);
    const double a = mu * cosi - sk;
    // out = mu d + a N
    const double ab = N[0] * ob[0] + N[1] * ob[1] + N[2] * ob[2];
    const double cb = ab * (mu - mu * mu * cosi / sk);
    double NbU[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        db[i] += mu * ob[i] - cb * N[i];          // cosi = -d . N
        NbU[i] = a * ob[i] - cb * d[i];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) Nb[i] += s * NbU[i];
}

// Adjoint of one surface.  XD: telescope-frame state entering it.  For the detector, fb is the adjoint of
// the final (x, y) in its frame and L the conversion length (the diffusion offset does not depend on the
// optics); otherwise Xb / Db carry the adjoint of the state leaving the surface in and of the state
// entering it out.
__device__ void surface_adjoint(const TraceParams& P, const GradParams& G, int si, const double XD[6], double lam,
                                bool detector, const double fb[2], double L, double Xb[3], double Db[3],
                                double* __restrict__ gacc) {
    const DSurface& S = P.surf[si];
    const double X[3] = {XD[0], XD[1], XD[2]}, D[3] = {XD[3], XD[4], XD[5]};
    double p[3], dl[3];
    to_surface(S, X, D, p, dl);
    double l, Nfwd[3];
    intersect(S, p, dl, l, Nfwd);
    const double h[3] = {fma(l, dl[0], p[0]), fma(l, dl[1], p[1]), fma(l, dl[2], p[2])};
    double zs, sx, sy, sxx, sxy, syy;
    sag_d2(S, nullptr, h[0], h[1], zs, sx, sy, sxx, sxy, syy);
    const double zx = sx, zy = sy;            // the slopes that define the normal, at the root
    const double q = sqrt(1.0 + zx * zx + zy * zy);
    const double iq = 1.0 / q;
    const double N[3] = {-zx * iq, -zy * iq, iq};
    const double n1 = material_index(P, G.mat_before[si], lam);
    // forward outgoing direction in the surface frame
    double out[3] = {dl[0], dl[1], dl[2]};
    double hb[3] = {0.0, 0.0, 0.0}, ob[3] = {0.0, 0.0, 0.0}, Mb[9], obv[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int k = 0; k < 9; ++k) Mb[k] = 0.0;
    if (detector) {
        hb[0] = fb[0];
        hb[1] = fb[1];
        if (P.flags & PHOSIM_SENSOR) {
            const double n2 = silicon_index(lam);
            refract(out, N[0], N[1], N[2], n1 / n2);
            ob[0] = L * fb[0];
            ob[1] = L * fb[1];
        }
    } else {
        if (S.kind == PHOSIM_MIRROR) {
            const double dn = dl[0] * N[0] + dl[1] * N[1] + dl[2] * N[2];
            out[0] = fma(-2.0 * dn, N[0], dl[0]);
            out[1] = fma(-2.0 * dn, N[1], dl[1]);
            out[2] = fma(-2.0 * dn, N[2], dl[2]);
        } else {
            refract(out, N[0], N[1], N[2], n1 / material_index(P, S.material, lam));
        }
        // X' = M^T h + o, D' = M^T out: adjoints into h, out, M and o
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            hb[i] = S.M[3 * i] * Xb[0] + S.M[3 * i + 1] * Xb[1] + S.M[3 * i + 2] * Xb[2];
            ob[i] = S.M[3 * i] * Db[0] + S.M[3 * i + 1] * Db[1] + S.M[3 * i + 2] * Db[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) Mb[3 * i + k] += h[i] * Xb[k] + out[i] * Db[k];
            obv[i] += Xb[i];
        }
    }
    // reflection / refraction adjoint: into dl and N
    double dlb[3] = {0.0, 0.0, 0.0}, Nb[3] = {0.0, 0.0, 0.0};
    if (detector) {
        if (P.flags & PHOSIM_SENSOR) refract_adjoint(dl, N, n1, silicon_index(lam), ob, dlb, Nb);
    } else if (S.kind == PHOSIM_MIRROR) {
        const double dn = dl[0] * N[0] + dl[1] * N[1] + dl[2] * N[2];
        const double Nob = N[0] * ob[0] + N[1] * ob[1] + N[2] * ob[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            dlb[i] += ob[i] - 2.0 * N[i] * Nob;
            Nb[i] += -2.0 * (dn * ob[i] + dl[i] * Nob);
        }
    } else {
        refract_adjoint(dl, N, n1, material_index(P, S.material, lam), ob, dlb, Nb);
    }
    // normal N = (-zx, -zy, 1) / q: adjoint into the slopes
    const double nu_dot = -Nb[0] * zx - Nb[1] * zy + Nb[2];
    const double iq3 = iq * iq * iq;
    const double zxb = -Nb[0] * iq - nu_dot * zx * iq3;
    const double zyb = -Nb[1] * iq - nu_dot * zy * iq3;
    // slopes of the sag at the hit: into h (second derivatives) and the Zernike coefficients
    hb[0] += sxx * zxb + sxy * zyb;
    hb[1] += sxy * zxb + syy * zyb;
    // h = p + l dl
    const double lb = hb[0] * dl[0] + hb[1] * dl[1] + hb[2] * dl[2];
    double pb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        pb[i] = hb[i];
        dlb[i] += l * hb[i];
    }
    // implicit intersection: F(l; p, dl, c) = p_z + l dl_z - S(p_xy + l dl_xy; c) = 0
    const double Fl = dl[2] - sx * dl[0] - sy * dl[1];
    const double w = -lb / Fl;
    pb[0] += -w * sx; pb[1] += -w * sy; pb[2] += w;
    dlb[0] += -w * l * sx; dlb[1] += -w * l * sy; dlb[2] += w * l;
    // Zernike coefficients: dF/dc_j = -Z_j(h), d(slopes)/dc_j = grad Z_j(h)
    for (int k = 0; k < G.n_zp[si]; ++k) {
        double Z, Zx, Zy;
        zern_term(G.zmono + (size_t)(G.zp_j[si][k] - 1) * kZPoly, S.zinv, h[0], h[1], Z, Zx, Zy);
        gacc[G.zp_p[si][k]] += Zx * zxb + Zy * zyb - w * Z;
    }
    // p = M (X - o), dl = M D
    const double r[3] = {X[0] - S.o[0], X[1] - S.o[1], X[2] - S.o[2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Xb[k] = S.M[k] * pb[0] + S.M[3 + k] * pb[1] + S.M[6 + k] * pb[2];
        Db[k] = S.M[k] * dlb[0] + S.M[3 + k] * dlb[1] + S.M[6 + k] * dlb[2];
        obv[k] -= Xb[k];
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) Mb[3 * i + k] += pb[i] * r[k] + dlb[i] * D[k];
    // vertex o = (dx, dy, z + dz); rotation M(tx, ty, tz)
#pragma unroll
    for (int f = 0; f < 3; ++f)
        if (G.pert_p[si][f] >= 0) gacc[G.pert_p[si][f]] += obv[f];
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        if (G.pert_p[si][3 + f] < 0) continue;
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < 9; ++k) acc = fma(Mb[k], G.dM[si][f][k], acc);
        gacc[G.pert_p[si][3 + f]] += acc;
    }
}

__global__ void __launch_bounds__(128) grad_kernel(const __grid_constant__ TraceParams P,
                                                    const __grid_constant__ GradParams G) {
    // As in the trace kernel, photons the dynamic transmission test removes are dropped first and the
    // survivors are queued per warp, so the recomputed forward pass and the reverse sweep run on full warps.
    __shared__ uint32_t queue_mem[4][64];
    const int lane = threadIdx.x & 31;
    uint32_t* queue = queue_mem[threadIdx.x >> 5];
    const unsigned lanes_below = (1u << lane) - 1u;
    const bool early = (P.flags & PHOSIM_EARLY_REJECT) != 0;
    double gacc[kMaxGradParams];
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(P.tile_counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= P.n_tiles) break;
        const int src = tile_source(P, t, lane);
        const DSource& s = P.sources[src];
        const uint64_t off = (t - P.tile_prefix[src]) * P.tile_photons;
        const uint32_t count = (uint32_t)min((uint64_t)P.tile_photons, s.count - off);
        const double* sd = G.seeds + (size_t)src * 8;
        const double Ax = sd[0], Ay = sd[1], Bxx = sd[2], Bxy = sd[3], Byy = sd[4], xm = sd[5], ym = sd[6];
        for (int p = 0; p < G.n_params; ++p) gacc[p] = 0.0;
        int queued = 0;
        uint32_t base = 0;
        for (;;) {
            if (base < count) {
                const uint32_t k = base + lane;
                bool go_on = k < count;
                if (early && go_on) {
                    double lam;
                    go_on = early_reject_surface<false>(P, s, src, s.first + off + k, lam) < 0;
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
                if (v) {
                    ForwardRecord fr;
                    PhotonOut R;
                    trace_photon<false, true>(P, s, src, s.first + off + kk, R, &fr);
                    if (R.flags & PHOSIM_F_DETECTED) {
                        const double dx = R.x - xm, dy = R.y - ym;
                        const double fb[2] = {Ax + Bxx * dx + Bxy * dy, Ay + Byy * dy + Bxy * dx};
                        double Xb[3] = {0.0, 0.0, 0.0}, Db[3] = {0.0, 0.0, 0.0};
                        const int last = P.n_surf - 1;
                        surface_adjoint(P, G, last, fr.XD[last], R.lam, true, fb, fr.L, Xb, Db, gacc);
                        for (int si = last - 1; si >= 0; --si)
                            surface_adjoint(P, G, si, fr.XD[si], R.lam, false, fb, 0.0, Xb, Db, gacc);
                    }
                }
            }
            if (drained && queued == 0) break;
        }
        double* out = G.grad + (size_t)src * G.n_params;
        for (int p = 0; p < G.n_params; ++p) {
            double v = gacc[p];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v != 0.0) atomicAdd(out + p, v);
        }
    }
}

cudaError_t launch_grad(const TraceParams& P, const GradParams& G, int blocks, cudaStream_t st) {
    grad_kernel<<<blocks, 128, 0, st>>>(P, G);
    return cudaGetLastError();
}

cudaError_t grad_occupancy(int* blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, grad_kernel, 128, 0);
}

}  // namespace phosim
