/*
 * CPU oracle of the photon Monte Carlo path of Peterson et al. (2015), "Simulation of Astronomical Images
 * from Optical Survey Telescopes using a Comprehensive Photon Monte Carlo Approach".
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's CPU-baseline leg load this
 * library; the product path never does.  It shares no code with the CUDA library: its own Philox, its own
 * data layout, its own sag / intersection / refraction / sensor code, written from the paper's Sec. 2.
 *
 * Everything is plain FP64 (the paper fixes no precision), one photon at a time, in the paper's order:
 *   Sec. 2.2   sample the photon: direction, time, pupil point, wavelength (+ Sersic / Gaussian shapes)
 *   Sec. 2.3   propagate through plane-parallel layers, refractive kick from the phase-screen gradient
 *   Sec. 2.4.1 surfaces: conic + asphere sag, Zernike figure, 6-DOF misalignment, Sellmeier / Si index
 *   Sec. 2.4.2 intersection (parabolic first guess, then iterate), reflection / Snell refraction,
 *              coating accept-reject, silicon conversion length
 *   Sec. 2.5   lateral Gaussian diffusion and pixel quantisation
 * The gradient entry point re-runs the optics with a forward-mode dual number per parameter, the accept
 * decisions being those of the value part.
 *
 * Readings of the paper that this file takes (each is listed with its reason in the design notes):
 *  - back-propagation to the top of the atmosphere moves the photon against its direction of travel;
 *  - the intersection iteration is Newton's method on F(l) = z + n_z l - S(x + n_x l, y + n_y l) from the
 *    root of the paraboloid of the same vertex curvature, iterated to convergence;
 *  - screen coordinate = position - wind * t; deflection = (lambda_ref / 2 pi) grad(phi) (lambda/lambda_ref)^(-1/5)
 *    with grad(phi) the bilinear interpolation of central-difference gradients;
 *  - misalignment rotation R = Rz(tz) Ry(ty) Rx(tx) about the displaced vertex;
 *  - Zernike terms in Noll's order and normalisation over the radius zern_rnorm;
 *  - the fringing back-side reflection probability is the reflectance of one absorbing silicon layer
 *    (Airy sum of its two interfaces' amplitudes, s and p averaged) between the medium in front of the
 *    detector and vacuum behind it, at the photon's angle, wavelength and the local layer thickness.
 * Parity pins live in tests/test_oracle_*.py; "parity unpinned" is stated there for the parts without one.
 */
#include <algorithm>
#include <complex>
#include <type_traits>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// ------------------------------------------------------------------------------------------------------
// forward-mode dual number (value + one tangent) for the gradient oracle
// ------------------------------------------------------------------------------------------------------
struct Dual {
    double v, d;
    Dual(double a = 0.0, double b = 0.0) : v(a), d(b) {}
};
inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
inline Dual sqrt(Dual a) { double s = std::sqrt(a.v); return Dual(s, a.d / (2.0 * s)); }
inline Dual sin(Dual a) { return Dual(std::sin(a.v), std::cos(a.v) * a.d); }
inline Dual cos(Dual a) { return Dual(std::cos(a.v), -std::sin(a.v) * a.d); }
inline Dual atan2(Dual y, Dual x) {
    double r2 = x.v * x.v + y.v * y.v;
    return Dual(std::atan2(y.v, x.v), (x.v * y.d - y.v * x.d) / r2);
}
inline Dual log(Dual a) { return Dual(std::log(a.v), a.d / a.v); }
inline Dual exp(Dual a) { double e = std::exp(a.v); return Dual(e, e * a.d); }
// ------------------------------------------------------------------------------------------------------
// operation counter: a double that counts the arithmetic done on it (the algorithmic work of a photon)
// ------------------------------------------------------------------------------------------------------
struct OpCount { double add = 0, mul = 0, div = 0, sqrt = 0, special = 0; };
thread_local OpCount g_ops;
struct Cnt {
    double v;
    Cnt(double a = 0.0) : v(a) {}
};
inline Cnt operator+(Cnt a, Cnt b) { g_ops.add += 1; return Cnt(a.v + b.v); }
inline Cnt operator-(Cnt a, Cnt b) { g_ops.add += 1; return Cnt(a.v - b.v); }
inline Cnt operator-(Cnt a) { return Cnt(-a.v); }
inline Cnt operator*(Cnt a, Cnt b) { g_ops.mul += 1; return Cnt(a.v * b.v); }
inline Cnt operator/(Cnt a, Cnt b) { g_ops.div += 1; return Cnt(a.v / b.v); }
inline Cnt sqrt(Cnt a) { g_ops.sqrt += 1; return Cnt(std::sqrt(a.v)); }
inline Cnt sin(Cnt a) { g_ops.special += 1; return Cnt(std::sin(a.v)); }
inline Cnt cos(Cnt a) { g_ops.special += 1; return Cnt(std::cos(a.v)); }
inline Cnt atan2(Cnt y, Cnt x) { g_ops.special += 1; return Cnt(std::atan2(y.v, x.v)); }
inline Cnt log(Cnt a) { g_ops.special += 1; return Cnt(std::log(a.v)); }
inline Cnt exp(Cnt a) { g_ops.special += 1; return Cnt(std::exp(a.v)); }
inline Cnt pow(Cnt a, Cnt b) { g_ops.special += 1; return Cnt(std::pow(a.v, b.v)); }
inline double val(const Cnt& a) { return a.v; }
inline bool is_zero(const Cnt& a) { return a.v == 0.0; }

inline double val(double a) { return a; }
inline double val(const Dual& a) { return a.v; }
inline bool is_zero(double a) { return a == 0.0; }
inline bool is_zero(const Dual& a) { return a.v == 0.0 && a.d == 0.0; }
using std::sqrt; using std::sin; using std::cos; using std::atan2; using std::log; using std::exp; using std::pow;

// ------------------------------------------------------------------------------------------------------
// Philox4x32-10, from the published definition (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications with the round keys bumped by the Weyl constants between rounds.
// ------------------------------------------------------------------------------------------------------
void philox4x32_10(const uint32_t in[4], uint32_t k0, uint32_t k1, uint32_t out[4]) {
    uint32_t c[4] = {in[0], in[1], in[2], in[3]};
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Random-word slots of one photon: counter = (photon lo, photon hi, source id, block), key = seed.
enum Slot {
    S_PUPIL_R = 0, S_PUPIL_PHI = 1, S_LAM_BIN = 2, S_LAM_BLUR = 3,
    S_TIME = 4, S_SHAPE_A = 5, S_SHAPE_B = 6, S_CONV = 7,
    S_DIFF_A = 8, S_DIFF_B = 9, S_COAT0 = 10,   // coated surface k uses slot 10 + k (k < 6)
    S_HF_R = 16, S_HF_PSI = 17,                 // high-frequency kick: magnitude, direction
    S_BACK = 18,                                // back-side reflection
    N_SLOTS = 20
};

inline double uniform01(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }  // (w + 1/2) 2^-32

// ------------------------------------------------------------------------------------------------------
// scene
// ------------------------------------------------------------------------------------------------------
enum { K_MIRROR = 0, K_REFRACT = 1, K_DETECTOR = 2 };
enum { M_VACUUM = 0, M_SELLMEIER = 1, M_SILICON = 2 };
enum { SRC_POINT = 0, SRC_SERSIC = 1, SRC_GAUSS = 2 };

// record flags
enum : uint32_t {
    F_DETECTED = 1u,
    LOST_VIGNETTED = 1u, LOST_MISSED = 2u, LOST_NEWTON = 3u, LOST_TIR = 4u, LOST_COATING = 5u,
    LOST_OFF_CHIP = 6u, LOST_NOT_CONVERTED = 7u, LOST_DEAD_LAYER = 8u,
};
inline uint32_t lost_flag(uint32_t reason, int surface) { return (reason << 8) | ((uint32_t)(surface & 0xff) << 16); }

struct Surf {
    int kind, material, coating;
    double R, kappa, alpha[8];     // alpha_3 .. alpha_10
    double z, r_in, r_out;
    double pert[6];                // dx, dy, dz, tx, ty, tz
    double rnorm;
    std::vector<double> zern;      // Noll c_1 ..
};
struct Mat { int kind; double B[3], C[3]; };
struct Coat { double lam0, dlam, th0, dth; int nl, nt; std::vector<double> T, R; };   // R empty: no reflection
struct Scale { double pixel; int N; std::vector<double> phase; };
struct Layer { double z, vx, vy; std::vector<Scale> scales; };

struct Scene {
    uint64_t seed = 1;
    double pr_in = 0, pr_out = 0, h_top = 1e8, lam_ref = 500.0, z_ent = 0;
    int atm_on = 1, sensor_on = 1, back_reflect = 0;
    double dead_layer = 0.0;
    // fringing (Sec. 2.4.2): back-side reflection from the single-layer interference calculation, with the
    // layer's optical thickness t_si + t_gx (x - x0) + t_gy (y - y0) at the photon's position
    int fringe = 0;
    double t_gx = 0.0, t_gy = 0.0;
    std::vector<Surf> surf;
    std::vector<Mat> mat;
    std::vector<Coat> coat;
    // detector
    int nx = 0, ny = 0;
    double pixel = 0.01, x0 = 0, y0 = 0, t_si = 0.1;
    double ell_lam0 = 300, ell_dlam = 1;
    std::vector<double> ell, sig;
    std::vector<Layer> layers;
    // spectra and shapes
    double sed_lam0 = 300, sed_dlam = 1;
    int n_bins = 0;
    std::vector<std::vector<double>> cdf;      // per SED, cumulative photon probability at bin ends
    int sersic_K = 0;
    std::vector<std::vector<double>> sersic;
    std::vector<double> hf;      // quantiles of the high-frequency kick angle at lam_ref, u = (k + 1/2) / K
    // background bundles (Sec. 3.2): per source, photons per ray (<= 1: one photon per ray) and the sigma (mm)
    // of the Gaussian spread of a ray's photons on the detector surface
    std::vector<int> bundle_n;
    std::vector<double> bundle_sigma;
};

// A photon of a bundle: its own Gaussian offset on the detector surface and its own sensor draws, from
// blocks 5 and 6 of its counter (the ray's path uses the draws of the ray's counter).
struct Member {
    double sx, sy;
    uint32_t conv, diff_a, diff_b, back;
};

struct Source {
    int kind, sed, table;
    double xi, eta, redshift, t0, t_exp, a, b, pa;
};

struct Record {
    double x, y, xc, yc, lam;
    uint32_t flags;
    int32_t pix;
    double margin_mm, margin_nm;
};

// ------------------------------------------------------------------------------------------------------
// surface shape (Sec. 2.4.1): conic + asphere + Zernike figure, with first derivatives
// ------------------------------------------------------------------------------------------------------
double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

// Noll index j (1-based) -> (n, m) with m signed: m > 0 cosine term, m < 0 sine term
void noll_nm(int j, int& n, int& m) {
    n = 0;
    while ((n + 1) * (n + 2) / 2 < j) ++n;
    int first = n * (n + 1) / 2 + 1;                 // first Noll index of radial order n
    int k = j - first;                               // 0 .. n
    // |m| values present at order n, in increasing order, each twice except m = 0
    std::vector<int> ms;
    for (int a = n % 2; a <= n; a += 2) { if (a == 0) ms.push_back(0); else { ms.push_back(a); ms.push_back(a); } }
    int am = ms[k];
    if (am == 0) { m = 0; return; }
    m = (j % 2 == 0) ? am : -am;                    // even j: cos, odd j: sin (Noll 1976)
}

template <class T>
void zernike_term(int j, T rho, T theta, T& Z, T& dZdrho, T& dZdtheta) {
    int n, m;
    noll_nm(j, n, m);
    int am = m < 0 ? -m : m;
    T R = T(0.0), dR = T(0.0);
    for (int k = 0; k <= (n - am) / 2; ++k) {
        double c = ((k % 2) ? -1.0 : 1.0) * factorial(n - k) /
                   (factorial(k) * factorial((n + am) / 2 - k) * factorial((n - am) / 2 - k));
        int p = n - 2 * k;
        T rp = T(1.0);
        for (int q = 0; q < p; ++q) rp = rp * rho;
        R = R + T(c) * rp;
        if (p > 0) {
            T rq = T(1.0);
            for (int q = 0; q < p - 1; ++q) rq = rq * rho;
            dR = dR + T(c * p) * rq;
        }
    }
    if (m == 0) {
        double N = std::sqrt((double)(n + 1));
        Z = T(N) * R; dZdrho = T(N) * dR; dZdtheta = T(0.0);
    } else {
        double N = std::sqrt(2.0 * (n + 1));
        T a = T((double)am) * theta;
        if (m > 0) { Z = T(N) * R * cos(a); dZdrho = T(N) * dR * cos(a); dZdtheta = -T(N * am) * R * sin(a); }
        else       { Z = T(N) * R * sin(a); dZdrho = T(N) * dR * sin(a); dZdtheta = T(N * am) * R * cos(a); }
    }
}

// Surface in its own frame with differentiable figure / alignment parameters.
template <class T>
struct SurfT {
    const Surf* s;
    T pert[6];
    std::vector<T> zern;
    T M[3][3];        // global -> local rotation
    T o[3];           // displaced vertex, global frame
};

template <class T>
void rot_matrix(const T& tx, const T& ty, const T& tz, T Rg[3][3]) {
    // R = Rz(tz) Ry(ty) Rx(tx) maps local directions to global ones
    T cx = cos(tx), sx = sin(tx), cy = cos(ty), sy = sin(ty), cz = cos(tz), sz = sin(tz);
    T Rx[3][3] = {{T(1.0), T(0.0), T(0.0)}, {T(0.0), cx, -sx}, {T(0.0), sx, cx}};
    T Ry[3][3] = {{cy, T(0.0), sy}, {T(0.0), T(1.0), T(0.0)}, {-sy, T(0.0), cy}};
    T Rz[3][3] = {{cz, -sz, T(0.0)}, {sz, cz, T(0.0)}, {T(0.0), T(0.0), T(1.0)}};
    T A[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            A[i][j] = T(0.0);
            for (int k = 0; k < 3; ++k) A[i][j] = A[i][j] + Ry[i][k] * Rx[k][j];
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Rg[i][j] = T(0.0);
            for (int k = 0; k < 3; ++k) Rg[i][j] = Rg[i][j] + Rz[i][k] * A[k][j];
        }
}

template <class T>
void setup_surface(const Surf& s, SurfT<T>& st) {
    st.s = &s;
    T Rg[3][3];
    rot_matrix(st.pert[3], st.pert[4], st.pert[5], Rg);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) st.M[i][j] = Rg[j][i];     // inverse of a rotation = transpose
    st.o[0] = st.pert[0];
    st.o[1] = st.pert[1];
    st.o[2] = T(s.z) + st.pert[2];
}

// sag z(x, y) and its partial derivatives; false outside the conic's domain
template <class T>
bool surface_sag(const SurfT<T>& st, T x, T y, T& z, T& zx, T& zy) {
    const Surf& s = *st.s;
    T r2 = x * x + y * y;
    z = T(0.0); zx = T(0.0); zy = T(0.0);
    if (s.R != 0.0) {
        double c = 1.0 / s.R;
        T arg = T(1.0) - T((1.0 + s.kappa) * c * c) * r2;
        if (val(arg) < 0.0) return false;
        T sq = sqrt(arg);
        z = T(c) * r2 / (T(1.0) + sq);
        zx = T(c) * x / sq;
        zy = T(c) * y / sq;
    }
    bool any_alpha = false;
    for (int i = 0; i < 8; ++i) any_alpha = any_alpha || s.alpha[i] != 0.0;
    if (any_alpha) {
        T r = sqrt(r2);
        for (int i = 3; i <= 10; ++i) {
            double a = s.alpha[i - 3];
            if (a == 0.0) continue;
            T ri = T(1.0), rim2 = T(1.0);
            for (int q = 0; q < i; ++q) ri = ri * r;
            for (int q = 0; q < i - 2; ++q) rim2 = rim2 * r;
            z = z + T(a) * ri;
            zx = zx + T(a * i) * rim2 * x;
            zy = zy + T(a * i) * rim2 * y;
        }
    }
    if (!st.zern.empty() && s.rnorm > 0.0) {
        T xr = x, yr = y;
        if (val(r2) == 0.0) xr = T(1e-150);     // its square stays a normal number
        T rr = sqrt(xr * xr + yr * yr);
        T rho = rr / T(s.rnorm);
        T th = atan2(yr, xr);
        T cth = xr / rr, sth = yr / rr;
        for (size_t j = 0; j < st.zern.size(); ++j) {
            if (is_zero(st.zern[j])) continue;
            T Z, dZr, dZt;
            zernike_term((int)j + 1, rho, th, Z, dZr, dZt);
            // d/dx = cos(th) d/dr - sin(th)/r d/dth, with d/dr = (1/rnorm) d/drho
            T dzdr = dZr / T(s.rnorm);
            z = z + st.zern[j] * Z;
            zx = zx + st.zern[j] * (cth * dzdr - sth * dZt / rr);
            zy = zy + st.zern[j] * (sth * dzdr + cth * dZt / rr);
        }
    }
    return true;
}

// ------------------------------------------------------------------------------------------------------
// ray-surface intersection (Sec. 2.4.2)
// ------------------------------------------------------------------------------------------------------
// Returns 0 on success with l the distance along d; LOST_MISSED or LOST_NEWTON otherwise.
template <class T>
uint32_t intersect(const SurfT<T>& st, const T p[3], const T d[3], T& l) {
    const Surf& s = *st.s;
    // first guess: the paraboloid of the same vertex curvature, solved exactly (nearest-vertex root)
    double c = (s.R != 0.0) ? 1.0 / s.R : 0.0;
    T qa = T(0.5 * c) * (d[0] * d[0] + d[1] * d[1]);
    T qb = T(c) * (p[0] * d[0] + p[1] * d[1]) - d[2];
    T qc = T(0.5 * c) * (p[0] * p[0] + p[1] * p[1]) - p[2];
    if (val(qa) == 0.0) {
        if (val(qb) == 0.0) return LOST_MISSED;
        l = -qc / qb;
    } else {
        T disc = qb * qb - T(4.0) * qa * qc;
        if (val(disc) < 0.0) {
            if (val(qb) == 0.0) return LOST_MISSED;
            l = -qc / qb;
        } else {
            T sq = sqrt(disc);
            T q = (val(qb) >= 0.0) ? T(-0.5) * (qb + sq) : T(-0.5) * (qb - sq);
            if (val(q) == 0.0) return LOST_MISSED;
            l = qc / q;
        }
    }
    // Newton's method on F(l) = p_z + l d_z - S(p_x + l d_x, p_y + l d_y); one extra step after
    // convergence makes the dual part the implicit-function derivative
    int converged_at = -1;
    for (int it = 0; it < 100; ++it) {
        T x = p[0] + l * d[0], y = p[1] + l * d[1];
        T zs, zx, zy;
        if (!surface_sag(st, x, y, zs, zx, zy)) return LOST_MISSED;
        T F = p[2] + l * d[2] - zs;
        T dF = d[2] - zx * d[0] - zy * d[1];
        if (val(dF) == 0.0) return LOST_NEWTON;
        T step = F / dF;
        l = l - step;
        if (converged_at >= 0) break;
        if (std::is_same<T, Cnt>::value) {
            if (std::fabs(val(step)) < 1e-5) { converged_at = it; break; }
        } else if (std::fabs(val(step)) < 1e-12 * (1.0 + std::fabs(val(l)))) {
            converged_at = it;
        }
    }
    if (converged_at < 0) return LOST_NEWTON;
    T x = p[0] + l * d[0], y = p[1] + l * d[1], zs, zx, zy;
    if (!surface_sag(st, x, y, zs, zx, zy)) return LOST_MISSED;
    if (std::fabs(val(p[2] + l * d[2] - zs)) > 1e-9) return LOST_NEWTON;
    return 0;
}

// ------------------------------------------------------------------------------------------------------
// media (Sec. 2.4.1)
// ------------------------------------------------------------------------------------------------------
template <class T>
T refractive_index_t(const Scene& sc, int material, T lam_nm) {
    const Mat& m = sc.mat[material];
    if (m.kind == M_VACUUM) return T(1.0);
    if (m.kind == M_SELLMEIER) {
        T lu = lam_nm * T(1e-3);
        T l2 = lu * lu;
        T n2 = T(1.0);
        for (int i = 0; i < 3; ++i) n2 = n2 + T(m.B[i]) * l2 / (l2 - T(m.C[i]));
        return sqrt(n2);
    }
    // silicon, E in eV
    T E = T(1239.841984) / lam_nm;
    return T(3.36) + T(0.211) * E + T(2.79) * exp((E - T(3.30)) / T(0.398));
}
double refractive_index(const Scene& sc, int material, double lam_nm) { return refractive_index_t<double>(sc, material, lam_nm); }

// reflection of d across the unit normal N
template <class T>
void reflect(T d[3], const T N[3]) {
    T dn = d[0] * N[0] + d[1] * N[1] + d[2] * N[2];
    for (int i = 0; i < 3; ++i) d[i] = d[i] - T(2.0) * dn * N[i];
}

// Snell's law in vector form from index n1 to n2; false on total internal reflection
template <class T>
bool refract(T d[3], const T Nin[3], T n1, T n2) {
    T N[3] = {Nin[0], Nin[1], Nin[2]};
    T cosi = -(d[0] * N[0] + d[1] * N[1] + d[2] * N[2]);
    if (val(cosi) < 0.0) { for (int i = 0; i < 3; ++i) N[i] = -N[i]; cosi = -cosi; }
    T mu = n1 / n2;
    T k = T(1.0) - mu * mu * (T(1.0) - cosi * cosi);
    if (val(k) < 0.0) return false;
    T a = mu * cosi - sqrt(k);
    for (int i = 0; i < 3; ++i) d[i] = mu * d[i] + a * N[i];
    return true;
}

// ------------------------------------------------------------------------------------------------------
// photon
// ------------------------------------------------------------------------------------------------------
struct Draws {
    uint32_t w[N_SLOTS];
    const Scene* sc;
    int src;
    uint64_t i;
};

Draws draw_photon(const Scene& sc, int src_id, uint64_t i) {
    Draws D;
    D.sc = &sc; D.src = src_id; D.i = i;
    for (uint32_t blk = 0; blk < 5; ++blk) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), (uint32_t)src_id, blk};
        philox4x32_10(ctr, (uint32_t)sc.seed, (uint32_t)(sc.seed >> 32), &D.w[4 * blk]);
    }
    return D;
}

// Photon i of a bundle of n photons per ray (Sec. 3.2): the ray is i / n; the photon's offset on the
// detector surface is a Gaussian of the given sigma drawn from block 5 of its own counter (Box-Muller), its
// sensor draws are the rest of blocks 5 and 6.
Member member_draws(const Scene& sc, int src_id, uint64_t i, double sigma) {
    uint32_t w[8];
    for (uint32_t blk = 5; blk < 7; ++blk) {
        uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), (uint32_t)src_id, blk};
        philox4x32_10(ctr, (uint32_t)sc.seed, (uint32_t)(sc.seed >> 32), &w[4 * (blk - 5)]);
    }
    Member m;
    const double g = std::sqrt(-2.0 * std::log(uniform01(w[0])));
    const double ph = 2.0 * M_PI * uniform01(w[1]);
    m.sx = sigma * g * std::cos(ph);
    m.sy = sigma * g * std::sin(ph);
    m.conv = w[2]; m.diff_a = w[3]; m.diff_b = w[4]; m.back = w[5];
    return m;
}

inline int bundle_of(const Scene& sc, int s) {
    return (s < (int)sc.bundle_n.size() && sc.bundle_n[s] > 1) ? sc.bundle_n[s] : 1;
}

// Ghosts (Sec. 2.4.2): after a photon's first reflection by a coating, each coated-surface decision takes the
// next word of blocks 7, 8, ... of its counter (word n of block 7 + n / 4).
uint32_t ghost_word(const Draws& D, int n) {
    uint32_t ctr[4] = {(uint32_t)D.i, (uint32_t)(D.i >> 32), (uint32_t)D.src, (uint32_t)(7 + n / 4)}, w[4];
    philox4x32_10(ctr, (uint32_t)D.sc->seed, (uint32_t)(D.sc->seed >> 32), w);
    return w[n % 4];
}
constexpr int kMaxGhostBounces = 8;

inline void min_margin(double& m, double v) { v = std::fabs(v); if (v < m) m = v; }

struct Pre {     // photon state entering the optics (after the atmosphere)
    double x[3], d[3], lam, t;
};

// central-difference phase gradient at a screen node: a table entry the paper precomputes (Sec. 3.2),
// so the operation counter does not see it
inline void node_gradient(const Scale& S, long long i, long long j, double& gx, double& gy) {
    const int N = S.N;
    auto wrap = [N](long long v) { long long m = v % N; return (int)(m < 0 ? m + N : m); };
    auto ph = [&](long long a, long long b) { return S.phase[(size_t)wrap(b) * N + wrap(a)]; };
    gx = (ph(i + 1, j) - ph(i - 1, j)) / (2.0 * S.pixel);
    gy = (ph(i, j + 1) - ph(i, j - 1)) / (2.0 * S.pixel);
}

// Sec. 2.2 + 2.3: everything before the first optical surface.  T = double, or the operation counter.
template <class T>
void sample_and_atmosphere_t(const Scene& sc, const Source& s, const Draws& D, T X[3], T Dir[3], T& lam, T& tt) {
    // time stamp (Sec. 2.2)
    tt = T(s.t0) + T(s.t_exp) * T(uniform01(D.w[S_TIME]));
    // wavelength: photon-number CDF, first bin with u < cdf, blurred uniformly within the bin, redshifted
    const std::vector<double>& cdf = sc.cdf[s.sed];
    double ub = uniform01(D.w[S_LAM_BIN]);
    int bin = 0;
    while (bin < sc.n_bins - 1 && !(ub < cdf[bin])) ++bin;
    lam = (T(sc.sed_lam0 + bin * sc.sed_dlam) + T(uniform01(D.w[S_LAM_BLUR])) * T(sc.sed_dlam)) * T(1.0 + s.redshift);
    // direction: tangent-plane components, perturbed paraxially by the source shape, renormalised
    T nx = T(s.xi), ny = T(s.eta);
    if (s.kind == SRC_SERSIC) {
        const std::vector<double>& tab = sc.sersic[s.table];
        int K = sc.sersic_K;
        T f = T(uniform01(D.w[S_SHAPE_A])) * T((double)K) - T(0.5);
        int k = (int)std::floor(val(f));
        if (k < 0) k = 0;
        if (k > K - 2) k = K - 2;
        T t = f - T((double)k);
        if (val(t) < 0.0) t = T(0.0);
        if (val(t) > 1.0) t = T(1.0);
        T r = T(tab[k]) * (T(1.0) - t) + T(tab[k + 1]) * t;
        T psi = T(2.0 * M_PI) * T(uniform01(D.w[S_SHAPE_B]));
        T dx = T(s.a) * r * cos(psi), dy = T(s.b) * r * sin(psi);
        T cpa = T(std::cos(s.pa)), spa = T(std::sin(s.pa));      // per source, not per photon
        nx = nx + (dx * cpa - dy * spa);
        ny = ny + (dx * spa + dy * cpa);
    } else if (s.kind == SRC_GAUSS) {
        T g = sqrt(T(-2.0) * log(T(uniform01(D.w[S_SHAPE_A]))));
        T ph = T(2.0 * M_PI) * T(uniform01(D.w[S_SHAPE_B]));
        nx = nx + T(s.a) * g * cos(ph);
        ny = ny + T(s.a) * g * sin(ph);
    }
    T nz = -sqrt(T(1.0) - nx * nx - ny * ny);
    // pupil point on the annulus, z from the (nominal) first surface, then back to the top of the atmosphere
    T u = T(uniform01(D.w[S_PUPIL_R]));
    T r = sqrt(u * T(sc.pr_out * sc.pr_out - sc.pr_in * sc.pr_in) + T(sc.pr_in * sc.pr_in));
    T phi = T(2.0 * M_PI) * T(uniform01(D.w[S_PUPIL_PHI]));
    T x = r * cos(phi), y = r * sin(phi);
    SurfT<T> m1;
    for (int q = 0; q < 6; ++q) m1.pert[q] = T(0.0);
    setup_surface(sc.surf[0], m1);
    T zs = T(0.0), zx, zy;
    surface_sag(m1, x, y, zs, zx, zy);
    T z = T(sc.surf[0].z) + zs;
    T l = (T(sc.h_top) - z) / (-nz);
    x = x - nx * l; y = y - ny * l; z = T(sc.h_top);
    // plane-parallel layers, top to bottom (Sec. 2.3.1, 2.3.2)
    if (sc.atm_on) {
        T kick = T(sc.lam_ref * 1e-6 / (2.0 * M_PI)) * pow(lam / T(sc.lam_ref), T(-0.2));
        for (const Layer& L : sc.layers) {
            T ll = (z - T(L.z)) / (-nz);
            x = x + nx * ll; y = y + ny * ll; z = T(L.z);
            T sx = x - T(L.vx) * tt, sy = y - T(L.vy) * tt;
            T gx = T(0.0), gy = T(0.0);
            for (const Scale& S : L.scales) {
                T fx = sx / T(S.pixel), fy = sy / T(S.pixel);
                double ix = std::floor(val(fx)), iy = std::floor(val(fy));
                T tx = fx - T(ix), ty = fy - T(iy);
                T w[2][2] = {{(T(1.0) - tx) * (T(1.0) - ty), tx * (T(1.0) - ty)}, {(T(1.0) - tx) * ty, tx * ty}};
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        double gxt, gyt;
                        node_gradient(S, (long long)ix + a, (long long)iy + b, gxt, gyt);
                        gx = gx + w[b][a] * T(gxt);
                        gy = gy + w[b][a] * T(gyt);
                    }
            }
            nx = nx + kick * gx;
            ny = ny + kick * gy;
            nz = -sqrt(T(1.0) - nx * nx - ny * ny);
        }
        // second kick (Sec. 2.3.2): a draw from the long-exposure PSF of the screens above kappa_crit,
        // scaled like the refractive kick by (lambda / lambda_ref)^(-1/5)
        if (!sc.hf.empty()) {
            const int K = (int)sc.hf.size();
            T f = T(uniform01(D.w[S_HF_R])) * T((double)K) - T(0.5);
            int k = (int)std::floor(val(f));
            if (k < 0) k = 0;
            if (k > K - 2) k = K - 2;
            T t = f - T((double)k);
            if (val(t) < 0.0) t = T(0.0);
            if (val(t) > 1.0) t = T(1.0);
            T ang = (T(sc.hf[k]) * (T(1.0) - t) + T(sc.hf[k + 1]) * t) * (kick / T(sc.lam_ref * 1e-6 / (2.0 * M_PI)));
            T psi = T(2.0 * M_PI) * T(uniform01(D.w[S_HF_PSI]));
            nx = nx + ang * cos(psi);
            ny = ny + ang * sin(psi);
            nz = -sqrt(T(1.0) - nx * nx - ny * ny);
        }
    }
    // straight on to the entrance plane of the telescope, where the raytrace starts
    T le = (z - T(sc.z_ent)) / (-nz);
    x = x + nx * le; y = y + ny * le; z = T(sc.z_ent);
    X[0] = x; X[1] = y; X[2] = z;
    Dir[0] = nx; Dir[1] = ny; Dir[2] = nz;
}

void sample_and_atmosphere(const Scene& sc, const Source& s, const Draws& D, Pre& P) {
    sample_and_atmosphere_t<double>(sc, s, D, P.x, P.d, P.lam, P.t);
}

// Sec. 2.4.2 fringing: the probability that a photon reaching the back of the silicon is reflected, from the
// electromagnetic calculation for a single layer.  The layer is silicon of complex index n1 + i k1 and
// thickness t (mm); in front of it a medium of real index n0, behind it vacuum.  s = n sin(theta) is the
// photon's invariant (the same in every medium).  In each medium q = N cos(theta) = sqrt(N^2 - s^2); the
// amplitude reflection coefficients of an interface from medium a to medium b are
//   s polarisation: (q_a - q_b) / (q_a + q_b),   p polarisation: (N_b^2 q_a - N_a^2 q_b) / (N_b^2 q_a + N_a^2 q_b);
// the layer's amplitude is the sum of the multiple reflections inside it (Airy),
//   r = (r01 + r12 e) / (1 + r01 r12 e),  e = exp(2 i beta),  beta = (2 pi / lambda) t q1,
// and the probability is |r|^2 averaged over the two polarisations (unpolarised light).
double film_reflectance(double lam_nm, double n0, double n1, double k1, double t_mm, double s) {
    typedef std::complex<double> C;
    const C N0(n0, 0.0), N1(n1, k1), N2(1.0, 0.0), s2(s * s, 0.0);
    const C q0 = std::sqrt(N0 * N0 - s2), q1 = std::sqrt(N1 * N1 - s2), q2 = std::sqrt(N2 * N2 - s2);
    const C rs01 = (q0 - q1) / (q0 + q1), rs12 = (q1 - q2) / (q1 + q2);
    const C rp01 = (N1 * N1 * q0 - N0 * N0 * q1) / (N1 * N1 * q0 + N0 * N0 * q1);
    const C rp12 = (N2 * N2 * q1 - N1 * N1 * q2) / (N2 * N2 * q1 + N1 * N1 * q2);
    const double lam_mm = lam_nm * 1e-6;
    const C e = std::exp(C(0.0, 2.0) * C(2.0 * M_PI / lam_mm * t_mm, 0.0) * q1);
    const C rs = (rs01 + rs12 * e) / (C(1.0, 0.0) + rs01 * rs12 * e);
    const C rp = (rp01 + rp12 * e) / (C(1.0, 0.0) + rp01 * rp12 * e);
    return 0.5 * (std::norm(rs) + std::norm(rp));
}

template <class T>
struct OpticsOut {
    T x, y;          // final position (detector frame)
    double xc, yc;   // at conversion (value)
    uint32_t flags;
    int32_t pix;
    double margin_mm, margin_nm;
};

// Sec. 2.4.2 + 2.5: surfaces in order, then the silicon sensor and the pixel
template <class T>
void optics_and_sensor(const Scene& sc, const std::vector<SurfT<T>>& ST, const Pre& P, const Draws* D,
                       OpticsOut<T>& out, const Member* M = nullptr) {
    T x[3] = {T(P.x[0]), T(P.x[1]), T(P.x[2])};
    T d[3] = {T(P.d[0]), T(P.d[1]), T(P.d[2])};
    const double lam = P.lam;
    const T lamT = T(P.lam);
    T n_cur = T(1.0);
    int coat_k = 0;
    out.flags = 0; out.pix = -1; out.margin_mm = 1e300; out.margin_nm = 1e300;
    out.x = T(0.0); out.y = T(0.0); out.xc = out.yc = 0.0;
    // Surfaces are met in order (dir = +1); a photon reflected by a refracting surface's coating (a ghost)
    // travels back through them (dir = -1) until another reflection turns it round again.
    int si = 0, dir = 1, bounces = 0, n_ghost = 0;
    const int n_surf = (int)ST.size();
    for (;;) {
        if (si < 0 || si >= n_surf) { out.flags = lost_flag(LOST_MISSED, si < 0 ? 0 : n_surf); return; }
        const SurfT<T>& st = ST[si];
        const Surf& s = *st.s;
        // into the frame of the optic
        T p[3], dl[3];
        for (int i = 0; i < 3; ++i) {
            p[i] = st.M[i][0] * (x[0] - st.o[0]) + st.M[i][1] * (x[1] - st.o[1]) + st.M[i][2] * (x[2] - st.o[2]);
            dl[i] = st.M[i][0] * d[0] + st.M[i][1] * d[1] + st.M[i][2] * d[2];
        }
        T l;
        uint32_t why = intersect(st, p, dl, l);
        if (why) { out.flags = lost_flag(why, (int)si); return; }
        // a ghost only meets surfaces ahead of it
        if (bounces > 0 && !(val(l) > 0.0)) { out.flags = lost_flag(LOST_MISSED, (int)si); return; }
        for (int i = 0; i < 3; ++i) p[i] = p[i] + l * dl[i];
        T zs, zx, zy;
        surface_sag(st, p[0], p[1], zs, zx, zy);
        T nn = sqrt(T(1.0) + zx * zx + zy * zy);
        T N[3] = {-zx / nn, -zy / nn, T(1.0) / nn};
        if (s.kind == K_DETECTOR) {
            if (M) {   // a bundle's photon: its Gaussian offset from the ray's hit on the detector surface
                p[0] = p[0] + T(M->sx);
                p[1] = p[1] + T(M->sy);
            }
            // the sensor's draws (none for the deterministic rays of the surface-only traces, D = null)
            const uint32_t w_conv = M ? M->conv : (D ? D->w[S_CONV] : 0u);
            const uint32_t w_back = M ? M->back : (D ? D->w[S_BACK] : 0u);
            const uint32_t w_diff_a = M ? M->diff_a : (D ? D->w[S_DIFF_A] : 0u);
            const uint32_t w_diff_b = M ? M->diff_b : (D ? D->w[S_DIFF_B] : 0u);
            double hx = val(p[0]) - (sc.x0 - 0.5 * sc.nx * sc.pixel);
            double hy = val(p[1]) - (sc.y0 - 0.5 * sc.ny * sc.pixel);
            min_margin(out.margin_mm, hx); min_margin(out.margin_mm, hx - sc.nx * sc.pixel);
            min_margin(out.margin_mm, hy); min_margin(out.margin_mm, hy - sc.ny * sc.pixel);
            if (!(hx >= 0.0 && hy >= 0.0 && hx < sc.nx * sc.pixel && hy < sc.ny * sc.pixel)) {
                out.flags = lost_flag(LOST_OFF_CHIP, (int)si); return;
            }
            T fx = p[0], fy = p[1];
            double xc = val(p[0]), yc = val(p[1]);
            if (sc.sensor_on) {
                // refraction into silicon, exponential conversion length, lateral diffusion (Sec. 2.4.2, 2.5)
                T n_si = refractive_index_t<T>(sc, s.material, lamT);
                if (!refract(dl, N, n_cur, n_si)) { out.flags = lost_flag(LOST_TIR, (int)si); return; }
                T fl = (lamT - T(sc.ell_lam0)) / T(sc.ell_dlam);
                int ne = (int)sc.ell.size();
                int k = (int)std::floor(val(fl));
                if (k < 0) k = 0;
                if (k > ne - 2) k = ne - 2;
                T t = fl - T((double)k);
                if (val(t) < 0.0) t = T(0.0);
                if (val(t) > 1.0) t = T(1.0);
                T ell = T(sc.ell[k]) * (T(1.0) - t) + T(sc.ell[k + 1]) * t;
                T Lt = ell * (-log(T(uniform01(w_conv))));
                T dz = dl[2];
                T deptht = Lt * (val(dz) < 0.0 ? -dz : dz);
                double depth = val(deptht), L = val(Lt);
                min_margin(out.margin_mm, depth - sc.t_si);
                if (!(depth <= sc.t_si)) {
                    // back-side reflection (Sec. 2.4.2) with the normal-incidence Fresnel probability of the
                    // Si/vacuum interface, or with fringing the single-layer interference calculation; the
                    // photon converts on its way back towards the entrance
                    bool back = false;
                    if (sc.back_reflect) {
                        double r_back;
                        if (sc.fringe) {
                            // the single-layer calculation at the photon's angle in the silicon, its
                            // wavelength and the layer's thickness where it entered the chip
                            const double ns = val(n_si), c1 = std::fabs(val(dz));
                            const double sinv = ns * std::sqrt(std::max(0.0, 1.0 - c1 * c1));
                            const double k1 = lam * 1e-6 / (4.0 * M_PI * val(ell));
                            const double thick = sc.t_si + sc.t_gx * (xc - sc.x0) + sc.t_gy * (yc - sc.y0);
                            r_back = film_reflectance(lam, val(n_cur), ns, k1, thick, sinv);
                        } else {
                            T rf = (n_si - T(1.0)) / (n_si + T(1.0));
                            r_back = val(rf * rf);
                        }
                        double u = uniform01(w_back);
                        if (std::fabs(u - r_back) < 1e-12) out.margin_mm = 0.0;
                        if (u < r_back) {
                            deptht = T(2.0 * sc.t_si) - deptht;
                            depth = val(deptht);
                            back = depth >= 0.0;
                            min_margin(out.margin_mm, depth);
                        }
                    }
                    if (!back) { out.flags = lost_flag(LOST_NOT_CONVERTED, (int)si); return; }
                }
                // charge converted in the field-free dead layer at the entrance is not collected
                if (sc.dead_layer > 0.0) min_margin(out.margin_mm, depth - sc.dead_layer);
                if (depth < sc.dead_layer) { out.flags = lost_flag(LOST_DEAD_LAYER, (int)si); return; }
                fx = fx + T(L) * dl[0];
                fy = fy + T(L) * dl[1];
                xc = val(fx); yc = val(fy);
                int ns = (int)sc.sig.size();
                T fs = deptht / T(sc.t_si) * T((double)(ns - 1));
                int ks = std::min(ns - 2, std::max(0, (int)std::floor(val(fs))));
                T ts = fs - T((double)ks);
                if (val(ts) < 0.0) ts = T(0.0);
                if (val(ts) > 1.0) ts = T(1.0);
                T sigma = T(sc.sig[ks]) * (T(1.0) - ts) + T(sc.sig[ks + 1]) * ts;
                T g = sqrt(T(-2.0) * log(T(uniform01(w_diff_a))));
                T ph = T(2.0 * M_PI) * T(uniform01(w_diff_b));
                fx = fx + T(val(sigma * g * cos(ph)));
                fy = fy + T(val(sigma * g * sin(ph)));
            }
            double ux = val(fx) - (sc.x0 - 0.5 * sc.nx * sc.pixel);
            double uy = val(fy) - (sc.y0 - 0.5 * sc.ny * sc.pixel);
            double px = std::floor(ux / sc.pixel), py = std::floor(uy / sc.pixel);
            min_margin(out.margin_mm, ux - px * sc.pixel); min_margin(out.margin_mm, ux - (px + 1) * sc.pixel);
            min_margin(out.margin_mm, uy - py * sc.pixel); min_margin(out.margin_mm, uy - (py + 1) * sc.pixel);
            out.x = fx; out.y = fy; out.xc = xc; out.yc = yc;
            if (!(px >= 0 && py >= 0 && px < sc.nx && py < sc.ny)) { out.flags = lost_flag(LOST_OFF_CHIP, (int)si); return; }
            out.pix = ((double)sc.nx * sc.ny < 2.0e9) ? (int32_t)(py * sc.nx + px) : -1;
            out.flags = F_DETECTED;
            return;
        }
        // clear aperture (vignetting)
        double r = std::sqrt(val(p[0]) * val(p[0]) + val(p[1]) * val(p[1]));
        min_margin(out.margin_mm, r - s.r_out);
        if (s.r_in > 0.0) min_margin(out.margin_mm, r - s.r_in);
        if (!(r <= s.r_out && r >= s.r_in)) { out.flags = lost_flag(LOST_VIGNETTED, (int)si); return; }
        // coating accept-reject at the incidence angle and wavelength
        if (s.coating >= 0) {
            const Coat& C = sc.coat[s.coating];
            double cosi = std::fabs(val(dl[0] * N[0] + dl[1] * N[1] + dl[2] * N[2]));
            double th = std::acos(std::min(1.0, cosi));
            double fl = (lam - C.lam0) / C.dlam, ft = (th - C.th0) / C.dth;
            min_margin(out.margin_nm, (fl - std::round(fl)) * C.dlam);
            int il = std::min(C.nl - 1, std::max(0, (int)std::floor(fl)));
            int it = std::min(C.nt - 1, std::max(0, (int)std::floor(ft)));
            const size_t ix = (size_t)il * C.nt + it;
            const double Tr = C.T[ix], Rr = C.R.empty() ? 0.0 : C.R[ix];
            // the first pass takes the coated surface's own slot; after a ghost reflection, the ghost words
            double u = 0.0;
            if (D) u = uniform01(bounces == 0 ? D->w[S_COAT0 + coat_k] : ghost_word(*D, n_ghost++));
            if (bounces == 0) ++coat_k;
            if (!(u < Tr)) {
                // reflected backwards (a ghost) with probability R, absorbed otherwise
                if (s.kind == K_MIRROR || !(u < Tr + Rr)) { out.flags = lost_flag(LOST_COATING, (int)si); return; }
                reflect(dl, N);
                dir = -dir;
                if (++bounces > kMaxGhostBounces) { out.flags = lost_flag(LOST_MISSED, (int)si); return; }
                for (int i = 0; i < 3; ++i) {
                    x[i] = st.M[0][i] * p[0] + st.M[1][i] * p[1] + st.M[2][i] * p[2] + st.o[i];
                    d[i] = st.M[0][i] * dl[0] + st.M[1][i] * dl[1] + st.M[2][i] * dl[2];
                }
                si += dir;
                continue;
            }
        }
        if (s.kind == K_MIRROR) {
            reflect(dl, N);
        } else {
            // the medium beyond the surface in the direction of travel
            int m_next = s.material;
            if (dir < 0) {
                m_next = -1;
                for (int j = 0; j < si; ++j)
                    if (sc.surf[j].kind != K_MIRROR) m_next = sc.surf[j].material;
            }
            T n_next = m_next < 0 ? T(1.0) : refractive_index_t<T>(sc, m_next, lamT);
            if (!refract(dl, N, n_cur, n_next)) { out.flags = lost_flag(LOST_TIR, (int)si); return; }
            n_cur = n_next;
        }
        // back to the telescope frame: x = M^T p + o
        for (int i = 0; i < 3; ++i) {
            x[i] = st.M[0][i] * p[0] + st.M[1][i] * p[1] + st.M[2][i] * p[2] + st.o[i];
            d[i] = st.M[0][i] * dl[0] + st.M[1][i] * dl[1] + st.M[2][i] * dl[2];
        }
        si += dir;
    }
}

template <class T>
void build_surfaces(const Scene& sc, std::vector<SurfT<T>>& ST) {
    ST.resize(sc.surf.size());
    for (size_t i = 0; i < sc.surf.size(); ++i) {
        const Surf& s = sc.surf[i];
        SurfT<T>& st = ST[i];
        for (int k = 0; k < 6; ++k) st.pert[k] = T(s.pert[k]);
        st.zern.assign(s.zern.size(), T(0.0));
        for (size_t k = 0; k < s.zern.size(); ++k) st.zern[k] = T(s.zern[k]);
        setup_surface(s, st);
    }
}

Source make_source(const int* kind, const int* sed, const int* table, const double* xi, const double* eta,
                   const double* z, const double* t0, const double* te, const double* a, const double* b,
                   const double* pa, int i) {
    Source s;
    s.kind = kind[i]; s.sed = sed[i]; s.table = table[i];
    s.xi = xi[i]; s.eta = eta[i]; s.redshift = z[i]; s.t0 = t0[i]; s.t_exp = te[i];
    s.a = a[i]; s.b = b[i]; s.pa = pa[i];
    return s;
}

}  // namespace

// ==========================================================================================================
// C interface (ctypes)
// ==========================================================================================================
extern "C" {

void oracle_philox(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out) { philox4x32_10(ctr, k0, k1, out); }

void* oracle_new(uint64_t seed, double pr_in, double pr_out, double h_top, double z_ent, double lam_ref, int atm_on,
                 int sensor_on) {
    Scene* s = new Scene();
    s->seed = seed; s->pr_in = pr_in; s->pr_out = pr_out; s->h_top = h_top; s->z_ent = z_ent; s->lam_ref = lam_ref;
    s->atm_on = atm_on; s->sensor_on = sensor_on;
    return s;
}
void oracle_free(void* p) { delete (Scene*)p; }

int oracle_add_surface(void* p, int kind, double R, double kappa, const double* alpha8, double z, double r_in,
                       double r_out, int material, int coating, const double* pert6, double rnorm, int nz,
                       const double* zern) {
    Scene* sc = (Scene*)p;
    Surf s;
    s.kind = kind; s.R = R; s.kappa = kappa; s.z = z; s.r_in = r_in; s.r_out = r_out;
    s.material = material; s.coating = coating; s.rnorm = rnorm;
    for (int i = 0; i < 8; ++i) s.alpha[i] = alpha8[i];
    for (int i = 0; i < 6; ++i) s.pert[i] = pert6[i];
    s.zern.assign(zern, zern + nz);
    sc->surf.push_back(s);
    return (int)sc->surf.size() - 1;
}
void oracle_set_perturbation(void* p, int surface, const double* pert6, int nz, const double* zern) {
    Scene* sc = (Scene*)p;
    Surf& s = sc->surf[surface];
    for (int i = 0; i < 6; ++i) s.pert[i] = pert6[i];
    s.zern.assign(zern, zern + nz);
}
int oracle_add_material(void* p, int kind, const double* B, const double* C) {
    Scene* sc = (Scene*)p;
    Mat m; m.kind = kind;
    for (int i = 0; i < 3; ++i) { m.B[i] = B[i]; m.C[i] = C[i]; }
    sc->mat.push_back(m);
    return (int)sc->mat.size() - 1;
}
int oracle_add_coating(void* p, double lam0, double dlam, double th0, double dth, int nl, int nt, const double* T,
                       const double* R) {
    Scene* sc = (Scene*)p;
    Coat c; c.lam0 = lam0; c.dlam = dlam; c.th0 = th0; c.dth = dth; c.nl = nl; c.nt = nt;
    c.T.assign(T, T + (size_t)nl * nt);
    if (R) c.R.assign(R, R + (size_t)nl * nt);
    sc->coat.push_back(c);
    return (int)sc->coat.size() - 1;
}
void oracle_set_detector(void* p, int nx, int ny, double pixel, double x0, double y0, double t_si, double ell_lam0,
                         double ell_dlam, int n_ell, const double* ell, int n_sig, const double* sig) {
    Scene* sc = (Scene*)p;
    sc->nx = nx; sc->ny = ny; sc->pixel = pixel; sc->x0 = x0; sc->y0 = y0; sc->t_si = t_si;
    sc->ell_lam0 = ell_lam0; sc->ell_dlam = ell_dlam;
    sc->ell.assign(ell, ell + n_ell);
    sc->sig.assign(sig, sig + n_sig);
}
int oracle_add_layer(void* p, double z, double vx, double vy) {
    Scene* sc = (Scene*)p;
    Layer L; L.z = z; L.vx = vx; L.vy = vy;
    sc->layers.push_back(L);
    return (int)sc->layers.size() - 1;
}
void oracle_add_scale(void* p, int layer, double pixel, int N, const double* phase) {
    Scene* sc = (Scene*)p;
    Scale S; S.pixel = pixel; S.N = N; S.phase.assign(phase, phase + (size_t)N * N);
    sc->layers[layer].scales.push_back(S);
}
// photon-number probability per bin = flux x wavelength x bin width (Sec. 2.2); cumulative sums in order
void oracle_set_seds(void* p, double lam0, double dlam, int n_sed, int n_bins, const double* flux) {
    Scene* sc = (Scene*)p;
    sc->sed_lam0 = lam0; sc->sed_dlam = dlam; sc->n_bins = n_bins;
    sc->cdf.assign(n_sed, std::vector<double>(n_bins));
    for (int s = 0; s < n_sed; ++s) {
        std::vector<double> acc(n_bins);
        double run = 0.0;
        for (int k = 0; k < n_bins; ++k) {
            double centre = lam0 + (k + 0.5) * dlam;
            double pk = flux[(size_t)s * n_bins + k] * centre;
            pk = pk * dlam;
            run = run + pk;
            acc[k] = run;
        }
        for (int k = 0; k < n_bins; ++k) sc->cdf[s][k] = acc[k] / run;
    }
}
void oracle_get_cdf(void* p, int sed, double* out) {
    Scene* sc = (Scene*)p;
    for (int k = 0; k < sc->n_bins; ++k) out[k] = sc->cdf[sed][k];
}
void oracle_set_sensor_options(void* p, int back_reflect, double dead_layer) {
    Scene* sc = (Scene*)p;
    sc->back_reflect = back_reflect;
    sc->dead_layer = dead_layer;
}
void oracle_set_fringe(void* p, int on, double t_gx, double t_gy) {
    Scene* sc = (Scene*)p;
    sc->fringe = on;
    sc->t_gx = t_gx;
    sc->t_gy = t_gy;
}
double oracle_film_reflectance(double lam_nm, double n0, double n1, double k1, double t_mm, double s) {
    return film_reflectance(lam_nm, n0, n1, k1, t_mm, s);
}

// Saturation and bleeding (Sec. 2.5) on a finished image: in each half of every row, pixels above the full
// well, visited left to right, give their excess electron by electron to the closest pixel of the half-row
// that is below the full well (the left one first at equal distance); what finds no room is removed.
uint64_t oracle_bleed(uint32_t* img, int nx, int ny, uint32_t w) {
    uint64_t removed = 0;
    for (int y = 0; y < ny; ++y) {
        for (int half = 0; half < 2; ++half) {
            const int lo = half ? nx / 2 : 0, hi = half ? nx : nx / 2;    // [lo, hi)
            uint32_t* row = img + (size_t)y * nx;
            for (int x = lo; x < hi; ++x) {
                if (row[x] <= w) continue;
                uint64_t excess = row[x] - w;
                row[x] = w;
                for (int d = 1; excess > 0; ++d) {
                    const bool has_l = x - d >= lo, has_r = x + d < hi;
                    if (!has_l && !has_r) { removed += excess; excess = 0; break; }
                    // electrons alternate left, right, left, ... while both sides have room
                    while (excess > 0) {
                        bool moved = false;
                        if (has_l && row[x - d] < w) { row[x - d] += 1; --excess; moved = true; }
                        if (excess > 0 && has_r && row[x + d] < w) { row[x + d] += 1; --excess; moved = true; }
                        if (!moved) break;
                    }
                }
            }
        }
    }
    return removed;
}

// Background bundles (Sec. 3.2): n[s] photons per ray of source s (<= 1: one), spread with sigma[s] mm.
void oracle_set_bundles(void* p, int n_src, const int* n, const double* sigma) {
    Scene* s = (Scene*)p;
    s->bundle_n.assign(n, n + n_src);
    s->bundle_sigma.assign(sigma, sigma + n_src);
}

void oracle_set_hf_kick(void* p, int K, const double* q) {
    Scene* sc = (Scene*)p;
    sc->hf.assign(q, q + K);
}
void oracle_set_sersic(void* p, int n_tab, int K, const double* r) {
    Scene* sc = (Scene*)p;
    sc->sersic_K = K;
    sc->sersic.assign(n_tab, std::vector<double>(K));
    for (int t = 0; t < n_tab; ++t)
        for (int k = 0; k < K; ++k) sc->sersic[t][k] = r[(size_t)t * K + k];
}

// Trace photons [first[s], first[s] + count[s]) of every source s.  Records are written in source order.
int oracle_trace(void* p, int n_src, const int* kind, const int* sed, const int* table, const double* xi,
                 const double* eta, const double* z, const double* t0, const double* te, const double* a,
                 const double* b, const double* pa, const uint64_t* first, const uint64_t* count,
                 double* rx, double* ry, double* rxc, double* ryc, double* rlam, uint32_t* rflags, int32_t* rpix,
                 double* rmargin_mm, double* rmargin_nm, uint32_t* image, int n_threads) {
    Scene* sc = (Scene*)p;
    if (sc->surf.empty() || sc->cdf.empty()) return -1;
    std::vector<uint64_t> off(n_src + 1, 0);
    for (int s = 0; s < n_src; ++s) off[s + 1] = off[s] + count[s];
    std::vector<SurfT<double>> ST;
    build_surfaces(*sc, ST);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
    for (int s = 0; s < n_src; ++s) {
        Source src = make_source(kind, sed, table, xi, eta, z, t0, te, a, b, pa, s);
        long long n = (long long)count[s];
#pragma omp parallel for schedule(static)
        for (long long k = 0; k < n; ++k) {
            uint64_t i = first[s] + (uint64_t)k;
            const int nb = bundle_of(*sc, s);
            // a bundle's photon follows its ray (index i / nb) to the detector surface
            Draws D = draw_photon(*sc, s, nb > 1 ? i / (uint64_t)nb : i);
            Pre P;
            sample_and_atmosphere(*sc, src, D, P);
            OpticsOut<double> o;
            if (nb > 1) {
                const Member M = member_draws(*sc, s, i, sc->bundle_sigma[s]);
                optics_and_sensor(*sc, ST, P, &D, o, &M);
            } else {
                optics_and_sensor(*sc, ST, P, &D, o);
            }
            size_t r = off[s] + (size_t)k;
            if (rx) { rx[r] = o.x; ry[r] = o.y; rxc[r] = o.xc; ryc[r] = o.yc; rlam[r] = P.lam; rflags[r] = o.flags;
                      rpix[r] = o.pix; rmargin_mm[r] = o.margin_mm; rmargin_nm[r] = o.margin_nm; }
            if (image && (o.flags & F_DETECTED)) {
#pragma omp atomic
                image[o.pix] += 1u;
            }
        }
    }
    return 0;
}

// Deterministic rays through the surfaces only (no atmosphere, coatings pass, no silicon): the position
// of each ray on the last surface in that surface's frame.
int oracle_trace_rays(void* p, int n, const double* pos, const double* dir, const double* lam, double* outx,
                      double* outy, double* outz, double* outd, uint32_t* flags) {
    Scene* sc = (Scene*)p;
    std::vector<SurfT<double>> ST;
    build_surfaces(*sc, ST);
    int saved = sc->sensor_on;
    sc->sensor_on = 0;
    std::vector<int> saved_coat;
    for (auto& s : sc->surf) { saved_coat.push_back(s.coating); s.coating = -1; }
    int saved_nx = sc->nx, saved_ny = sc->ny;
    double saved_x0 = sc->x0, saved_y0 = sc->y0, saved_pix = sc->pixel;
    // a very large chip so that every ray reaching the last surface is reported
    sc->nx = sc->ny = 1 << 30; sc->pixel = 1.0; sc->x0 = 0; sc->y0 = 0;
    for (int i = 0; i < n; ++i) {
        Pre P;
        for (int k = 0; k < 3; ++k) { P.x[k] = pos[3 * i + k]; P.d[k] = dir[3 * i + k]; }
        P.lam = lam[i]; P.t = 0;
        OpticsOut<double> o;
        optics_and_sensor(*sc, ST, P, nullptr, o);
        outx[i] = o.x; outy[i] = o.y;
        if (outz) outz[i] = 0.0;
        if (outd) outd[i] = 0.0;
        flags[i] = o.flags;
    }
    sc->nx = saved_nx; sc->ny = saved_ny; sc->x0 = saved_x0; sc->y0 = saved_y0; sc->pixel = saved_pix;
    for (size_t k = 0; k < sc->surf.size(); ++k) sc->surf[k].coating = saved_coat[k];
    sc->sensor_on = saved;
    return 0;
}

// One surface: intersection distance, hit point, unit normal of a single ray given in the surface frame.
int oracle_intersect(void* p, int surface, const double* pos, const double* dir, double* l, double* hit, double* normal) {
    Scene* sc = (Scene*)p;
    SurfT<double> st;
    const Surf& s = sc->surf[surface];
    for (int k = 0; k < 6; ++k) st.pert[k] = 0.0;
    st.zern.assign(s.zern.begin(), s.zern.end());
    setup_surface(s, st);
    double pp[3] = {pos[0], pos[1], pos[2]}, dd[3] = {dir[0], dir[1], dir[2]}, ll;
    uint32_t why = intersect(st, pp, dd, ll);
    if (why) return (int)why;
    *l = ll;
    for (int k = 0; k < 3; ++k) hit[k] = pp[k] + ll * dd[k];
    double zs, zx, zy;
    surface_sag(st, hit[0], hit[1], zs, zx, zy);
    double nn = std::sqrt(1.0 + zx * zx + zy * zy);
    normal[0] = -zx / nn; normal[1] = -zy / nn; normal[2] = 1.0 / nn;
    return 0;
}

int oracle_sag(void* p, int surface, int n, const double* x, const double* y, double* z, double* zx, double* zy) {
    Scene* sc = (Scene*)p;
    SurfT<double> st;
    const Surf& s = sc->surf[surface];
    for (int k = 0; k < 6; ++k) st.pert[k] = 0.0;
    st.zern.assign(s.zern.begin(), s.zern.end());
    setup_surface(s, st);
    for (int i = 0; i < n; ++i)
        if (!surface_sag(st, x[i], y[i], z[i], zx[i], zy[i])) z[i] = NAN;
    return 0;
}

void oracle_zernike(int j, int n, const double* rho, const double* theta, double* Z) {
    for (int i = 0; i < n; ++i) {
        double a, b, c;
        zernike_term(j, rho[i], theta[i], a, b, c);
        Z[i] = a;
    }
}

int oracle_refract(const double* d, const double* N, double n1, double n2, double* out) {
    double dd[3] = {d[0], d[1], d[2]}, NN[3] = {N[0], N[1], N[2]};
    if (!refract<double>(dd, NN, n1, n2)) return 1;
    for (int i = 0; i < 3; ++i) out[i] = dd[i];
    return 0;
}
int oracle_reflect(const double* d, const double* N, double* out) {
    double dd[3] = {d[0], d[1], d[2]}, NN[3] = {N[0], N[1], N[2]};
    reflect(dd, NN);
    for (int i = 0; i < 3; ++i) out[i] = dd[i];
    return 0;
}
double oracle_index(void* p, int material, double lam_nm) { return refractive_index(*(Scene*)p, material, lam_nm); }

// Photon state after sampling and the atmosphere (for pins of Sec. 2.2 and 2.3).
int oracle_pre_optics(void* p, int n_src, const int* kind, const int* sed, const int* table, const double* xi,
                      const double* eta, const double* z, const double* t0, const double* te, const double* a,
                      const double* b, const double* pa, int src_index, uint64_t first, uint64_t count, double* pos,
                      double* dir, double* lam, double* t) {
    Scene* sc = (Scene*)p;
    if (src_index < 0 || src_index >= n_src) return -1;
    Source src = make_source(kind, sed, table, xi, eta, z, t0, te, a, b, pa, src_index);
    for (uint64_t k = 0; k < count; ++k) {
        Draws D = draw_photon(*sc, src_index, first + k);
        Pre P;
        sample_and_atmosphere(*sc, src, D, P);
        for (int q = 0; q < 3; ++q) { pos[3 * k + q] = P.x[q]; dir[3 * k + q] = P.d[q]; }
        lam[k] = P.lam; t[k] = P.t;
    }
    return 0;
}

// Pathwise gradient (Sec. 2.4 optics, parameters of the misalignments and Zernike figures).
// param_surface[p], param_field[p]: field 0..5 = dx, dy, dz, tx, ty, tz; field 100 + j = Noll c_(j+1).
// Outputs, for photons [first[s], first[s] + count[s]) of every source: the detected positions' tangent
// dx/dtheta_p and dy/dtheta_p in dxdp/dydp (records x n_params, zero for undetected photons), with the
// values in rx/ry and the detection flags in rflags.
int oracle_trace_tangents(void* p, int n_src, const int* kind, const int* sed, const int* table, const double* xi,
                          const double* eta, const double* z, const double* t0, const double* te, const double* a,
                          const double* b, const double* pa, const uint64_t* first, const uint64_t* count,
                          int n_params, const int* param_surface, const int* param_field, double* rx, double* ry,
                          uint32_t* rflags, double* dxdp, double* dydp, int n_threads) {
    Scene* sc = (Scene*)p;
    std::vector<uint64_t> off(n_src + 1, 0);
    for (int s = 0; s < n_src; ++s) off[s + 1] = off[s] + count[s];
    std::vector<std::vector<SurfT<Dual>>> STs(n_params);
    for (int q = 0; q < n_params; ++q) {
        std::vector<SurfT<Dual>>& ST = STs[q];
        ST.resize(sc->surf.size());
        for (size_t i = 0; i < sc->surf.size(); ++i) {
            const Surf& s = sc->surf[i];
            for (int k = 0; k < 6; ++k) ST[i].pert[k] = Dual(s.pert[k], 0.0);
            ST[i].zern.assign(s.zern.size(), Dual());
            for (size_t k = 0; k < s.zern.size(); ++k) ST[i].zern[k] = Dual(s.zern[k], 0.0);
        }
        int ps = param_surface[q], pf = param_field[q];
        if (ps < 0 || ps >= (int)sc->surf.size()) return -2;
        if (pf < 6) ST[ps].pert[pf].d = 1.0;
        else {
            int j = pf - 100;
            if (j < 0) return -3;
            if ((int)ST[ps].zern.size() <= j) ST[ps].zern.resize(j + 1, Dual());
            ST[ps].zern[j].d = 1.0;
        }
        for (size_t i = 0; i < sc->surf.size(); ++i) setup_surface(sc->surf[i], ST[i]);
    }
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#endif
    for (int s = 0; s < n_src; ++s) {
        Source src = make_source(kind, sed, table, xi, eta, z, t0, te, a, b, pa, s);
        long long n = (long long)count[s];
#pragma omp parallel for schedule(static)
        for (long long k = 0; k < n; ++k) {
            uint64_t i = first[s] + (uint64_t)k;
            Draws D = draw_photon(*sc, s, i);
            Pre P;
            sample_and_atmosphere(*sc, src, D, P);
            size_t r = off[s] + (size_t)k;
            for (int q = 0; q < n_params; ++q) {
                OpticsOut<Dual> o;
                optics_and_sensor(*sc, STs[q], P, &D, o);
                if (q == 0) { rx[r] = o.x.v; ry[r] = o.y.v; rflags[r] = o.flags; }
                bool det = (o.flags & F_DETECTED) != 0;
                dxdp[r * n_params + q] = det ? o.x.d : 0.0;
                dydp[r * n_params + q] = det ? o.y.d : 0.0;
            }
        }
    }
    return 0;
}

// Algorithmic operation counts of the photon path (per photon, averaged over the given photons):
// out[0..4] = add/sub, mul, div, sqrt, transcendental of sampling + atmosphere; out[5..9] the same for the
// optics and sensor; out[10] = photons counted; out[11] = fraction not removed by the early test.  Newton stops at the paper's 0.01 um step here; the
// central-difference screen gradients are table reads (precomputed, Sec. 3.2) and are not counted.
int oracle_count_ops(void* p, int n_src, const int* kind, const int* sed, const int* table, const double* xi,
                     const double* eta, const double* z, const double* t0, const double* te, const double* a,
                     const double* b, const double* pa, const uint64_t* first, const uint64_t* count, int early,
                     double* out) {
    Scene* sc = (Scene*)p;
    OpCount pre, opt;
    double n = 0, survivors = 0;
    std::vector<SurfT<Cnt>> ST;
    build_surfaces(*sc, ST);
    for (int s = 0; s < n_src; ++s) {
        Source src = make_source(kind, sed, table, xi, eta, z, t0, te, a, b, pa, s);
        for (uint64_t k = 0; k < count[s]; ++k) {
            Draws D = draw_photon(*sc, s, first[s] + k);
            n += 1;
            if (early) {
                // dynamic transmission (Sec. 3.2): a photon whose coating draw is not below the largest
                // transmission over angles at its wavelength is dropped before any propagation
                Pre P0;
                sample_and_atmosphere(*sc, src, D, P0);
                bool rejected = false;
                int kq = 0;
                for (const Surf& sf : sc->surf) {
                    if (sf.coating < 0 || sf.kind == K_DETECTOR) continue;
                    const Coat& C = sc->coat[sf.coating];
                    int il = std::min(C.nl - 1, std::max(0, (int)std::floor((P0.lam - C.lam0) / C.dlam)));
                    double tmax = 0.0;
                    for (int it = 0; it < C.nt; ++it) tmax = std::max(tmax, C.T[(size_t)il * C.nt + it]);
                    if (!(uniform01(D.w[S_COAT0 + kq]) < tmax)) rejected = true;
                    ++kq;
                }
                if (rejected) continue;
            }
            survivors += 1;
            g_ops = OpCount();
            Cnt X[3], Dir[3], lam, tt;
            sample_and_atmosphere_t<Cnt>(*sc, src, D, X, Dir, lam, tt);
            pre.add += g_ops.add; pre.mul += g_ops.mul; pre.div += g_ops.div; pre.sqrt += g_ops.sqrt; pre.special += g_ops.special;
            Pre P;
            for (int q = 0; q < 3; ++q) { P.x[q] = X[q].v; P.d[q] = Dir[q].v; }
            P.lam = lam.v; P.t = tt.v;
            g_ops = OpCount();
            OpticsOut<Cnt> o;
            optics_and_sensor(*sc, ST, P, &D, o);
            opt.add += g_ops.add; opt.mul += g_ops.mul; opt.div += g_ops.div; opt.sqrt += g_ops.sqrt; opt.special += g_ops.special;
        }
    }
    if (n == 0) return -1;
    double v[10] = {pre.add, pre.mul, pre.div, pre.sqrt, pre.special, opt.add, opt.mul, opt.div, opt.sqrt, opt.special};
    for (int i = 0; i < 10; ++i) out[i] = v[i] / n;
    out[10] = n;
    out[11] = survivors / n;
    return 0;
}

}  // extern "C"
