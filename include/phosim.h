/*
 * phosim.h — C ABI of the GB300 photon Monte Carlo library.
 *
 * The library traces astrophysical photons one by one through frozen-flow atmospheric phase screens, an
 * aspheric multi-surface telescope/camera and a silicon sensor into a pixel histogram, as described in
 * Peterson et al. 2015 (PhoSim), Sec. 2.  Every per-photon step runs in CUDA kernels for sm_103a on the
 * caller's stream; nothing in this interface uses C++ or PyTorch types.
 *
 * Conventions
 *   - Units: mm for lengths, rad for angles, nm for wavelengths, s for times, rad (at lambda_ref) for phase.
 *   - The telescope frame has z along the optical axis; photons arrive travelling towards -z (Sec. 2.2).
 *   - Ownership: the caller owns every input and output buffer.  A scene owns device copies of everything
 *     loaded into it; load calls copy synchronously and may be called again to replace what they load.
 *   - Errors: every call returns a phosim_status (0 = success, negative = error) and never throws or aborts.
 *     A failed call leaves the scene as it was before the call, except where noted.  Per-photon events
 *     (vignetting, total internal reflection, a non-converged intersection, leaving the chip) are not
 *     errors: such photons are dropped and counted (phosim_get_counters).
 *   - Thread safety: calls on different scenes may run concurrently; calls on one scene must not overlap.
   - Devices: a scene lives on the CUDA device that was current when it was created; every call on it must be
     made with that device current (else INVALID_ARGUMENT), and device buffers passed to it must be on it.
 */
#ifndef PHOSIM_H
#define PHOSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int phosim_status;
#define PHOSIM_OK 0
#define PHOSIM_ERR_INVALID_ARGUMENT (-1)
#define PHOSIM_ERR_OUT_OF_MEMORY (-2)
#define PHOSIM_ERR_CUDA (-3)
#define PHOSIM_ERR_UNSUPPORTED (-4)
#define PHOSIM_ERR_NOT_READY (-5)    /* a required load (optics, SEDs) has not been done */
#define PHOSIM_ERR_LIMIT (-6)        /* a size exceeds a documented maximum */

#define PHOSIM_MAX_SURFACES 16
#define PHOSIM_MAX_LAYERS 8
#define PHOSIM_MAX_SCALES 2
#define PHOSIM_MAX_ZERNIKE 28        /* Noll j <= 28: radial order <= 6 */
#define PHOSIM_MAX_COATED 6          /* coated surfaces with an accept-reject draw */
#define PHOSIM_MAX_BUNDLE 4096       /* photons per ray of a background bundle */
#define PHOSIM_MAX_GHOST_BOUNCES 8   /* coating reflections a ghost photon may undergo */

/* surface kinds, materials, source kinds (Sec. 2.4.1, 2.2) */
enum { PHOSIM_MIRROR = 0, PHOSIM_REFRACT = 1, PHOSIM_DETECTOR = 2 };
enum { PHOSIM_VACUUM = 0, PHOSIM_SELLMEIER = 1, PHOSIM_SILICON = 2 };
enum { PHOSIM_POINT = 0, PHOSIM_SERSIC = 1, PHOSIM_GAUSS = 2 };

/* precision of the photon path */
enum {
    PHOSIM_PLAIN_FP64 = 0,   /* every step in FP64 */
    PHOSIM_MIXED = 1,        /* FP64 for positions, surface transforms and intersections; FP32 for the
                                wavelength blur, screen-gradient deflections, source shapes, silicon
                                conversion and diffusion; FP32 moment partials with compensated sums */
    PHOSIM_MIXED_DS = 2      /* PHOSIM_MIXED with its FP64 parts (positions, directions, surface transforms,
                                intersections, focal-plane position) in double-single arithmetic: pairs of
                                FP32 numbers carrying about 48 significant bits, on the FP32 pipes, which
                                issue about seventy times the FP64 rate on this GPU.  The pupil azimuth and
                                the Sellmeier index are double-single too; coating decisions compare the
                                integer draw with integer thresholds.  phosim_grad runs the FP64 path
                                whatever the scene's precision. */
};

/* scene flags */
#define PHOSIM_ATMOSPHERE 1u     /* apply the phase-screen layers */
#define PHOSIM_SENSOR 2u         /* silicon conversion and diffusion; otherwise the detector-surface hit */
#define PHOSIM_GRAPH 8u          /* launch each phosim_trace call's kernels as one CUDA graph: the chief rays and the
                                    trace kernel, or in the two-kernel double-single path the chief rays, then per
                                    chunk of the state buffer the counter resets and the entry, optics and bundle
                                    stages, then the moment-stripe sum.  Built on the first call of a given shape
                                    (number of chunks, kernel list) and replayed with each call's parameters */
#define PHOSIM_BACK_REFLECT 16u  /* back-side reflection (Sec. 2.4.2): a photon whose conversion length takes it
                                    past the back of the silicon is reflected there with the Fresnel probability
                                    of the silicon / vacuum interface at normal incidence, ((n - 1) / (n + 1))^2
                                    (with PHOSIM_FRINGE: the single-layer interference result), and converts on
                                    its way back */
#define PHOSIM_FRINGE 32u       /* with PHOSIM_BACK_REFLECT, fringing (Sec. 2.4.2): the back-side reflection probability is
                                    the single-layer electromagnetic result instead, the reflectance of one layer of
                                    silicon (index n + i k, k = lambda / (4 pi ell(lambda)) from the absorption-length
                                    table) between the medium in front of the detector and vacuum behind it: the Airy
                                    sum of its two interfaces' amplitude reflection coefficients at the photon's angle,
                                    averaged over the s and p polarisations, with the layer's optical thickness
                                    t_si + t_si_gx (x - x0) + t_si_gy (y - y0) at the photon's entry point (x, y) */
#define PHOSIM_EARLY_REJECT 4u   /* dynamic transmission (Sec. 3.2): decide each coating's accept draw against
                                    the largest transmission over incidence angles at the photon's wavelength
                                    before propagating it.  The detected photons, image and moments are
                                    unchanged; a photon rejected this way is reported as a COATING loss at
                                    that surface even if an earlier surface would have vignetted it. */

/* record flags (phosim_photon_record.flags): bit 0 = detected; otherwise bits 8..15 hold the reason the
   photon was dropped and bits 16..23 the index of the surface where it happened */
#define PHOSIM_F_DETECTED 1u
enum {
    PHOSIM_LOST_VIGNETTED = 1, PHOSIM_LOST_MISSED = 2, PHOSIM_LOST_NEWTON = 3, PHOSIM_LOST_TIR = 4,
    PHOSIM_LOST_COATING = 5, PHOSIM_LOST_OFF_CHIP = 6, PHOSIM_LOST_NOT_CONVERTED = 7, PHOSIM_LOST_DEAD_LAYER = 8
};

/* Scene description (Sec. 2.2 pupil and top of the atmosphere; Sec. 2.4.1 detector device; Sec. 2.4.2
   absorption length; Sec. 2.5 diffusion).  Tables are host pointers, copied at creation. */
typedef struct phosim_scene_desc {
    uint64_t seed;              /* Philox4x32-10 key */
    int32_t precision;          /* PHOSIM_PLAIN_FP64, PHOSIM_MIXED or PHOSIM_MIXED_DS */
    uint32_t flags;             /* PHOSIM_ATMOSPHERE | PHOSIM_SENSOR */
    double pupil_r_in, pupil_r_out;   /* annulus sampled on the first surface (Sec. 2.2), mm */
    double h_top;               /* top of the atmosphere, telescope-frame z, mm (100 km) */
    double z_entrance;          /* plane below every layer and above every optic where the raytrace starts */
    double lambda_ref;          /* wavelength of the screen phases, nm */
    int32_t nx, ny;             /* pixels of the chip */
    double pixel;               /* mm */
    double x0, y0;              /* chip centre in the detector surface frame, mm */
    double t_si;                /* silicon thickness, mm */
    double ell_lam0, ell_dlam;  /* absorption length table: lambda_k = ell_lam0 + k ell_dlam (nm) */
    int32_t n_ell;              /* >= 2 */
    const double* ell;          /* mm, linear interpolation, clamped at the ends */
    int32_t n_sigma;            /* >= 2 */
    const double* sigma;        /* diffusion sigma (mm) at depths k t_si / (n_sigma - 1) below the entrance */
    double dead_layer;          /* field-free layer at the entrance (Sec. 2.4.2), mm: photons converting in it
                                   are lost; 0 = none */
    double t_si_gx, t_si_gy;    /* PHOSIM_FRINGE: gradient of the silicon's optical thickness across the chip (mm
                                   per mm of the detector surface frame, about the chip centre); the conversion
                                   geometry keeps t_si */
} phosim_scene_desc;

/* One optical surface (Sec. 2.4.1, Table 1): z(r) = r^2 / (R (1 + sqrt(1 - (1 + kappa) r^2 / R^2)))
   + sum_{i=3..10} alpha_i r^i + sum_j zern[j-1] Z_j(x / zern_rnorm, y / zern_rnorm) (Noll order and
   normalisation), about a vertex at (pert[0], pert[1], z + pert[2]) rotated by
   Rz(pert[5]) Ry(pert[4]) Rx(pert[3]).  R = 0 means flat.  Surfaces are met in array order. */
typedef struct phosim_surface {
    int32_t kind;               /* PHOSIM_MIRROR, PHOSIM_REFRACT or PHOSIM_DETECTOR (last surface only) */
    int32_t material;           /* medium after a refracting surface / the silicon of the detector */
    int32_t coating;            /* index of the coating table, -1 = none */
    int32_t n_zern;             /* number of Zernike coefficients used, <= PHOSIM_MAX_ZERNIKE */
    double R, kappa;
    double alpha[8];            /* alpha_3 .. alpha_10 */
    double z;
    double r_in, r_out;         /* clear aperture radius bounds in the surface frame */
    double pert[6];             /* dx, dy, dz (mm), tx, ty, tz (rad) */
    double zern_rnorm;
    double zern[PHOSIM_MAX_ZERNIKE];
} phosim_surface;

typedef struct phosim_material {
    int32_t kind;               /* PHOSIM_VACUUM, PHOSIM_SELLMEIER (lambda in um, C in um^2), PHOSIM_SILICON */
    double B[3], C[3];
} phosim_material;

/* transmission probability, piecewise constant in (lambda, incidence angle) (Sec. 2.4.2), and optionally the
   reflection probability on the same grid (the four-column coating interface: T and R against wavelength and
   angle).  A photon meeting a coated refracting surface is transmitted with probability T, reflected with
   probability R (a ghost: it travels back through the surfaces, refracting and meeting coatings on its way,
   until another reflection turns it round; after a photon's first reflection each coating decision draws the
   next word of Philox blocks 7, 8, ... of the photon's (or its ray's) counter; a photon reflected more than
   PHOSIM_MAX_GHOST_BOUNCES times, leaving the first surface backwards or missing a surface is MISSED) and
   absorbed otherwise; on a mirror T is the reflectance and the rest is absorbed.  Ghosts are not available to
   phosim_grad (UNSUPPORTED). */
typedef struct phosim_coating {
    double lam0, dlam;          /* nm */
    double theta0, dtheta;      /* rad */
    int32_t n_lambda, n_theta;
    const double* table;        /* host, n_lambda x n_theta, row-major */
    const double* reflect;      /* host, n_lambda x n_theta, or NULL (no reflection); table + reflect <= 1 */
} phosim_coating;

/* One frozen-flow layer (Sec. 2.3.1): up to two screen scales whose gradients add. */
typedef struct phosim_screen_scale {
    double pixel;               /* mm */
    int32_t n;                  /* n x n periodic screen, n >= 3 */
    const double* phase;        /* host, row-major (row = y), rad at lambda_ref */
} phosim_screen_scale;

typedef struct phosim_layer {
    double z;                   /* telescope-frame height, mm; layers must be given top to bottom */
    double vx, vy;              /* wind, mm/s: the screen sampled at time t is the one at position - v t */
    int32_t n_scales;
    phosim_screen_scale scales[PHOSIM_MAX_SCALES];
} phosim_layer;

/* A source (Sec. 2.2): its direction's tangent-plane components, spectrum, time window and shape. */
typedef struct phosim_source {
    int32_t kind;               /* PHOSIM_POINT, PHOSIM_SERSIC, PHOSIM_GAUSS */
    int32_t sed;                /* index of the SED table */
    int32_t table;              /* Sersic radial table index */
    int32_t bundle;             /* photons per ray, the background optimisation of Sec. 3.2 (0 or 1: one photon
                                   per ray, <= PHOSIM_MAX_BUNDLE): photon i follows ray i / bundle through the
                                   atmosphere and the optics to the detector surface, then lands at a Gaussian
                                   offset of sigma bundle_sigma from the ray's hit and goes through the sensor
                                   with its own draws (Philox blocks 5 and 6 of its own counter) */
    double xi, eta;             /* n_x, n_y of the undisturbed photon */
    double redshift;
    double t0, t_exp;
    double a, b, pa;            /* Sersic semi-axes at the half-light radius and position angle (rad);
                                   PHOSIM_GAUSS: a = sigma (rad) */
    double bundle_sigma;        /* mm on the detector surface, >= 0 (used when bundle > 1) */
} phosim_source;

/* Per-photon record, written only when a record buffer is given (debugging / parity). */
typedef struct phosim_photon_record {
    double x, y;                /* final position in the detector surface frame (after diffusion), mm */
    double xc, yc;              /* lateral position where the photon converted, mm */
    double lambda;              /* nm */
    uint32_t flags;
    int32_t pix;                /* y * nx + x, or -1 */
} phosim_photon_record;

/* Per-source moment sums, PHOSIM_MOMENT_WORDS doubles per source, additive across calls:
   [0] detected count, [1] sum dx, [2] sum dy, [3] sum dx^2, [4] sum dx dy, [5] sum dy^2,
   [6] ref_x, [7] ref_y, with dx = x - ref_x, dy = y - ref_y and (ref_x, ref_y) the detector-plane
   position of the source's chief ray at lambda_ref (written, not added). */
#define PHOSIM_MOMENT_WORDS 8

typedef struct phosim_scene phosim_scene;

/* Create a scene from its description (copies the tables).  Errors: INVALID_ARGUMENT (null pointers,
   sizes < 2, non-positive pixel or thickness, unknown precision), OUT_OF_MEMORY, CUDA. */
phosim_status phosim_create_scene(const phosim_scene_desc* desc, phosim_scene** out);

/* Load the surfaces in the order photons meet them (Sec. 2.4.1-2.4.2) with their media and coatings.
   The last surface must be the only PHOSIM_DETECTOR.  At most PHOSIM_MAX_SURFACES surfaces and
   PHOSIM_MAX_COATED coated surfaces.  Errors: INVALID_ARGUMENT, LIMIT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_load_optics(phosim_scene* scene, const phosim_surface* surfaces, int n_surfaces,
                                 const phosim_material* materials, int n_materials,
                                 const phosim_coating* coatings, int n_coatings);

/* Load the atmosphere (Sec. 2.3): layers top to bottom; the central-difference gradient screens are
   built on the device.  n_layers = 0 removes the atmosphere.  Errors: INVALID_ARGUMENT, LIMIT,
   OUT_OF_MEMORY, CUDA. */
phosim_status phosim_load_screens(phosim_scene* scene, const phosim_layer* layers, int n_layers);

/* Load the SEDs (Sec. 2.2): flux per unit wavelength at bin centres lam0 + (k + 1/2) dlam, n_sed x n_bins,
   host, row-major.  The photon-number cumulative tables are built on the device.
   Errors: INVALID_ARGUMENT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_load_seds(phosim_scene* scene, const double* flux, int n_sed, int n_bins, double lam0,
                               double dlam);

/* Load Sersic radial tables (Sec. 2.2.1): radius / half-light radius at u = (k + 1/2) / n_nodes,
   n_tables x n_nodes, host.  Errors: INVALID_ARGUMENT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_load_sersic(phosim_scene* scene, const double* table, int n_tables, int n_nodes);

/* Load the second, statistical atmospheric kick (Sec. 2.3.2): the kick angle's quantiles (rad, at
   lambda_ref) at u = (k + 1/2) / n of the long-exposure PSF of the screens above kappa_crit (including the
   unscattered part as zero angles), non-decreasing.  Each photon that crossed the layers then draws an
   angle (linear interpolation, scaled by (lambda / lambda_ref)^(-1/5)) and a uniform direction.  n = 0
   removes it.  Errors: INVALID_ARGUMENT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_load_hf_kick(phosim_scene* scene, const double* quantiles, int n);

/* Trace photons first[s] .. first[s] + n_photons[s] - 1 of every source s (first = NULL: from 0).
   sources, n_photons and first are host arrays.  Photon i of source s always draws the same random
   numbers (counter = (i, s, block), key = seed), whatever the batching.
   image: nx * ny uint32 counts, ADDED to (device or host pointer; a host pointer is staged through a
          scene-owned device buffer and the call returns after the copy back; another device's memory is
          INVALID_ARGUMENT).
   records: NULL or a device array of sum(n_photons) records in source order.
   moments: NULL or a device array of n_src * PHOSIM_MOMENT_WORDS doubles; sums are added.
   records and moments must be device (or managed) memory of the scene's device: a host pointer returns
   INVALID_ARGUMENT before anything is launched.
   stream: a cudaStream_t (NULL = legacy default stream); all device work is ordered on it.
   Errors: INVALID_ARGUMENT, NOT_READY, LIMIT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_trace(phosim_scene* scene, const phosim_source* sources, int n_src,
                           const uint64_t* n_photons, const uint64_t* first, uint32_t* image,
                           phosim_photon_record* records, double* moments, void* stream);

/* Pathwise gradient (adjoint raytrace) of L = sum_s sum_k dL_dmoments[s][k] M_s[k] with respect to the
   listed surface parameters, where M_s = (mean x, mean y, Ixx, Ixy, Iyy) of the detected photons of
   source s (central second moments).  Common random numbers, accept decisions of the forward pass held.
   param_surface[p], param_field[p]: field 0..5 = pert[0..5], field 100 + j = zern[j].
   dL_dmoments: host, n_src x 5.  grad: host, n_src x n_params, written (per-source contributions).
   moments_out: NULL or host n_src x 6 (count, mean x, mean y, Ixx, Ixy, Iyy).
   Errors: INVALID_ARGUMENT, NOT_READY, LIMIT, OUT_OF_MEMORY, CUDA. */
phosim_status phosim_grad(phosim_scene* scene, const phosim_source* sources, int n_src,
                          const uint64_t* n_photons, const double* dL_dmoments, const int32_t* param_surface,
                          const int32_t* param_field, int n_params, double* grad, double* moments_out,
                          void* stream);

/* Launch shape of the trace kernel: threads per block and photons per warp tile (0 = keep current).  In the
   two-kernel double-single path it applies to the entry and bundle stages; the optics stage keeps blocks of
   256 threads, whose warps take the surfaces together. */
phosim_status phosim_set_schedule(phosim_scene* scene, int threads_per_block, int tile_photons);

/* The launch shape phosim_trace uses now (after phosim_set_schedule or phosim_autotune): threads per block
   and photons per warp tile (0 = chosen per call from the workload).  Errors: INVALID_ARGUMENT (null). */
phosim_status phosim_get_schedule(const phosim_scene* scene, int* threads_per_block, int* tile_photons);

/* Per-source detected count, centroid and central second moments from the additive sums phosim_trace writes
   (the number of photons detected from every source and their mean coordinate, Sec. 3.1, and the second
   moments the image-quality comparisons use): out[6 s + 0] = n, [1] = ref_x + sum dx / n, [2] = ref_y +
   sum dy / n, [3] = sum dx^2 / n - (sum dx / n)^2, [4] = sum dx dy / n - (sum dx / n)(sum dy / n),
   [5] = sum dy^2 / n - (sum dy / n)^2; NaN for a source with no detected photon.  sums: host, n_src *
   PHOSIM_MOMENT_WORDS doubles; out: host, n_src * 6.  Pure host arithmetic.  Errors: INVALID_ARGUMENT. */
phosim_status phosim_moments_derive(const double* sums, int n_src, double* out);

/* Autotuner of the trace launch: traces a sample of the workload (about sample_photons photons, spread
   over the sources in proportion to their counts) with each candidate (threads per block in {64, 128, 256},
   photons per warp tile in {64, 256, 1024, 4096}), times each on the stream with CUDA events (best of
   two), and keeps the fastest through phosim_set_schedule.  Results never depend on the schedule (the
   random numbers are counter-based), only the speed does.  A sample should give every resident warp several
   tiles of the largest candidate (on a GB300 with the double-single path, 2e8 photons: with 2e7 the large
   tiles' trials end on a ragged last round and small tiles win that the whole workload runs slower).
   out_threads / out_tile may be NULL.
   Errors: as phosim_trace. */
phosim_status phosim_autotune(phosim_scene* scene, const phosim_source* sources, int n_src,
                              const uint64_t* n_photons, uint64_t sample_photons, void* stream,
                              int* out_threads, int* out_tile);

/* Totals of the last phosim_trace: out[0] = photons traced, out[1] = detected, out[1 + r] = dropped for
   reason r = 1..8 (PHOSIM_LOST_*).  n >= 10.  Synchronises the scene's last stream. */
phosim_status phosim_get_counters(phosim_scene* scene, uint64_t* out, int n);

/* Allocation-free variant of phosim_trace (the paper has no counterpart; it exists for callers of this
   library that cannot call cudaMalloc, for example an application whose device memory is owned by an
   outside pool that budgets every byte, or a latency-critical loop where an allocation would synchronise
   the device and stall other work).  Same photons, same kernels and same results as phosim_trace, with
   these differences:
   - its per-call scratch (source list, tile prefix, work counters) lives in one file-scope device array of
     PHOSIM_NOALLOC_SCRATCH_BYTES held by every GPU that loads the library until the process exits; it
     allocates no memory and calls no allocating routine;
   - n_src must be <= PHOSIM_NOALLOC_MAX_SOURCES (else PHOSIM_ERR_LIMIT), and image must be device memory
     (else PHOSIM_ERR_INVALID_ARGUMENT: a host image would need a staging buffer);
   - the first call on a device looks up the array's device address on that device (set-up, once per
     device, with that device current); make that first call before any stream capture;
   - the call copies its source list and tile prefix from host memory that it frees on return, so on a
     stream that is being captured it returns PHOSIM_ERR_INVALID_ARGUMENT and enqueues nothing;
   - every call shares the array and leaves its contents behind; each call clears the counters it needs.
     Calls whose GPU work overlaps (different streams, or different threads on one device) race on the
     array and must be serialised by the caller;
   - records and moments, like image, must be device memory of the scene's device (else INVALID_ARGUMENT);
   - phosim_get_counters does not report its photons, and per-kernel stage timing does not cover it (after
     it, phosim_stage_times reads zero).
   Errors: as phosim_trace, plus LIMIT above. */
#define PHOSIM_NOALLOC_MAX_SOURCES 4096
#define PHOSIM_NOALLOC_SCRATCH_BYTES (1u << 20)
phosim_status phosim_trace_noalloc(phosim_scene* scene, const phosim_source* sources, int n_src,
                                   const uint64_t* n_photons, const uint64_t* first, uint32_t* image,
                                   phosim_photon_record* records, double* moments, void* stream);

/* Saturation and bleeding (Sec. 2.5) as a pass over a finished image: in each half of every row (the halves
   meet at the centre implant, column nx / 2), pixels are visited left to right and electrons above
   full_well move to the closest pixels below full well in that half-row, alternating left then right at
   equal distance; electrons that find no room in the half-row are removed.  image: device, nx * ny,
   updated in place on stream.  removed: NULL or a device uint64 that receives the count of removed
   electrons (added to).  Errors: INVALID_ARGUMENT, CUDA. */
phosim_status phosim_bleed(uint32_t* image, int nx, int ny, uint32_t full_well, unsigned long long* removed,
                           void* stream);

void phosim_destroy_scene(phosim_scene* scene);
const char* phosim_status_string(phosim_status status);

#ifdef __cplusplus
}
#endif
#endif /* PHOSIM_H */
