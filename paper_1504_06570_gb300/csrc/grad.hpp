// Parameters of the adjoint kernel (grad.cu), filled by phosim_grad.
#pragma once

#include "phosim_device.cuh"

namespace phosim {

constexpr int kMaxGradParams = 128;

struct GradParams {
    int n_params;
    int pert_p[PHOSIM_MAX_SURFACES][6];                  // parameter index of misalignment field f, or -1
    int n_zp[PHOSIM_MAX_SURFACES];                       // Zernike parameters of each surface
    int zp_j[PHOSIM_MAX_SURFACES][PHOSIM_MAX_ZERNIKE];   // their Noll index j (1-based)
    int zp_p[PHOSIM_MAX_SURFACES][PHOSIM_MAX_ZERNIKE];   // their parameter index
    int mat_before[PHOSIM_MAX_SURFACES];                 // medium in front of each surface (-1 = vacuum)
    double dM[PHOSIM_MAX_SURFACES][3][9];                // dM/dtx, dM/dty, dM/dtz of each surface
    const double* zmono;                                 // PHOSIM_MAX_ZERNIKE x kZPoly monomials of Z_j
    const double* seeds;                                 // per source: Ax, Ay, Bxx, Bxy, Byy, mean x, mean y, 0
    double* grad;                                        // n_src x n_params, added to
};

cudaError_t launch_grad(const TraceParams& P, const GradParams& G, int blocks, cudaStream_t st);
cudaError_t grad_occupancy(int* blocks_per_sm);

}  // namespace phosim
