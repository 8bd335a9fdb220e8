// Internal interface between the binary-fluid host code (binary2d.cu) and the
// D3Q19 kernels (binary3d.cu).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "binary_common.cuh"

namespace lbb {

// One D3Q19 step from a.src into a.dst: the phi pass into `phi` (one value
// per site), then the fused step; both launches on `st`.
cudaError_t binary_step3(bool forcing, const StepArgs<float>& a, float* phi, cudaStream_t st);
cudaError_t binary_step3(bool forcing, const StepArgs<double>& a, double* phi, cudaStream_t st);

// f = f^eq, g = g^eq of float64 fields rho [N], phi [N], u [3][N] (NULL: 0) into
// the population set `dst` (float32 if f32, else float64).
cudaError_t binary_init3(bool forcing, bool f32, const double* rho, const double* phi, const double* u, void* dst,
                         unsigned pitch, int nx, int ny, int nz, double A, double B, double kappa, double Gamma,
                         cudaStream_t st);

// Observables of the set `src` into the workspace w (15 N doubles): rho, phi,
// u [3], v [3], mu, and (forcing) the six M' fields of the body force.
cudaError_t binary_fields3(bool forcing, bool f32, const void* src, unsigned pitch, int nx, int ny, int nz, double A,
                           double B, double kappa, double* w, cudaStream_t st);

}  // namespace lbb
