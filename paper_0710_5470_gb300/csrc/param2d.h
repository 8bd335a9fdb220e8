// Internal interface of the run-time-parameter D2Q9 step (param2d.cu).  Not
// part of the C ABI.
#pragma once
#include <cuda_runtime.h>

namespace lbk {

// Per-velocity weights of Eq. 5 (w, w^p, w^t, w^xx, w^yy, w^xy; index 0
// unused) and the coefficients of the gradient (A, B), Laplacian (C, D) and
// force (E, F) stencils.
struct Free2D {
    double w[9], wp[9], wt[9], wxx[9], wyy[9], wxy[9];
    double gA, gB, lC, lD, fE, fF;
};

struct Phys2 {
    double a, b, T, kappa, omega, nu;
};

// Weights and stencils from the free parameters w^p_{5-8}, w^t_{5-8},
// w^xx_{5-8}, B, D, F and the constraints of Secs. II-III.
Free2D free2d_weights(double wp58, double wt58, double wxx58, double B, double D, double F);

// One time step src -> dst (float64 SoA, population i at i * pitch).  rho (N),
// gl (3N) and mp (2N) are scratch; status bit 0 is set on a non-finite or
// non-positive density.
cudaError_t free2d_step(const Free2D& w, const Phys2& ph, int forcing, const double* src, double* dst,
                        long long pitch, int nx, int ny, double* rho, double* gl, double* mp, unsigned* status,
                        cudaStream_t st);

// dst = f^eq(rho, u) with these weights and stencils (u may be null: u = 0).
cudaError_t free2d_init(const Free2D& w, const Phys2& ph, int forcing, double* dst, long long pitch, int nx, int ny,
                        const double* rho, const double* u, double* gl, double* mp, cudaStream_t st);

// v = u + g/(2 rho) (Eq. 40) with the force stencil of w.
cudaError_t free2d_velocity_v(const Free2D& w, double kappa, const double* rho, const double* u, int nx, int ny,
                              double* gl, double* mp, double* v, cudaStream_t st);

}  // namespace lbk
