// D2Q9 float64 time step with the free parameters of the equilibrium and of
// the stencils given at run time (Sec. III, Eq. 16; the scans of Fig. 2 and
// the prior-art choices of Sec. III).  Three plain kernels per step:
//   rho       rho = sum_i f_i (Eq. 3);
//   stencils  d_x rho, d_y rho (Eq. 10 with A, B), lap rho (Eq. 11 with C, D)
//             and, for the forcing scheme, M'_xx = kappa (G_x^2 - G_y^2)/2,
//             M'_xy = kappa G_x G_y (Sec. VI);
//   collide   f^eq (Eqs. 5, 6) with per-velocity weights w, w^p, w^t, w^ab,
//             g = -div M' with the force stencil (E, F) (Eq. 28), F_i
//             (Eq. 27), BGK relaxation (Eq. 4) and push streaming.
// Used for parameter studies, not for throughput: the fused kernels serve the
// optimum weights.
#include <cuda_runtime.h>

#include "param2d.h"

namespace lbk {
namespace {

// D2Q9 velocities in the paper's order (Sec. II): host copy and device copy
constexpr int EX[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
constexpr int EY[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
__constant__ int c_ex[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
__constant__ int c_ey[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};

__device__ __forceinline__ int wrap(int v, int n) {
    const int r = v % n;
    return r < 0 ? r + n : r;
}

// A field on the 3x3 neighbourhood of a site (periodic lattice).
struct Nbr {
    double c, e, w, n, s, ne, nw, se, sw;
};

__device__ __forceinline__ Nbr gather(const double* a, int x, int y, int nx, int ny) {
    const int xp = wrap(x + 1, nx), xm = wrap(x - 1, nx), yp = wrap(y + 1, ny) * nx, ym = wrap(y - 1, ny) * nx;
    const int yc = y * nx;
    return Nbr{a[yc + x], a[yc + xp], a[yc + xm], a[yp + x], a[ym + x], a[yp + xp], a[yp + xm], a[ym + xp], a[ym + xm]};
}

// Gradient stencil with c1 on the axis neighbours and c2 on the diagonals.
__device__ __forceinline__ double dx_of(const Nbr& v, double c1, double c2) {
    return c1 * (v.e - v.w) + c2 * ((v.ne - v.nw) + (v.se - v.sw));
}

__device__ __forceinline__ double dy_of(const Nbr& v, double c1, double c2) {
    return c1 * (v.n - v.s) + c2 * ((v.ne - v.se) + (v.nw - v.sw));
}

__global__ void p2_rho_kernel(const double* f, long long pitch, int n, double* rho) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        double r = 0.0;
        for (int i = 0; i < 9; ++i) r += f[i * pitch + s];
        rho[s] = r;
    }
}

__global__ void p2_stencil_kernel(const double* rho, int nx, int ny, Free2D w, double kappa, int forcing,
                                  double* gl, double* mp) {
    const int n = nx * ny;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int x = s % nx, y = s / nx;
        const Nbr v = gather(rho, x, y, nx, ny);
        const double gx = dx_of(v, w.gA, w.gB), gy = dy_of(v, w.gA, w.gB);
        const double lap = w.lC * ((v.e + v.w) + (v.n + v.s)) + w.lD * ((v.ne + v.nw) + (v.se + v.sw)) -
                           4.0 * (w.lC + w.lD) * v.c;
        gl[s] = gx;
        gl[n + s] = gy;
        gl[2 * n + s] = lap;
        if (forcing) {
            mp[s] = 0.5 * kappa * (gx * gx - gy * gy);
            mp[n + s] = kappa * gx * gy;
        }
    }
}

// g = -div M' at (x, y) with the force stencil (Eq. 28); M'_yy = -M'_xx.
__device__ __forceinline__ void body_force(const double* mp, int x, int y, int nx, int ny, const Free2D& w,
                                           double& gx, double& gy) {
    const int n = nx * ny;
    const Nbr mxx = gather(mp, x, y, nx, ny), mxy = gather(mp + n, x, y, nx, ny);
    gx = -(dx_of(mxx, w.fE, w.fF) + dy_of(mxy, w.fE, w.fF));
    gy = -(dx_of(mxy, w.fE, w.fF) - dy_of(mxx, w.fE, w.fF));
}

// f^eq_i (i >= 1) of Eq. 5 at one site; feq[0] by Eq. 6.
__device__ __forceinline__ void equilibrium(double rho, const double (&u)[2], double gx, double gy, double lap,
                                            const Free2D& w, const Phys2& ph, int forcing, double (&feq)[9]) {
    const double ib = 1.0 / (1.0 - ph.b * rho);
    const double p0 = rho * ph.T * ib - ph.a * rho * rho;                      // Eq. 2
    const double lam = ph.nu * (1.0 - 3.0 * (ph.T * ib * ib - 2.0 * ph.a * rho));   // Eq. 36
    const double G[2] = {gx, gy};
    const double udg = u[0] * gx + u[1] * gy;
    double S[2][2];
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            S[a][b] = rho * u[a] * u[b] + lam * (u[a] * G[b] + u[b] * G[a] + (a == b ? udg : 0.0));
    double sum = 0.0;
    for (int i = 1; i < 9; ++i) {
        const double e[2] = {double(c_ex[i]), double(c_ey[i])};
        double quad = 0.0;
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) quad += (e[a] * e[b] - (a == b ? 1.0 / 3.0 : 0.0)) * S[a][b];
        double v = w.w[i] * (rho * (e[0] * u[0] + e[1] * u[1]) + 1.5 * quad);
        v += w.wp[i] * p0 - w.wt[i] * ph.kappa * rho * lap;
        if (!forcing) v += ph.kappa * (w.wxx[i] * gx * gx + w.wyy[i] * gy * gy + w.wxy[i] * gx * gy);
        feq[i] = v;
        sum += v;
    }
    feq[0] = rho - sum;
}

__global__ void p2_collide_kernel(const double* src, double* dst, long long pitch, int nx, int ny, const double* rho_a,
                                  const double* gl, const double* mp, Free2D w, Phys2 ph, int forcing,
                                  unsigned* status) {
    const int n = nx * ny;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const int x = s % nx, y = s / nx;
        double f[9];
        for (int i = 0; i < 9; ++i) f[i] = src[i * pitch + s];
        const double rho = rho_a[s];
        if (!(rho > 0.0) || !(rho < 1e30)) atomicOr(status, 1u);
        double j[2] = {0.0, 0.0};
        for (int i = 1; i < 9; ++i) {
            j[0] += f[i] * c_ex[i];
            j[1] += f[i] * c_ey[i];
        }
        const double u[2] = {j[0] / rho, j[1] / rho};
        double feq[9];
        equilibrium(rho, u, gl[s], gl[n + s], gl[2 * n + s], w, ph, forcing, feq);
        double F[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        if (forcing) {
            double g[2];
            body_force(mp, x, y, nx, ny, w, g[0], g[1]);
            double sumF = 0.0;
            for (int i = 1; i < 9; ++i) {
                const double e[2] = {double(c_ex[i]), double(c_ey[i])};
                double quad = 0.0;
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b)
                        quad += (e[a] * e[b] - (a == b ? 1.0 / 3.0 : 0.0)) * (u[a] * g[b] + u[b] * g[a]);
                F[i] = w.w[i] * ((e[0] * g[0] + e[1] * g[1]) + 1.5 * quad);   // Eq. 27
                sumF += F[i];
            }
            F[0] = -sumF;
        }
        for (int i = 0; i < 9; ++i) {
            const double out = f[i] + ph.omega * (feq[i] - f[i]) + F[i];
            const int xd = wrap(x + c_ex[i], nx), yd = wrap(y + c_ey[i], ny);
            dst[i * pitch + yd * nx + xd] = out;
        }
    }
}

__global__ void p2_init_kernel(double* dst, long long pitch, int nx, int ny, const double* rho_a, const double* u_a,
                               const double* gl, Free2D w, Phys2 ph, int forcing) {
    const int n = nx * ny;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        const double u[2] = {u_a ? u_a[s] : 0.0, u_a ? u_a[n + s] : 0.0};
        double feq[9];
        equilibrium(rho_a[s], u, gl[s], gl[n + s], gl[2 * n + s], w, ph, forcing, feq);
        for (int i = 0; i < 9; ++i) dst[i * pitch + s] = feq[i];
    }
}

__global__ void p2_velocity_v_kernel(const double* rho_a, const double* u_a, const double* mp, int nx, int ny,
                                     Free2D w, double* v) {
    const int n = nx * ny;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        double g[2];
        body_force(mp, s % nx, s / nx, nx, ny, w, g[0], g[1]);
        const double h = 0.5 / rho_a[s];                 // v = u + g/(2 rho), Eq. 40
        v[s] = u_a[s] + h * g[0];
        v[n + s] = u_a[n + s] + h * g[1];
    }
}

unsigned blocks_for(int n) {
    int b = (n + 255) / 256;
    return unsigned(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

Free2D free2d_weights(double wp58, double wt58, double wxx58, double B, double D, double F) {
    Free2D w{};
    for (int i = 1; i < 9; ++i) {
        const bool diag = EX[i] != 0 && EY[i] != 0;
        const bool xaxis = !diag && EX[i] != 0;
        // velocity weights (after Eq. 5); w^p, w^t with 2 w_{1-4} + 4 w_{5-8} = 1 (after Eq. 15)
        w.w[i] = diag ? 1.0 / 12.0 : 1.0 / 3.0;
        w.wp[i] = diag ? wp58 : 0.5 - 2.0 * wp58;
        w.wt[i] = diag ? wt58 : 0.5 - 2.0 * wt58;
        // w^xx: 2 w^xx_{1,2} + 4 w^xx_{5-8} = 1/2, w^yy: 2 w^yy_{1,2} + 4 w^yy_{5-8} = -1/2 with
        // w^yy_{5-8} = w^xx_{5-8}; w^xx on the y axis equals w^yy on the x axis (after Eq. 14)
        const double own = 0.25 - 2.0 * wxx58, other = -0.25 - 2.0 * wxx58;
        w.wxx[i] = diag ? wxx58 : (xaxis ? own : other);
        w.wyy[i] = diag ? wxx58 : (xaxis ? other : own);
        w.wxy[i] = diag ? 0.25 * EX[i] * EY[i] : 0.0;     // sign(e_x e_y)/4 (Sec. II)
    }
    // stencils: 2A + 4B = 1 (Eq. 10), C + 2D = 1 (Eq. 11), force stencil 2E + 4F = 1
    w.gB = B;
    w.gA = 0.5 - 2.0 * B;
    w.lD = D;
    w.lC = 1.0 - 2.0 * D;
    w.fF = F;
    w.fE = 0.5 - 2.0 * F;
    return w;
}

cudaError_t free2d_step(const Free2D& w, const Phys2& ph, int forcing, const double* src, double* dst,
                        long long pitch, int nx, int ny, double* rho, double* gl, double* mp, unsigned* status,
                        cudaStream_t st) {
    const int n = nx * ny;
    const unsigned nb = blocks_for(n);
    p2_rho_kernel<<<nb, 256, 0, st>>>(src, pitch, n, rho);
    p2_stencil_kernel<<<nb, 256, 0, st>>>(rho, nx, ny, w, ph.kappa, forcing, gl, mp);
    p2_collide_kernel<<<nb, 256, 0, st>>>(src, dst, pitch, nx, ny, rho, gl, mp, w, ph, forcing, status);
    return cudaGetLastError();
}

cudaError_t free2d_init(const Free2D& w, const Phys2& ph, int forcing, double* dst, long long pitch, int nx, int ny,
                        const double* rho, const double* u, double* gl, double* mp, cudaStream_t st) {
    const int n = nx * ny;
    const unsigned nb = blocks_for(n);
    p2_stencil_kernel<<<nb, 256, 0, st>>>(rho, nx, ny, w, ph.kappa, 0, gl, mp);
    p2_init_kernel<<<nb, 256, 0, st>>>(dst, pitch, nx, ny, rho, u, gl, w, ph, forcing);
    return cudaGetLastError();
}

cudaError_t free2d_velocity_v(const Free2D& w, double kappa, const double* rho, const double* u, int nx, int ny,
                              double* gl, double* mp, double* v, cudaStream_t st) {
    const int n = nx * ny;
    const unsigned nb = blocks_for(n);
    p2_stencil_kernel<<<nb, 256, 0, st>>>(rho, nx, ny, w, kappa, 1, gl, mp);
    p2_velocity_v_kernel<<<nb, 256, 0, st>>>(rho, u, mp, nx, ny, w, v);
    return cudaGetLastError();
}

}  // namespace lbk
