// Binary-fluid free-energy lattice Boltzmann on D3Q19 (the model stated in
// include/lb.h beside lb_binary_params; Sec. VII's weights and stencils, the
// forcing scheme in 3D by reading R7).
//
// Two launches per time step:
//   binary_phi_kernel     phi = sum_i g_i of every site (19 reads, one write);
//   binary_step_kernel3   one CTA per 32 x 4 x 2 brick, one site per thread:
//     the brick's phi plus a halo (1 site for the equilibrium scheme, 2 for
//     the forcing scheme) from the phi field into shared memory; the own
//     site's 19 f and 19 g into registers; (forcing) M'_ab - delta_ab M'_cc / 2
//     with M'_ab = kappa d_a phi d_b phi on the brick plus one ring; the
//     gradient and Laplacian of phi (Eq. 29 with A = 1/6, B = 1/12, C = 1/3,
//     D = 1/6); rho, u, mu, p0, f^eq, the body force g_a = -d_b (M'_ab -
//     delta_ab M'_cc / 2) with F_i (Eq. 27) and v (Eq. 40), g^eq with v, both
//     relaxations and the push of f* and g* to r + e_i in the other buffer.
// A site's phi depends on the g that 18 neighbours push into it, so it cannot
// be formed by the step that writes them: the phi pass adds one read of the
// 19 g and a write of phi per update (HBM: 2 x 38 x s + 19 s + s bytes, s the
// element size; 384 B per update in float32 against the 304 B the step moves).
#include <cuda_runtime.h>

#include "binary_common.cuh"
#include "binary_launch.h"

namespace lbb {

constexpr int Q3 = 19;
constexpr int BX = 32, BY = 4;
// Brick depth: 2 planes (256 threads).  Measured on GB300 at 128^3, float32:
// forcing 8.7 GLUPS (1711 instructions per update), equilibrium 11.2; 4 planes
// (512 threads, one CTA of 16 warps per SM; less halo and ring per site) ran
// 7.8 / 9.6.  float64 (238 registers a thread) has room for 256 threads only.
template <class real>
constexpr int brick_z() { return 2; }

template <class real>
__global__ void binary_phi_kernel(const real* src, unsigned pitch, unsigned n, real* phi) {
    for (unsigned s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        real p = 0;
#pragma unroll
        for (int i = 0; i < Q3; ++i) p += src[(Q3 + i) * pitch + s];
        phi[s] = p;
    }
}

// d_A of a field stored with strides 1, SY_ (y) and SZ_ (z) at index c: the
// gradient stencil of Eq. 29 (A = 1/6 on the axis pair, B = 1/12 on the four
// diagonal pairs with e_A != 0), opposite velocities differenced first.
template <int A, int SY_, int SZ_, class real>
__device__ __forceinline__ real dgrad(const real* p, int c) {
    real ax = real(0), dg = real(0);
    static_for<1, Q3>([&](auto K) {
        constexpr int i = decltype(K)::value;
        constexpr int ex = D3Q19::ex(i), ey = D3Q19::ey(i), ez = D3Q19::ez(i);
        constexpr int e = A == 0 ? ex : (A == 1 ? ey : ez);
        if constexpr (e > 0) {   // i with e_A = +1; its opposite is -e_i
            constexpr int off = ex + ey * SY_ + ez * SZ_;
            const real d = p[c + off] - p[c - off];
            if constexpr (ex * ex + ey * ey + ez * ez == 1) ax = ax + d;
            else dg = dg + d;
        }
    });
    return real(1.0 / 6.0) * ax + real(1.0 / 12.0) * dg;
}

// Laplacian of Eq. 29: 2 sum_i w_i (p(r + e_i) - p(r)) = 1/3 sum_axis + 1/6 sum_diag - 4 p(r).
template <int SY_, int SZ_, class real>
__device__ __forceinline__ real dlap(const real* p, int c) {
    real ax = real(0), dg = real(0);
    static_for<1, Q3>([&](auto K) {
        constexpr int i = decltype(K)::value;
        constexpr int ex = D3Q19::ex(i), ey = D3Q19::ey(i), ez = D3Q19::ez(i);
        constexpr int off = ex + ey * SY_ + ez * SZ_;
        if constexpr (ex * ex + ey * ey + ez * ez == 1) ax = ax + p[c + off];
        else dg = dg + p[c + off];
    });
    return real(1.0 / 3.0) * ax + real(1.0 / 6.0) * dg - real(4) * p[c];
}

// Body force of the forcing scheme from the six fields Mt_ab = M'_ab - delta_ab
// M'_cc / 2 (xx, yy, zz, xy, xz, yz, each `sn` long): g_a = -sum_b d_b Mt_ab.
template <int SY_, int SZ_, class real>
__device__ __forceinline__ void body_force3(const real* mt, int sn, int k, real (&g)[3]) {
    const real* xx = mt;
    const real* yy = mt + sn;
    const real* zz = mt + 2 * sn;
    const real* xy = mt + 3 * sn;
    const real* xz = mt + 4 * sn;
    const real* yz = mt + 5 * sn;
    g[0] = -((dgrad<0, SY_, SZ_>(xx, k) + dgrad<1, SY_, SZ_>(xy, k)) + dgrad<2, SY_, SZ_>(xz, k));
    g[1] = -((dgrad<0, SY_, SZ_>(xy, k) + dgrad<1, SY_, SZ_>(yy, k)) + dgrad<2, SY_, SZ_>(yz, k));
    g[2] = -((dgrad<0, SY_, SZ_>(xz, k) + dgrad<1, SY_, SZ_>(yz, k)) + dgrad<2, SY_, SZ_>(zz, k));
}

template <bool FORCING, class real>
struct Step3Layout {
    static constexpr int H = FORCING ? 2 : 1;
    static constexpr int BZ = brick_z<real>(), NT = BX * BY * BZ;
    static constexpr int RX = BX + 2 * H, RY = BY + 2 * H, RZ = BZ + 2 * H, RN = RX * RY * RZ;
    static constexpr int SX = BX + 2, SY = BY + 2, SZ = BZ + 2, SN = SX * SY * SZ;
    static constexpr size_t BYTES = sizeof(real) * (RN + (FORCING ? 6 * SN : 0));
};

// float32: three resident CTAs per SM (80 registers, no spills; the collision
// streams population by population so f^eq, F and g^eq are never held as
// arrays); float64 has room for one.
template <bool FORCING, class real>
__global__ void __launch_bounds__(BX * BY * brick_z<real>(), sizeof(real) == 4 ? 3 : 1)
    binary_step_kernel3(const StepArgs<real> a) {
    using Lay = Step3Layout<FORCING, real>;
    constexpr int H = Lay::H, RX = Lay::RX, RY = Lay::RY, RN = Lay::RN;
    constexpr int SX = Lay::SX, SY = Lay::SY, SN = Lay::SN;
    extern __shared__ __align__(16) unsigned char smem3[];
    real* phs = reinterpret_cast<real*>(smem3);
    real* mt = phs + RN;

    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const unsigned pitch = a.pitch;
    const int tx = threadIdx.x % BX, ty = (threadIdx.x / BX) % BY, tz = threadIdx.x / (BX * BY);
    constexpr int BZ = Lay::BZ, NT3 = Lay::NT;
    const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY, z0 = blockIdx.z * BZ;
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool own = x < nx && y < ny && z < nz;

    real f[Q3], g[Q3];
    if (own) {
        const unsigned s = (unsigned(z) * unsigned(ny) + unsigned(y)) * unsigned(nx) + unsigned(x);
#pragma unroll
        for (int i = 0; i < Q3; ++i) {
            f[i] = a.src[i * pitch + s];
            g[i] = a.src[(Q3 + i) * pitch + s];
        }
    }
    {
        // a warp per region row (y, z), its lanes along x: row offsets and wraps
        // once per row, the x wrap per element
        const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
        constexpr int NW = NT3 / 32;
        static_assert(RX <= 64, "two elements per lane cover a region row");
        const unsigned xa = unsigned(wrapc(x0 - H + lane, nx));
        const unsigned xb = lane + 32 < RX ? unsigned(wrapc(x0 - H + lane + 32, nx)) : 0u;
        for (int row = warp; row < RY * Lay::RZ; row += NW) {
            const int ry = row % RY, rz = row / RY;
            const unsigned base = (unsigned(wrapc(z0 - H + rz, nz)) * unsigned(ny) + unsigned(wrapc(y0 - H + ry, ny))) *
                                  unsigned(nx);
            phs[row * RX + lane] = a.phi[base + xa];
            if (lane + 32 < RX) phs[row * RX + lane + 32] = a.phi[base + xb];
        }
    }
    __syncthreads();

    if constexpr (FORCING) {
        for (int k = threadIdx.x; k < SN; k += NT3) {
            const int sx = k % SX, sy = (k / SX) % SY, sz = k / (SX * SY);
            const int c = ((sz - 1 + H) * RY + (sy - 1 + H)) * RX + (sx - 1 + H);
            const real gx = dgrad<0, RX, RX * RY>(phs, c), gy = dgrad<1, RX, RX * RY>(phs, c),
                       gz = dgrad<2, RX, RX * RY>(phs, c);
            const real htr = real(0.5) * ((gx * gx + gy * gy) + gz * gz);
            mt[k] = a.kappa * (gx * gx - htr);
            mt[SN + k] = a.kappa * (gy * gy - htr);
            mt[2 * SN + k] = a.kappa * (gz * gz - htr);
            mt[3 * SN + k] = a.kappa * (gx * gy);
            mt[4 * SN + k] = a.kappa * (gx * gz);
            mt[5 * SN + k] = a.kappa * (gy * gz);
        }
    }
    const int c = ((tz + H) * RY + ty + H) * RX + tx + H;
    const real gr[3] = {dgrad<0, RX, RX * RY>(phs, c), dgrad<1, RX, RX * RY>(phs, c), dgrad<2, RX, RX * RY>(phs, c)};
    const real lap = dlap<RX, RX * RY>(phs, c);
    const real phi = phs[c];
    if constexpr (FORCING) __syncthreads();

    bool bad = false;
    if (own) {
        real rho = 0, j[3] = {0, 0, 0};
        static_for<0, Q3>([&](auto K) {
            constexpr int i = decltype(K)::value;
            rho += f[i];
            j[0] = signed_add<D3Q19::ex(i)>(j[0], f[i]);
            j[1] = signed_add<D3Q19::ey(i)>(j[1], f[i]);
            j[2] = signed_add<D3Q19::ez(i)>(j[2], f[i]);
        });
        bad = !(rho > real(0)) || !isfinite(rho);
        const real ir = real(1) / rho;
        const real u[3] = {j[0] * ir, j[1] * ir, j[2] * ir};
        const real mu = a.A * phi + a.B * phi * phi * phi - a.kappa * lap;
        real v[3] = {u[0], u[1], u[2]}, bf[3] = {0, 0, 0};
        if constexpr (FORCING) {
            const int k = ((tz + 1) * SY + ty + 1) * SX + tx + 1;
            body_force3<SX, SX * SY>(mt, SN, k, bf);
            const real hir = real(0.5) * ir;
#pragma unroll
            for (int d = 0; d < 3; ++d) v[d] = u[d] + bf[d] * hir;   // Eq. 40
        }
        const int xw[3] = {wrapc(x - 1, nx), x, wrapc(x + 1, nx)};
        const unsigned yz[3][3] = {
            {(unsigned(wrapc(z - 1, nz)) * ny + unsigned(wrapc(y - 1, ny))) * unsigned(nx),
             (unsigned(wrapc(z - 1, nz)) * ny + unsigned(y)) * unsigned(nx),
             (unsigned(wrapc(z - 1, nz)) * ny + unsigned(wrapc(y + 1, ny))) * unsigned(nx)},
            {(unsigned(z) * ny + unsigned(wrapc(y - 1, ny))) * unsigned(nx), (unsigned(z) * ny + unsigned(y)) * unsigned(nx),
             (unsigned(z) * ny + unsigned(wrapc(y + 1, ny))) * unsigned(nx)},
            {(unsigned(wrapc(z + 1, nz)) * ny + unsigned(wrapc(y - 1, ny))) * unsigned(nx),
             (unsigned(wrapc(z + 1, nz)) * ny + unsigned(y)) * unsigned(nx),
             (unsigned(wrapc(z + 1, nz)) * ny + unsigned(wrapc(y + 1, ny))) * unsigned(nx)}};
        collide_stream<D3Q19, FORCING>(f, g, rho, u, phi, gr, lap, bf, v, mu, a.A, a.B, a.kappa, a.Gamma, a.omega,
                                       a.omega_phi, [&](auto K, real fs, real gs) {
                                           constexpr int i = decltype(K)::value;
                                           constexpr int ex = D3Q19::ex(i), ey = D3Q19::ey(i), ez = D3Q19::ez(i);
                                           const unsigned d = yz[1 + ez][1 + ey] + unsigned(xw[1 + ex]);
                                           a.dst[i * pitch + d] = fs;
                                           a.dst[(Q3 + i) * pitch + d] = gs;
                                       });
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x % 32) == 0) atomicOr(a.status, 1u);
}

// Reads the 3 x 3 x 3 periodic neighbourhood of site (x, y, z) of a float64 field.
__device__ __forceinline__ void neighbourhood(const double* f, int x, int y, int z, int nx, int ny, int nz,
                                              double (&p)[27]) {
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                p[((dz + 1) * 3 + dy + 1) * 3 + dx + 1] =
                    f[(size_t(wrapc(z + dz, nz)) * ny + wrapc(y + dy, ny)) * nx + wrapc(x + dx, nx)];
}

template <bool FORCING, class real>
__global__ void binary_init_kernel3(const double* rho, const double* phi, const double* u, real* dst, unsigned pitch,
                                    int nx, int ny, int nz, double A, double B, double kappa, double Gamma) {
    const size_t n = size_t(nx) * ny * nz;
    for (size_t s = blockIdx.x * size_t(blockDim.x) + threadIdx.x; s < n; s += size_t(gridDim.x) * blockDim.x) {
        const int x = int(s % nx), y = int((s / nx) % ny), z = int(s / (size_t(nx) * ny));
        double p[27];
        neighbourhood(phi, x, y, z, nx, ny, nz, p);
        const double gr[3] = {dgrad<0, 3, 9>(p, 13), dgrad<1, 3, 9>(p, 13), dgrad<2, 3, 9>(p, 13)};
        const double lap = dlap<3, 9>(p, 13);
        const double mu = A * p[13] + B * p[13] * p[13] * p[13] - kappa * lap;
        const double uu[3] = {u ? u[s] : 0.0, u ? u[n + s] : 0.0, u ? u[2 * n + s] : 0.0};
        double fe[Q3], ge[Q3];
        f_equilibrium<D3Q19, !FORCING>(rho[s], uu, p[13], gr, lap, A, B, kappa, fe);
        g_equilibrium<D3Q19>(p[13], uu, mu, Gamma, ge);
        for (int i = 0; i < Q3; ++i) {
            dst[i * size_t(pitch) + s] = real(fe[i]);
            dst[(Q3 + i) * size_t(pitch) + s] = real(ge[i]);
        }
    }
}

// Observables in float64: rho, phi, u (3 components) of the stored state.
template <class real>
__global__ void binary_moments_kernel3(const real* src, unsigned pitch, size_t n, double* rho, double* phi, double* u) {
    for (size_t s = blockIdx.x * size_t(blockDim.x) + threadIdx.x; s < n; s += size_t(gridDim.x) * blockDim.x) {
        double r = 0, p = 0, j[3] = {0, 0, 0};
        for (int i = 0; i < Q3; ++i) {
            const double fi = double(src[i * size_t(pitch) + s]);
            r += fi;
            j[0] += D3Q19::ex(i) * fi;
            j[1] += D3Q19::ey(i) * fi;
            j[2] += D3Q19::ez(i) * fi;
            p += double(src[(Q3 + i) * size_t(pitch) + s]);
        }
        rho[s] = r;
        phi[s] = p;
        for (int d = 0; d < 3; ++d) u[d * n + s] = j[d] / r;
    }
}

// mu and (forcing) the six Mt_ab fields.
__global__ void binary_mu_kernel3(const double* phi, int nx, int ny, int nz, double A, double B, double kappa,
                                  double* mu, double* mt) {
    const size_t n = size_t(nx) * ny * nz;
    for (size_t s = blockIdx.x * size_t(blockDim.x) + threadIdx.x; s < n; s += size_t(gridDim.x) * blockDim.x) {
        const int x = int(s % nx), y = int((s / nx) % ny), z = int(s / (size_t(nx) * ny));
        double p[27];
        neighbourhood(phi, x, y, z, nx, ny, nz, p);
        mu[s] = A * p[13] + B * p[13] * p[13] * p[13] - kappa * dlap<3, 9>(p, 13);
        if (mt) {
            const double gx = dgrad<0, 3, 9>(p, 13), gy = dgrad<1, 3, 9>(p, 13), gz = dgrad<2, 3, 9>(p, 13);
            const double htr = 0.5 * ((gx * gx + gy * gy) + gz * gz);
            mt[s] = kappa * (gx * gx - htr);
            mt[n + s] = kappa * (gy * gy - htr);
            mt[2 * n + s] = kappa * (gz * gz - htr);
            mt[3 * n + s] = kappa * (gx * gy);
            mt[4 * n + s] = kappa * (gx * gz);
            mt[5 * n + s] = kappa * (gy * gz);
        }
    }
}

// v = u + g / (2 rho) (Eq. 40) with g = -d_b Mt_ab from the Mt fields.
__global__ void binary_velocity_kernel3(const double* rho, const double* u, const double* mt, int nx, int ny, int nz,
                                        double* v) {
    const size_t n = size_t(nx) * ny * nz;
    for (size_t s = blockIdx.x * size_t(blockDim.x) + threadIdx.x; s < n; s += size_t(gridDim.x) * blockDim.x) {
        const int x = int(s % nx), y = int((s / nx) % ny), z = int(s / (size_t(nx) * ny));
        double m[6 * 27];
        for (int c = 0; c < 6; ++c) {
            double p[27];
            neighbourhood(mt + c * n, x, y, z, nx, ny, nz, p);
            for (int k = 0; k < 27; ++k) m[c * 27 + k] = p[k];
        }
        double g[3];
        body_force3<3, 9>(m, 27, 13, g);
        for (int d = 0; d < 3; ++d) v[d * n + s] = u[d * n + s] + g[d] / (2.0 * rho[s]);
    }
}

namespace {
inline unsigned blocks3(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 8192) b = 8192;
    return unsigned(b < 1 ? 1 : b);
}

template <bool FORCING, class real>
cudaError_t step3_impl(const StepArgs<real>& a, real* phi_buf, cudaStream_t st) {
    using Lay = Step3Layout<FORCING, real>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(binary_step_kernel3<FORCING, real>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(Lay::BYTES));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const unsigned n = unsigned(a.nx) * unsigned(a.ny) * unsigned(a.nz);
    binary_phi_kernel<real><<<blocks3(n), 256, 0, st>>>(a.src, a.pitch, n, phi_buf);
    StepArgs<real> b = a;
    b.phi = phi_buf;
    const dim3 grid((a.nx + BX - 1) / BX, (a.ny + BY - 1) / BY, (a.nz + Lay::BZ - 1) / Lay::BZ);
    binary_step_kernel3<FORCING, real><<<grid, Lay::NT, Lay::BYTES, st>>>(b);
    return cudaGetLastError();
}
}  // namespace

cudaError_t binary_step3(bool forcing, const StepArgs<float>& a, float* phi, cudaStream_t st) {
    return forcing ? step3_impl<true>(a, phi, st) : step3_impl<false>(a, phi, st);
}
cudaError_t binary_step3(bool forcing, const StepArgs<double>& a, double* phi, cudaStream_t st) {
    return forcing ? step3_impl<true>(a, phi, st) : step3_impl<false>(a, phi, st);
}

cudaError_t binary_init3(bool forcing, bool f32, const double* rho, const double* phi, const double* u, void* dst,
                         unsigned pitch, int nx, int ny, int nz, double A, double B, double kappa, double Gamma,
                         cudaStream_t st) {
    const unsigned nb = blocks3(size_t(nx) * ny * nz);
    if (f32) {
        float* d = static_cast<float*>(dst);
        if (forcing) binary_init_kernel3<true, float><<<nb, 256, 0, st>>>(rho, phi, u, d, pitch, nx, ny, nz, A, B, kappa, Gamma);
        else binary_init_kernel3<false, float><<<nb, 256, 0, st>>>(rho, phi, u, d, pitch, nx, ny, nz, A, B, kappa, Gamma);
    } else {
        double* d = static_cast<double*>(dst);
        if (forcing) binary_init_kernel3<true, double><<<nb, 256, 0, st>>>(rho, phi, u, d, pitch, nx, ny, nz, A, B, kappa, Gamma);
        else binary_init_kernel3<false, double><<<nb, 256, 0, st>>>(rho, phi, u, d, pitch, nx, ny, nz, A, B, kappa, Gamma);
    }
    return cudaGetLastError();
}

cudaError_t binary_fields3(bool forcing, bool f32, const void* src, unsigned pitch, int nx, int ny, int nz, double A,
                           double B, double kappa, double* w, cudaStream_t st) {
    const size_t n = size_t(nx) * ny * nz;
    const unsigned nb = blocks3(n);
    double *rho = w, *phi = w + n, *u = w + 2 * n, *v = w + 5 * n, *mu = w + 8 * n, *mt = w + 9 * n;
    if (f32) binary_moments_kernel3<float><<<nb, 256, 0, st>>>(static_cast<const float*>(src), pitch, n, rho, phi, u);
    else binary_moments_kernel3<double><<<nb, 256, 0, st>>>(static_cast<const double*>(src), pitch, n, rho, phi, u);
    binary_mu_kernel3<<<nb, 256, 0, st>>>(phi, nx, ny, nz, A, B, kappa, mu, forcing ? mt : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (forcing) {
        binary_velocity_kernel3<<<nb, 256, 0, st>>>(rho, u, mt, nx, ny, nz, v);
        return cudaGetLastError();
    }
    return cudaMemcpyAsync(v, u, 3 * n * sizeof(double), cudaMemcpyDeviceToDevice, st);
}

}  // namespace lbb
