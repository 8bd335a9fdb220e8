// Per-run and diagnostic kernels around the fused step: drop initialisation,
// equilibrium initialisation, moments, the body force for v (Eq. 40),
// population import/export and float64 reductions.  None of these is on the
// per-step path; they read and write global memory directly.
#pragma once
#include "field_reduce.cuh"
#include "step_kernel.cuh"

namespace lbk {

// Population arrays of one buffer.  aos = 0: population i is one array,
// element q at p[i] + q * size.  aos = 1 (16-bit deviations, nx a multiple of
// 32): populations 1..18 are interleaved in blocks of 32 sites (the 18 rows
// of 32 values of a block contiguous, 1152 bytes), p[i] points at population
// i's row of block 0, and element q is at half index aos_index(q) from it;
// population 0 stays one float32 array.
struct PopPtrs {
    char* p[MAXQ];
    float fref[MAXQ];
    int aos = 0;
};

constexpr int AOS_SITES = 32;                        // sites per block
constexpr int AOS_BLOCK_HALVES = 18 * AOS_SITES;     // 16-bit values per block

__host__ __device__ __forceinline__ size_t aos_index(size_t q) {
    return (q / AOS_SITES) * AOS_BLOCK_HALVES + (q % AOS_SITES);
}

// element index of population i at site q in its array pointer's units
__host__ __device__ __forceinline__ size_t pop_index(const PopPtrs& pp, int i, size_t q) {
    return (pp.aos && i > 0) ? aos_index(q) : q;
}

struct Grid3 {
    int nx, ny, nz;
    __device__ __forceinline__ size_t n() const { return size_t(nx) * ny * nz; }
    __device__ __forceinline__ void xyz(size_t idx, int& x, int& y, int& z) const {
        x = int(idx % nx);
        y = int((idx / nx) % ny);
        z = int(idx / (size_t(nx) * ny));
    }
    __device__ __forceinline__ size_t at(int x, int y, int z) const {
        return (size_t(wrapi(z, nz)) * ny + wrapi(y, ny)) * nx + wrapi(x, nx);
    }
};

// Density of one or more drops: rho_g + (rho_l - rho_g) max_k 1/2 (1 + tanh((R_k - d_k)/w)),
// d_k the periodic minimum-image distance of the site from centre k.
static __global__ void drop_density_kernel(double* rho, Grid3 g, int dim, int ndrops, const double* centres,
                                    const double* radii, double width, double rho_l, double rho_g) {
    const size_t n = g.n();
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < n; idx += size_t(gridDim.x) * blockDim.x) {
        int x, y, z;
        g.xyz(idx, x, y, z);
        const double c[3] = {double(x), double(y), double(z)};
        const double sz[3] = {double(g.nx), double(g.ny), double(g.nz)};
        double prof = 0.0;
        for (int k = 0; k < ndrops; ++k) {
            double d2 = 0.0;
            for (int a = 0; a < dim; ++a) {
                double dd = fabs(c[a] - centres[k * dim + a]);
                dd = fmin(dd, sz[a] - dd);
                d2 += dd * dd;
            }
            const double pk = 0.5 * (1.0 + tanh((radii[k] - sqrt(d2)) / width));
            prof = fmax(prof, pk);
        }
        rho[idx] = rho_g + (rho_l - rho_g) * prof;
    }
}

// Gradient and Laplacian of a float64 field at one site (stencils of
// Eq. 32 / Eq. 29 written as weighted sums over the velocity set).
template <class L>
__device__ __forceinline__ void stencils_global(const double* rho, Grid3 g, int x, int y, int z, double (&G)[3],
                                                double& lap) {
    G[0] = G[1] = G[2] = 0.0;
    lap = 0.0;
    const double r0 = rho[g.at(x, y, z)];
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
        const double rn = rho[g.at(x + L::ex(i), y + L::ey(i), z + L::ez(i))];
        const double wi = w_vel<L>(i);
#pragma unroll
        for (int c = 0; c < L::D; ++c) {
            if (e_comp<L>(i, c) == 1) G[c] += wi * rn;
            if (e_comp<L>(i, c) == -1) G[c] -= wi * rn;
        }
        lap += wi * (rn - r0);
    }
    lap *= 2.0;
}

struct Phys {
    double a, b, T, kappa, nu;
};

// f = f^eq(rho, u) of the chosen scheme (no force applied), float64 math.
template <class L, bool FORCING, class S>
__global__ void init_feq_kernel(const double* rho, const double* u, PopPtrs dst, Grid3 g, Phys ph) {
    const size_t n = g.n();
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < n; idx += size_t(gridDim.x) * blockDim.x) {
        int x, y, z;
        g.xyz(idx, x, y, z);
        double G[3], lap;
        stencils_global<L>(rho, g, x, y, z, G, lap);
        const double r = rho[idx];
        double uu[3] = {0.0, 0.0, 0.0}, j[3] = {0.0, 0.0, 0.0};
        if (u) {
            for (int c = 0; c < L::D; ++c) {
                uu[c] = u[c * n + idx];
                j[c] = r * uu[c];
            }
        }
        double feq[L::Q];
        equilibrium<L, FORCING, double>(r, j, uu, G, lap, ph.a, ph.b, ph.T, ph.kappa, ph.nu, feq);
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            S::store(i, dst.p[i], pop_index(dst, i, idx), typename S::real(feq[i]), dst.fref[i]);
    }
}

// rho, u (Eq. 3) of the stored populations, float64 outputs.
template <class L, class S>
__global__ void moments_kernel(PopPtrs src, Grid3 g, double* rho, double* u) {
    const size_t n = g.n();
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < n; idx += size_t(gridDim.x) * blockDim.x) {
        double f[L::Q];
        double r = 0.0;
#pragma unroll
        for (int i = 0; i < L::Q; ++i) {
            f[i] = double(S::load(i, src.p[i], pop_index(src, i, idx), src.fref[i]));
            r += f[i];
        }
        double j[3];
        momentum<L, double>(f, j);
        rho[idx] = r;
        for (int c = 0; c < L::D; ++c) u[c * n + idx] = j[c] / r;
    }
}

// M'_ab = kappa (G_a G_b - delta_ab |G|^2 / 2) of the density field.
template <class L>
__global__ void mprime_kernel(const double* rho, Grid3 g, double kappa, double* mp) {
    const size_t n = g.n();
    constexpr int NMC = L::D == 3 ? 6 : 3;
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < n; idx += size_t(gridDim.x) * blockDim.x) {
        int x, y, z;
        g.xyz(idx, x, y, z);
        double G[3], lap;
        stencils_global<L>(rho, g, x, y, z, G, lap);
        double g2 = 0.0;
        for (int c = 0; c < L::D; ++c) g2 += G[c] * G[c];
        for (int c = 0; c < L::D; ++c)
            for (int d = c; d < L::D; ++d) {
                double v = kappa * G[c] * G[d];
                if (c == d) v -= 0.5 * kappa * g2;
                mp[size_t(mcomp<L::D>(c, d)) * n + idx] = v;
            }
        (void)NMC;
    }
}

// g = -div M' (Eq. 28) and v = u + g/(2 rho) (Eq. 40).
template <class L>
__global__ void velocity_v_kernel(const double* rho, const double* u, const double* mp, Grid3 g, double* v) {
    const size_t n = g.n();
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < n; idx += size_t(gridDim.x) * blockDim.x) {
        int x, y, z;
        g.xyz(idx, x, y, z);
        double gf[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            const size_t nb = g.at(x + L::ex(i), y + L::ey(i), z + L::ez(i));
            const double wi = w_vel<L>(i);
#pragma unroll
            for (int c = 0; c < L::D; ++c)
#pragma unroll
                for (int d = 0; d < L::D; ++d) {
                    const int ed = e_comp<L>(i, d);
                    if (ed != 0) gf[c] -= wi * ed * mp[size_t(mcomp<L::D>(c, d)) * n + nb];
                }
        }
        const double r = rho[idx];
        for (int c = 0; c < L::D; ++c) v[c * n + idx] = u[c * n + idx] + gf[c] / (2.0 * r);
    }
}

template <class L, class S>
__global__ void get_pops_kernel(PopPtrs src, size_t n, double* out) {
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < n; idx += size_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i) out[i * n + idx] = double(S::load(i, src.p[i], pop_index(src, i, idx), src.fref[i]));
    }
}

// Populations of the box [x0, x0 + bx) x [y0, y0 + by) x [z0, z0 + bz) of the
// periodic lattice (coordinates wrapped), decoded to float64, [i][z][y][x] of the box.
template <class L, class S>
__global__ void get_box_kernel(PopPtrs src, Grid3 g, int x0, int y0, int z0, int bx, int by, int bz, double* out) {
    const size_t n = size_t(bx) * by * bz;
    for (size_t k = blockIdx.x * size_t(blockDim.x) + threadIdx.x; k < n; k += size_t(gridDim.x) * blockDim.x) {
        const int x = int(k % bx), y = int((k / bx) % by), z = int(k / (size_t(bx) * by));
        // origins are in [0, n) and box sizes at most n: one subtraction wraps (64-bit sums)
        long long xx = (long long)x0 + x, yy = (long long)y0 + y, zz = (long long)z0 + z;
        if (xx >= g.nx) xx -= g.nx;
        if (yy >= g.ny) yy -= g.ny;
        if (zz >= g.nz) zz -= g.nz;
        const size_t idx = (size_t(zz) * g.ny + size_t(yy)) * g.nx + size_t(xx);
#pragma unroll
        for (int i = 0; i < L::Q; ++i) out[i * n + k] = double(S::load(i, src.p[i], pop_index(src, i, idx), src.fref[i]));
    }
}

template <class L, class S>
__global__ void set_pops_kernel(PopPtrs dst, size_t n, const double* in) {
    for (size_t idx = blockIdx.x * size_t(blockDim.x) + threadIdx.x; idx < n; idx += size_t(gridDim.x) * blockDim.x) {
#pragma unroll
        for (int i = 0; i < L::Q; ++i)
            S::store(i, dst.p[i], pop_index(dst, i, idx), typename S::real(in[i * n + idx]), dst.fref[i]);
    }
}

// ---------------------------------------------------------------- reductions
// The float64 field reductions of lb_stats_get: field_reduce.cuh.
constexpr int STAT_THREADS = FR_THREADS;

}  // namespace lbk
