// Binary-fluid free-energy lattice Boltzmann: the D2Q9 kernels and the C ABI
// of both lattices (the D3Q19 kernels are in binary3d.cu).  The liquid-gas
// construction of Pooley & Furtado (Secs. II-VI) carried over to a symmetric
// binary fluid with an order parameter phi, as the paper says it applies
// (Sec. I).  The model (free energy, mu, p0, f^eq, g^eq, forcing) is stated
// in include/lb.h beside lb_binary_params.
//
// One fused kernel per time step.  A CTA owns a 32 x 8 tile, one site per
// thread:
//   stage A  the tile's f_i and g_i (18 loads per site, kept in registers)
//            and phi = sum_i g_i on the tile plus a halo (1 site for the
//            equilibrium scheme, 2 for the forcing scheme: Eq. 28 takes
//            differences of M' at the neighbours), halo sites reading g only;
//   stage B  (forcing) M'_xx - M'_yy and M'_xy on the tile plus one ring;
//            the gradient (Eq. 10) and Laplacian (Eq. 11) of phi at each site;
//   stage C  rho, u (Eq. 3), mu, p0, f^eq (Eqs. 5, 6), body force (Eq. 28)
//            and F_i (Eq. 27), v (Eq. 40), g^eq, both BGK relaxations and the
//            push of f*_i and g*_i to r + e_i in the other buffer.
// HBM traffic: one read and one write of the 18 populations per site
// (288 B per lattice update in float64, 144 B in float32); the halo sites'
// g are re-read by neighbouring CTAs from L2.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "../../include/lb.h"
#include "binary_common.cuh"
#include "binary_launch.h"

// Sets the thread-local message returned by lb_last_error (defined in lb_api.cu).
void lb_internal_set_error(const char* msg);

namespace lbb {

constexpr int Q = 9;
constexpr int TX = 32, TY = 8, NT = TX * TY;
constexpr int GRAPH_STEPS = 64;   // steps per captured graph (even: a replay ends in its start buffer)

// Gradient (Eq. 10, A = 1/3, B = 1/12) and Laplacian (Eq. 11, C = 2/3,
// D = 1/6) of a field on a row-major shared-memory region of row length RX
// at index c; the same sums give the force stencil (Eq. 28 with F = 1/12).
template <int RX, class real>
__device__ __forceinline__ void stencil(const real* p, int c, real& gx, real& gy) {
    const real a = real(1.0 / 3.0), b = real(1.0 / 12.0);
    gx = a * (p[c + 1] - p[c - 1]) + b * ((p[c + 1 + RX] - p[c - 1 + RX]) + (p[c + 1 - RX] - p[c - 1 - RX]));
    gy = a * (p[c + RX] - p[c - RX]) + b * ((p[c + RX + 1] - p[c - RX + 1]) + (p[c + RX - 1] - p[c - RX - 1]));
}
template <int RX, class real>
__device__ __forceinline__ real laplacian(const real* p, int c) {
    const real C = real(2.0 / 3.0), D = real(1.0 / 6.0);
    return C * ((p[c + 1] + p[c - 1]) + (p[c + RX] + p[c - RX])) +
           D * ((p[c + RX + 1] + p[c + RX - 1]) + (p[c - RX + 1] + p[c - RX - 1])) - real(10.0 / 3.0) * p[c];
}

template <bool FORCING, class real>
__global__ void __launch_bounds__(NT) binary_step_kernel(const StepArgs<real> a) {
    constexpr int H = FORCING ? 2 : 1;
    constexpr int RX = TX + 2 * H, RY = TY + 2 * H, RN = RX * RY;
    constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY;
    __shared__ real phs[RN];
    __shared__ real mdiff[FORCING ? SN : 1], mxy_s[FORCING ? SN : 1];

    const int nx = a.nx, ny = a.ny;
    const unsigned pitch = a.pitch;
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int x = x0 + tx, y = y0 + ty;
    const bool own = x < nx && y < ny;

    // ---- stage A: own populations; phi on the tile and the halo
    real f[Q], g[Q];
    {
        const int sx = own ? x : wrapc(x, nx), sy = own ? y : wrapc(y, ny);
        const unsigned s = unsigned(sy) * unsigned(nx) + unsigned(sx);
        real phi = 0;
        if (own) {
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = a.src[i * pitch + s];
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            g[i] = a.src[(Q + i) * pitch + s];
            phi += g[i];
        }
        phs[(ty + H) * RX + tx + H] = phi;
    }
    for (int h = threadIdx.x; h < RN - NT; h += NT) {
        int rx, ry;
        if (h < 2 * H * RX) {          // rows above and below the tile
            const int r = h / RX;
            rx = h % RX;
            ry = r < H ? r : r + TY;
        } else {                       // H columns left and right of every tile row
            const int k = h - 2 * H * RX;
            ry = H + k / (2 * H);
            const int c = k % (2 * H);
            rx = c < H ? c : c + TX;
        }
        const unsigned s = unsigned(wrapc(y0 - H + ry, ny)) * unsigned(nx) + unsigned(wrapc(x0 - H + rx, nx));
        real phi = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) phi += a.src[(Q + i) * pitch + s];
        phs[ry * RX + rx] = phi;
    }
    __syncthreads();

    // ---- stage B: M' on the tile + one ring (forcing); own gradient and Laplacian
    if constexpr (FORCING) {
        for (int k = threadIdx.x; k < SN; k += NT) {
            const int c = (k / SX - 1 + H) * RX + (k % SX - 1 + H);
            real gx, gy;
            stencil<RX>(phs, c, gx, gy);
            mdiff[k] = a.kappa * (gx * gx - gy * gy);
            mxy_s[k] = a.kappa * (gx * gy);
        }
    }
    const int c = (ty + H) * RX + tx + H;
    real gx, gy;
    stencil<RX>(phs, c, gx, gy);
    const real lap = laplacian<RX>(phs, c);
    const real phi = phs[c];
    if constexpr (FORCING) __syncthreads();

    // ---- stage C: collision and push of the own site
    bool bad = false;
    if (own) {
        real rho = 0, jx = 0, jy = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            rho += f[i];
            jx += real(D2Q9::ex(i)) * f[i];
            jy += real(D2Q9::ey(i)) * f[i];
        }
        bad = !(rho > real(0)) || !isfinite(rho);
        const real ir = real(1) / rho;
        const real ux = jx * ir, uy = jy * ir;
        const real mu = a.A * phi + a.B * phi * phi * phi - a.kappa * lap;
        const real u[2] = {ux, uy}, gr[2] = {gx, gy};
        real bf[2] = {real(0), real(0)}, v[2] = {ux, uy};
        if constexpr (FORCING) {
            // Eq. 28: g_x = -1/2 d_x (M'_xx - M'_yy) - d_y M'_xy, g_y = 1/2 d_y (M'_xx - M'_yy) - d_x M'_xy
            const int k = (ty + 1) * SX + tx + 1;
            real dDx, dDy, dXx, dXy;
            stencil<SX>(mdiff, k, dDx, dDy);
            stencil<SX>(mxy_s, k, dXx, dXy);
            bf[0] = real(-0.5) * dDx - dXy;
            bf[1] = real(0.5) * dDy - dXx;
            v[0] = ux + bf[0] * (real(0.5) * ir);   // Eq. 40
            v[1] = uy + bf[1] * (real(0.5) * ir);
        }
        const int xw[3] = {wrapc(x - 1, nx), x, wrapc(x + 1, nx)};
        const int yw[3] = {wrapc(y - 1, ny), y, wrapc(y + 1, ny)};
        collide_stream<D2Q9, FORCING>(f, g, rho, u, phi, gr, lap, bf, v, mu, a.A, a.B, a.kappa, a.Gamma, a.omega,
                                      a.omega_phi, [&](auto K, real fs, real gs) {
            constexpr int i = decltype(K)::value;
            constexpr int ex = D2Q9::ex(i), ey = D2Q9::ey(i);
            const unsigned d = unsigned(yw[1 + ey]) * unsigned(nx) + unsigned(xw[1 + ex]);
            a.dst[i * pitch + d] = fs;
            a.dst[(Q + i) * pitch + d] = gs;
        });
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x % 32) == 0) atomicOr(a.status, 1u);
}

// The same step with two adjacent x sites per thread (x even; nx even) for
// float32 storage: each population of the pair is one aligned 8-byte access,
// and every arithmetic step of stage C runs as packed float32 pair
// instructions.  CTA: a 32 x 8 tile, 128 threads; the phi halo is 2 sites in
// x (one pair) and 1 (equilibrium) or 2 (forcing) rows in y.
// Population k of a set (0 .. Q-1: f_k, Q .. 2Q-1: g_{k-Q}).  A float32 set holds
// 2Q float arrays of `pitch` elements.  A 16-bit set (fp16 deviations) holds
// f_0 and g_0 as float32 (at 0 and 4 pitch bytes) and the other 2Q - 2 as fp16
// arrays from 8 pitch bytes on: f_i - w_i pref (i >= 1; w_i pref is the rest
// equilibrium of a bulk phase) and g_i (i >= 1; zero at rest in a bulk phase).
__host__ __device__ constexpr unsigned set16_half_offset(int k, unsigned pitch) {
    return 8u * pitch + unsigned(k < Q ? k - 1 : Q - 1 + (k - Q - 1)) * 2u * pitch;
}
__host__ __device__ constexpr size_t set16_bytes(size_t pitch) { return 8 * pitch + size_t(2 * Q - 2) * 2 * pitch; }

// The pair of sites at pair index s2 (site 2 s2, x even) of population k, as
// float32 values; fref = w_k pref for f_k of a 16-bit set, else 0.
template <bool F16>
__device__ __forceinline__ P2 ld_pair(const char* set, unsigned pitch, int k, unsigned s2, float fref) {
    if constexpr (!F16) {
        return P2{reinterpret_cast<const float2*>(set)[unsigned(k) * (pitch >> 1) + s2]};
    } else {
        if (k == 0 || k == Q) return P2{reinterpret_cast<const float2*>(set + (k == 0 ? 0u : 4u * pitch))[s2]};
        const float2 v = __half22float2(reinterpret_cast<const __half2*>(set + set16_half_offset(k, pitch))[s2]);
        return pp(v.x + fref, v.y + fref);
    }
}
// Stores the pair v at sites idx, idx + 1 (idx even) / one value at site idx.
template <bool F16>
__device__ __forceinline__ void st_pair(char* set, unsigned pitch, int k, unsigned idx, P2 v, float fref) {
    if constexpr (!F16) {
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(set) + (unsigned(k) * pitch + idx)) = v.v;
    } else if (k == 0 || k == Q) {
        *reinterpret_cast<float2*>(reinterpret_cast<float*>(set + (k == 0 ? 0u : 4u * pitch)) + idx) = v.v;
    } else {
        *reinterpret_cast<__half2*>(reinterpret_cast<__half*>(set + set16_half_offset(k, pitch)) + idx) =
            __floats2half2_rn(v.v.x - fref, v.v.y - fref);
    }
}
template <bool F16>
__device__ __forceinline__ void st_one(char* set, unsigned pitch, int k, unsigned idx, float v, float fref) {
    if constexpr (!F16) {
        reinterpret_cast<float*>(set)[unsigned(k) * pitch + idx] = v;
    } else if (k == 0 || k == Q) {
        reinterpret_cast<float*>(set + (k == 0 ? 0u : 4u * pitch))[idx] = v;
    } else {
        reinterpret_cast<__half*>(set + set16_half_offset(k, pitch))[idx] = __float2half_rn(v - fref);
    }
}

constexpr int PTX_ = 32, PTY = 8, PTXP = PTX_ / 2, PNT = PTXP * PTY;
// Six resident CTAs per SM (at most 80 registers; the forcing form spills 20
// bytes): with the collision streamed population by population, measured on
// GB300 at 2048^2: forcing 38.8 GLUPS against 37.2 at five CTAs, equilibrium
// 38.1 against 35.7 (the array form at five CTAs: 36.7 / 35.8; unbounded,
// 118 registers and four CTAs: 34.0 / 33.4-36.0).
constexpr int PAIR_MINB = 6;
// 16-bit storage: five (at six its fp16 decodes spilled 32-68 bytes).
constexpr int PAIR_MINB16 = 5;

// Gradient (Eq. 10) and Laplacian (Eq. 11) of both sites of a pair from the
// 4 x 3 neighbourhood columns x-1 .. x+2 (c[r][0..3]) of rows y-1, y, y+1
// (r = 0, 1, 2): the scalar stencils of each site, lane by lane.
__device__ __forceinline__ void pair_stencil(const float (&c)[3][4], P2& gx, P2& gy, P2* lap) {
    const P2 a = pp(1.0f / 3.0f), b = pp(1.0f / 12.0f);
    P2 L[3], M[3], R[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        L[r] = pp(c[r][0], c[r][1]);
        M[r] = pp(c[r][1], c[r][2]);
        R[r] = pp(c[r][2], c[r][3]);
    }
    gx = a * (R[1] - L[1]) + b * ((R[2] - L[2]) + (R[0] - L[0]));
    gy = a * (M[2] - M[0]) + b * ((R[2] - R[0]) + (L[2] - L[0]));
    if (lap)
        *lap = pp(2.0f / 3.0f) * ((R[1] + L[1]) + (M[2] + M[0])) + pp(1.0f / 6.0f) * ((R[2] + L[2]) + (R[0] + L[0])) -
               pp(10.0f / 3.0f) * M[1];
}

template <bool FORCING, int MINB, bool F16 = false>
__global__ void __launch_bounds__(PNT, MINB) binary_step_kernel_pair(const StepArgs<float> a) {
    constexpr int H = FORCING ? 2 : 1, HX = 2;
    constexpr int RX = PTX_ + 2 * HX, RY = PTY + 2 * H, RN = RX * RY, RXP = RX / 2;
    constexpr int SX = PTX_ + 2, SY = PTY + 2, SN = SX * SY;
    constexpr int NHALO = 2 * H * RXP + 2 * PTY;        // halo pairs: H rows above and below, one pair each side
    constexpr int NRING = 2 * SX + 2 * PTY;             // M' ring sites around the tile
    static_assert(NHALO <= PNT && NRING <= PNT, "one halo pair and one ring site per thread at most");
    __shared__ __align__(8) float phs[RN];
    __shared__ float mdiff[FORCING ? SN : 1], mxy_s[FORCING ? SN : 1];

    const int nx = a.nx, ny = a.ny;
    const unsigned pitch = a.pitch;
    const int tid = threadIdx.x;
    const int px = tid % PTXP, py = tid / PTXP;
    const int x0 = blockIdx.x * PTX_, y0 = blockIdx.y * PTY;
    const int x = x0 + 2 * px, y = y0 + py;
    const bool own = x < nx && y < ny;
    const char* srcb = reinterpret_cast<const char*>(a.src);
    // w_i pref of the 16-bit deviations (f_i, i >= 1), formed where used
    auto fref = [&](int i) { return F16 && i > 0 ? float(lbk::w_vel<D2Q9>(i)) * a.pref : 0.0f; };

    // ---- stage A: the own pair's populations; phi pairs on the tile and halo
    P2 f[Q], g[Q];
    {
        const int sx = own ? x : wrapc(x, nx), sy = own ? y : wrapc(y, ny);
        const unsigned s2 = (unsigned(sy) * unsigned(nx) + unsigned(sx)) >> 1;   // pair index (x even)
        const float2* src = reinterpret_cast<const float2*>(a.src);
        const unsigned p2 = pitch >> 1;
        if (own) {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (F16) f[i] = ld_pair<F16>(srcb, pitch, i, s2, fref(i));
                else f[i].v = src[i * p2 + s2];
            }
        }
        P2 phi = pp(0.0f);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if constexpr (F16) g[i] = ld_pair<F16>(srcb, pitch, Q + i, s2, 0.0f);
            else g[i].v = src[(Q + i) * p2 + s2];
            phi += g[i];
        }
        *reinterpret_cast<float2*>(&phs[(py + H) * RX + 2 * px + HX]) = phi.v;
        if (tid < NHALO) {
            int rxp, ry;
            if (tid < 2 * H * RXP) {
                const int r = tid / RXP;
                rxp = tid % RXP;
                ry = r < H ? r : r + PTY;
            } else {
                const int k = tid - 2 * H * RXP;
                ry = H + (k >> 1);
                rxp = (k & 1) ? RXP - 1 : 0;
            }
            const unsigned h2 = (unsigned(wrapc(y0 - H + ry, ny)) * unsigned(nx) +
                                 unsigned(wrapc(x0 - HX + 2 * rxp, nx))) >> 1;
            P2 ph = pp(0.0f);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (F16) ph += ld_pair<F16>(srcb, pitch, Q + i, h2, 0.0f);
                else ph += P2{reinterpret_cast<const float2*>(a.src)[(Q + i) * (pitch >> 1) + h2]};
            }
            *reinterpret_cast<float2*>(&phs[ry * RX + 2 * rxp]) = ph.v;
        }
    }
    __syncthreads();

    // ---- stage B: the pair's gradient and Laplacian; M' on the tile and its ring
    float nb[3][4];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const int c = (py + H - 1 + r) * RX + 2 * px + HX;
        const float2 m = *reinterpret_cast<const float2*>(&phs[c]);
        nb[r][0] = phs[c - 1];
        nb[r][1] = m.x;
        nb[r][2] = m.y;
        nb[r][3] = phs[c + 2];
    }
    P2 gx, gy, lap;
    pair_stencil(nb, gx, gy, &lap);
    const P2 phi = pp(nb[1][1], nb[1][2]);
    if constexpr (FORCING) {
        const P2 kp = pp(a.kappa);
        const P2 md = kp * (gx * gx - gy * gy), mx = kp * (gx * gy);
        const int k = (py + 1) * SX + 2 * px + 1;
        mdiff[k] = md.v.x;
        mdiff[k + 1] = md.v.y;
        mxy_s[k] = mx.v.x;
        mxy_s[k + 1] = mx.v.y;
        if (tid < NRING) {
            int sx, sy;
            if (tid < 2 * SX) {
                sx = tid % SX;
                sy = tid < SX ? 0 : SY - 1;
            } else {
                const int q = tid - 2 * SX;
                sy = 1 + (q >> 1);
                sx = (q & 1) ? SX - 1 : 0;
            }
            const int c = (sy - 1 + H) * RX + (sx - 1 + HX);
            const float rgx = (1.0f / 3.0f) * (phs[c + 1] - phs[c - 1]) +
                              (1.0f / 12.0f) * ((phs[c + 1 + RX] - phs[c - 1 + RX]) + (phs[c + 1 - RX] - phs[c - 1 - RX]));
            const float rgy = (1.0f / 3.0f) * (phs[c + RX] - phs[c - RX]) +
                              (1.0f / 12.0f) * ((phs[c + RX + 1] - phs[c - RX + 1]) + (phs[c + RX - 1] - phs[c - RX - 1]));
            mdiff[sy * SX + sx] = a.kappa * (rgx * rgx - rgy * rgy);
            mxy_s[sy * SX + sx] = a.kappa * (rgx * rgy);
        }
        __syncthreads();
    }

    // ---- stage C: collision of the pair and push
    bool bad = false;
    if (own) {
        P2 rho = pp(0.0f), jx = pp(0.0f), jy = pp(0.0f);
        static_for<0, Q>([&](auto K) {
            constexpr int i = decltype(K)::value;
            rho += f[i];
            if constexpr (D2Q9::ex(i) > 0) jx += f[i];
            if constexpr (D2Q9::ex(i) < 0) jx -= f[i];
            if constexpr (D2Q9::ey(i) > 0) jy += f[i];
            if constexpr (D2Q9::ey(i) < 0) jy -= f[i];
        });
        bad = !(rho.v.x > 0.0f) || !(rho.v.y > 0.0f) || !isfinite(rho.v.x) || !isfinite(rho.v.y);
        const P2 ir = pp(1.0f / rho.v.x, 1.0f / rho.v.y);
        const P2 ux = jx * ir, uy = jy * ir;
        const P2 A = pp(a.A), B = pp(a.B), kp = pp(a.kappa);
        const P2 mu = A * phi + B * phi * phi * phi - kp * lap;
        const P2 u[2] = {ux, uy}, gr[2] = {gx, gy};
        P2 bf[2] = {pp(0.0f), pp(0.0f)}, v[2] = {ux, uy};
        if constexpr (FORCING) {
            // Eq. 28 from the 4 x 3 neighbourhoods of M'_xx - M'_yy and M'_xy
            float dn[3][4], xn[3][4];
#pragma unroll
            for (int r = 0; r < 3; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = (py + r) * SX + 2 * px + c;
                    dn[r][c] = mdiff[k];
                    xn[r][c] = mxy_s[k];
                }
            P2 dDx, dDy, dXx, dXy;
            pair_stencil(dn, dDx, dDy, nullptr);
            pair_stencil(xn, dXx, dXy, nullptr);
            bf[0] = pp(-0.5f) * dDx - dXy;
            bf[1] = pp(0.5f) * dDy - dXx;
            const P2 hir = pp(0.5f) * ir;
            v[0] = ux + bf[0] * hir;   // Eq. 40
            v[1] = uy + bf[1] * hir;
        }
        const unsigned xm = unsigned(wrapc(x - 1, nx)), xp2 = unsigned(wrapc(x + 2, nx));
        const unsigned row[3] = {unsigned(wrapc(y - 1, ny)) * unsigned(nx), unsigned(y) * unsigned(nx),
                                 unsigned(wrapc(y + 1, ny)) * unsigned(nx)};
        collide_stream<D2Q9, FORCING>(f, g, rho, u, phi, gr, lap, bf, v, mu, A, B, kp, pp(a.Gamma), pp(a.omega),
                                      pp(a.omega_phi), [&](auto K, P2 fs, P2 gs) {
            constexpr int i = decltype(K)::value;
            constexpr int ex = D2Q9::ex(i), ey = D2Q9::ey(i);
            const unsigned r = row[1 + ey];
            if constexpr (!F16) {
                float* df = a.dst + i * pitch + r;
                float* dg = a.dst + (Q + i) * pitch + r;
                if constexpr (ex == 0) {
                    *reinterpret_cast<float2*>(df + x) = fs.v;
                    *reinterpret_cast<float2*>(dg + x) = gs.v;
                } else if constexpr (ex > 0) {
                    df[x + 1] = fs.v.x;
                    df[xp2] = fs.v.y;
                    dg[x + 1] = gs.v.x;
                    dg[xp2] = gs.v.y;
                } else {
                    df[xm] = fs.v.x;
                    df[x] = fs.v.y;
                    dg[xm] = gs.v.x;
                    dg[x] = gs.v.y;
                }
                return;
            }
            char* db = reinterpret_cast<char*>(a.dst);
            if constexpr (ex == 0) {
                st_pair<F16>(db, pitch, i, r + x, fs, fref(i));
                st_pair<F16>(db, pitch, Q + i, r + x, gs, 0.0f);
            } else if constexpr (ex > 0) {
                st_one<F16>(db, pitch, i, r + x + 1, fs.v.x, fref(i));
                st_one<F16>(db, pitch, i, r + xp2, fs.v.y, fref(i));
                st_one<F16>(db, pitch, Q + i, r + x + 1, gs.v.x, 0.0f);
                st_one<F16>(db, pitch, Q + i, r + xp2, gs.v.y, 0.0f);
            } else {
                st_one<F16>(db, pitch, i, r + xm, fs.v.x, fref(i));
                st_one<F16>(db, pitch, i, r + x, fs.v.y, fref(i));
                st_one<F16>(db, pitch, Q + i, r + xm, gs.v.x, 0.0f);
                st_one<F16>(db, pitch, Q + i, r + x, gs.v.y, 0.0f);
            }
        });
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x % 32) == 0) atomicOr(a.status, 1u);
}

// f = f^eq, g = g^eq of float64 fields (rho, phi, u), stencils of phi read
// from the periodic field; one thread per site.
template <bool FORCING, class real>
__global__ void binary_init_kernel(const double* rho, const double* phi, const double* ux, const double* uy,
                                   real* dst, long long pitch, int nx, int ny, double A, double B, double kappa,
                                   double Gamma) {
    const long long n = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int x = int(s % nx), y = int(s / nx);
        double p[9];   // 3 x 3 neighbourhood, row-major, centre p[4]
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                p[(dy + 1) * 3 + dx + 1] = phi[(long long)wrapc(y + dy, ny) * nx + wrapc(x + dx, nx)];
        double gx, gy;
        stencil<3>(p, 4, gx, gy);
        const double lap = laplacian<3>(p, 4);
        const double mu = A * p[4] + B * p[4] * p[4] * p[4] - kappa * lap;
        const double u0 = ux ? ux[s] : 0.0, u1 = uy ? uy[s] : 0.0;
        double fe[Q], ge[Q];
        const double u[2] = {u0, u1}, gr[2] = {gx, gy};
        f_equilibrium<D2Q9, !FORCING>(rho[s], u, p[4], gr, lap, A, B, kappa, fe);
        g_equilibrium<D2Q9>(p[4], u, mu, Gamma, ge);
        for (int i = 0; i < Q; ++i) {
            dst[i * pitch + s] = real(fe[i]);
            dst[(Q + i) * pitch + s] = real(ge[i]);
        }
    }
}

// Observables in float64: rho, phi, u (Eq. 3) and mu; in the forcing scheme
// also M'_xx - M'_yy and M'_xy for binary_velocity_kernel.
template <class real>
__global__ void binary_moments_kernel(const real* src, long long pitch, int nx, int ny, double* rho, double* phi,
                                      double* ux, double* uy) {
    const long long n = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        double r = 0, p = 0, jx = 0, jy = 0;
        for (int i = 0; i < Q; ++i) {
            const double fi = double(src[i * pitch + s]);
            r += fi;
            jx += D2Q9::ex(i) * fi;
            jy += D2Q9::ey(i) * fi;
            p += double(src[(Q + i) * pitch + s]);
        }
        rho[s] = r;
        phi[s] = p;
        ux[s] = jx / r;
        uy[s] = jy / r;
    }
}

__global__ void binary_mu_kernel(const double* phi, int nx, int ny, double A, double B, double kappa, double* mu,
                                 double* mdiff, double* mxy) {
    const long long n = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int x = int(s % nx), y = int(s / nx);
        double p[9];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx)
                p[(dy + 1) * 3 + dx + 1] = phi[(long long)wrapc(y + dy, ny) * nx + wrapc(x + dx, nx)];
        double gx, gy;
        stencil<3>(p, 4, gx, gy);
        mu[s] = A * p[4] + B * p[4] * p[4] * p[4] - kappa * laplacian<3>(p, 4);
        if (mdiff) {
            mdiff[s] = kappa * (gx * gx - gy * gy);
            mxy[s] = kappa * (gx * gy);
        }
    }
}

// v = u + g / (2 rho) (Eq. 40) with g of Eq. 28 from the M' fields.
__global__ void binary_velocity_kernel(const double* rho, const double* ux, const double* uy, const double* mdiff,
                                       const double* mxy, int nx, int ny, double* vx, double* vy) {
    const long long n = (long long)nx * ny;
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
        const int x = int(s % nx), y = int(s / nx);
        double d[9], m[9];
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const long long t = (long long)wrapc(y + dy, ny) * nx + wrapc(x + dx, nx);
                d[(dy + 1) * 3 + dx + 1] = mdiff[t];
                m[(dy + 1) * 3 + dx + 1] = mxy[t];
            }
        double dDx, dDy, dXx, dXy;
        stencil<3>(d, 4, dDx, dDy);
        stencil<3>(m, 4, dXx, dXy);
        vx[s] = ux[s] + (-0.5 * dDx - dXy) / (2.0 * rho[s]);
        vy[s] = uy[s] + (0.5 * dDy - dXx) / (2.0 * rho[s]);
    }
}

template <class real>
__global__ void binary_convert_kernel(const real* src, double* out, long long pitch, long long n, int q2,
                                      int to_double, const double* in, real* dst) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < q2 * n;
         t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / n, s = t % n;
        if (to_double) out[t] = double(src[k * pitch + s]);
        else dst[k * pitch + s] = real(in[t]);
    }
}

// Conversion between a 16-bit set and float64 populations [2Q][n] (f then g);
// to_double: set -> buf, else buf -> set (deviations rounded to fp16 from float64).
__global__ void binary_convert16_kernel(char* set, unsigned pitch, unsigned n, int to_double, double* buf, float pref) {
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < 2u * Q * n; t += gridDim.x * blockDim.x) {
        const int k = int(t / n);
        const unsigned s = t % n;
        if (k == 0 || k == Q) {
            float* p = reinterpret_cast<float*>(set + (k == 0 ? 0u : 4u * pitch));
            if (to_double) buf[t] = double(p[s]);
            else p[s] = float(buf[t]);
        } else {
            __half* h = reinterpret_cast<__half*>(set + set16_half_offset(k, pitch));
            const double fref = k < Q ? lbk::w_vel<D2Q9>(k) * double(pref) : 0.0;
            if (to_double) buf[t] = double(__half2float(h[s])) + fref;
            else h[s] = __float2half_rn(float(buf[t] - fref));
        }
    }
}

// rho, phi, u of a 16-bit set in float64.
__global__ void binary_moments16_kernel(const char* set, unsigned pitch, unsigned n, float pref, double* rho,
                                        double* phi, double* ux, double* uy) {
    for (unsigned s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x) {
        double r = double(reinterpret_cast<const float*>(set)[s]);
        double p = double(reinterpret_cast<const float*>(set + 4u * pitch)[s]);
        double jx = 0, jy = 0;
        for (int i = 1; i < Q; ++i) {
            const double fi = double(__half2float(reinterpret_cast<const __half*>(set + set16_half_offset(i, pitch))[s])) +
                              lbk::w_vel<D2Q9>(i) * double(pref);
            r += fi;
            jx += D2Q9::ex(i) * fi;
            jy += D2Q9::ey(i) * fi;
            p += double(__half2float(reinterpret_cast<const __half*>(set + set16_half_offset(Q + i, pitch))[s]));
        }
        rho[s] = r;
        phi[s] = p;
        ux[s] = jx / r;
        uy[s] = jy / r;
    }
}

inline unsigned blocks_for(long long n) {
    long long b = (n + 255) / 256;
    if (b > 8192) b = 8192;
    return unsigned(b < 1 ? 1 : b);
}

}  // namespace lbb

using namespace lbb;

struct lb_binary {
    lb_binary_params p{};
    cudaStream_t stream = nullptr;       // the caller's stream (NULL: the legacy default stream)
    cudaStream_t cap_stream = nullptr;   // private stream the step graphs are captured on
    int D = 2, Qn = 9;            // lattice dimension and velocities
    long long N = 0, pitch = 0;
    size_t esize = 8;
    void* pop = nullptr;          // 2 sets x 2 Q populations x pitch elements
    void* phi = nullptr;          // D3Q19: phi of the current set (one value per site, storage type)
    int cur = 0;                  // set holding the current populations
    bool initialised = false;
    long long step = 0;
    unsigned* d_status = nullptr;
    double* work = nullptr;       // float64 observables: 9 fields of N (D2Q9), 15 (D3Q19)
    double* d_in = nullptr;       // staging of host float64 inputs (2 Q N)
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_failed = false;
    bool pair = false;            // float32 / 16-bit with an even nx: the two-sites-per-thread kernel
    bool f16 = false;             // LB_F16DEV: f_0, g_0 float32, the rest fp16 (f_i as deviations)
    float pref = 0.0f;            // the deviations' reference p0 of a bulk phase at rho = 1
    size_t set_bytes = 0;         // bytes of one population set
    lb_status sticky = LB_OK;
};

namespace {

lb_status bfail(lb_status s, const std::string& msg) {
    lb_internal_set_error(msg.c_str());
    return s;
}

lb_status brecord(lb_binary* c, cudaError_t e, const char* where) {
    cudaGetLastError();
    c->sticky = LB_ECUDA;
    return bfail(LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

lb_status bcheck(lb_binary* c) {
    if (!c) return bfail(LB_EINVAL, "null context");
    if (c->sticky != LB_OK) return bfail(c->sticky, "binary context is in an error state");
    return LB_OK;
}

char* set_ptr(lb_binary* c, int set) {
    return static_cast<char*>(c->pop) + size_t(set) * c->set_bytes;
}

template <class real>
cudaError_t launch_step(lb_binary* c, int from, cudaStream_t st) {
    StepArgs<real> a;
    a.src = reinterpret_cast<const real*>(set_ptr(c, from));
    a.dst = reinterpret_cast<real*>(set_ptr(c, 1 - from));
    a.phi = nullptr;
    a.pitch = unsigned(c->pitch);
    a.nx = c->p.nx;
    a.ny = c->p.ny;
    a.nz = c->p.nz;
    a.A = real(c->p.A);
    a.B = real(c->p.B);
    a.kappa = real(c->p.kappa);
    a.Gamma = real(c->p.Gamma);
    a.omega = real(1.0 / c->p.tau);
    a.omega_phi = real(1.0 / c->p.tau_phi);
    a.status = c->d_status;
    a.pref = c->pref;
    const bool forcing = c->p.scheme == LB_SCHEME_FORCING;
    if (c->D == 3) return binary_step3(forcing, a, static_cast<real*>(c->phi), st);
    if constexpr (sizeof(real) == 4) {
        if (c->pair) {   // float32 or 16-bit, even nx: two sites per thread
            const dim3 grid((c->p.nx + PTX_ - 1) / PTX_, (c->p.ny + PTY - 1) / PTY);
            if (c->f16) {
                if (forcing) binary_step_kernel_pair<true, PAIR_MINB16, true><<<grid, PNT, 0, st>>>(a);
                else binary_step_kernel_pair<false, PAIR_MINB16, true><<<grid, PNT, 0, st>>>(a);
            } else {
                if (forcing) binary_step_kernel_pair<true, PAIR_MINB><<<grid, PNT, 0, st>>>(a);
                else binary_step_kernel_pair<false, PAIR_MINB><<<grid, PNT, 0, st>>>(a);
            }
            return cudaGetLastError();
        }
    }
    const dim3 grid((c->p.nx + TX - 1) / TX, (c->p.ny + TY - 1) / TY);
    if (forcing) binary_step_kernel<true, real><<<grid, NT, 0, st>>>(a);
    else binary_step_kernel<false, real><<<grid, NT, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t step_once(lb_binary* c, int from, cudaStream_t st) {
    return c->p.storage == LB_F64 ? launch_step<double>(c, from, st) : launch_step<float>(c, from, st);
}

lb_status sync_status(lb_binary* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return brecord(c, e, "cudaStreamSynchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return brecord(c, e, "status read");
    if (st) {
        c->sticky = LB_EUNSTABLE;
        return bfail(LB_EUNSTABLE, "a density became non-finite or non-positive");
    }
    return LB_OK;
}

lb_status ensure_work(lb_binary* c) {
    if (c->work) return LB_OK;
    cudaError_t e = cudaMalloc(&c->work, size_t(c->D == 3 ? 15 : 9) * c->N * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->work = nullptr;
        return bfail(LB_ENOMEM, "field workspace");
    }
    return LB_OK;
}

lb_status ensure_in(lb_binary* c) {
    if (c->d_in) return LB_OK;
    cudaError_t e = cudaMalloc(&c->d_in, size_t(2) * c->Qn * c->N * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->d_in = nullptr;
        return bfail(LB_ENOMEM, "input staging");
    }
    return LB_OK;
}

void drop_graphs(lb_binary* c) {
    for (auto& g : c->graph)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
}

lb_status reset_after_set(lb_binary* c) {
    c->cur = 0;
    c->step = 0;
    c->initialised = true;
    cudaError_t e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return brecord(c, e, "status reset");
    return sync_status(c);
}

// Observables of the current state into the workspace:
// rho, phi, ux, uy, vx, vy, mu, mdiff, mxy (each N doubles).
lb_status compute_fields(lb_binary* c) {
    lb_status s = ensure_work(c);
    if (s != LB_OK) return s;
    if (c->D == 3) {
        cudaError_t e = binary_fields3(c->p.scheme == LB_SCHEME_FORCING, c->p.storage == LB_F32, set_ptr(c, c->cur),
                                       unsigned(c->pitch), c->p.nx, c->p.ny, c->p.nz, c->p.A, c->p.B, c->p.kappa,
                                       c->work, c->stream);
        if (e != cudaSuccess) return brecord(c, e, "binary fields");
        return LB_OK;
    }
    const long long N = c->N;
    double* w = c->work;
    double *rho = w, *phi = w + N, *ux = w + 2 * N, *uy = w + 3 * N, *vx = w + 4 * N, *vy = w + 5 * N,
           *mu = w + 6 * N, *md = w + 7 * N, *mx = w + 8 * N;
    const unsigned nb = blocks_for(N);
    const int nx = c->p.nx, ny = c->p.ny;
    if (c->f16)
        binary_moments16_kernel<<<nb, 256, 0, c->stream>>>(set_ptr(c, c->cur), unsigned(c->pitch), unsigned(N), c->pref,
                                                           rho, phi, ux, uy);
    else if (c->p.storage == LB_F64)
        binary_moments_kernel<double><<<nb, 256, 0, c->stream>>>(
            reinterpret_cast<const double*>(set_ptr(c, c->cur)), c->pitch, nx, ny, rho, phi, ux, uy);
    else
        binary_moments_kernel<float><<<nb, 256, 0, c->stream>>>(
            reinterpret_cast<const float*>(set_ptr(c, c->cur)), c->pitch, nx, ny, rho, phi, ux, uy);
    const bool forcing = c->p.scheme == LB_SCHEME_FORCING;
    binary_mu_kernel<<<nb, 256, 0, c->stream>>>(phi, nx, ny, c->p.A, c->p.B, c->p.kappa, mu, forcing ? md : nullptr,
                                                 forcing ? mx : nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return brecord(c, e, "binary moments");
    if (forcing) {
        binary_velocity_kernel<<<nb, 256, 0, c->stream>>>(rho, ux, uy, md, mx, nx, ny, vx, vy);
        e = cudaGetLastError();
    } else {
        e = cudaMemcpyAsync(vx, ux, size_t(2) * N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e != cudaSuccess) return brecord(c, e, "binary velocity");
    return LB_OK;
}

bool is_fin(double v) { return std::isfinite(v); }

}  // namespace

extern "C" {

lb_status lb_binary_create(const lb_binary_params* p, void* stream, lb_binary** out) {
    if (!p || !out) return bfail(LB_EINVAL, "null argument");
    *out = nullptr;
    if (p->lattice != LB_D2Q9 && p->lattice != LB_D3Q19) return bfail(LB_EINVAL, "lattice");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return bfail(LB_EINVAL, "nx, ny and nz must be >= 1");
    if (p->lattice == LB_D2Q9 && p->nz != 1) return bfail(LB_EINVAL, "D2Q9 needs nz = 1");
    if ((long long)p->nx * p->ny * p->nz > 0x7fffffffLL) return bfail(LB_EINVAL, "more than 2^31 - 1 sites");
    if (!is_fin(p->A) || !is_fin(p->B) || !is_fin(p->kappa) || !is_fin(p->Gamma) || !is_fin(p->tau) ||
        !is_fin(p->tau_phi))
        return bfail(LB_EINVAL, "non-finite parameter");
    if (p->B < 0 || p->kappa < 0) return bfail(LB_EINVAL, "B and kappa must be >= 0");
    if (!(p->Gamma > 0)) return bfail(LB_EINVAL, "Gamma must be > 0");
    if (!(p->tau > 0.5) || !(p->tau_phi > 0.5)) return bfail(LB_EINVAL, "tau and tau_phi must be > 1/2");
    if (p->scheme != LB_SCHEME_EQUILIBRIUM && p->scheme != LB_SCHEME_FORCING) return bfail(LB_EINVAL, "scheme");
    if (p->storage != LB_F64 && p->storage != LB_F32 && p->storage != LB_F16DEV)
        return bfail(LB_EINVAL, "storage must be LB_F64, LB_F32 or LB_F16DEV");
    if (p->storage == LB_F16DEV && (p->lattice != LB_D2Q9 || p->nx % 2 != 0))
        return bfail(LB_EINVAL, "LB_F16DEV binary storage needs D2Q9 and an even nx");
    lb_binary* c = new (std::nothrow) lb_binary;
    if (!c) return bfail(LB_ENOMEM, "context");
    c->p = *p;
    c->D = p->lattice == LB_D2Q9 ? 2 : 3;
    c->Qn = p->lattice == LB_D2Q9 ? 9 : 19;
    c->N = (long long)p->nx * p->ny * p->nz;
    c->esize = p->storage == LB_F64 ? 8 : 4;
    c->f16 = p->storage == LB_F16DEV;
    // LB_BINARY_SITE=1 keeps the one-site kernel for float32 (comparisons)
    c->pair = c->f16 || (c->D == 2 && p->storage == LB_F32 && p->nx % 2 == 0 && !std::getenv("LB_BINARY_SITE"));
    c->pitch = (c->N + 63) / 64 * 64;
    if (2 * c->Qn * c->pitch >= (1LL << 32) || (c->f16 && set16_bytes(size_t(c->pitch)) >= (1ULL << 32))) {
        delete c;
        return bfail(LB_EINVAL, "lattice too large: offsets within a population set must fit 32 bits "
                                "(at most 238,609,280 sites for D2Q9, 107,374,144 with LB_F16DEV, "
                                "113,025,408 for D3Q19)");
    }
    c->set_bytes = c->f16 ? set16_bytes(size_t(c->pitch)) : size_t(2) * c->Qn * c->pitch * c->esize;
    // the rest equilibrium w_i p0 of a bulk phase at rho = 1, phi = +-phi* (the same in both)
    const double ps2 = (p->A < 0 && p->B > 0) ? -p->A / p->B : 0.0;
    c->pref = float(1.0 / 3.0 + 0.5 * p->A * ps2 + 0.75 * p->B * ps2 * ps2);
    c->stream = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMalloc(&c->pop, 2 * c->set_bytes);
    if (e == cudaSuccess && c->D == 3) e = cudaMalloc(&c->phi, size_t(c->N) * c->esize);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        lb_binary_destroy(c);
        return bfail(e == cudaErrorMemoryAllocation ? LB_ENOMEM : LB_ECUDA, std::string("create: ") + cudaGetErrorString(e));
    }
    *out = c;
    return LB_OK;
}

lb_status lb_binary_destroy(lb_binary* c) {
    if (!c) return LB_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    drop_graphs(c);
    cudaFree(c->pop);
    cudaFree(c->phi);
    cudaFree(c->d_status);
    cudaFree(c->work);
    cudaFree(c->d_in);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return LB_OK;
}

lb_status lb_binary_init_fields(lb_binary* c, const double* rho, const double* phi, const double* u) {
    lb_status s = bcheck(c);
    if (s != LB_OK) return s;
    if (!rho || !phi) return bfail(LB_EINVAL, "rho and phi are required");
    for (long long i = 0; i < c->N; ++i)
        if (!(rho[i] > 0) || !is_fin(rho[i]) || !is_fin(phi[i])) return bfail(LB_EINVAL, "rho must be positive and finite, phi finite");
    if ((s = ensure_in(c)) != LB_OK) return s;
    const long long N = c->N;
    double* d = c->d_in;
    const size_t nb = size_t(N) * sizeof(double);
    cudaError_t e = cudaMemcpyAsync(d, rho, nb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d + N, phi, nb, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(d + 2 * N, u, c->D * nb, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return brecord(c, e, "field upload");
    if (c->D == 3) {
        e = binary_init3(c->p.scheme == LB_SCHEME_FORCING, c->p.storage == LB_F32, d, d + N, u ? d + 2 * N : nullptr,
                         set_ptr(c, 0), unsigned(c->pitch), c->p.nx, c->p.ny, c->p.nz, c->p.A, c->p.B, c->p.kappa,
                         c->p.Gamma, c->stream);
        if (e != cudaSuccess) return brecord(c, e, "binary init");
        return reset_after_set(c);
    }
    const double* ux = u ? d + 2 * N : nullptr;
    const double* uy = u ? d + 3 * N : nullptr;
    const unsigned nbk = blocks_for(N);
    const bool forcing = c->p.scheme == LB_SCHEME_FORCING;
    const lb_binary_params& p = c->p;
    if (c->f16) {   // float64 equilibria into a staging array, then rounded into the 16-bit set
        double* tmp = nullptr;
        e = cudaMalloc(&tmp, size_t(2) * Q * N * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(LB_ENOMEM, "init staging");
        }
        if (forcing) binary_init_kernel<true, double><<<nbk, 256, 0, c->stream>>>(d, d + N, ux, uy, tmp, N, p.nx, p.ny, p.A, p.B, p.kappa, p.Gamma);
        else binary_init_kernel<false, double><<<nbk, 256, 0, c->stream>>>(d, d + N, ux, uy, tmp, N, p.nx, p.ny, p.A, p.B, p.kappa, p.Gamma);
        binary_convert16_kernel<<<blocks_for(2 * Q * N), 256, 0, c->stream>>>(set_ptr(c, 0), unsigned(c->pitch),
                                                                            unsigned(N), 0, tmp, c->pref);
        e = cudaGetLastError();
        cudaError_t e2 = cudaStreamSynchronize(c->stream);
        cudaFree(tmp);
        if (e == cudaSuccess) e = e2;
        if (e != cudaSuccess) return brecord(c, e, "binary init");
        return reset_after_set(c);
    }
    if (p.storage == LB_F64) {
        double* dst = reinterpret_cast<double*>(set_ptr(c, 0));
        if (forcing) binary_init_kernel<true, double><<<nbk, 256, 0, c->stream>>>(d, d + N, ux, uy, dst, c->pitch, p.nx, p.ny, p.A, p.B, p.kappa, p.Gamma);
        else binary_init_kernel<false, double><<<nbk, 256, 0, c->stream>>>(d, d + N, ux, uy, dst, c->pitch, p.nx, p.ny, p.A, p.B, p.kappa, p.Gamma);
    } else {
        float* dst = reinterpret_cast<float*>(set_ptr(c, 0));
        if (forcing) binary_init_kernel<true, float><<<nbk, 256, 0, c->stream>>>(d, d + N, ux, uy, dst, c->pitch, p.nx, p.ny, p.A, p.B, p.kappa, p.Gamma);
        else binary_init_kernel<false, float><<<nbk, 256, 0, c->stream>>>(d, d + N, ux, uy, dst, c->pitch, p.nx, p.ny, p.A, p.B, p.kappa, p.Gamma);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return brecord(c, e, "binary init");
    return reset_after_set(c);
}

lb_status lb_binary_set_populations(lb_binary* c, const double* f, const double* g) {
    lb_status s = bcheck(c);
    if (s != LB_OK) return s;
    if (!f || !g) return bfail(LB_EINVAL, "null populations");
    if ((s = ensure_in(c)) != LB_OK) return s;
    const size_t half = size_t(c->Qn) * c->N;
    cudaError_t e = cudaMemcpyAsync(c->d_in, f, half * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->d_in + half, g, half * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return brecord(c, e, "population upload");
    const unsigned nb = blocks_for(2 * half);
    if (c->f16)
        binary_convert16_kernel<<<nb, 256, 0, c->stream>>>(set_ptr(c, 0), unsigned(c->pitch), unsigned(c->N), 0, c->d_in,
                                                           c->pref);
    else if (c->p.storage == LB_F64)
        binary_convert_kernel<double><<<nb, 256, 0, c->stream>>>(nullptr, nullptr, c->pitch, c->N, 2 * c->Qn, 0, c->d_in,
                                                                  reinterpret_cast<double*>(set_ptr(c, 0)));
    else
        binary_convert_kernel<float><<<nb, 256, 0, c->stream>>>(nullptr, nullptr, c->pitch, c->N, 2 * c->Qn, 0, c->d_in,
                                                                 reinterpret_cast<float*>(set_ptr(c, 0)));
    e = cudaGetLastError();
    if (e != cudaSuccess) return brecord(c, e, "set populations");
    return reset_after_set(c);
}

lb_status lb_binary_get_populations(lb_binary* c, double* f, double* g) {
    lb_status s = bcheck(c);
    if (s != LB_OK) return s;
    if (!f || !g) return bfail(LB_EINVAL, "null output");
    if (!c->initialised) return bfail(LB_ESTATE, "state not initialised");
    if ((s = ensure_in(c)) != LB_OK) return s;
    const size_t half = size_t(c->Qn) * c->N;
    const unsigned nb = blocks_for(2 * half);
    if (c->f16)
        binary_convert16_kernel<<<nb, 256, 0, c->stream>>>(set_ptr(c, c->cur), unsigned(c->pitch), unsigned(c->N), 1,
                                                           c->d_in, c->pref);
    else if (c->p.storage == LB_F64)
        binary_convert_kernel<double><<<nb, 256, 0, c->stream>>>(
            reinterpret_cast<const double*>(set_ptr(c, c->cur)), c->d_in, c->pitch, c->N, 2 * c->Qn, 1, nullptr, nullptr);
    else
        binary_convert_kernel<float><<<nb, 256, 0, c->stream>>>(
            reinterpret_cast<const float*>(set_ptr(c, c->cur)), c->d_in, c->pitch, c->N, 2 * c->Qn, 1, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, c->d_in, half * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(g, c->d_in + half, half * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return brecord(c, e, "get populations");
    return sync_status(c);
}

lb_status lb_binary_step(lb_binary* c, int nsteps) {
    lb_status s = bcheck(c);
    if (s != LB_OK) return s;
    if (nsteps < 0) return bfail(LB_EINVAL, "nsteps must be >= 0");
    if (!c->initialised) return bfail(LB_ESTATE, "step before init");
    int k = 0;
    // long runs: replay a graph of GRAPH_STEPS launches per start buffer, captured
    // on a private stream (the legacy default stream cannot be captured) and
    // launched on the context's stream
    if (!c->graph_failed && nsteps >= GRAPH_STEPS) {
        if (!c->graph[c->cur]) {
            cudaGraph_t graph = nullptr;
            cudaError_t e = cudaSuccess;
            if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
            const bool capturing = e == cudaSuccess;
            for (int j = 0; e == cudaSuccess && j < GRAPH_STEPS; ++j) e = step_once(c, (c->cur + j) & 1, c->cap_stream);
            if (capturing) {
                cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &graph);
                if (e == cudaSuccess) e = e2;
            }
            cudaGraphExec_t exec = nullptr;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (e == cudaSuccess) c->graph[c->cur] = exec;
            else {
                cudaGetLastError();
                c->graph_failed = true;
            }
        }
        for (cudaGraphExec_t g = c->graph[c->cur]; g && k + GRAPH_STEPS <= nsteps; k += GRAPH_STEPS) {
            cudaError_t e = cudaGraphLaunch(g, c->stream);
            if (e != cudaSuccess) return brecord(c, e, "binary step graph");
            c->step += GRAPH_STEPS;
        }
    }
    for (; k < nsteps; ++k) {
        cudaError_t e = step_once(c, c->cur, c->stream);
        if (e != cudaSuccess) return brecord(c, e, "binary step");
        c->cur = 1 - c->cur;
        ++c->step;
    }
    return LB_OK;
}

lb_status lb_binary_synchronize(lb_binary* c) {
    lb_status s = bcheck(c);
    if (s != LB_OK) return s;
    return sync_status(c);
}

lb_status lb_binary_fields(lb_binary* c, double* rho, double* phi, double* u, double* v, double* mu) {
    lb_status s = bcheck(c);
    if (s != LB_OK) return s;
    if (!c->initialised) return bfail(LB_ESTATE, "state not initialised");
    if ((s = compute_fields(c)) != LB_OK) return s;
    const long long N = c->N;
    const size_t nb = size_t(N) * sizeof(double);
    const double* w = c->work;
    cudaError_t e = cudaSuccess;
    if (rho) e = cudaMemcpyAsync(rho, w, nb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && phi) e = cudaMemcpyAsync(phi, w + N, nb, cudaMemcpyDeviceToHost, c->stream);
    const int D = c->D;   // workspace: rho, phi, u [D], v [D], mu, ...
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, w + 2 * N, D * nb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, w + (2 + D) * N, D * nb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && mu) e = cudaMemcpyAsync(mu, w + (2 + 2 * D) * N, nb, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return brecord(c, e, "field download");
    return sync_status(c);
}

lb_status lb_binary_stats_get(lb_binary* c, lb_binary_stats* out) {
    lb_status s = bcheck(c);
    if (s != LB_OK) return s;
    if (!out) return bfail(LB_EINVAL, "null output");
    if (!c->initialised) return bfail(LB_ESTATE, "state not initialised");
    const long long N = c->N;
    const int D = c->D;
    std::vector<double> h;
    try {
        h.resize(size_t(2 + 2 * D) * N);
    } catch (...) {
        return bfail(LB_ENOMEM, "host buffer");
    }
    const double* hu = h.data() + 2 * N;
    const double* hv = h.data() + (2 + D) * N;
    s = lb_binary_fields(c, h.data(), h.data() + N, h.data() + 2 * N, h.data() + (2 + D) * N, nullptr);
    if (s != LB_OK && s != LB_EUNSTABLE) return s;
    lb_binary_stats r{};
    r.min_phi = h[N];
    r.max_phi = h[N];
    for (long long i = 0; i < N; ++i) {
        const double rh = h[i], ph = h[N + i];
        double u2 = 0, v2 = 0;
        for (int d = 0; d < D; ++d) {
            r.momentum[d] += rh * hu[d * N + i];
            u2 += hu[d * N + i] * hu[d * N + i];
            v2 += hv[d * N + i] * hv[d * N + i];
        }
        r.mass += rh;
        r.phi_total += ph;
        r.max_u = std::fmax(r.max_u, std::sqrt(u2));
        r.max_v = std::fmax(r.max_v, std::sqrt(v2));
        r.min_phi = std::fmin(r.min_phi, ph);
        r.max_phi = std::fmax(r.max_phi, ph);
    }
    r.step = c->step;
    r.status = s == LB_EUNSTABLE ? LB_EUNSTABLE : 0;
    *out = r;
    return s;
}

}  // extern "C"
