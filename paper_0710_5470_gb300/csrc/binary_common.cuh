// Shared pieces of the binary-fluid kernels (binary2d.cu: D2Q9 and the C ABI,
// binary3d.cu: D3Q19): periodic wrap, the argument block of a step and the
// per-site arithmetic of the model (stated in include/lb.h beside
// lb_binary_params): f^eq (Eqs. 5, 6 with the binary p0 and phi's gradient
// terms), g^eq, and the force populations of Eq. 27.  The arithmetic is
// written once for a scalar (float, double) and for a packed pair of float32
// sites (lbk::P2: FADD2 / FMUL2 / FFMA2, one instruction for two sites), and
// once for both lattices (every velocity component and weight a compile-time
// constant inside static_for).
#pragma once
#include <cuda_runtime.h>

#include "aux_kernels.cuh"
#include "lattice.cuh"
#include "step3d_pk.cuh"   // lbk::P2: packed float32 pairs

namespace lbb {

using lbk::D2Q9;
using lbk::D3Q19;
using lbk::P2;
using lbk::pp;
using lbk::static_for;

// Periodic wrap of an offset coordinate: one compare-and-add for v in
// [-n, 2n), the integer modulo otherwise (lattices narrower than a tile).
__host__ __device__ __forceinline__ int wrapc(int v, int n) {
    if (v < 0) v += n;
    else if (v >= n) v -= n;
    if (unsigned(v) >= unsigned(n)) {
        v %= n;
        if (v < 0) v += n;
    }
    return v;
}

template <class real>
struct StepArgs {
    const real* src;     // populations after streaming: f_0..f_{Q-1} then g_0..g_{Q-1}, each `pitch` elements
    real* dst;
    const real* phi;     // D3Q19: phi = sum_i g_i of src, one value per site (binary_phi_kernel)
    unsigned pitch;      // 2 Q pitch < 2^32: element offsets within a set are 32-bit
    int nx, ny, nz;
    real A, B, kappa, Gamma, omega, omega_phi;   // omega = 1/tau, omega_phi = 1/tau_phi
    float pref;          // 16-bit sets: f_i (i >= 1) are stored as f_i - w_i pref
    unsigned* status;
};

template <class real>
__device__ __forceinline__ real cst(double d) { return real(d); }
template <>
__device__ __forceinline__ P2 cst<P2>(double d) { return pp(float(d)); }

// Weights of the optimum: w_i = w^p_i = w^t_i (Sec. VIII; Eq. 31 with R4).
template <class L, int I>
__device__ __forceinline__ constexpr double W() { return lbk::w_vel<L>(I); }

template <int E, class real>
__device__ __forceinline__ real signed_add(real acc, real v) {
    if constexpr (E > 0) return acc + v;
    else if constexpr (E < 0) return acc - v;
    else return acc;
}

// e_I . u for a velocity with components in {-1, 0, 1}: adds only.
template <class L, int I, class real>
__device__ __forceinline__ real edot(const real (&u)[L::D]) {
    constexpr int ex = L::ex(I), ey = L::ey(I), ez = L::ez(I);
    if constexpr (ex != 0) {
        real a = ex > 0 ? u[0] : -u[0];
        a = signed_add<ey>(a, u[1]);
        if constexpr (L::D == 3) a = signed_add<ez>(a, u[2]);
        return a;
    } else if constexpr (ey != 0) {
        real a = ey > 0 ? u[1] : -u[1];
        if constexpr (L::D == 3) a = signed_add<ez>(a, u[2]);
        return a;
    } else if constexpr (L::D == 3 && ez != 0) {
        return ez > 0 ? u[2] : -u[2];
    } else {
        return cst<real>(0.0);
    }
}

template <class L, class real>
__device__ __forceinline__ real dot(const real (&a)[L::D], const real (&b)[L::D]) {
    real s = a[0] * b[0] + a[1] * b[1];
    if constexpr (L::D == 3) s = s + a[2] * b[2];
    return s;
}

// The velocity part of Eq. 5 with lambda = 0 for population I of a density
// `dens` moving with u: w_I (dens e.u + 3/2 [dens (e.u)^2 - dens |u|^2 / 3]).
template <class L, int I, class real>
__device__ __forceinline__ real velocity_part(real dens, const real (&u)[L::D], real usq3) {
    const real eu = edot<L, I>(u);
    const real de = dens * eu;
    return cst<real>(W<L, I>()) * (de + cst<real>(1.5) * (de * eu - dens * usq3));
}

// f^eq_i, i >= 1, of the binary model (Eq. 5 with p0 = rho/3 + A/2 phi^2 +
// 3B/4 phi^4, w^t kappa phi lap(phi) and, in the equilibrium scheme,
// sum_{a<=b} w^ab kappa d_a phi d_b phi); f^eq_0 = rho - sum (Eq. 6).
template <class L, bool MTERMS, class real>
__device__ __forceinline__ void f_equilibrium(real rho, const real (&u)[L::D], real phi, const real (&gr)[L::D],
                                              real lap, real A, real B, real kappa, real (&fe)[L::Q]) {
    const real phi2 = phi * phi;
    const real p0 = rho * cst<real>(1.0 / 3.0) + cst<real>(0.5) * A * phi2 + cst<real>(0.75) * B * phi2 * phi2;
    const real iso = p0 - kappa * phi * lap;
    const real usq3 = dot<L>(u, u) * cst<real>(1.0 / 3.0);
    real sum = cst<real>(0.0);
    static_for<1, L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        real pr = cst<real>(W<L, i>()) * iso;
        if constexpr (MTERMS) {
            static_for<0, L::D>([&](auto AA) {
                constexpr int a = decltype(AA)::value;
                static_for<a, L::D>([&](auto BB) {
                    constexpr int b = decltype(BB)::value;
                    constexpr double wab = lbk::w_m<L>(i, a, b);
                    if constexpr (wab != 0.0) pr += cst<real>(wab) * (kappa * gr[a] * gr[b]);
                });
            });
        }
        fe[i] = velocity_part<L, i>(rho, u, usq3) + pr;
        sum += fe[i];
    });
    fe[0] = rho - sum;
}

// g^eq_i = velocity part of phi moving with v + w_i Gamma mu (i >= 1),
// g^eq_0 = phi - sum: sum g = phi, sum g e = phi v, sum g e e = Gamma mu I + phi v v.
template <class L, class real>
__device__ __forceinline__ void g_equilibrium(real phi, const real (&v)[L::D], real mu, real Gamma,
                                              real (&ge)[L::Q]) {
    const real gm = Gamma * mu;
    const real usq3 = dot<L>(v, v) * cst<real>(1.0 / 3.0);
    real sum = cst<real>(0.0);
    static_for<1, L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        ge[i] = velocity_part<L, i>(phi, v, usq3) + cst<real>(W<L, i>()) * gm;
        sum += ge[i];
    });
    ge[0] = phi - sum;
}

// Force populations of Eq. 27, F_i = w_i (e.g + 3/2 [2 (e.u)(e.g) - 2 u.g / 3]),
// F_0 = -sum (reading R8: sum_i F_i = 0).
template <class L, class real>
__device__ __forceinline__ void force_populations(const real (&u)[L::D], const real (&g)[L::D], real (&F)[L::Q]) {
    const real ug23 = dot<L>(u, g) * cst<real>(2.0 / 3.0);
    real sum = cst<real>(0.0);
    static_for<1, L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        const real eg = edot<L, i>(g);
        const real eu = edot<L, i>(u);
        F[i] = cst<real>(W<L, i>()) * (eg + cst<real>(1.5) * (cst<real>(2.0) * eu * eg - ug23));
        sum += F[i];
    });
    F[0] = -sum;
}

// The collision of one site (or a packed pair) streamed population by
// population: for i = 1 .. Q-1 it forms f^eq_i, (forcing) F_i and g^eq_i with
// the arithmetic of f_equilibrium, force_populations and g_equilibrium,
// relaxes f_i with omega and g_i with omega_phi and hands f*_i, g*_i to
// push(integral_constant<int, i>, f*_i, g*_i) at once; i = 0 follows from the
// running sums (f^eq_0 = rho - sum, Eq. 6; F_0 = -sum, reading R8; g^eq_0 =
// phi - sum).  No population array beyond f and g is ever live, which keeps a
// thread's registers low enough for more resident CTAs.
template <class L, bool FORCING, class real, class Push>
__device__ __forceinline__ void collide_stream(const real (&f)[L::Q], const real (&g)[L::Q], real rho,
                                               const real (&u)[L::D], real phi, const real (&gr)[L::D], real lap,
                                               const real (&bf)[L::D], const real (&v)[L::D], real mu, real A,
                                               real B, real kappa, real Gamma, real omega, real omega_phi,
                                               Push&& push) {
    const real phi2 = phi * phi;
    const real p0 = rho * cst<real>(1.0 / 3.0) + cst<real>(0.5) * A * phi2 + cst<real>(0.75) * B * phi2 * phi2;
    const real iso = p0 - kappa * phi * lap;
    const real usq3 = dot<L>(u, u) * cst<real>(1.0 / 3.0);
    const real vsq3 = dot<L>(v, v) * cst<real>(1.0 / 3.0);
    const real gm = Gamma * mu;
    real ug23 = cst<real>(0.0);
    if constexpr (FORCING) ug23 = dot<L>(u, bf) * cst<real>(2.0 / 3.0);
    real sfe = cst<real>(0.0), sF = cst<real>(0.0), sge = cst<real>(0.0);
    static_for<1, L::Q>([&](auto K) {
        constexpr int i = decltype(K)::value;
        real pr = cst<real>(W<L, i>()) * iso;
        if constexpr (!FORCING) {
            static_for<0, L::D>([&](auto AA) {
                constexpr int a = decltype(AA)::value;
                static_for<a, L::D>([&](auto BB) {
                    constexpr int b = decltype(BB)::value;
                    constexpr double wab = lbk::w_m<L>(i, a, b);
                    if constexpr (wab != 0.0) pr += cst<real>(wab) * (kappa * gr[a] * gr[b]);
                });
            });
        }
        const real fe = velocity_part<L, i>(rho, u, usq3) + pr;
        sfe += fe;
        real fs = f[i] + omega * (fe - f[i]);
        if constexpr (FORCING) {
            const real eg = edot<L, i>(bf), eu = edot<L, i>(u);
            const real Fi = cst<real>(W<L, i>()) * (eg + cst<real>(1.5) * (cst<real>(2.0) * eu * eg - ug23));
            sF += Fi;
            fs += Fi;
        }
        const real ge = velocity_part<L, i>(phi, v, vsq3) + cst<real>(W<L, i>()) * gm;
        sge += ge;
        push(K, fs, g[i] + omega_phi * (ge - g[i]));
    });
    real fs0 = f[0] + omega * ((rho - sfe) - f[0]);
    if constexpr (FORCING) fs0 += -sF;
    push(std::integral_constant<int, 0>{}, fs0, g[0] + omega_phi * ((phi - sge) - g[0]));
}

}  // namespace lbb
