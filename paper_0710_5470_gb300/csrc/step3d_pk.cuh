// Fused D3Q19 forcing-scheme time step, two adjacent x sites per thread.
//
// Same physics and plane pipeline as step_kernel3d (step3d.cuh): a CTA owns a
// TX x TY column tile and marches through a chunk of z planes; the density
// halo is recomputed from the populations of the neighbouring columns; the
// gradient / Laplacian stencils (Eq. 29 with A = 1/6, B = 1/12, C = 1/3,
// D = 1/6) and the divergence of M' (Eq. 28, read in 3D as
// g_a = -d_b (M_ab - delta_ab M_cc / 2)) are split by e_z and carried along
// the march.  What differs is the work split:
//
//   * every thread owns one pair of sites (x, x+1), x even.  The collision
//     (Eqs. 2, 3, 5, 6, 27, 36 and Eq. 4) runs on the pair as packed float32
//     pairs, one paired instruction (FADD2 / FMUL2 / FFMA2) for both sites;
//   * stage A sums the density of 16-bit deviations with mixed-precision
//     adds (float32 accumulator, fp16 / bf16 operand), so a halo site costs
//     one instruction per population besides its load; the own pair's
//     momentum is summed the same way;
//   * the owner thread loads its own pair in stage A and keeps the raw
//     populations in a thread-private shared-memory stash (128-bit accesses)
//     until its collision two planes later, so the stash needs no barrier;
//   * the own sites' gradient, Laplacian and density stay in registers from
//     stage B / stage A to the collision; stage B forms the own pair's
//     stencil parts as packed pairs from one aligned 2-vector and two scalars
//     per row.
//
// Two barriers per plane: after stage A (densities of the plane visible) and
// after stage B (M' of the plane visible).
#pragma once
#include "bounds.cuh"
#include "step3d.cuh"

namespace lbk {

// ------------------------------------------------------------ packed float pairs
struct P2 {
    float2 v;
};
__device__ __forceinline__ P2 pp(float a) { return P2{make_float2(a, a)}; }
__device__ __forceinline__ P2 pp(float a, float b) { return P2{make_float2(a, b)}; }
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2{__fadd2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2 operator-(P2 a) { return P2{make_float2(-a.v.x, -a.v.y)}; }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2{__fadd2_rn(a.v, make_float2(-b.v.x, -b.v.y))}; }
__device__ __forceinline__ P2 operator*(P2 a, P2 b) { return P2{__fmul2_rn(a.v, b.v)}; }
__device__ __forceinline__ P2 fma(P2 a, P2 b, P2 c) { return P2{__ffma2_rn(a.v, b.v, c.v)}; }
__device__ __forceinline__ P2& operator+=(P2& a, P2 b) { return a = a + b; }
__device__ __forceinline__ P2& operator-=(P2& a, P2 b) { return a = a - b; }

template <int E>
__device__ __forceinline__ void add_signed2(P2& acc, P2 v) {
    if constexpr (E == 1) acc += v;
    if constexpr (E == -1) acc -= v;
}

// ------------------------------------------------------------ storage of a pair
// raw 32-bit word of a 16-bit pair and the float32 sum of the two halves into
// two accumulators: one mixed-precision add per value (PTX add.f32.f16 /
// add.f32.bf16, sm_100 and later).
__device__ __forceinline__ void madd_f16x2(float& a, float& b, unsigned w) {
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "add.rn.f32.f16 %0, lo, %0;\n\tadd.rn.f32.f16 %1, hi, %1;\n\t}"
        : "+f"(a), "+f"(b)
        : "r"(w));
}
__device__ __forceinline__ void madd_bf16x2(float& a, float& b, unsigned w) {
    asm("{\n\t.reg .b16 lo, hi;\n\tmov.b32 {lo, hi}, %2;\n\t"
        "add.rn.f32.bf16 %0, lo, %0;\n\tadd.rn.f32.bf16 %1, hi, %1;\n\t}"
        : "+f"(a), "+f"(b)
        : "r"(w));
}

// Pair traits of a storage format: W = raw word of population i >= 1 for two
// sites; decode / encode and the density sum.
template <class S>
struct PairIO;

template <>
struct PairIO<StF32> {
    using W = float2;
    static constexpr bool RAW16 = false;
    __device__ __forceinline__ static W ld(const char* p, unsigned e) { return reinterpret_cast<const float2*>(p)[e >> 1]; }
    __device__ __forceinline__ static P2 dec(W w) { return P2{w}; }
    __device__ __forceinline__ static void st2(char* p, unsigned e, P2 v) { reinterpret_cast<float2*>(p)[e >> 1] = v.v; }
    __device__ __forceinline__ static void st1(char* p, unsigned e, float v) { reinterpret_cast<float*>(p)[e] = v; }
    // rho = (rsum + f_0) + sum_i d_i, balanced tree of paired adds
    __device__ __forceinline__ static P2 rho(float2 f0, const W (&d)[18], float rsum) {
        P2 t[18];
#pragma unroll
        for (int i = 0; i < 18; ++i) t[i] = P2{d[i]};
        return (pp(rsum) + P2{f0}) + tree_sum<0, 18>(t);
    }
};

template <>
struct PairIO<StF16> {
    using W = unsigned;
    static constexpr bool RAW16 = true;
    __device__ __forceinline__ static W ld(const char* p, unsigned e) { return reinterpret_cast<const unsigned*>(p)[e >> 1]; }
    __device__ __forceinline__ static P2 dec(W w) {
        __half2 h;
        *reinterpret_cast<unsigned*>(&h) = w;
        return P2{__half22float2(h)};
    }
    __device__ __forceinline__ static void st2(char* p, unsigned e, P2 v) {
        reinterpret_cast<__half2*>(p)[e >> 1] = __float22half2_rn(v.v);
    }
    __device__ __forceinline__ static void st1(char* p, unsigned e, float v) {
        reinterpret_cast<__half*>(p)[e] = __float2half_rn(v);
    }
    __device__ __forceinline__ static void st2p(char* p, P2 v) { *reinterpret_cast<__half2*>(p) = __float22half2_rn(v.v); }
    __device__ __forceinline__ static void st1p(char* p, float v) { *reinterpret_cast<__half*>(p) = __float2half_rn(v); }
    // rho = (rsum + f_0) + (d_1 + ... + d_9) + (d_10 + ... + d_18), each run of
    // nine summed in order into a float32 accumulator
    __device__ __forceinline__ static P2 rho(float2 f0, const W (&d)[18], float rsum) {
        const P2 a = pp(rsum) + P2{f0};
        float a0 = a.v.x, a1 = a.v.y, b0 = 0.0f, b1 = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            madd_f16x2(a0, a1, d[i]);
            madd_f16x2(b0, b1, d[i + 9]);
        }
        return pp(a0, a1) + pp(b0, b1);
    }
};

template <>
struct PairIO<StBF16> {
    using W = unsigned;
    static constexpr bool RAW16 = true;
    __device__ __forceinline__ static W ld(const char* p, unsigned e) { return reinterpret_cast<const unsigned*>(p)[e >> 1]; }
    __device__ __forceinline__ static P2 dec(W w) {
        __nv_bfloat162 h;
        *reinterpret_cast<unsigned*>(&h) = w;
        return P2{__bfloat1622float2(h)};
    }
    __device__ __forceinline__ static void st2(char* p, unsigned e, P2 v) {
        reinterpret_cast<__nv_bfloat162*>(p)[e >> 1] = __float22bfloat162_rn(v.v);
    }
    __device__ __forceinline__ static void st1(char* p, unsigned e, float v) {
        reinterpret_cast<__nv_bfloat16*>(p)[e] = __float2bfloat16_rn(v);
    }
    __device__ __forceinline__ static void st2p(char* p, P2 v) {
        *reinterpret_cast<__nv_bfloat162*>(p) = __float22bfloat162_rn(v.v);
    }
    __device__ __forceinline__ static void st1p(char* p, float v) { *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v); }
    __device__ __forceinline__ static P2 rho(float2 f0, const W (&d)[18], float rsum) {
        const P2 a = pp(rsum) + P2{f0};
        float a0 = a.v.x, a1 = a.v.y, b0 = 0.0f, b1 = 0.0f;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            madd_bf16x2(a0, a1, d[i]);
            madd_bf16x2(b0, b1, d[i + 9]);
        }
        return pp(a0, a1) + pp(b0, b1);
    }
};


// Density of a pair from its raw populations in the order every item of the
// kernel uses (so that a site's density is bitwise the same in every CTA that
// computes it): MIXED = mixed-precision adds (16-bit storage), otherwise the
// decoded deviations summed as a balanced tree of paired adds.
template <class S, bool MIXED>
__device__ __forceinline__ P2 pair_rho(float2 f0, const typename PairIO<S>::W (&w)[18], float rsum) {
    using IO = PairIO<S>;
    if constexpr (MIXED && IO::RAW16) {
        return IO::rho(f0, w, rsum);
    } else {
        P2 d[18];
#pragma unroll
        for (int i = 0; i < 18; ++i) d[i] = IO::dec(w[i]);
        return (pp(rsum) + P2{f0}) + tree_sum<0, 18>(d);
    }
}

// Momentum j = sum_i d_i e_i of a pair (Eq. 3; sum_i w_i e_i = 0, so the
// deviations give the momentum), opposite velocities differenced first.
template <class S>
__device__ __forceinline__ void pair_momentum(const typename PairIO<S>::W (&w)[18], P2 (&j)[3]) {
    using L = D3Q19;
    using IO = PairIO<S>;
    j[0] = j[1] = j[2] = pp(0.0f);
    static_for<1, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int o = opposite<L>(i);
        if constexpr (i < o) {
            const P2 df = IO::dec(w[i - 1]) - IO::dec(w[o - 1]);
            add_signed2<L::ex(i)>(j[0], df);
            add_signed2<L::ey(i)>(j[1], df);
            add_signed2<L::ez(i)>(j[2], df);
        }
    });
}

// The same momentum from the raw 16-bit words by mixed-precision adds: for
// every axis the populations with e_a = +1 and with e_a = -1 are summed into
// float32 accumulators (one add per value, no decode) and differenced once.
template <class S>
__device__ __forceinline__ void pair_momentum_mixed(const typename PairIO<S>::W (&w)[18], P2 (&j)[3]) {
    using L = D3Q19;
    static_assert(PairIO<S>::RAW16, "16-bit storage");
    float pl[3][2] = {}, mi[3][2] = {};
    static_for<1, 19>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int e[3] = {L::ex(i), L::ey(i), L::ez(i)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if (e[a] == 0) continue;
            float* acc = e[a] > 0 ? pl[a] : mi[a];
            if constexpr (std::is_same<S, StF16>::value) madd_f16x2(acc[0], acc[1], w[i - 1]);
            else madd_bf16x2(acc[0], acc[1], w[i - 1]);
        }
    });
#pragma unroll
    for (int a = 0; a < 3; ++a) j[a] = pp(pl[a][0], pl[a][1]) - pp(mi[a][0], mi[a][1]);
}

// ------------------------------------------------------------ collision of a pair
// collide() of step_kernel.cuh (forcing scheme, deviation space) for two
// sites at once, split into the per-site coefficients (PairColl::prep) and the
// per-population update (PairColl::out).  f^eq of Eqs. 5, 6 with the optimal
// D3Q19 weights, F_i of Eq. 27 with F_0 = -sum F_i, BGK of Eq. 4:
//   omega f^eq_i + F_i = w_i [e.(omega j + g) + e.T.e + omega A0 - u.g]
//   T_cd = 3/2 (omega Q_cd + u_c g_d + u_d g_c),  A0 = p0 - kappa rho lap - trQ/2,
//   Q_cd = rho u_c u_d + lambda (u_c G_d + u_d G_c + delta_cd u.G);
// d_i = f_i - w_i pref (pref = 0: f_i itself); the collided deviation is
// (1 - omega) d_i + w_i [... - omega pref].  Opposite velocities share the
// even part and differ in the sign of w_i e_i.(omega j + g).
struct PairPhys {
    float a, b, T, kappa, omega, nu, pref, rsum;
};

__device__ __forceinline__ P2 rcp2(P2 x) { return pp(__fdividef(1.0f, x.v.x), __fdividef(1.0f, x.v.y)); }

// ------------------------------------------------------------ stencils of a pair
// plane_parts / finish / start of step3d.cuh for the two sites of a pair at
// once: the 3 x 4 density neighbourhood of the pair is read as one aligned
// 2-vector and two scalars per row (9 shared loads instead of 18) and the
// parts are formed with paired float32 instructions.
struct PlaneParts2 {
    P2 dx, dy, s;            // Dx, Dy, S of the plane
    P2 gx, gy, lin, c;       // in-plane parts of d_x, d_y, sum w rho, and rho
};
struct StencilAcc2 {
    P2 gx, gy, gz, lap;
    P2 dx, dy, s;
};

// rc: region index of site 0 of the pair (even); RX even
__device__ __forceinline__ PlaneParts2 plane_parts2(const float* rho, int rc, int RX) {
    const float2 C = *reinterpret_cast<const float2*>(rho + rc);
    const float2 U = *reinterpret_cast<const float2*>(rho + rc + RX);
    const float2 D = *reinterpret_cast<const float2*>(rho + rc - RX);
    const P2 c{C}, yp{U}, ym{D};
    const P2 xm = pp(rho[rc - 1], C.x), xp = pp(C.y, rho[rc + 2]);
    const P2 ppp = pp(U.y, rho[rc + RX + 2]), pm = pp(D.y, rho[rc - RX + 2]);
    const P2 mp = pp(rho[rc + RX - 1], U.x), mm = pp(rho[rc - RX - 1], D.x);
    const P2 sixth = pp(1.0f / 6.0f), twelfth = pp(1.0f / 12.0f);
    PlaneParts2 o;
    o.dx = xp - xm;
    o.dy = yp - ym;
    const P2 f = (xp + xm) + (yp + ym);
    o.s = fma(sixth, c, twelfth * f);
    o.gx = fma(sixth, o.dx, twelfth * ((ppp + pm) - (mp + mm)));
    o.gy = fma(sixth, o.dy, twelfth * ((ppp + mp) - (pm + mm)));
    o.lin = fma(sixth, f, twelfth * ((ppp + pm) + (mp + mm)));
    o.c = c;
    return o;
}

__device__ __forceinline__ void finish2(const StencilAcc2& a, const PlaneParts2& hi, P2 (&G)[3], P2& lap) {
    const P2 twelfth = pp(1.0f / 12.0f);
    G[0] = fma(twelfth, hi.dx, a.gx);
    G[1] = fma(twelfth, hi.dy, a.gy);
    G[2] = a.gz + hi.s;
    lap = fma(pp(2.0f), hi.s, a.lap);
}

__device__ __forceinline__ void start2(StencilAcc2& a, const PlaneParts2& cur) {
    const P2 twelfth = pp(1.0f / 12.0f);
    a.gx = fma(twelfth, a.dx, cur.gx);
    a.gy = fma(twelfth, a.dy, cur.gy);
    a.gz = -a.s;
    a.lap = fma(pp(2.0f), cur.lin + a.s, pp(-4.0f) * cur.c);
    a.dx = cur.dx;
    a.dy = cur.dy;
    a.s = cur.s;
}

struct PairColl {
    P2 Jw[3];      // omega j + g
    P2 E[3];       // even part of the axis pairs (before the weight 1/6)
    P2 WP[3], WT[3];   // diagonal planes xy, xz, yz: w (E_c + T_dd) and w 2T_cd
    P2 omw;        // 1 - omega
    P2 c0;         // omega (rho - rsum) - 2 sum_i (even parts): f_0 gain

    __device__ __forceinline__ void prep(P2 rho, const P2 (&j)[3], const P2 (&G)[3], P2 lap, const P2 (&g)[3],
                                         const PairPhys& ph) {
        const P2 irho = rcp2(rho);
        const P2 u[3] = {j[0] * irho, j[1] * irho, j[2] * irho};
        const P2 ib = rcp2(fma(pp(-ph.b), rho, pp(1.0f)));
        const P2 p0 = fma(rho * pp(ph.T), ib, -(pp(ph.a) * rho * rho));      // Eq. 2
        const P2 cs2 = fma(pp(ph.T) * ib, ib, pp(-2.0f * ph.a) * rho);       // dp0/drho
        const P2 lam = fma(pp(-3.0f * ph.nu), cs2, pp(ph.nu));                // Eq. 36
        P2 lu[3], g3[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            lu[c] = lam * u[c];
            g3[c] = pp(3.0f) * g[c];
        }
        const P2 udg = fma(u[0], G[0], fma(u[1], G[1], u[2] * G[2]));
        const P2 ug = fma(u[0], g[0], fma(u[1], g[1], u[2] * g[2]));
        const P2 w15 = pp(1.5f * ph.omega), w3 = pp(3.0f * ph.omega);
        const P2 ludg = lam * udg;
        P2 Td[3], trQ = pp(0.0f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const P2 q = fma(j[c], u[c], fma(pp(2.0f) * lu[c], G[c], ludg));
            trQ += q;
            Td[c] = fma(w15, q, u[c] * g3[c]);
        }
        constexpr int cc[3] = {0, 0, 1}, dd[3] = {1, 2, 2};
        P2 To[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = cc[k], e = dd[k];
            const P2 q = fma(j[c], u[e], fma(lu[c], G[e], lu[e] * G[c]));
            To[k] = fma(w3, q, fma(u[c], g3[e], u[e] * g3[c]));
        }
        const P2 A0 = (p0 - pp(ph.kappa) * rho * lap) - pp(0.5f) * trQ;
        const P2 Aw = fma(pp(ph.omega), A0 - pp(ph.pref), -ug);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Jw[c] = fma(pp(ph.omega), j[c], g[c]);
            E[c] = Aw + Td[c];
        }
        constexpr float wdg = 1.0f / 12.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            WP[k] = pp(wdg) * (E[cc[k]] + Td[dd[k]]);
            WT[k] = pp(wdg) * To[k];
        }
        omw = pp(1.0f - ph.omega);
        // sum over the pairs of the even parts: axis pairs E_c / 6, diagonal planes 2 WP
        const P2 sum = fma(pp(1.0f / 6.0f), E[0] + E[1] + E[2], pp(2.0f) * (WP[0] + WP[1] + WP[2]));
        c0 = fma(pp(ph.omega), rho - pp(ph.rsum), pp(-2.0f) * sum);   // Eq. 6, sum F_i = 0
    }

    // collided deviations of the opposite pair (i, o), i < o
    template <int i>
    __device__ __forceinline__ void out(P2 di, P2 dn, P2& oi, P2& on) const {
        using L = D3Q19;
        constexpr int c = first_axis<L>(i), e2 = second_axis<L>(i);
        P2 odd;
        if constexpr (e2 < 0) {
            odd = (e_comp<L>(i, c) > 0) ? Jw[c] : -Jw[c];
        } else {
            constexpr int sc = e_comp<L>(i, c), se = e_comp<L>(i, e2);
            odd = (sc > 0) ? ((se > 0) ? Jw[c] + Jw[e2] : Jw[c] - Jw[e2]) : ((se > 0) ? Jw[e2] - Jw[c] : -(Jw[c] + Jw[e2]));
        }
        P2 ev;
        if constexpr (e2 < 0) {
            ev = pp(1.0f / 6.0f) * E[c];
        } else {
            constexpr int k = (c == 0 && e2 == 1) ? 0 : ((c == 0 && e2 == 2) ? 1 : 2);
            constexpr int sg = e_comp<L>(i, c) * e_comp<L>(i, e2);
            ev = (sg > 0) ? WP[k] + WT[k] : WP[k] - WT[k];
        }
        const P2 wo = pp(float(w_vel<L>(i))) * odd;
        oi = fma(omw, di, ev + wo);
        on = fma(omw, dn, ev - wo);
    }
};

// ------------------------------------------------------------ layout
template <int TX, int TY, bool RAW16>
struct LayoutPK {
    static constexpr int H = 2;                     // density halo in y (forcing)
    static constexpr int HX = 2;                    // density halo in x (pairs start on even x)
    static constexpr int TXP = TX / 2;              // pairs per tile row
    static constexpr int NTH = TXP * TY;            // threads: one own pair each
    static constexpr int RX = TX + 2 * HX, RY = TY + 2 * H, RN = RX * RY;
    static constexpr int RXP = RX / 2, NIT = RXP * RY;
    static constexpr int NHALO = NIT - NTH;         // region pairs outside the tile
    static constexpr int NAH = (NHALO + NTH - 1) / NTH;
    static constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY;   // tile + 1 ring
    static constexpr int SXH = SX / 2;
    static constexpr int NRING = SN - TX * TY;      // ring sites (stage B, one site per item)
    static constexpr int NBR = (NRING + NTH - 1) / NTH;
    static constexpr int NRHO = 2;                  // density slots (planes p, p + 1)
    static constexpr int NST = 3;                   // stash slots (planes p, p - 1, p - 2)
    // raw stash words per pair: f_0 pair + 18 raw pairs (16-bit: 20 words as
    // 5 x 16 B; float32: 38 words as 19 float2)
    static constexpr int STW = RAW16 ? 20 : 38;
    static constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }
    static constexpr size_t OFF_RHO = 0;
    static constexpr size_t OFF_ST = al16(OFF_RHO + size_t(NRHO) * RN * 4);
    // moments stash: (rho, j_x, j_y, j_z) pairs per slot, thread-private
    static constexpr size_t OFF_MOM = al16(OFF_ST + size_t(NST) * STW * 4 * NTH);
    static constexpr size_t OFF_MPA = al16(OFF_MOM + size_t(NST) * 4 * 8 * NTH);
    static constexpr size_t OFF_MPB = al16(OFF_MPA + size_t(SN) * 16);
    static constexpr size_t BYTES = al16(OFF_MPB + size_t(SN) * 8);
    static_assert(TX % 4 == 0, "tile width");
    static_assert(NAH <= 2 && NBR <= 2, "items per thread");
    // M' index of ring site (sx, sy): even and odd columns in separate halves
    // so that the pair neighbourhoods of consecutive threads are conflict-free
    __host__ __device__ static constexpr int mp_index(int sx, int sy) { return (sx & 1) * (SY * SXH) + sy * SXH + (sx >> 1); }
};

// Byte offset of site q in the interleaved 16-bit layout (PopPtrs aos = 1):
// blocks of AOS_SITES sites, 18 rows of AOS_SITES values each.
__host__ __device__ __forceinline__ unsigned aos_bytes(unsigned q) {
    return (q / AOS_SITES) * (2 * AOS_BLOCK_HALVES) + (q % AOS_SITES) * 2;
}

// PF: items whose next-plane loads are issued one plane ahead into registers
// (0 none, 1 the own pair, 2 every item); the others load at the start of
// stage A.  MIXED: densities by mixed-precision adds (16-bit storage).
// AOS: populations 1..18 in the interleaved block layout (nx a multiple of
// AOS_SITES): one address per site, the 18 rows at fixed offsets from it;
// args.src[1] / args.dst[1] point at the first block.  PB: stage B of the own
// pair with the paired stencils (plane_parts2) instead of site by site.
template <class S, int TX, int TY, int MINB, int PF, bool MIXED, bool AOS = false, bool PB = false>
__global__ void __launch_bounds__((TX / 2) * TY, MINB) step_kernel3d_pk(const StepArgs args) {
    using L = D3Q19;
    using IO = PairIO<S>;
    using Wd = typename IO::W;
    constexpr bool RAW16 = IO::RAW16;
    using Lay = LayoutPK<TX, TY, RAW16>;
    constexpr int H = Lay::H, HX = Lay::HX, TXP = Lay::TXP, NTH = Lay::NTH;
    constexpr int RX = Lay::RX, RXP = Lay::RXP, SX = Lay::SX;
    constexpr int NAH = Lay::NAH, NBR = Lay::NBR;
    static_assert(!AOS || RAW16, "interleaved layout: 16-bit storage only");
    constexpr int ROWB = 2 * AOS_SITES;             // bytes of one population row of a block

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* rho_s = reinterpret_cast<float*>(smem_raw + Lay::OFF_RHO);
    unsigned char* stash = smem_raw + Lay::OFF_ST;
    float2* mom_s = reinterpret_cast<float2*>(smem_raw + Lay::OFF_MOM);
    float4* mpA = reinterpret_cast<float4*>(smem_raw + Lay::OFF_MPA);   // (Mxx, Mxy, Mxz, Myy)
    float2* mpB = reinterpret_cast<float2*>(smem_raw + Lay::OFF_MPB);   // (Myz, Mzz)

    const int nx = args.nx, ny = args.ny, nz = args.nz;
    const int tid = threadIdx.x;
    const int px = tid % TXP, py = tid / TXP;
    const int4 wk = args.work[blockIdx.x];
    const int x0 = wk.x, y0 = wk.y, z0 = wk.z, z1 = wk.w;
    const int plane = nx * ny;
#ifdef LB_DEBUG_BOUNDS
    const size_t nsites = size_t(plane) * nz;   // sites of the lattice
#endif
    const PairPhys ph{args.fa, args.fb, args.fT, args.fkappa, args.fomega, args.fnu, args.pref, args.rsum};
    const float pk = args.fkappa;

    // ---- stage-A items: the own pair, then halo pairs (rows above / below the
    // tile, then the left and right pair of every tile row); in-plane element
    // index of the first site (even) and the density slot index
    const int xo = x0 + 2 * px, yo = y0 + py;
    const bool own = xo < nx && yo < ny;
    unsigned a_in[1 + NAH];
    int a_rs[1 + NAH];
    a_in[0] = unsigned(wrapi(yo, ny) * nx + wrapi(xo, nx));
    a_rs[0] = (py + H) * RX + 2 * px + HX;
#pragma unroll
    for (int m = 0; m < NAH; ++m) {
        const int h = tid + m * NTH;
        a_rs[1 + m] = -1;
        a_in[1 + m] = 0;
        if (h < Lay::NHALO) {
            int rxp, ry;
            if (h < 2 * H * RXP) {
                const int r = h / RXP;
                rxp = h % RXP;
                ry = r < H ? r : r + TY;
            } else {
                const int k = h - 2 * H * RXP;
                ry = H + (k >> 1);
                rxp = (k & 1) ? RXP - 1 : 0;
            }
            a_rs[1 + m] = ry * RX + 2 * rxp;
            a_in[1 + m] = unsigned(wrapi(y0 - H + ry, ny) * nx + wrapi(x0 - HX + 2 * rxp, nx));
        }
    }
    // ---- stage-B items: own site 0, own site 1, ring sites; region index of
    // the site and its M' index
    constexpr int NB = 2 + NBR;
    int b_rc[NB], b_mp[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) {
        int sx = 0, sy = 0;
        bool ok = true;
        if (m < 2) {
            sx = 2 * px + 1 + m;
            sy = py + 1;
        } else {
            const int r = tid + (m - 2) * NTH;
            ok = r < Lay::NRING;
            if (r < 2 * SX) {
                sx = r % SX;
                sy = r < SX ? 0 : Lay::SY - 1;
            } else {
                const int k = r - 2 * SX;
                sy = 1 + (k >> 1);
                sx = (k & 1) ? SX - 1 : 0;
            }
        }
        b_rc[m] = ok ? (sy + H - 1) * RX + (sx + HX - 1) : -1;
        b_mp[m] = Lay::mp_index(sx, sy);
    }
    // push targets: x columns of the pair's neighbours, row offsets of the pair
    const unsigned xm1 = unsigned(wrapi(xo - 1, nx)), xc = unsigned(wrapi(xo, nx));
    const unsigned xp2 = unsigned(wrapi(xo + 2, nx));
    const unsigned yr[3] = {unsigned(wrapi(yo - 1, ny) * nx), unsigned(wrapi(yo, ny) * nx),
                            unsigned(wrapi(yo + 1, ny) * nx)};

    const int pstart = z0 - 2, pend = z1 + 2;
    const int vol = nz * plane;
    int ld_off = wrapi(pstart, nz) * plane;
    int zr[3] = {wrapi(z0 - 1, nz) * plane, wrapi(z0, nz) * plane, wrapi(z0 + 1, nz) * plane};
    auto advance = [&](int& v) {
        v += plane;
        if (v == vol) v = 0;
    };

    // interleaved layout: byte offset of each item within its plane (planes
    // start on a block: nx * ny is a multiple of AOS_SITES)
    unsigned a_h[1 + NAH];
#pragma unroll
    for (int m = 0; m < 1 + NAH; ++m) a_h[m] = AOS ? aos_bytes(a_in[m]) : 0u;
    // raw populations of the items of plane ld_off
    float2 r0[1 + NAH];
    Wd ri[1 + NAH][18];
    auto issue = [&](int mb, int me) {
#pragma unroll
        for (int m = 0; m < 1 + NAH; ++m) {
            if (m >= mb && m < me && (m == 0 || a_rs[m] >= 0)) {
                const unsigned q = unsigned(ld_off) + a_in[m];
                LB_GUARD(size_t(q) + 1 < nsites, BK_PK_LOAD, q, r0[m] = make_float2(0.f, 0.f);
                         for (int i = 0; i < 18; ++i) ri[m][i] = Wd{}; continue)
                r0[m] = reinterpret_cast<const float2*>(args.src[0])[q >> 1];
                if constexpr (AOS) {
                    const char* b = args.src[1] + (size_t(unsigned(ld_off)) / AOS_SITES) * (2 * AOS_BLOCK_HALVES) + a_h[m];
#pragma unroll
                    for (int i = 1; i < 19; ++i) ri[m][i - 1] = *reinterpret_cast<const unsigned*>(b + (i - 1) * ROWB);
                } else {
                    static_for<1, 19>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        ri[m][i - 1] = IO::ld(args.src[i], q);
                    });
                }
            }
        }
    };
    constexpr int NPF = PF == 0 ? 0 : (PF == 1 ? 1 : 1 + NAH);   // items prefetched
    issue(0, NPF);

    StencilAcc<float> acc[NB];
#pragma unroll
    for (int m = 0; m < NB; ++m) acc[m] = StencilAcc<float>{0, 0, 0, 0, 0, 0, 0};
    StencilAcc2 acc2{pp(0.f), pp(0.f), pp(0.f), pp(0.f), pp(0.f), pp(0.f), pp(0.f)};
    // body force carries of the own pair: -(U0(q-1) + U-(q-2)) and -U-(q-1)
    P2 gacc1[3] = {pp(0.f), pp(0.f), pp(0.f)}, gacc2[3] = {pp(0.f), pp(0.f), pp(0.f)};
    // G, lap of the own pair: of plane q - 1 (Gc, for this plane's collision) and of q (Gn)
    P2 Gc[3] = {pp(0.f), pp(0.f), pp(0.f)}, lapc = pp(0.f);
    bool bad = false;

    for (int p = pstart; p < pend; ++p) {
        const int it = p - pstart;
        // ---------------- stage A: density of plane p on the region
        {
            if (NPF < 1 + NAH) issue(NPF, 1 + NAH);
            advance(ld_off);
            float* rho_w = rho_s + (it & 1) * Lay::RN;
            const int slot = it % Lay::NST;
#pragma unroll
            for (int m = 0; m < 1 + NAH; ++m) {
                if (m == 0 || a_rs[m] >= 0) {
                    const P2 r = pair_rho<S, MIXED>(r0[m], ri[m], ph.rsum);
                    LB_GUARD(a_rs[m] >= 0 && a_rs[m] + 1 < Lay::RN, BK_PK_SHARED, a_rs[m], continue)
                    *reinterpret_cast<float2*>(rho_w + a_rs[m]) = r.v;
                    if (m == 0) {
                        // thread-private stash of the own pair: raw populations and (rho, j)
                        float2* mo = mom_s + slot * 4 * NTH + tid;
                        mo[0] = r.v;
                        P2 j[3];
                        if constexpr (MIXED && RAW16) pair_momentum_mixed<S>(ri[0], j);
                        else pair_momentum<S>(ri[0], j);
                        mo[NTH] = j[0].v;
                        mo[2 * NTH] = j[1].v;
                        mo[3 * NTH] = j[2].v;
                        unsigned char* st = stash + size_t(slot) * Lay::STW * 4 * NTH;
                        if constexpr (RAW16) {
                            uint4* s4 = reinterpret_cast<uint4*>(st) + tid;
                            s4[0] = make_uint4(__float_as_uint(r0[0].x), __float_as_uint(r0[0].y), ri[0][0], ri[0][1]);
#pragma unroll
                            for (int c = 1; c < 5; ++c)
                                s4[c * NTH] = make_uint4(ri[0][4 * c - 2], ri[0][4 * c - 1], ri[0][4 * c], ri[0][4 * c + 1]);
                        } else {
                            float2* s2 = reinterpret_cast<float2*>(st) + tid;
                            s2[0] = r0[0];
#pragma unroll
                            for (int i = 1; i < 19; ++i) s2[i * NTH] = *reinterpret_cast<const float2*>(&ri[0][i - 1]);
                        }
                    }
                }
            }
            if (NPF > 0 && p + 1 < pend) issue(0, NPF);
        }
        __syncthreads();

        // ---------------- stage B: stencil parts of plane p; G, lap, M' of plane q = p - 1
        const bool assemble = it >= 2;
        float Go[2][4];
        P2 Gn[3], lapn;
        {
            const float* rho_p = rho_s + (it & 1) * Lay::RN;
            if constexpr (PB) {
                const PlaneParts2 cur = plane_parts2(rho_p, b_rc[0], RX);
                if (assemble) {
                    finish2(acc2, cur, Gn, lapn);
#pragma unroll
                    for (int m = 0; m < 2; ++m) {
                        const float G[3] = {m ? Gn[0].v.y : Gn[0].v.x, m ? Gn[1].v.y : Gn[1].v.x,
                                            m ? Gn[2].v.y : Gn[2].v.x};
                        const float g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
                        const float hk = 0.5f * pk * g2;
                        LB_GUARD(b_mp[m] >= 0 && b_mp[m] < Lay::SN, BK_PK_SHARED, b_mp[m], continue)
                        mpA[b_mp[m]] = make_float4(pk * G[0] * G[0] - hk, pk * G[0] * G[1], pk * G[0] * G[2],
                                                   pk * G[1] * G[1] - hk);
                        mpB[b_mp[m]] = make_float2(pk * G[1] * G[2], pk * G[2] * G[2] - hk);
                    }
                }
                start2(acc2, cur);
            }
#pragma unroll
            for (int m = PB ? 2 : 0; m < NB; ++m) {
                if (b_rc[m] < 0) continue;
                const PlaneParts<float> cur = plane_parts(rho_p, b_rc[m], RX);
                if (assemble) {
                    float G[3], lap;
                    finish(acc[m], cur, G, lap);
                    const float g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
                    const float hk = 0.5f * pk * g2;
                    LB_GUARD(b_mp[m] >= 0 && b_mp[m] < Lay::SN, BK_PK_SHARED, b_mp[m], continue)
                    mpA[b_mp[m]] = make_float4(pk * G[0] * G[0] - hk, pk * G[0] * G[1], pk * G[0] * G[2],
                                               pk * G[1] * G[1] - hk);
                    mpB[b_mp[m]] = make_float2(pk * G[1] * G[2], pk * G[2] * G[2] - hk);
                    if (m < 2) {
                        Go[m][0] = G[0]; Go[m][1] = G[1]; Go[m][2] = G[2]; Go[m][3] = lap;
                    }
                }
                start(acc[m], cur);
            }
        }
        __syncthreads();

        // ---------------- body force of the own pair: parts of plane q (Eq. 28)
        P2 gf[3] = {pp(0.f), pp(0.f), pp(0.f)};
        if (assemble) {
            // neighbourhood columns c = 0..3 (sites x-1 .. x+2) and rows -1, 0, +1 of the
            // ring; site 0 of the pair is column 1, site 1 column 2
            float sp[2][3] = {}, sz[2][3] = {}, se[2][3] = {}, zc[2][3];
            const int cx0 = 2 * px, cy = py + 1;
#pragma unroll
            for (int r = -1; r <= 1; ++r) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = Lay::mp_index(cx0 + c, cy + r);
                    const float4 A = mpA[k];
                    const float2 B = mpB[k];
#pragma unroll
                    for (int s = 0; s < 2; ++s) {
                        const int dx = c - 1 - s;   // column offset from site s
                        if (dx < -1 || dx > 1) continue;
                        if (r == 0 && dx == 0) {
                            zc[s][0] = A.z; zc[s][1] = B.x; zc[s][2] = B.y;
                        } else if (r == 0) {        // x neighbour, sign dx
                            if (dx > 0) {
                                sp[s][0] += A.x; sp[s][1] += A.y; sp[s][2] += A.z;
                            } else {
                                sp[s][0] -= A.x; sp[s][1] -= A.y; sp[s][2] -= A.z;
                            }
                            sz[s][0] += A.z; sz[s][1] += B.x; sz[s][2] += B.y;
                        } else if (dx == 0) {       // y neighbour, sign r
                            if (r > 0) {
                                sp[s][0] += A.y; sp[s][1] += A.w; sp[s][2] += B.x;
                            } else {
                                sp[s][0] -= A.y; sp[s][1] -= A.w; sp[s][2] -= B.x;
                            }
                            sz[s][0] += A.z; sz[s][1] += B.x; sz[s][2] += B.y;
                        } else {                    // xy diagonal (dx, r)
                            const float ax = dx > 0 ? A.x : -A.x, ay = dx > 0 ? A.y : -A.y, az = dx > 0 ? A.z : -A.z;
                            const float by = r > 0 ? A.y : -A.y, bw = r > 0 ? A.w : -A.w, bx = r > 0 ? B.x : -B.x;
                            se[s][0] += ax + by;
                            se[s][1] += ay + bw;
                            se[s][2] += az + bx;
                        }
                    }
                }
            }
            constexpr float sixth = 1.0f / 6.0f, twelfth = 1.0f / 12.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const P2 SP = pp(sp[0][c], sp[1][c]), SZ = pp(sz[0][c], sz[1][c]), SE = pp(se[0][c], se[1][c]);
                const P2 ZC = pp(zc[0][c], zc[1][c]);
                const P2 u0 = fma(pp(sixth), SP, pp(twelfth) * SE);
                const P2 up = fma(pp(twelfth), SP + SZ, pp(sixth) * ZC);
                const P2 um = fma(pp(twelfth), SP - SZ, -(pp(sixth) * ZC));
                // g(q-1) = -(U+(q) + U0(q-1) + U-(q-2))
                gf[c] = gacc1[c] - up;
                gacc1[c] = gacc2[c] - u0;
                gacc2[c] = -um;
            }
        }

        // ---------------- stage C: collide and push plane s = p - 2
        const int s = p - 2;
        if (s >= z0) {
            const int slot = (it - 2) % Lay::NST;
            const float2* mo = mom_s + slot * 4 * NTH + tid;
            const P2 rho = P2{mo[0]};
            const P2 G[3] = {Gc[0], Gc[1], Gc[2]};
            const P2 lap = lapc;
            if (own) bad |= !(rho.v.x > 0.f) || !(rho.v.x < 1e30f) || !(rho.v.y > 0.f) || !(rho.v.y < 1e30f);
            const unsigned char* st = stash + size_t(slot) * Lay::STW * 4 * NTH;
            // raw stashed populations: the f_0 pair, then one word per population
            Wd w[19];
            float2 f0;
            if constexpr (RAW16) {
                const uint4* s4 = reinterpret_cast<const uint4*>(st) + tid;
                unsigned u[20];
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const uint4 v = s4[c * NTH];
                    u[4 * c] = v.x; u[4 * c + 1] = v.y; u[4 * c + 2] = v.z; u[4 * c + 3] = v.w;
                }
                f0 = make_float2(__uint_as_float(u[0]), __uint_as_float(u[1]));
#pragma unroll
                for (int i = 1; i < 19; ++i) w[i] = u[i + 1];
            } else {
                const float2* s2 = reinterpret_cast<const float2*>(st) + tid;
                f0 = s2[0];
#pragma unroll
                for (int i = 1; i < 19; ++i) w[i] = s2[i * NTH];
            }
            const P2 j[3] = {P2{mo[NTH]}, P2{mo[2 * NTH]}, P2{mo[3 * NTH]}};
            PairColl K;
            K.prep(rho, j, G, lap, gf, ph);
            if (own) {
                // push f*_i(r) to r + e_i: populations with e_x = 0 as aligned pairs,
                // the others site by site
                // interleaved layout: block-row byte offsets of the destination
                // planes (64-bit) and rows, block byte offsets of the x columns
                size_t zb[3] = {0, 0, 0};
                unsigned yb[3] = {0, 0, 0}, cb[4] = {0, 0, 0, 0};
                if constexpr (AOS) {
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        zb[k] = size_t(unsigned(zr[k])) / AOS_SITES * (2 * AOS_BLOCK_HALVES);
                        yb[k] = yr[k] / AOS_SITES * (2 * AOS_BLOCK_HALVES);
                    }
                    cb[0] = aos_bytes(xm1);
                    cb[1] = aos_bytes(xc);
                    cb[2] = aos_bytes(xc + 1);
                    cb[3] = aos_bytes(xp2);
                }
                auto store = [&](auto I, P2 v) {
                    constexpr int i = decltype(I)::value;
                    constexpr int ex = L::ex(i), ey = L::ey(i), ez = L::ez(i);
#ifdef LB_DEBUG_BOUNDS
                    {
                        const size_t row0 = size_t(unsigned(zr[1 + ez])) + yr[1 + ey];
                        const size_t xa = ex == 0 ? xc : (ex == 1 ? xc + 1 : xm1);
                        const size_t xb = ex == 0 ? xc + 1 : (ex == 1 ? xp2 : xc);
                        LB_GUARD(row0 + xa < nsites && row0 + xb < nsites, BK_PK_STORE, row0 + xa, return)
                    }
#endif
                    if constexpr (AOS) {
                        char* b = args.dst[1] + zb[1 + ez] + yb[1 + ey] + (i - 1) * ROWB;
                        if constexpr (ex == 0) {
                            IO::st2p(b + cb[1], v);
                        } else if constexpr (ex == 1) {
                            IO::st1p(b + cb[2], v.v.x);
                            IO::st1p(b + cb[3], v.v.y);
                        } else {
                            IO::st1p(b + cb[0], v.v.x);
                            IO::st1p(b + cb[1], v.v.y);
                        }
                    } else {
                        const unsigned row = unsigned(zr[1 + ez]) + yr[1 + ey];
                        if constexpr (ex == 0) {
                            IO::st2(args.dst[i], row + xc, v);
                        } else if constexpr (ex == 1) {
                            IO::st1(args.dst[i], row + xc + 1, v.v.x);
                            IO::st1(args.dst[i], row + xp2, v.v.y);
                        } else {
                            IO::st1(args.dst[i], row + xm1, v.v.x);
                            IO::st1(args.dst[i], row + xc, v.v.y);
                        }
                    }
                };
                const P2 o0 = fma(K.omw, P2{f0}, K.c0);
#ifdef LB_DEBUG_BOUNDS
                const size_t q0 = size_t(unsigned(zr[1])) + yr[1] + xc;
                if (lbk::in_bounds(q0 + 1 < nsites, BK_PK_STORE, q0))
#endif
                    reinterpret_cast<float2*>(args.dst[0])[(unsigned(zr[1]) + yr[1] + xc) >> 1] = o0.v;
                static_for<1, 19>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    constexpr int o = opposite<L>(i);
                    if constexpr (i < o) {
                        P2 oi, on;
                        K.template out<i>(IO::dec(w[i]), IO::dec(w[o]), oi, on);
                        store(std::integral_constant<int, i>{}, oi);
                        store(std::integral_constant<int, o>{}, on);
                    }
                });
            }
            advance(zr[0]);
            advance(zr[1]);
            advance(zr[2]);
        }
        if (assemble) {
            if constexpr (PB) {
#pragma unroll
                for (int c = 0; c < 3; ++c) Gc[c] = Gn[c];
                lapc = lapn;
            } else {
#pragma unroll
                for (int c = 0; c < 3; ++c) Gc[c] = pp(Go[0][c], Go[1][c]);
                lapc = pp(Go[0][3], Go[1][3]);
            }
        }
    }
    if (bad) atomicOr(args.status, 1u);
}

}  // namespace lbk
