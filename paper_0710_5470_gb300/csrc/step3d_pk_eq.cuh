// Fused D3Q19 equilibrium-scheme time step, two adjacent x sites per thread.
//
// The equilibrium scheme of Secs. II-V in 3D (Sec. VII): f^eq of Eq. 5 with
// the pressure-tensor terms M_ab = kappa d_a rho d_b rho weighted by the
// optimal w^ab_i, f_0 by Eq. 6, BGK and push-streaming (Eq. 4); no body force.
// The work is split as in the forcing scheme's pair kernel (step3d_pk.cuh):
// a CTA owns a TX x TY column tile and marches through a chunk of z planes,
// every thread owns one pair of x sites, densities and the own momentum are
// summed from the raw 16-bit words by mixed-precision adds, the own pair's
// raw populations wait in a thread-private shared-memory stash for their
// collision, and the stencils (Eq. 29) are split by e_z and carried along the
// march, the own pair's parts formed as pairs.  Without the body force the
// collision of plane p - 1 follows the density of plane p directly: a density
// halo of one row in y, two stash slots, one barrier per plane.
#pragma once
#include "step3d_pk.cuh"

namespace lbk {

template <int TX, int TY, bool RAW16>
struct LayoutPKE {
    static constexpr int H = 1;                     // density halo in y
    static constexpr int HX = 2;                    // density halo in x (pairs start on even x)
    static constexpr int TXP = TX / 2;
    static constexpr int NTH = TXP * TY;
    static constexpr int RX = TX + 2 * HX, RY = TY + 2 * H, RN = RX * RY;
    static constexpr int RXP = RX / 2, NIT = RXP * RY;
    static constexpr int NHALO = NIT - NTH;
    static constexpr int NAH = (NHALO + NTH - 1) / NTH;
    static constexpr int NRHO = 2;                  // density slots (planes p, p - 1)
    static constexpr int NST = 2;                   // stash slots (planes p, p - 1)
    static constexpr int STW = RAW16 ? 20 : 38;     // raw stash words per pair
    static constexpr size_t al16(size_t x) { return (x + 15) / 16 * 16; }
    static constexpr size_t OFF_RHO = 0;
    static constexpr size_t OFF_ST = al16(OFF_RHO + size_t(NRHO) * RN * 4);
    static constexpr size_t OFF_MOM = al16(OFF_ST + size_t(NST) * STW * 4 * NTH);
    static constexpr size_t BYTES = al16(OFF_MOM + size_t(NST) * 4 * 8 * NTH);
    static_assert(TX % 4 == 0, "tile width");
    static_assert(NAH <= 2, "items per thread");
};

// collide() of step_kernel.cuh for the D3Q19 equilibrium scheme and two sites
// at once (deviation space): the forcing-free even and odd parts of PairColl
// plus the M terms of the optimal weights: axis direction along c: 5/12 Mw_cc
// - 1/3 (Mw_dd + Mw_ee); diagonal in the plane (c, d): -1/24 (Mw_cc + Mw_dd)
// + 1/12 Mw_ee + sign(e_c e_d) / 4 Mw_cd; Mw = omega kappa d rho d rho.
struct PairCollEq {
    P2 Jw[3];          // omega j
    P2 EA[3];          // even part of the axis pairs, weight and M terms included
    P2 WE[3], WO[3];   // diagonal planes xy, xz, yz: even parts WP + MD and sign-odd parts WT + MO
    P2 omw, c0;

    __device__ __forceinline__ void prep(P2 rho, const P2 (&j)[3], const P2 (&G)[3], P2 lap, const PairPhys& ph) {
        const P2 irho = rcp2(rho);
        const P2 u[3] = {j[0] * irho, j[1] * irho, j[2] * irho};
        const P2 ib = rcp2(fma(pp(-ph.b), rho, pp(1.0f)));
        const P2 p0 = fma(rho * pp(ph.T), ib, -(pp(ph.a) * rho * rho));      // Eq. 2
        const P2 cs2 = fma(pp(ph.T) * ib, ib, pp(-2.0f * ph.a) * rho);       // dp0/drho
        const P2 lam = fma(pp(-3.0f * ph.nu), cs2, pp(ph.nu));                // Eq. 36
        P2 lu[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) lu[c] = lam * u[c];
        const P2 udg = fma(u[0], G[0], fma(u[1], G[1], u[2] * G[2]));
        const P2 ludg = lam * udg;
        const P2 w15 = pp(1.5f * ph.omega), w3 = pp(3.0f * ph.omega);
        P2 Td[3], trQ = pp(0.0f);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const P2 q = fma(j[c], u[c], fma(pp(2.0f) * lu[c], G[c], ludg));
            trQ += q;
            Td[c] = w15 * q;
        }
        constexpr int cc[3] = {0, 0, 1}, dd[3] = {1, 2, 2};
        P2 To[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int c = cc[k], e = dd[k];
            To[k] = w3 * fma(j[c], u[e], fma(lu[c], G[e], lu[e] * G[c]));
        }
        const P2 A0 = (p0 - pp(ph.kappa) * rho * lap) - pp(0.5f) * trQ;
        const P2 Aw = pp(ph.omega) * (A0 - pp(ph.pref));
        const P2 ok = pp(ph.omega * ph.kappa);
        P2 Md[3], Mo[3];   // Mw_cc and Mw_cd (planes xy, xz, yz)
#pragma unroll
        for (int c = 0; c < 3; ++c) Md[c] = ok * G[c] * G[c];
#pragma unroll
        for (int k = 0; k < 3; ++k) Mo[k] = ok * G[cc[k]] * G[dd[k]];
        const P2 Msum = Md[0] + Md[1] + Md[2];
        constexpr float wax = 1.0f / 6.0f, wdg = 1.0f / 12.0f;
        // axis: 5/12 Mw_cc - 1/3 (Msum - Mw_cc) = 3/4 Mw_cc - 1/3 Msum
        static_assert(w_m<D3Q19>(1, 0, 0) == 5.0 / 12.0 && w_m<D3Q19>(1, 1, 1) == -1.0 / 3.0 &&
                          w_m<D3Q19>(1, 0, 1) == 0.0,
                      "D3Q19 axis M weights");
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            Jw[c] = pp(ph.omega) * j[c];
            EA[c] = fma(pp(wax), Aw + Td[c], fma(pp(0.75f), Md[c], pp(-1.0f / 3.0f) * Msum));
        }
        // diagonal (c, d): -1/24 (Mw_cc + Mw_dd) + 1/12 Mw_ee = 1/12 Msum - 1/8 (Mw_cc + Mw_dd)
        static_assert(w_m<D3Q19>(7, 0, 0) == -1.0 / 24.0 && w_m<D3Q19>(7, 2, 2) == 1.0 / 12.0 &&
                          w_m<D3Q19>(7, 0, 1) == 0.25 * D3Q19::ex(7) * D3Q19::ey(7),
                      "D3Q19 diagonal M weights");
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const P2 WP = pp(wdg) * ((Aw + Td[cc[k]]) + Td[dd[k]]);
            WE[k] = WP + fma(pp(wdg), Msum, pp(-0.125f) * (Md[cc[k]] + Md[dd[k]]));
            WO[k] = fma(pp(wdg), To[k], pp(0.25f) * Mo[k]);
        }
        omw = pp(1.0f - ph.omega);
        // Eq. 6: every pair's even part counted twice; the two diagonal pairs of a plane add to 2 WE
        const P2 sum = (EA[0] + EA[1] + EA[2]) + pp(2.0f) * (WE[0] + WE[1] + WE[2]);
        c0 = fma(pp(ph.omega), rho - pp(ph.rsum), pp(-2.0f) * sum);
    }

    template <int i>
    __device__ __forceinline__ void out(P2 di, P2 dn, P2& oi, P2& on) const {
        using L = D3Q19;
        constexpr int c = first_axis<L>(i), e2 = second_axis<L>(i);
        P2 odd, ev;
        if constexpr (e2 < 0) {
            odd = (e_comp<L>(i, c) > 0) ? Jw[c] : -Jw[c];
            ev = EA[c];
        } else {
            constexpr int sc = e_comp<L>(i, c), se = e_comp<L>(i, e2);
            odd = (sc > 0) ? ((se > 0) ? Jw[c] + Jw[e2] : Jw[c] - Jw[e2]) : ((se > 0) ? Jw[e2] - Jw[c] : -(Jw[c] + Jw[e2]));
            constexpr int k = (c == 0 && e2 == 1) ? 0 : ((c == 0 && e2 == 2) ? 1 : 2);
            ev = (sc * se > 0) ? WE[k] + WO[k] : WE[k] - WO[k];
        }
        const P2 wo = pp(float(w_vel<L>(i))) * odd;
        oi = fma(omw, di, ev + wo);
        on = fma(omw, dn, ev - wo);
    }
};

template <class S, int TX, int TY, int MINB, bool AOS>
__global__ void __launch_bounds__((TX / 2) * TY, MINB) step_kernel3d_pk_eq(const StepArgs args) {
    using L = D3Q19;
    using IO = PairIO<S>;
    using Wd = typename IO::W;
    constexpr bool RAW16 = IO::RAW16;
    using Lay = LayoutPKE<TX, TY, RAW16>;
    constexpr int H = Lay::H, HX = Lay::HX, TXP = Lay::TXP, NTH = Lay::NTH;
    constexpr int RX = Lay::RX, RXP = Lay::RXP, NAH = Lay::NAH;
    static_assert(!AOS || RAW16, "interleaved layout: 16-bit storage only");
    constexpr int ROWB = 2 * AOS_SITES;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* rho_s = reinterpret_cast<float*>(smem_raw + Lay::OFF_RHO);
    unsigned char* stash = smem_raw + Lay::OFF_ST;
    float2* mom_s = reinterpret_cast<float2*>(smem_raw + Lay::OFF_MOM);

    const int nx = args.nx, ny = args.ny, nz = args.nz;
    const int tid = threadIdx.x;
    const int px = tid % TXP, py = tid / TXP;
    const int4 wk = args.work[blockIdx.x];
    const int x0 = wk.x, y0 = wk.y, z0 = wk.z, z1 = wk.w;
    const int plane = nx * ny;
#ifdef LB_DEBUG_BOUNDS
    const size_t nsites = size_t(plane) * nz;
#endif
    const PairPhys ph{args.fa, args.fb, args.fT, args.fkappa, args.fomega, args.fnu, args.pref, args.rsum};

    // ---- stage-A items: own pair, then halo pairs (row below, row above, then the
    // left and right pair of every tile row)
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
    const unsigned xm1 = unsigned(wrapi(xo - 1, nx)), xc = unsigned(wrapi(xo, nx));
    const unsigned xp2 = unsigned(wrapi(xo + 2, nx));
    const unsigned yr[3] = {unsigned(wrapi(yo - 1, ny) * nx), unsigned(wrapi(yo, ny) * nx),
                            unsigned(wrapi(yo + 1, ny) * nx)};

    // planes z0 - 1 .. z1 (loads) ; collisions of z0 .. z1 - 1, one plane behind
    const int pstart = z0 - 1, pend = z1 + 1;
    const int vol = nz * plane;
    int ld_off = wrapi(pstart, nz) * plane;
    int zr[3] = {wrapi(z0 - 1, nz) * plane, wrapi(z0, nz) * plane, wrapi(z0 + 1, nz) * plane};
    auto advance = [&](int& v) {
        v += plane;
        if (v == vol) v = 0;
    };
    unsigned a_h[1 + NAH];
#pragma unroll
    for (int m = 0; m < 1 + NAH; ++m) a_h[m] = AOS ? aos_bytes(a_in[m]) : 0u;
    float2 r0[1 + NAH];
    Wd ri[1 + NAH][18];
    auto issue = [&]() {
#pragma unroll
        for (int m = 0; m < 1 + NAH; ++m) {
            if (m == 0 || a_rs[m] >= 0) {
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
    issue();

    StencilAcc2 acc2{pp(0.f), pp(0.f), pp(0.f), pp(0.f), pp(0.f), pp(0.f), pp(0.f)};
    bool bad = false;

    for (int p = pstart; p < pend; ++p) {
        const int it = p - pstart;
        // ---------------- stage A: density of plane p; own pair into the stash
        {
            advance(ld_off);
            float* rho_w = rho_s + (it & 1) * Lay::RN;
            const int slot = it & 1;
#pragma unroll
            for (int m = 0; m < 1 + NAH; ++m) {
                if (m == 0 || a_rs[m] >= 0) {
                    const P2 r = pair_rho<S, true>(r0[m], ri[m], ph.rsum);
                    LB_GUARD(a_rs[m] >= 0 && a_rs[m] + 1 < Lay::RN, BK_PK_SHARED, a_rs[m], continue)
                    *reinterpret_cast<float2*>(rho_w + a_rs[m]) = r.v;
                    if (m == 0) {
                        float2* mo = mom_s + slot * 4 * NTH + tid;
                        mo[0] = r.v;
                        P2 j[3];
                        if constexpr (RAW16) pair_momentum_mixed<S>(ri[0], j);
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
            if (p + 1 < pend) issue();
        }
        __syncthreads();

        // ---------------- stage B: stencil parts of plane p; G, lap of plane q = p - 1
        const PlaneParts2 cur = plane_parts2(rho_s + (it & 1) * Lay::RN, a_rs[0], RX);
        P2 G[3], lap;
        const bool assemble = it >= 1;
        if (assemble) finish2(acc2, cur, G, lap);
        start2(acc2, cur);

        // ---------------- stage C: collide and push plane s = p - 1
        const int s = p - 1;
        if (assemble && s >= z0) {
            const int slot = (it - 1) & 1;
            const float2* mo = mom_s + slot * 4 * NTH + tid;
            const P2 rho = P2{mo[0]};
            const P2 j[3] = {P2{mo[NTH]}, P2{mo[2 * NTH]}, P2{mo[3 * NTH]}};
            if (own) bad |= !(rho.v.x > 0.f) || !(rho.v.x < 1e30f) || !(rho.v.y > 0.f) || !(rho.v.y < 1e30f);
            const unsigned char* st = stash + size_t(slot) * Lay::STW * 4 * NTH;
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
            PairCollEq K;
            K.prep(rho, j, G, lap, ph);
            if (own) {
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
    }
    if (bad) atomicOr(args.status, 1u);
}

}  // namespace lbk
