// Fused D2Q9 time step, two adjacent x sites per thread.
//
// The same step as step2d_tile (step_kernel.cuh) - Eq. 3 moments, the
// gradient and Laplacian of Eq. 32 (w = 1/3 on the axes, 1/12 on the
// diagonals), p0 and lambda (Eqs. 2, 36), the equilibrium of Eqs. 5, 6 (with
// the M terms of the optimal weights in the equilibrium scheme), or the
// forcing scheme's g = -div M' (Eq. 28) and F_i (Eq. 27), BGK and
// push-streaming (Eq. 4) - with the work of the pair kernel of step3d_pk.cuh:
//
//   * every thread owns one pair of sites (x, x+1), x even; its collision runs
//     as packed float32 pairs (FADD2 / FMUL2 / FFMA2);
//   * the density of every region pair (own and halo) is summed from the raw
//     16-bit deviations by mixed-precision adds, and the own pair's momentum
//     the same way; the own pair's raw populations stay in registers from
//     their load to the collision (one plane: no stash);
//   * the own pair's stencil parts are formed as pairs from one aligned
//     2-vector and two scalars per density row.
//
// AL: nx even, so every pair is one aligned 2-vector in every population array
// and never split by the periodic wrap; otherwise (odd nx) every site of a
// pair is loaded and stored on its own, wrapped on its own, and a pair whose
// second site lies beyond the lattice stores its first site only.
#pragma once
#include "bounds.cuh"
#include "step3d_pk.cuh"
#include "step_kernel.cuh"

namespace lbk {

template <bool FORCING, int TX, int TY>
struct Layout2PK {
    static constexpr int H = FORCING ? 2 : 1;       // density halo in y
    static constexpr int HX = 2;                    // density halo in x (pairs start on even x)
    static constexpr int TXP = TX / 2;              // pairs per tile row
    static constexpr int NTH = TXP * TY;            // threads: one own pair each
    static constexpr int RX = TX + 2 * HX, RY = TY + 2 * H, RN = RX * RY, RXP = RX / 2;
    static constexpr int NHALO = RXP * RY - NTH;    // region pairs outside the tile
    static constexpr int NAH = (NHALO + NTH - 1) / NTH;
    static constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY, SXH = SX / 2;   // tile + 1 ring (M')
    static constexpr int NRING = SN - TX * TY;
    static constexpr int NBR = (NRING + NTH - 1) / NTH;
    static constexpr size_t OFF_RHO = 0;
    static constexpr size_t OFF_MP = (size_t(RN) * 4 + 15) / 16 * 16;
    static constexpr size_t BYTES = FORCING ? OFF_MP + size_t(SN) * 16 : OFF_MP;
    static_assert(TX % 4 == 0, "tile width");
    static_assert(NAH <= 2 && NBR <= 2, "items per thread");
    // M' (Mxx, Myy, Mxy) of ring site (sx, sy): even and odd columns in separate
    // halves, so that the pair neighbourhoods of consecutive threads are conflict-free
    __host__ __device__ static constexpr int mp_index(int sx, int sy) { return (sx & 1) * (SY * SXH) + sy * SXH + (sx >> 1); }
};

// Raw word of population i >= 1 of the two sites qa, qb (odd nx: not one aligned pair).
template <class S>
__device__ __forceinline__ typename PairIO<S>::W ld_split(const char* p, size_t qa, size_t qb) {
    if constexpr (PairIO<S>::RAW16) {
        const unsigned short* h = reinterpret_cast<const unsigned short*>(p);
        return unsigned(h[qa]) | (unsigned(h[qb]) << 16);
    } else {
        const float* f = reinterpret_cast<const float*>(p);
        return make_float2(f[qa], f[qb]);
    }
}

// Density of a pair from f_0 and the raw words of populations 1..8: mixed-
// precision adds (16-bit), else the decoded values as a balanced tree.
template <class S>
__device__ __forceinline__ P2 pair_rho9(float2 f0, const typename PairIO<S>::W (&w)[8], float rsum) {
    using IO = PairIO<S>;
    const P2 a = pp(rsum) + P2{f0};
    if constexpr (IO::RAW16) {
        float a0 = a.v.x, a1 = a.v.y, b0 = 0.0f, b1 = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if constexpr (std::is_same<S, StF16>::value) {
                madd_f16x2(a0, a1, w[i]);
                madd_f16x2(b0, b1, w[i + 4]);
            } else {
                madd_bf16x2(a0, a1, w[i]);
                madd_bf16x2(b0, b1, w[i + 4]);
            }
        }
        return pp(a0, a1) + pp(b0, b1);
    } else {
        P2 d[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) d[i] = IO::dec(w[i]);
        return a + tree_sum<0, 8>(d);
    }
}

// Momentum j = sum_i d_i e_i of a pair (Eq. 3; sum_i w_i e_i = 0): per axis the
// populations with e_a = +1 and with e_a = -1 summed, then differenced.
template <class S>
__device__ __forceinline__ void pair_momentum9(const typename PairIO<S>::W (&w)[8], P2 (&j)[2]) {
    using L = D2Q9;
    using IO = PairIO<S>;
    if constexpr (IO::RAW16) {
        float pl[2][2] = {}, mi[2][2] = {};
        static_for<1, 9>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int e[2] = {L::ex(i), L::ey(i)};
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                if (e[a] == 0) continue;
                float* acc = e[a] > 0 ? pl[a] : mi[a];
                if constexpr (std::is_same<S, StF16>::value) madd_f16x2(acc[0], acc[1], w[i - 1]);
                else madd_bf16x2(acc[0], acc[1], w[i - 1]);
            }
        });
#pragma unroll
        for (int a = 0; a < 2; ++a) j[a] = pp(pl[a][0], pl[a][1]) - pp(mi[a][0], mi[a][1]);
    } else {
        j[0] = j[1] = pp(0.0f);
        static_for<1, 9>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int o = opposite<L>(i);
            if constexpr (i < o) {
                const P2 df = IO::dec(w[i - 1]) - IO::dec(w[o - 1]);
                add_signed2<L::ex(i)>(j[0], df);
                add_signed2<L::ey(i)>(j[1], df);
            }
        });
    }
}

// Gradient and Laplacian (Eq. 32) of the pair whose site 0 has region index
// rc (even; RX even): per row one aligned 2-vector and two scalars.
__device__ __forceinline__ void pair_stencil9(const float* rho, int rc, int RX, P2 (&G)[2], P2& lap) {
    const float2 C = *reinterpret_cast<const float2*>(rho + rc);
    const float2 U = *reinterpret_cast<const float2*>(rho + rc + RX);
    const float2 D = *reinterpret_cast<const float2*>(rho + rc - RX);
    const P2 c{C}, up{U}, dn{D};
    const P2 xm = pp(rho[rc - 1], C.x), xp = pp(C.y, rho[rc + 2]);
    const P2 upp = pp(U.y, rho[rc + RX + 2]), upm = pp(rho[rc + RX - 1], U.x);
    const P2 dnp = pp(D.y, rho[rc - RX + 2]), dnm = pp(rho[rc - RX - 1], D.x);
    const P2 third = pp(1.0f / 3.0f), twelfth = pp(1.0f / 12.0f);
    G[0] = fma(third, xp - xm, twelfth * ((upp - upm) + (dnp - dnm)));
    G[1] = fma(third, up - dn, twelfth * ((upp + upm) - (dnp + dnm)));
    const P2 ax = (xp + xm) + (up + dn), dg = (upp + upm) + (dnp + dnm);
    // 2 sum_i w_i (rho_i - rho) = 2 [(1/3) ax + (1/12) dg - (4/3 + 4/12) rho]
    lap = pp(2.0f) * (fma(third, ax, twelfth * dg) - pp(5.0f / 3.0f) * c);
}

// Gradient and Laplacian of one site at region index rc (ring sites).
__device__ __forceinline__ void site_stencil9(const float* rho, int rc, int RX, float (&G)[2], float& lap) {
    const float r0 = rho[rc];
    G[0] = G[1] = 0.0f;
    lap = 0.0f;
    static_for<1, 9>([&](auto I) {
        constexpr int i = decltype(I)::value;
        const float rn = rho[rc + D2Q9::ey(i) * RX + D2Q9::ex(i)];
        constexpr float wi = float(w_vel<D2Q9>(i));
        add_signed<D2Q9::ex(i)>(G[0], wi * rn);
        add_signed<D2Q9::ey(i)>(G[1], wi * rn);
        lap += wi * (rn - r0);
    });
    lap *= 2.0f;
}

// collide() of step_kernel.cuh for D2Q9 and two sites at once (deviation
// space, d_i = f_i - w_i pref): per-site coefficients in prep, the collided
// deviations of an opposite pair (i, o) in out, f_0 in out0.
template <bool FORCING>
struct PairColl2D {
    P2 Jw[2];          // omega j + g
    P2 EA[2];          // even part of the axis pairs (weight included)
    P2 ED[2];          // even part of the diagonal pairs e = (1, 1) / (-1, 1) (weight included)
    P2 omw, c0;        // 1 - omega; f_0 gain

    __device__ __forceinline__ void prep(P2 rho, const P2 (&j)[2], const P2 (&G)[2], P2 lap, const P2 (&g)[2],
                                         const PairPhys& ph) {
        const P2 irho = rcp2(rho);
        const P2 u[2] = {j[0] * irho, j[1] * irho};
        const P2 ib = rcp2(fma(pp(-ph.b), rho, pp(1.0f)));
        const P2 p0 = fma(rho * pp(ph.T), ib, -(pp(ph.a) * rho * rho));      // Eq. 2
        const P2 cs2 = fma(pp(ph.T) * ib, ib, pp(-2.0f * ph.a) * rho);       // dp0/drho
        const P2 lam = fma(pp(-3.0f * ph.nu), cs2, pp(ph.nu));                // Eq. 36
        const P2 lu[2] = {lam * u[0], lam * u[1]};
        const P2 udg = fma(u[0], G[0], u[1] * G[1]);
        const P2 ludg = lam * udg;
        const P2 w15 = pp(1.5f * ph.omega), w3 = pp(3.0f * ph.omega);
        P2 Td[2], trQ = pp(0.0f);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const P2 q = fma(j[c], u[c], fma(pp(2.0f) * lu[c], G[c], ludg));
            trQ += q;
            Td[c] = FORCING ? fma(w15, q, pp(3.0f) * u[c] * g[c]) : w15 * q;
        }
        const P2 qo = fma(j[0], u[1], fma(lu[0], G[1], lu[1] * G[0]));
        const P2 To = FORCING ? fma(w3, qo, pp(3.0f) * fma(u[0], g[1], u[1] * g[0])) : w3 * qo;
        const P2 A0 = (p0 - pp(ph.kappa) * rho * lap) - pp(0.5f) * trQ;
        P2 Aw = pp(ph.omega) * (A0 - pp(ph.pref));
        if constexpr (FORCING) Aw -= fma(u[0], g[0], u[1] * g[1]);
#pragma unroll
        for (int c = 0; c < 2; ++c) Jw[c] = FORCING ? fma(pp(ph.omega), j[c], g[c]) : pp(ph.omega) * j[c];
        const P2 E0 = Aw + Td[0], E1 = Aw + Td[1];
        constexpr float wax = 1.0f / 3.0f, wdg = 1.0f / 12.0f;
        EA[0] = pp(wax) * E0;
        EA[1] = pp(wax) * E1;
        const P2 WP = pp(wdg) * (E0 + Td[1]), WT = pp(wdg) * To;
        ED[0] = WP + WT;   // e = (1, 1): sign e_x e_y = +1
        ED[1] = WP - WT;   // e = (-1, 1)
        if constexpr (!FORCING) {
            // M terms of the equilibrium scheme, w^ab_i omega kappa d_a rho d_b rho
            const P2 ok = pp(ph.omega * ph.kappa);
            const P2 Mxx = ok * G[0] * G[0], Myy = ok * G[1] * G[1], Mxy = ok * G[0] * G[1];
            constexpr float wa = float(w_m<D2Q9>(1, 0, 0)), wb = float(w_m<D2Q9>(1, 1, 1));
            constexpr float wd = float(w_m<D2Q9>(5, 0, 0)), wo = float(w_m<D2Q9>(5, 0, 1));
            static_assert(w_m<D2Q9>(3, 1, 1) == w_m<D2Q9>(1, 0, 0) && w_m<D2Q9>(3, 0, 0) == w_m<D2Q9>(1, 1, 1) &&
                              w_m<D2Q9>(5, 1, 1) == w_m<D2Q9>(5, 0, 0) && w_m<D2Q9>(7, 0, 1) == -w_m<D2Q9>(5, 0, 1) &&
                              w_m<D2Q9>(1, 0, 1) == 0.0 && w_m<D2Q9>(3, 0, 1) == 0.0,
                          "D2Q9 M weights");
            EA[0] += fma(pp(wa), Mxx, pp(wb) * Myy);
            EA[1] += fma(pp(wb), Mxx, pp(wa) * Myy);
            const P2 md = pp(wd) * (Mxx + Myy);
            ED[0] += fma(pp(wo), Mxy, md);
            ED[1] += fma(pp(-wo), Mxy, md);
        }
        omw = pp(1.0f - ph.omega);
        // Eq. 6: f_0 = rho - sum_{i>=1} f_i (and sum_i F_i = 0); every pair's even part counted twice
        const P2 sum = (EA[0] + EA[1]) + (ED[0] + ED[1]);
        c0 = fma(pp(ph.omega), rho - pp(ph.rsum), pp(-2.0f) * sum);
    }

    // collided deviations of the opposite pair (i, o), i < o
    template <int i>
    __device__ __forceinline__ void out(P2 di, P2 dn, P2& oi, P2& on) const {
        using L = D2Q9;
        constexpr int ex = L::ex(i), ey = L::ey(i);
        P2 odd, ev;
        if constexpr (ey == 0) {
            odd = ex > 0 ? Jw[0] : -Jw[0];
            ev = EA[0];
        } else if constexpr (ex == 0) {
            odd = ey > 0 ? Jw[1] : -Jw[1];
            ev = EA[1];
        } else {
            odd = (ex > 0 ? Jw[0] : -Jw[0]) + (ey > 0 ? Jw[1] : -Jw[1]);
            ev = (ex * ey > 0) ? ED[0] : ED[1];
        }
        const P2 wo = pp(float(w_vel<L>(i))) * odd;
        oi = fma(omw, di, ev + wo);
        on = fma(omw, dn, ev - wo);
    }
};

// One D2Q9 time step of the TX x TY tile at (x0, y0), (TX / 2) * TY threads.
template <bool FORCING, class S, int TX, int TY, bool AL>
__device__ __forceinline__ void step2d_pair_tile(const Tile2DArgs& args, int x0, int y0, unsigned char* smem) {
    using L = D2Q9;
    using IO = PairIO<S>;
    using Wd = typename IO::W;
    using Lay = Layout2PK<FORCING, TX, TY>;
    constexpr int H = Lay::H, HX = Lay::HX, TXP = Lay::TXP, NTH = Lay::NTH;
    constexpr int RX = Lay::RX, RXP = Lay::RXP, SX = Lay::SX;
    float* rho_s = reinterpret_cast<float*>(smem + Lay::OFF_RHO);
    float4* mp_s = reinterpret_cast<float4*>(smem + Lay::OFF_MP);

    const int nx = args.nx, ny = args.ny;
#ifdef LB_DEBUG_BOUNDS
    const size_t nsites = size_t(nx) * ny;
#endif
    const int tid = threadIdx.x;
    const int px = tid % TXP, py = tid / TXP;
    const PairPhys ph{args.fa, args.fb, args.fT, args.fkappa, args.fomega, args.fnu, args.pref, args.rsum};
    const float pk = args.fkappa;
    const char* src = args.src;
    char* dst = args.dst;
    const long long pitch = args.pitch;

    // raw populations of the pair whose site 0 is at (x, y) of the lattice
    // (wrap_near: one compare-and-add for offsets up to a lattice width outside)
    auto load = [&](int x, int y, float2& f0, Wd (&w)[8]) {
        const size_t row = size_t(wrap_near(y, ny)) * nx;
        if constexpr (AL) {
            const size_t q = row + wrap_near(x, nx);   // even
            LB_GUARD(q + 1 < nsites, BK_2D_LOAD, q, f0 = make_float2(0.f, 0.f); for (int i = 0; i < 8; ++i) w[i] = Wd{};
                     return)
            f0 = reinterpret_cast<const float2*>(src)[q >> 1];
            static_for<1, 9>([&](auto I) {
                constexpr int i = decltype(I)::value;
                w[i - 1] = IO::ld(src + S::pop_offset(i, pitch), unsigned(q));
            });
        } else {
            const size_t qa = row + wrap_near(x, nx), qb = row + wrap_near(x + 1, nx);
            LB_GUARD(qa < nsites && qb < nsites, BK_2D_LOAD, qa, f0 = make_float2(0.f, 0.f);
                     for (int i = 0; i < 8; ++i) w[i] = Wd{}; return)
            const float* f = reinterpret_cast<const float*>(src);
            f0 = make_float2(f[qa], f[qb]);
            static_for<1, 9>([&](auto I) {
                constexpr int i = decltype(I)::value;
                w[i - 1] = ld_split<S>(src + S::pop_offset(i, pitch), qa, qb);
            });
        }
    };

    // ---------------- stage A: density of the region; own pair kept in registers
    const int xo = x0 + 2 * px, yo = y0 + py;
    const bool v0 = xo < nx && yo < ny, v1 = xo + 1 < nx && yo < ny;
    float2 f0o;
    Wd wo[8];
    load(xo, yo, f0o, wo);
    const P2 rho = pair_rho9<S>(f0o, wo, ph.rsum);
    *reinterpret_cast<float2*>(rho_s + (py + H) * RX + 2 * px + HX) = rho.v;
    P2 j[2];
    pair_momentum9<S>(wo, j);
#pragma unroll
    for (int m = 0; m < Lay::NAH; ++m) {
        const int h = tid + m * NTH;
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
            float2 f0;
            Wd w[8];
            load(x0 - HX + 2 * rxp, y0 - H + ry, f0, w);
            const P2 r = pair_rho9<S>(f0, w, ph.rsum);
            *reinterpret_cast<float2*>(rho_s + ry * RX + 2 * rxp) = r.v;
        }
    }
    __syncthreads();

    // ---------------- stage B: gradient / Laplacian (and, forcing, M' on the tile + 1 ring)
    const int rc = (py + H) * RX + 2 * px + HX;
    P2 G[2], lap;
    pair_stencil9(rho_s, rc, RX, G, lap);
    P2 g[2] = {pp(0.f), pp(0.f)};
    if constexpr (FORCING) {
        auto put_mp = [&](int k, float gx, float gy) {
            const float hk = 0.5f * pk * (gx * gx + gy * gy);
            LB_GUARD(k >= 0 && k < Lay::SN, BK_2D_SHARED, k, return)
            mp_s[k] = make_float4(pk * gx * gx - hk, pk * gy * gy - hk, pk * gx * gy, 0.0f);
        };
        put_mp(Lay::mp_index(2 * px + 1, py + 1), G[0].v.x, G[1].v.x);
        put_mp(Lay::mp_index(2 * px + 2, py + 1), G[0].v.y, G[1].v.y);
#pragma unroll
        for (int m = 0; m < Lay::NBR; ++m) {
            const int r = tid + m * NTH;
            if (r < Lay::NRING) {
                int sx, sy;
                if (r < 2 * SX) {
                    sx = r % SX;
                    sy = r < SX ? 0 : Lay::SY - 1;
                } else {
                    const int k = r - 2 * SX;
                    sy = 1 + (k >> 1);
                    sx = (k & 1) ? SX - 1 : 0;
                }
                float Gs[2], ls;
                site_stencil9(rho_s, (sy + H - 1) * RX + (sx + HX - 1), RX, Gs, ls);
                put_mp(Lay::mp_index(sx, sy), Gs[0], Gs[1]);
            }
        }
        __syncthreads();
        // g_a = -sum_i w_i sum_b e_ib M'_ab(r + e_i) (Eq. 28): neighbourhood columns
        // c = 0..3 (sites x-1 .. x+2) and rows -1, 0, +1 of the ring frame
        float gs[2][2] = {};
#pragma unroll
        for (int r = -1; r <= 1; ++r) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 M = mp_s[Lay::mp_index(2 * px + c, py + 1 + r)];
#pragma unroll
                for (int s = 0; s < 2; ++s) {
                    const int dx = c - 1 - s;
                    if (dx < -1 || dx > 1 || (dx == 0 && r == 0)) continue;
                    const float wi = (dx == 0 || r == 0) ? 1.0f / 3.0f : 1.0f / 12.0f;
                    // sum_b e_b M'_ab: a = x: e_x Mxx + e_y Mxy; a = y: e_x Mxy + e_y Myy
                    const float ax = float(dx) * M.x + float(r) * M.z;
                    const float ay = float(dx) * M.z + float(r) * M.y;
                    gs[s][0] -= wi * ax;
                    gs[s][1] -= wi * ay;
                }
            }
        }
        g[0] = pp(gs[0][0], gs[1][0]);
        g[1] = pp(gs[0][1], gs[1][1]);
    }

    // ---------------- stage C: collide and push the own pair
    if ((v0 && (!(rho.v.x > 0.f) || !(rho.v.x < 1e30f))) || (v1 && (!(rho.v.y > 0.f) || !(rho.v.y < 1e30f))))
        atomicOr(args.status, 1u);
    PairColl2D<FORCING> K;
    K.prep(rho, j, G, lap, g, ph);
    const P2 o0 = fma(K.omw, P2{f0o}, K.c0);
    const int xm1 = wrap_near(xo - 1, nx), xp1 = wrap_near(xo + 1, nx), xp2 = wrap_near(xo + 2, nx);
    const size_t yr[3] = {size_t(wrap_near(yo - 1, ny)) * nx, size_t(yo) * nx, size_t(wrap_near(yo + 1, ny)) * nx};
    // destination column of site s moved by ex (site 0 at xo, site 1 at xo + 1)
    const int col[2][3] = {{xm1, xo, xp1}, {xo, xp1, xp2}};
    auto store = [&](auto I, P2 v) {
        constexpr int i = decltype(I)::value;
        constexpr int ex = L::ex(i), ey = L::ey(i);
        char* p = dst + S::pop_offset(i, pitch);
        const size_t row = yr[1 + ey];
#ifdef LB_DEBUG_BOUNDS
        LB_GUARD(row + col[0][1 + ex] < nsites && row + col[1][1 + ex] < nsites, BK_2D_STORE, row, return)
#endif
        if constexpr (AL && ex == 0) {
            if (v0) IO::st2(p, unsigned(row + xo), v);
        } else {
            if (v0) IO::st1(p, unsigned(row + col[0][1 + ex]), v.v.x);
            if (v1) IO::st1(p, unsigned(row + col[1][1 + ex]), v.v.y);
        }
    };
    if (v0) {
        float* f0d = reinterpret_cast<float*>(dst);
        if constexpr (AL) {
            reinterpret_cast<float2*>(dst)[(yr[1] + xo) >> 1] = o0.v;
        } else {
            f0d[yr[1] + xo] = o0.v.x;
            if (v1) f0d[yr[1] + xp1] = o0.v.y;
        }
        static_for<1, 9>([&](auto I) {
            constexpr int i = decltype(I)::value;
            constexpr int o = opposite<L>(i);
            if constexpr (i < o) {
                P2 oi, on;
                K.template out<i>(IO::dec(wo[i - 1]), IO::dec(wo[o - 1]), oi, on);
                store(std::integral_constant<int, i>{}, oi);
                store(std::integral_constant<int, o>{}, on);
            }
        });
    }
}

// One step of a single D2Q9 lattice: one CTA of (TX / 2) * TY threads per tile.
// Resident CTAs of 128 threads per SM: 10 for 16-bit storage (48 registers;
// measured on GB300 at 2048^2 against the unbounded 56 registers: fp16
// deviations forcing 73.6 against 71.6 GLUPS, equilibrium 94.1 against 89.9),
// 8 for float32 (64 registers, what the unbounded form takes; 10 cost it 12%,
// a bound of 1 let it grow to 89 registers and cost 11%).
template <bool FORCING, class S, int TX, int TY>
__global__ void __launch_bounds__((TX / 2) * TY, (PairIO<S>::RAW16 ? 1280 : 1024) / ((TX / 2) * TY))
    step_kernel2d_pk(const Tile2DArgs args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (args.pair) step2d_pair_tile<FORCING, S, TX, TY, true>(args, blockIdx.x * TX, blockIdx.y * TY, smem_raw);
    else step2d_pair_tile<FORCING, S, TX, TY, false>(args, blockIdx.x * TX, blockIdx.y * TY, smem_raw);
}

}  // namespace lbk
