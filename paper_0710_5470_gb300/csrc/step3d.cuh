// Fused D3Q19 time step with the z-split stencils.
//
// Same plane pipeline as the generic kernel (step_kernel.cuh): a CTA owns a
// TX x TY column of the lattice and marches through a chunk of z planes.  The
// 3D stencils are split by the z component of the velocity: with the D3Q19
// weights (1/6 on axes, 1/12 on diagonals) every stencil over the 18
// neighbours of r is the sum of an in-plane part (e_z = 0) and one part from
// each adjacent plane (e_z = +-1).  A plane's parts are computed once, from 9
// values of that plane, and carried in registers along the march:
//
//   grad rho (Eq. 29, A = 1/6, B = 1/12), on a plane q' with
//     Dx = rho(x+1) - rho(x-1), Dy = rho(y+1) - rho(y-1),
//     S  = rho/6 + (rho(x+-1) + rho(y+-1))/12:
//       d_x rho(q) = Dx(q)/6 + Ex(q)/12 + (Dx(q+1) + Dx(q-1))/12   (Ex: xy diagonals)
//       d_z rho(q) = S(q+1) - S(q-1)
//   lap rho (C = 1/3, D = 1/6) = 2 sum_i w_i rho(r + e_i) - 4 rho(r), with the
//     same split of sum_i w_i rho(r + e_i).
//   g = -div M' (Eq. 28, forcing scheme, reading for 3D: M'_ab = M_ab - delta_ab M_cc/2)
//     = -(U+(q+1) + U0(q) + U-(q-1)), U+/0/- the contributions of one plane's
//     M' e_i to the plane above / itself / below (43 values per site).
#pragma once
#include <type_traits>

#include "bounds.cuh"
#include "step_kernel.cuh"

namespace lbk {

// RAW: 16-bit deviation storage; the stash keeps f_0 (float) and the raw
// 16-bit deviations as loaded, and stage C decodes them.
template <bool FORCING, int TX, int TY, class real, bool RAW = false>
struct Layout3D {
    static constexpr int Q = 19;
    // density halo: 2 sites in x for both schemes (pairs of sites start on an
    // even x), H in y (2 forcing: the divergence of M' on the tile needs the
    // gradient on ring 1; 1 equilibrium)
    static constexpr int H = FORCING ? 2 : 1;
    static constexpr int HX = 2, HY = H;
    static constexpr int RX = TX + 2 * HX, RY = TY + 2 * HY, RN = RX * RY;
    static constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY;
    static constexpr int NT = TX * TY;
    static constexpr int NB = FORCING ? (SN + NT - 1) / NT : 1;
    static constexpr int LAG_C = FORCING ? 2 : 1;   // stage C trails stage A by LAG_C planes
    // rho and stash slots.  Float stash: planes p .. p - LAG_C are live and a barrier closes
    // each plane.  RAW (smaller) stash: LAG_C + 2 slots and no closing barrier: stage A of
    // plane p+1 writes a slot no stage of plane p reads, and the barrier after that stage A
    // orders this plane's stage C before the next stage B (measured: +4% for 16-bit storage;
    // with the float stash the extra slots cost more than the barrier saves).
    static constexpr bool OPEN = RAW;
    static constexpr int NRHO = OPEN ? LAG_C + 2 : 3;
    static constexpr int NSTASH = OPEN ? LAG_C + 2 : (FORCING ? 3 : 2);
    static constexpr int al4(int x) { return (x + 3) / 4 * 4; }
    static constexpr int OFF_RHO = 0;
    // stash: the tile's populations, [slot][population][site] (a site-major
    // layout would let stage C read a site with 128-bit loads, but the paired
    // stage-A writes then conflict on banks: measured slower)
    static constexpr int OFF_STASH = al4(OFF_RHO + NRHO * RN);
    // reals per stash slot: Q per site, or with RAW one f_0 and Q - 1 half-size deviations
    static constexpr int SLOT = RAW ? NT + (Q - 1) * NT / 2 : Q * NT;
    // M' of one plane on the tile + 1 ring: (Mxx, Mxy, Mxz, Myy) per site, then (Myz, Mzz) per site
    static constexpr int OFF_MP = al4(OFF_STASH + NSTASH * SLOT);
    // G and the Laplacian of the tile for two planes: (G_x, G_y, G_z, lap) per site
    static constexpr int OFF_G = al4(OFF_MP + (FORCING ? 6 * SN : 0));
    static constexpr int TOTAL = OFF_G + (FORCING ? 2 * 4 * NT : 0);
    static constexpr size_t BYTES = size_t(TOTAL) * sizeof(real);
};

// 4- and 2-vectors of reals in shared memory (16-byte / 8- or 16-byte aligned).
template <class real>
__device__ __forceinline__ void st4(real* p, real a, real b, real c, real d) {
    if constexpr (sizeof(real) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
    } else {
        reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
        reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
    }
}
template <class real>
__device__ __forceinline__ void ld4(const real* p, real& a, real& b, real& c, real& d) {
    if constexpr (sizeof(real) == 4) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        a = v.x; b = v.y; c = v.z; d = v.w;
    } else {
        const double2 v0 = reinterpret_cast<const double2*>(p)[0], v1 = reinterpret_cast<const double2*>(p)[1];
        a = v0.x; b = v0.y; c = v1.x; d = v1.y;
    }
}
template <class real>
__device__ __forceinline__ void ld2(const real* p, real& a, real& b) {
    if constexpr (sizeof(real) == 4) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        a = v.x; b = v.y;
    } else {
        const double2 v = *reinterpret_cast<const double2*>(p);
        a = v.x; b = v.y;
    }
}
// Per-plane parts of the gradient / Laplacian stencil at one site.
template <class real>
struct PlaneParts {
    real dx, dy, s;          // Dx, Dy, S of the plane (used by the planes above and below)
    real gx, gy, lin, c;     // in-plane parts of d_x, d_y, sum w rho, and rho itself
};

template <class real>
__device__ __forceinline__ PlaneParts<real> plane_parts(const real* rho, int rc, int RX) {
    const real c = rho[rc];
    const real xp = rho[rc + 1], xm = rho[rc - 1], yp = rho[rc + RX], ym = rho[rc - RX];
    const real pp = rho[rc + RX + 1], pm = rho[rc - RX + 1], mp = rho[rc + RX - 1], mm = rho[rc - RX - 1];
    const real sixth = real(1) / real(6), twelfth = real(1) / real(12);
    PlaneParts<real> o;
    o.dx = xp - xm;
    o.dy = yp - ym;
    const real f = (xp + xm) + (yp + ym);
    o.s = sixth * c + twelfth * f;
    o.gx = sixth * o.dx + twelfth * ((pp + pm) - (mp + mm));
    o.gy = sixth * o.dy + twelfth * ((pp + mp) - (pm + mm));
    o.lin = sixth * f + twelfth * ((pp + pm) + (mp + mm));
    o.c = c;
    return o;
}

// Carried stencil state of one site along the march: the gradient and
// Laplacian of plane q with the contributions of planes q-1 and q summed,
// and Dx, Dy, S of plane q (for plane q+1).
template <class real>
struct StencilAcc {
    real gx, gy, gz, lap;
    real dx, dy, s;
};

// Gradient and Laplacian of plane q: its accumulated parts plus plane q+1's (hi).
template <class real>
__device__ __forceinline__ void finish(const StencilAcc<real>& a, const PlaneParts<real>& hi, real (&G)[3],
                                       real& lap) {
    const real twelfth = real(1) / real(12);
    G[0] = a.gx + twelfth * hi.dx;
    G[1] = a.gy + twelfth * hi.dy;
    G[2] = a.gz + hi.s;
    lap = a.lap + real(2) * hi.s;
}

// Start plane q+1 (cur) from its in-plane parts and plane q's Dx, Dy, S.
template <class real>
__device__ __forceinline__ void start(StencilAcc<real>& a, const PlaneParts<real>& cur) {
    const real twelfth = real(1) / real(12);
    a.gx = cur.gx + twelfth * a.dx;
    a.gy = cur.gy + twelfth * a.dy;
    a.gz = -a.s;
    a.lap = real(2) * (cur.lin + a.s) - real(4) * cur.c;
    a.dx = cur.dx;
    a.dy = cur.dy;
    a.s = cur.s;
}

// PAIR: stage A moves two adjacent x sites per thread with 2-vector loads
// (requires an even nx); otherwise one site per thread.
template <bool FORCING, class S, int TX, int TY, bool PAIR>
__global__ void __launch_bounds__(TX* TY, (sizeof(typename S::real) == 4 && TX * TY <= 256) ? 2 : 1) step_kernel3d(const StepArgs args) {
    using L = D3Q19;
    using real = typename S::real;
    constexpr bool RAW = sizeof(typename S::rawi) == 2;
    using Lay = Layout3D<FORCING, TX, TY, real, RAW>;
    constexpr int Q = 19, HX = Lay::HX, HY = Lay::HY, NT = Lay::NT;
    constexpr int RX = Lay::RX, RN = Lay::RN, SX = Lay::SX, SN = Lay::SN;
    constexpr int W = PAIR ? 2 : 1;                 // sites per stage-A item
    constexpr int RXW = RX / W, NIT = RN / W;       // items per region row, per region
    constexpr int NA = (NIT + NT - 1) / NT;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sm = reinterpret_cast<real*>(smem_raw);
    real* rho_s = sm + Lay::OFF_RHO;
    real* stash = sm + Lay::OFF_STASH;
    real* mpA = sm + Lay::OFF_MP;              // (Mxx, Mxy, Mxz, Myy) per ring-1 site
    real* mpB = sm + Lay::OFF_MP + 4 * SN;     // (Myz, Mzz) per ring-1 site
    real* gl_s = sm + Lay::OFF_G;              // [slot][site](G_x, G_y, G_z, lap)

    const int nx = args.nx, ny = args.ny, nz = args.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int4 wk = args.work[blockIdx.x];    // this CTA's tile and z chunk
    const int x0 = wk.x, y0 = wk.y;
    const int z0 = wk.z, z1 = wk.w;
    const int plane = nx * ny;

    const real pa = arg_param<real>(args.a, args.fa), pb = arg_param<real>(args.b, args.fb);
    const real pT = arg_param<real>(args.T, args.fT), pk = arg_param<real>(args.kappa, args.fkappa);
    const real om = arg_param<real>(args.omega, args.fomega), nu = arg_param<real>(args.nu, args.fnu);
    const real pref = real(args.pref), rsum = real(args.rsum);

    // stage-A items: W adjacent region sites each; a_in = in-plane element
    // index of the first (even when PAIR: x0 - HX is even and nx is even),
    // a_st = its stash index if the item lies in the tile (items never
    // straddle the tile edge since HX is even); rho slot index = k * W
    int a_in[NA], a_st[NA];
#pragma unroll
    for (int m = 0; m < NA; ++m) {
        const int k = tid + m * NT;
        a_in[m] = -1;
        a_st[m] = -1;
        if (k < NIT) {
            const int rx = (k % RXW) * W, ry = k / RXW;
            a_in[m] = wrapi(y0 - HY + ry, ny) * nx + wrapi(x0 - HX + rx, nx);
            if (rx >= HX && rx < HX + TX && ry >= HY && ry < HY + TY) a_st[m] = (ry - HY) * TX + (rx - HX);
        }
    }
    // stage-B items: the tile + 1 ring (forcing) or the thread's own site
    int b_rc[Lay::NB], b_k[Lay::NB], b_r0[Lay::NB];
#pragma unroll
    for (int m = 0; m < Lay::NB; ++m) {
        if (FORCING) {
            const int k = tid + m * NT;
            const int sx = k % SX, sy = k / SX;
            b_k[m] = k < SN ? k : -1;
            b_rc[m] = (sy + HY - 1) * RX + (sx + HX - 1);
            b_r0[m] = (k < SN && sx >= 1 && sx <= TX && sy >= 1 && sy <= TY) ? (sy - 1) * TX + (sx - 1) : -1;
        } else {
            b_k[m] = tid;
            b_rc[m] = (ty + HY) * RX + (tx + HX);
            b_r0[m] = tid;
        }
    }
    const int xs = x0 + tx, ys = y0 + ty;
    const bool own = xs < nx && ys < ny;
    const int xw[3] = {wrapi(xs - 1, nx), wrapi(xs, nx), wrapi(xs + 1, nx)};
    const int yr[3] = {wrapi(ys - 1, ny) * nx, wrapi(ys, ny) * nx, wrapi(ys + 1, ny) * nx};

    const int pstart = z0 - Lay::LAG_C;
    const int pend = z1 + Lay::LAG_C;
    const int vol = nz * plane;
    // plane offsets wrapped once here and advanced by one plane per use
    // (v + plane wraps to 0 at vol): the plane loaded next, and planes s-1,
    // s, s+1 of the next stage C
    int ld_off = wrapi(pstart, nz) * plane;
    int zr[3] = {wrapi(z0 - 1, nz) * plane, wrapi(z0, nz) * plane, wrapi(z0 + 1, nz) * plane};
    auto advance = [&](int& v) {
        v += plane;
        if (v == vol) v = 0;
    };

    using R0 = std::conditional_t<PAIR, typename S::raw0x2, typename S::raw0>;
    using RI = std::conditional_t<PAIR, typename S::rawix2, typename S::rawi>;
    R0 r0[NA];
    RI ri[NA][Q - 1];
    // load plane ld_off of the halo region into r0/ri, then advance ld_off
    auto issue = [&]() {
#pragma unroll
        for (int m = 0; m < NA; ++m) {
            if (a_in[m] >= 0) {
                const size_t q = size_t(ld_off + a_in[m]);
                LB_GUARD(q + (PAIR ? 1 : 0) < size_t(vol), BK_3D_LOAD, q, r0[m] = R0{};
                         for (int i = 0; i < Q - 1; ++i) ri[m][i] = RI{}; continue)
                if constexpr (PAIR) r0[m] = S::ld0x2(args.src[0], q);
                else r0[m] = S::ld0(args.src[0], q);
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    if constexpr (PAIR) ri[m][i - 1] = S::ldix2(args.src[i], q);
                    else ri[m][i - 1] = S::ldi(args.src[i], q);
                });
            }
        }
        advance(ld_off);
    };
    constexpr bool PREFETCH = sizeof(real) == 4;
    if (PREFETCH) issue();

    // carried stencil state of the stage-B items (plane p-1 accumulated)
    StencilAcc<real> acc[Lay::NB];
#pragma unroll
    for (int m = 0; m < Lay::NB; ++m) acc[m] = StencilAcc<real>{0, 0, 0, 0, 0, 0, 0};
    // carried body force of the tile site: -(U0(q-1) + U-(q-2)) and -U-(q-1)
    real gacc1[3] = {0, 0, 0}, gacc2[3] = {0, 0, 0};
    // equilibrium scheme: G, lap of plane p-1 assembled in stage B
    real Geq[3] = {0, 0, 0}, lapeq = 0;
    // a density that is not positive and finite at any collided site (reported once at the end)
    bool bad = false;

    for (int p = pstart; p < pend; ++p) {
        const int it = p - pstart;
        // ---------------- stage A: density of plane p on the halo region
        {
            if (!PREFETCH) issue();
            real* rho_w = rho_s + (it % Lay::NRHO) * RN;
            real* st_w = stash + (it % Lay::NSTASH) * Lay::SLOT;
            typename S::rawi* sd_w = reinterpret_cast<typename S::rawi*>(st_w + NT);   // RAW deviations
            const bool keep = p >= z0 && p < z1;
#pragma unroll
            for (int m = 0; m < NA; ++m) {
                if (a_in[m] >= 0) {
                    if constexpr (PAIR) {
                        pair_t<real> f2[Q];   // f_0 and the deviations d_i of the two sites
                        S::dec0x2(r0[m], f2[0].x, f2[0].y);
                        static_for<1, Q>([&](auto I) {
                            constexpr int i = decltype(I)::value;
                            S::devix2(ri[m][i - 1], f2[i].x, f2[i].y);
                        });
                        const pair_t<real> r2 = site_rho_pair(f2, rsum);
                        st_pair(rho_w + 2 * (tid + m * NT), r2.x, r2.y);
                        if (keep && a_st[m] >= 0) {
                            if constexpr (RAW) {
                                st_pair(st_w + a_st[m], f2[0].x, f2[0].y);
                                static_for<1, Q>([&](auto I) {
                                    constexpr int i = decltype(I)::value;
                                    *reinterpret_cast<RI*>(sd_w + (i - 1) * NT + a_st[m]) = ri[m][i - 1];
                                });
                            } else {
                                static_for<0, Q>([&](auto I) {
                                    constexpr int i = decltype(I)::value;
                                    st_pair(st_w + i * NT + a_st[m], f2[i].x, f2[i].y);
                                });
                            }
                        }
                    } else {
                        real f[Q];           // f_0 and the deviations d_i
                        f[0] = S::dec0(r0[m]);
                        static_for<1, Q>([&](auto I) {
                            constexpr int i = decltype(I)::value;
                            f[i] = S::devi(ri[m][i - 1]);
                        });
                        rho_w[tid + m * NT] = site_rho(f, rsum);
                        if (keep && a_st[m] >= 0) {
                            if constexpr (RAW) {
                                st_w[a_st[m]] = f[0];
                                static_for<1, Q>([&](auto I) {
                                    constexpr int i = decltype(I)::value;
                                    sd_w[(i - 1) * NT + a_st[m]] = ri[m][i - 1];
                                });
                            } else {
                                static_for<0, Q>([&](auto I) {
                                    constexpr int i = decltype(I)::value;
                                    st_w[i * NT + a_st[m]] = f[i];
                                });
                            }
                        }
                    }
                }
            }
            if (PREFETCH && p + 1 < pend) issue();
        }
        __syncthreads();

        // ---------------- stage B: stencil parts of plane p; G, lap (and M') of plane q = p-1
        const int q = p - 1;
        const bool assemble_q = q >= z0 - (FORCING ? 1 : 0) && it >= 2;
        {
            const real* rho_p = rho_s + (it % Lay::NRHO) * RN;
#pragma unroll
            for (int m = 0; m < Lay::NB; ++m) {
                if (b_k[m] < 0) continue;
                const PlaneParts<real> cur = plane_parts(rho_p, b_rc[m], RX);
                if (assemble_q) {
                    real G[3], lap;
                    finish(acc[m], cur, G, lap);
                    if constexpr (FORCING) {
                        const real g2 = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
                        const real hk = real(0.5) * pk * g2;
                        const int k = b_k[m];
                        st4(mpA + 4 * k, pk * G[0] * G[0] - hk, pk * G[0] * G[1], pk * G[0] * G[2],
                            pk * G[1] * G[1] - hk);
                        st_pair(mpB + 2 * k, pk * G[1] * G[2], pk * G[2] * G[2] - hk);
                        if (b_r0[m] >= 0) {
                            real* gl = gl_s + ((q - pstart) & 1) * 4 * NT;
                            st4(gl + 4 * b_r0[m], G[0], G[1], G[2], lap);
                        }
                    } else {
                        Geq[0] = G[0];
                        Geq[1] = G[1];
                        Geq[2] = G[2];
                        lapeq = lap;
                    }
                }
                start(acc[m], cur);
            }
        }
        if constexpr (FORCING) __syncthreads();

        // ---------------- body-force parts of plane q (forcing)
        real gf[3] = {0, 0, 0};
        if constexpr (FORCING) {
            if (assemble_q) {
                const int kc = (ty + 1) * SX + (tx + 1);
                real sp[3] = {0, 0, 0}, sz[3] = {0, 0, 0}, se[3] = {0, 0, 0};
                real xx, xy, xz, yy, yz, zz;
#pragma unroll
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const int kx = kc + sgn, ky = kc + sgn * SX;
                    const real s = real(sgn);
                    // x faces: s (Mxx, Mxy, Mxz); z parts (Mxz, Myz, Mzz)
                    ld4(mpA + 4 * kx, xx, xy, xz, yy);
                    ld2(mpB + 2 * kx, yz, zz);
                    sp[0] += s * xx; sp[1] += s * xy; sp[2] += s * xz;
                    sz[0] += xz; sz[1] += yz; sz[2] += zz;
                    // y faces: s (Mxy, Myy, Myz)
                    ld4(mpA + 4 * ky, xx, xy, xz, yy);
                    ld2(mpB + 2 * ky, yz, zz);
                    sp[0] += s * xy; sp[1] += s * yy; sp[2] += s * yz;
                    sz[0] += xz; sz[1] += yz; sz[2] += zz;
                    // xy diagonals (sx = sgn, sy = +-1)
#pragma unroll
                    for (int sgy = -1; sgy <= 1; sgy += 2) {
                        const int ke = kc + sgn + sgy * SX;
                        const real ty_ = real(sgy);
                        ld4(mpA + 4 * ke, xx, xy, xz, yy);
                        ld2(mpB + 2 * ke, yz, zz);
                        se[0] += s * xx + ty_ * xy;
                        se[1] += s * xy + ty_ * yy;
                        se[2] += s * xz + ty_ * yz;
                    }
                }
                ld4(mpA + 4 * kc, xx, xy, xz, yy);
                ld2(mpB + 2 * kc, yz, zz);
                const real zc[3] = {xz, yz, zz};
                const real sixth = real(1) / real(6), twelfth = real(1) / real(12);
                real up[3], u0[3], um[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    u0[c] = sixth * sp[c] + twelfth * se[c];
                    up[c] = twelfth * (sp[c] + sz[c]) + sixth * zc[c];
                    um[c] = twelfth * (sp[c] - sz[c]) - sixth * zc[c];
                }
                // g(q-1) = -(U+(q) + U0(q-1) + U-(q-2))   (Eq. 28)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    gf[c] = gacc1[c] - up[c];
                    gacc1[c] = gacc2[c] - u0[c];
                    gacc2[c] = -um[c];
                }
            }
        }

        // ---------------- stage C: collide and push plane s
        const int s = p - Lay::LAG_C;
        if (s >= z0 && own) {
            const int is = s - pstart;
            const real* st_r = stash + (is % Lay::NSTASH) * Lay::SLOT;
            real f[Q];
            if constexpr (RAW) {
                const typename S::rawi* sd_r = reinterpret_cast<const typename S::rawi*>(st_r + NT);
                f[0] = st_r[tid];
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    f[i] = S::devi(sd_r[(i - 1) * NT + tid]);
                });
            } else {
                static_for<0, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    f[i] = st_r[i * NT + tid];
                });
            }
            const real rho = rho_s[(is % Lay::NRHO) * RN + (ty + HY) * RX + (tx + HX)];
            real G[3], lap;
            if constexpr (FORCING) {
                const real* gl = gl_s + ((s - pstart) & 1) * 4 * NT;
                ld4(gl + 4 * tid, G[0], G[1], G[2], lap);
            } else {
                G[0] = Geq[0];
                G[1] = Geq[1];
                G[2] = Geq[2];
                lap = lapeq;
            }
            bad |= !(rho > real(0)) || !(rho < real(1e30));
            real out[Q];
            collide<L, FORCING, real>(f, rho, G, lap, gf, pa, pb, pT, pk, om, nu, pref, rsum, out);
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const int idx = zr[1 + L::ez(i)] + yr[1 + L::ey(i)] + xw[1 + L::ex(i)];
                LB_GUARD(idx >= 0 && idx < vol, BK_3D_STORE, idx, return)
                if constexpr (i == 0) S::st0(args.dst[0], size_t(idx), out[0]);
                else S::sti(args.dst[i], size_t(idx), out[i]);
            });
        }
        if (s >= z0) {
            advance(zr[0]);
            advance(zr[1]);
            advance(zr[2]);
        }
        if constexpr (!Lay::OPEN) __syncthreads();
    }
    if (bad) atomicOr(args.status, 1u);
}

}  // namespace lbk
