// Fused free-energy lattice Boltzmann time step (Pooley & Furtado, Eq. 4).
//
// One launch advances the whole lattice by one step.  The populations in HBM
// hold f_i(r, t) after streaming; each CTA owns a TX x TY tile of the xy plane
// and marches through a chunk of z planes (3D) keeping a short window of
// planes in shared memory:
//
//   stage A  plane p:   read every f_i at the tile plus a density halo (2
//                       sites in x; in y 1 for the equilibrium scheme, 2 for
//                       the forcing scheme, Sec. VI), sum rho (Eq. 3); the
//                       populations of the tile's own sites are kept in
//                       shared memory.  With an even nx a thread moves two
//                       adjacent x sites per access.
//   stage B  plane p-1: (forcing) gradient of rho on the tile plus one ring,
//                       M'_ab = kappa (d_a rho d_b rho - delta_ab |d rho|^2/2),
//                       gradient and Laplacian on the tile.
//   stage C  plane p-2: (p-1 for the equilibrium scheme) per site: u (Eq. 3),
//                       p0 (Eq. 2), lambda (Eq. 36), f^eq (Eqs. 5, 6), force
//                       g = -div M' (Eq. 28) and F_i (Eq. 27), BGK, and the
//                       push of f*_i(r) to r + e_i in the other buffer.
//
// HBM traffic is one read and one write of every population per step; the
// density halo is recomputed from populations that neighbouring CTAs read at
// the same time (served by L2).  2D lattices use the same code with a single
// plane and no lag between the stages.  Every loop over velocities is
// expanded at compile time (static_for), so velocity components and weights
// are literals in the generated code.
#pragma once
#include "lattice.cuh"
#include "storage.cuh"
#include "bounds.cuh"

namespace lbk {

constexpr int MAXQ = 19;

struct StepArgs {
    const char* src[MAXQ];
    char* dst[MAXQ];
    const char* src_base;   // population 0 of src; population i at pop_offset(i, pitch)
    char* dst_base;
    long long pitch;        // elements per population array
    float fref[MAXQ];
    float pref, rsum;  // deviation storage: fref_i = w_i pref, rsum = pref sum_{i>=1} w_i
    int nx, ny, nz;
    int lz;  // longest z chunk of a CTA (3D)
    const int4* work;  // 3D: per CTA (x0, y0, z0, z1) of its column tile and z chunk
    int pair2d;  // 2D: two sites per halo load (nx even, 32-bit arithmetic)
    double a, b, T, kappa, omega, nu;
    // the same parameters rounded to float32 (rounded on the host, so a
    // 32-bit kernel reads them as constant operands instead of converting
    // doubles inside its loops)
    float fa, fb, fT, fkappa, fomega, fnu;
    unsigned int* status;
};

// A parameter in the arithmetic type: the double, or its float32 rounding.
template <class real>
__device__ __forceinline__ real arg_param(double d, float f) {
    if constexpr (sizeof(real) == 4) return f;
    else return d;
}

__host__ __device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

// wrapi for the per-site offsets of the tile kernels: one compare-and-add
// covers v in [-n, 2n) (a lattice offset at most n outside [0, n)); anything
// further out (lattices narrower than the halo) takes the integer modulo.
// Same result as wrapi for every v.
__host__ __device__ __forceinline__ int wrap_near(int v, int n) {
    if (v < 0) v += n;
    else if (v >= n) v -= n;
    if (unsigned(v) >= unsigned(n)) v = wrapi(v, n);
    return v;
}

// Sum of a[B], ..., a[E-1] as a balanced tree (short dependency chains).
template <int B, int E, class real>
__device__ __forceinline__ real tree_sum(const real* a) {
    if constexpr (E - B == 1) return a[B];
    else {
        constexpr int M = B + (E - B) / 2;
        return tree_sum<B, M>(a) + tree_sum<M, E>(a);
    }
}

// Density of one site from f_0 and the deviations d_1..d_18 (Eq. 3):
// rho = (rsum + f_0) + sum_i d_i.
template <int Q, class real>
__device__ __forceinline__ real site_rho(const real (&f)[Q], real rsum) {
    return (rsum + f[0]) + tree_sum<1, Q>(f);
}

// Two adjacent sites' values of one population: a packed pair, whose float32
// adds run as one paired instruction.
template <class real>
using pair_t = std::conditional_t<sizeof(real) == 4, float2, double2>;

__device__ __forceinline__ float2 pair_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ double2 pair_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

template <int B, int E, class P>
__device__ __forceinline__ P tree_sum_pair(const P* a) {
    if constexpr (E - B == 1) return a[B];
    else {
        constexpr int M = B + (E - B) / 2;
        return pair_add(tree_sum_pair<B, M>(a), tree_sum_pair<M, E>(a));
    }
}

// site_rho of two sites at once, the same order of additions in each lane.
template <int Q, class P, class real>
__device__ __forceinline__ P site_rho_pair(const P (&f)[Q], real rsum) {
    return pair_add(pair_add(P{rsum, rsum}, f[0]), tree_sum_pair<1, Q>(f));
}

template <class real>
__device__ __forceinline__ void st_pair(real* p, real a, real b) {
    if constexpr (sizeof(real) == 4) *reinterpret_cast<float2*>(p) = make_float2(a, b);
    else *reinterpret_cast<double2*>(p) = make_double2(a, b);
}

template <class L, bool FORCING, int TX, int TY, class real>
struct StepLayout {
    static constexpr bool D3 = L::D == 3;
    static constexpr int Q = L::Q;
    static constexpr int H = FORCING ? 2 : 1;                 // density halo in y
    static constexpr int HX = 2, HY = H;                      // x halo even: pairs start on even x
    static constexpr int RX = TX + 2 * HX, RY = TY + 2 * HY, RN = RX * RY;
    static constexpr int SX = TX + 2, SY = TY + 2, SN = SX * SY;  // tile + one ring
    static constexpr int NT = TX * TY;
    static constexpr int NA = (RN + NT - 1) / NT;
    static constexpr int NB = (SN + NT - 1) / NT;
    static constexpr int NRHO = D3 ? 3 : 1;
    static constexpr int NSTASH = D3 ? (FORCING ? 3 : 2) : 1;
    static constexpr int NMC = D3 ? 6 : 3;                    // components of M'
    static constexpr int NMP = FORCING ? (D3 ? 3 : 1) : 0;
    static constexpr int NGL = FORCING ? (D3 ? 2 : 1) : 0;
    static constexpr int LAG_B = (D3 && FORCING) ? 1 : 0;
    static constexpr int LAG_C = D3 ? (FORCING ? 2 : 1) : 0;
    static constexpr int OFF_RHO = 0;
    static constexpr int OFF_STASH = OFF_RHO + NRHO * RN;
    static constexpr int OFF_MP = OFF_STASH + NSTASH * Q * NT;
    static constexpr int OFF_G = OFF_MP + NMP * NMC * SN;
    static constexpr int OFF_L = OFF_G + NGL * L::D * NT;
    static constexpr int TOTAL = OFF_L + NGL * NT;
    static constexpr size_t BYTES = size_t(TOTAL) * sizeof(real);
};

// index of the M' component (a, b) in shared memory
template <int D>
__host__ __device__ constexpr int mcomp(int a, int b) {
    return a == b ? a : (D == 2 ? 2 : ((a + b == 1) ? 3 : ((a + b == 3) ? 4 : 5)));
}

template <int E, class real>
__device__ __forceinline__ void add_signed(real& acc, real v) {
    if constexpr (E == 1) acc += v;
    if constexpr (E == -1) acc -= v;
}

// Momentum j = sum_i f_i e_i (Eq. 3).
template <class L, class real>
__device__ __forceinline__ void momentum(const real (&f)[L::Q], real (&j)[3]) {
    j[0] = j[1] = j[2] = real(0);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        add_signed<L::ex(i)>(j[0], f[i]);
        add_signed<L::ey(i)>(j[1], f[i]);
        if constexpr (L::D == 3) add_signed<L::ez(i)>(j[2], f[i]);
    });
}

// Tuned equilibrium (Eqs. 5, 6) of one site from rho, j = rho u, u, the
// gradient G and Laplacian lap of rho.  The M_ab = kappa d_a rho d_b rho terms
// are included in the equilibrium scheme only (Sec. VI).  feq[0] closes the
// sum: sum_i feq_i = rho.  Used to initialise populations.
template <class L, bool FORCING, class real>
__device__ __forceinline__ void equilibrium(real rho, const real (&j)[3], const real (&u)[3],
                                            const real (&G)[3], real lap, real a, real b, real T,
                                            real kappa, real nu, real (&feq)[L::Q]) {
    constexpr int D = L::D;
    const real ib = real(1) / (real(1) - b * rho);
    const real p0 = rho * T * ib - a * rho * rho;            // Eq. 2
    const real cs2 = T * ib * ib - real(2) * a * rho;        // dp0/drho
    const real lam = nu * (real(1) - real(3) * cs2);         // Eq. 36
    real udg = real(0);
    for (int c = 0; c < D; ++c) udg += u[c] * G[c];
    real Qt[3][3];
    for (int c = 0; c < D; ++c)
        for (int d = c; d < D; ++d) {
            real v = rho * u[c] * u[d] + lam * (u[c] * G[d] + u[d] * G[c]);
            if (c == d) v += lam * udg;
            Qt[c][d] = v;
            Qt[d][c] = v;
        }
    real trQ = real(0);
    for (int c = 0; c < D; ++c) trQ += Qt[c][c];
    const real A0 = (p0 - kappa * rho * lap) - real(0.5) * trQ;
    real sum = real(0);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        real s = A0;
        real qe = real(0);
        static_for<0, D>([&](auto C) {
            constexpr int c = decltype(C)::value;
            add_signed<e_comp<L>(i, c)>(s, j[c]);
            static_for<0, D>([&](auto Dd) {
                constexpr int d = decltype(Dd)::value;
                add_signed<e_comp<L>(i, c) * e_comp<L>(i, d)>(qe, Qt[c][d]);
            });
        });
        real fe = real(w_vel<L>(i)) * (s + real(1.5) * qe);
        if constexpr (!FORCING) {
            static_for<0, D>([&](auto C) {
                constexpr int c = decltype(C)::value;
                static_for<c, D>([&](auto Dd) {
                    constexpr int d = decltype(Dd)::value;
                    constexpr double wm = w_m<L>(i, c, d);
                    if constexpr (wm != 0.0) fe += real(wm) * kappa * G[c] * G[d];
                });
            });
        }
        feq[i] = fe;
        sum += fe;
    });
    feq[0] = rho - sum;                                       // Eq. 6
}

template <class real>
__device__ __forceinline__ real fast_rcp(real x) {
    if constexpr (sizeof(real) == 4) return __fdividef(1.0f, x);
    else return real(1) / x;
}

// BGK collision with force, Eq. 4: f*_i = (1 - omega) f_i + omega f^eq_i + F_i,
// with f^eq of Eqs. 5, 6 and, for the forcing scheme, F_i of Eq. 27 and
// F_0 = -sum F_i.  Written as one quadratic form in e_i per site:
//   omega f^eq_i + F_i = w_i [e.(omega j + g) + e.T.e + omega A0 - u.g] (+ omega M-part)
//   T_cd = 3/2 (omega Q_cd + u_c g_d + u_d g_c),  A0 = p0 - kappa rho lap - trQ/2,
//   Q_cd = rho u_c u_d + lambda (u_c G_d + u_d G_c + delta_cd u.G).
// Populations i >= 1 are deviations d_i = f_i - w_i pref from the rest state
// w_i pref (pref = 0 stores f_i itself); since sum_i w_i e_i = 0 the momentum
// is sum_i d_i e_i, and the collided deviation is (1 - omega) d_i + v_i with
// v_i = w_i [... - omega pref].  rsum = pref sum_{i>=1} w_i.  Opposite
// velocities i, -i share the even part of v and differ in the sign of e.J.
template <class L, bool FORCING, class real>
__device__ __forceinline__ void collide(const real (&f)[L::Q], real rho, const real (&G)[3], real lap,
                                        const real (&g)[3], real a, real b, real T, real kappa,
                                        real omega, real nu, real pref, real rsum, real (&out)[L::Q]) {
    constexpr int D = L::D;
    real j[3] = {real(0), real(0), real(0)};
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int o = opposite<L>(i);
        if constexpr (i < o) {
            const real df = f[i] - f[o];
            add_signed<L::ex(i)>(j[0], df);
            add_signed<L::ey(i)>(j[1], df);
            if constexpr (D == 3) add_signed<L::ez(i)>(j[2], df);
        }
    });
    const real irho = fast_rcp(rho);
    real u[3] = {j[0] * irho, j[1] * irho, D == 3 ? j[2] * irho : real(0)};
    const real ib = fast_rcp(real(1) - b * rho);
    const real p0 = rho * T * ib - a * rho * rho;            // Eq. 2
    const real cs2 = T * ib * ib - real(2) * a * rho;        // dp0/drho
    const real lam = nu * (real(1) - real(3) * cs2);         // Eq. 36
    real lu[3], udg = real(0), ug = real(0), g3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lu[c] = lam * u[c];
        g3[c] = FORCING ? real(3) * g[c] : real(0);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) {
        udg += u[c] * G[c];
        if (FORCING) ug += u[c] * g[c];
    }
    const real w15 = real(1.5) * omega, w3 = real(3) * omega;
    real Tq[3][3];          // T_cd (diagonal) and 2 T_cd (off-diagonal)
    real trQ = real(0);
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d = c; d < D; ++d) {
            if (c == d) {
                const real q = j[c] * u[c] + real(2) * lu[c] * G[c] + lam * udg;
                trQ += q;
                Tq[c][c] = w15 * q + (FORCING ? u[c] * g3[c] : real(0));
            } else {
                const real q = j[c] * u[d] + lu[c] * G[d] + lu[d] * G[c];
                Tq[c][d] = w3 * q + (FORCING ? u[c] * g3[d] + u[d] * g3[c] : real(0));
            }
        }
    const real A0 = (p0 - kappa * rho * lap) - real(0.5) * trQ;
    const real Aw = omega * (A0 - pref) - ug;
    real Jw[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) Jw[c] = omega * j[c] + (FORCING ? g[c] : real(0));
    real Mw[3][3];
    if constexpr (!FORCING) {
        const real ok = omega * kappa;
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int d = c; d < D; ++d) Mw[c][d] = ok * G[c] * G[d];
    }
    const real omw = real(1) - omega;
    // Even part of pair (i, -i): Aw plus T_cc of every nonzero component c of
    // e_i plus e_ic e_id T_cd.  Per axis E_c = Aw + T_cc; per plane of
    // diagonals, weighted, WP_cd = w_diag (E_c + T_dd) and WT_cd = w_diag T_cd,
    // so a diagonal pair's even part is WP_cd +- WT_cd.
    constexpr real wax = real(L::D == 2 ? 1.0 / 3.0 : 1.0 / 6.0), wdg = real(1.0 / 12.0);
    real E[3], WP[3][3], WT[3][3];
#pragma unroll
    for (int c = 0; c < D; ++c) E[c] = Aw + Tq[c][c];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d = c + 1; d < D; ++d) {
            WP[c][d] = wdg * (E[c] + Tq[d][d]);
            WT[c][d] = wdg * Tq[c][d];
        }
    real sum = real(0);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int o = opposite<L>(i);
        if constexpr (i < o) {
            constexpr int c = first_axis<L>(i), d = second_axis<L>(i);
            real odd = real(0);
            static_for<0, D>([&](auto C) {
                constexpr int cc = decltype(C)::value;
                add_signed<e_comp<L>(i, cc)>(odd, Jw[cc]);
            });
            constexpr real wi = real(w_vel<L>(i));
            real ev;
            if constexpr (d < 0) {
                ev = wax * E[c];
            } else {
                ev = WP[c][d];
                add_signed<e_comp<L>(i, c) * e_comp<L>(i, d)>(ev, WT[c][d]);
            }
            if constexpr (!FORCING) {
                static_for<0, D>([&](auto C) {
                    constexpr int c2 = decltype(C)::value;
                    static_for<c2, D>([&](auto Dd) {
                        constexpr int d2 = decltype(Dd)::value;
                        constexpr double wm = w_m<L>(i, c2, d2);
                        if constexpr (wm != 0.0) ev += real(wm) * Mw[c2][d2];
                    });
                });
                sum += ev;
            }
            out[i] = omw * f[i] + (ev + wi * odd);
            out[o] = omw * f[o] + (ev - wi * odd);
        }
    });
    if constexpr (FORCING) {
        // sum over pairs of the even parts: the two diagonal pairs of a plane add to 2 WP_cd
        real se = E[0];
#pragma unroll
        for (int c = 1; c < D; ++c) se += E[c];
        real sp = real(0);
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int d = c + 1; d < D; ++d) sp += WP[c][d];
        sum = wax * se + real(2) * sp;
    }
    out[0] = omw * f[0] + (omega * (rho - rsum) - real(2) * sum);  // Eq. 6 and sum_i F_i = 0
}

// Per-tile arguments of the 2D step: population buffers as one base pointer
// each (population i at byte offset S::pop_offset(i, pitch)), grid size and
// physical parameters.
struct Tile2DArgs {
    const char* src;
    char* dst;
    long long pitch;
    int nx, ny;
    int pair;            // 1: two sites per halo load (nx even, 32-bit arithmetic)
    double a, b, T, kappa, omega, nu;
    float fa, fb, fT, fkappa, fomega, fnu;   // their float32 roundings
    float pref, rsum;
    unsigned int* status;
};

// One D2Q9 time step of the TX x TY tile at (x0, y0) (Eq. 4): stage A sums
// rho on the tile plus its density halo, stage B (forcing) computes the
// gradient and M' on the tile plus one ring, stage C collides and pushes the
// tile's sites.  smem holds StepLayout<L, FORCING, TX, TY, real>::TOTAL reals.
template <class L, bool FORCING, class S, int TX, int TY>
__device__ __forceinline__ void step2d_tile(const Tile2DArgs& args, int x0, int y0, typename S::real* sm) {
    static_assert(L::D == 2, "2D tile step");
    using real = typename S::real;
    using Lay = StepLayout<L, FORCING, TX, TY, real>;
    constexpr int Q = L::Q, D = 2, HX = Lay::HX, HY = Lay::HY, NT = Lay::NT;
    constexpr int RX = Lay::RX, RN = Lay::RN, SX = Lay::SX, SN = Lay::SN;
    real* rho_s = sm + Lay::OFF_RHO;
    real* stash = sm + Lay::OFF_STASH;
    real* mp_s = sm + Lay::OFF_MP;
    real* g0_s = sm + Lay::OFF_G;
    real* l0_s = sm + Lay::OFF_L;

    const int nx = args.nx, ny = args.ny;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const real pa = arg_param<real>(args.a, args.fa), pb = arg_param<real>(args.b, args.fb);
    const real pT = arg_param<real>(args.T, args.fT), pk = arg_param<real>(args.kappa, args.fkappa);
    const real om = arg_param<real>(args.omega, args.fomega), nu = arg_param<real>(args.nu, args.fnu);
    const real pref = real(args.pref), rsum = real(args.rsum);
    const long long pitch = args.pitch;

    // ---------------- stage A: density on the halo region (2 columns in x, HY rows in y)
    if (sizeof(real) == 4 && args.pair) {
        // two adjacent sites per item, 2-vector loads (x0 - HX and nx even: aligned, never split by the wrap)
        constexpr int NIT = RN / 2, NA2 = (NIT + NT - 1) / NT;
#pragma unroll
        for (int m = 0; m < NA2; ++m) {
            const int k = tid + m * NT;
            if (k < NIT) {
                const int rx = (k % (RX / 2)) * 2, ry = k / (RX / 2);
                const size_t q = size_t(wrap_near(y0 - HY + ry, ny)) * nx + wrap_near(x0 - HX + rx, nx);
                pair_t<real> f2[Q];
                LB_GUARD(q + 1 < size_t(nx) * ny, BK_2D_LOAD, q, continue)
                S::dec0x2(S::ld0x2(args.src, q), f2[0].x, f2[0].y);
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    S::devix2(S::ldix2(args.src + S::pop_offset(i, pitch), q), f2[i].x, f2[i].y);
                });
                const pair_t<real> r2 = site_rho_pair(f2, rsum);
                st_pair(rho_s + 2 * k, r2.x, r2.y);
                if (rx >= HX && rx < HX + TX && ry >= HY && ry < HY + TY) {
                    const int st = (ry - HY) * TX + (rx - HX);
                    static_for<0, Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        st_pair(stash + i * NT + st, f2[i].x, f2[i].y);
                    });
                }
            }
        }
    } else {
#pragma unroll
        for (int m = 0; m < Lay::NA; ++m) {
            const int k = tid + m * NT;
            if (k < RN) {
                const int rx = k % RX, ry = k / RX;
                const size_t q = size_t(wrap_near(y0 - HY + ry, ny)) * nx + wrap_near(x0 - HX + rx, nx);
                real f[Q];
                LB_GUARD(q < size_t(nx) * ny, BK_2D_LOAD, q, continue)
                f[0] = S::dec0(S::ld0(args.src, q));
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    f[i] = S::devi(S::ldi(args.src + S::pop_offset(i, pitch), q));
                });
                rho_s[k] = site_rho(f, rsum);
                if (rx >= HX && rx < HX + TX && ry >= HY && ry < HY + TY) {
                    const int st = (ry - HY) * TX + (rx - HX);
                    static_for<0, Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        stash[i * NT + st] = f[i];
                    });
                }
            }
        }
    }
    __syncthreads();

    // ---------------- stage B (forcing): G, M' on the tile + 1 ring
    if constexpr (FORCING) {
#pragma unroll
        for (int m = 0; m < Lay::NB; ++m) {
            const int k = tid + m * NT;
            if (k < SN) {
                const int sx = k % SX, sy = k / SX;
                const int rc = (sy + HY - 1) * RX + (sx + HX - 1);
                const real r0 = rho_s[rc];
                real G[2] = {real(0), real(0)};
                real lap = real(0);
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    const real rn = rho_s[rc + L::ey(i) * RX + L::ex(i)];
                    constexpr real wi = real(w_vel<L>(i));
                    add_signed<L::ex(i)>(G[0], wi * rn);
                    add_signed<L::ey(i)>(G[1], wi * rn);
                    lap += wi * (rn - r0);
                });
                const real hk = real(0.5) * pk * (G[0] * G[0] + G[1] * G[1]);
                mp_s[0 * SN + k] = pk * G[0] * G[0] - hk;
                mp_s[1 * SN + k] = pk * G[1] * G[1] - hk;
                mp_s[2 * SN + k] = pk * G[0] * G[1];
                if (sx >= 1 && sx <= TX && sy >= 1 && sy <= TY) {
                    const int r0i = (sy - 1) * TX + (sx - 1);
                    g0_s[r0i] = G[0];
                    g0_s[NT + r0i] = G[1];
                    l0_s[r0i] = real(2) * lap;
                }
            }
        }
        __syncthreads();
    }

    // ---------------- stage C: collide and push
    const int xs = x0 + tx, ys = y0 + ty;
    if (xs < nx && ys < ny) {
        real f[Q];
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            f[i] = stash[i * NT + tid];
        });
        const int rc = (ty + HY) * RX + (tx + HX);
        const real rho = rho_s[rc];
        real G[3] = {real(0), real(0), real(0)};
        real g[3] = {real(0), real(0), real(0)};
        real lap = real(0);
        if constexpr (FORCING) {
            G[0] = g0_s[tid];
            G[1] = g0_s[NT + tid];
            lap = l0_s[tid];
            // g_a = -sum_i w_i sum_b e_ib M'_ab(r + e_i)   (Eq. 28)
            const int kc = (ty + 1) * SX + (tx + 1);
            static_for<1, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const real* mp = mp_s + kc + L::ey(i) * SX + L::ex(i);
                constexpr real wi = real(w_vel<L>(i));
                static_for<0, D>([&](auto C) {
                    constexpr int c = decltype(C)::value;
                    real acc = real(0);
                    static_for<0, D>([&](auto Dd) {
                        constexpr int d = decltype(Dd)::value;
                        add_signed<e_comp<L>(i, d)>(acc, mp[mcomp<D>(c, d) * SN]);
                    });
                    g[c] -= wi * acc;
                });
            });
        } else {
            static_for<1, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const real rn = rho_s[rc + L::ey(i) * RX + L::ex(i)];
                constexpr real wi = real(w_vel<L>(i));
                add_signed<L::ex(i)>(G[0], wi * rn);
                add_signed<L::ey(i)>(G[1], wi * rn);
                lap += wi * (rn - rho);
            });
            lap *= real(2);
        }
        if (!(rho > real(0)) || !(rho < real(1e30))) atomicOr(args.status, 1u);
        real out[Q];
        collide<L, FORCING, real>(f, rho, G, lap, g, pa, pb, pT, pk, om, nu, pref, rsum, out);
        const int xw[3] = {wrap_near(xs - 1, nx), xs, wrap_near(xs + 1, nx)};
        const int yr[3] = {wrap_near(ys - 1, ny) * nx, ys * nx, wrap_near(ys + 1, ny) * nx};
        static_for<0, Q>([&](auto I) {
            constexpr int i = decltype(I)::value;
            const size_t idx = size_t(yr[1 + L::ey(i)] + xw[1 + L::ex(i)]);
            LB_GUARD(idx < size_t(nx) * ny, BK_2D_STORE, idx, return)
            if constexpr (i == 0) S::st0(args.dst, idx, out[0]);
            else S::sti(args.dst + S::pop_offset(i, pitch), idx, out[i]);
        });
    }
}

// One step of a single D2Q9 lattice: one CTA per tile.
template <class L, bool FORCING, class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) step_kernel(const Tile2DArgs args) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step2d_tile<L, FORCING, S, TX, TY>(args, blockIdx.x * TX, blockIdx.y * TY,
                                       reinterpret_cast<typename S::real*>(smem_raw));
}

}  // namespace lbk
