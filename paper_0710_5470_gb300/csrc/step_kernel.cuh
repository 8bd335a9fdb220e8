// Fused free-energy lattice Boltzmann time step (Pooley & Furtado, Eq. 4).
//
// One launch advances the whole lattice by one step.  The populations in HBM
// hold f_i(r, t) after streaming; each CTA owns a TX x TY tile of the xy plane
// and marches through a chunk of z planes (3D) keeping a short window of
// planes in shared memory:
//
//   stage A  plane p:   read every f_i at the tile plus a density halo of H
//                       sites (H = 1 equilibrium scheme, H = 2 forcing
//                       scheme, Sec. VI), sum rho (Eq. 3); the populations of
//                       the tile's own sites are kept in shared memory.
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

namespace lbk {

constexpr int MAXQ = 19;

struct StepArgs {
    const char* src[MAXQ];
    char* dst[MAXQ];
    float fref[MAXQ];
    float pref, rsum;  // deviation storage: fref_i = w_i pref, rsum = pref sum_{i>=1} w_i
    int nx, ny, nz;
    int lz;  // z planes per CTA (3D)
    double a, b, T, kappa, omega, nu;
    unsigned int* status;
};

__host__ __device__ __forceinline__ int wrapi(int v, int n) {
    int r = v % n;
    return r < 0 ? r + n : r;
}

template <class L, bool FORCING, int TX, int TY, class real>
struct StepLayout {
    static constexpr bool D3 = L::D == 3;
    static constexpr int Q = L::Q;
    static constexpr int H = FORCING ? 2 : 1;                 // density halo
    static constexpr int RX = TX + 2 * H, RY = TY + 2 * H, RN = RX * RY;
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
    real sum = real(0);
    static_for<1, L::Q>([&](auto I) {
        constexpr int i = decltype(I)::value;
        constexpr int o = opposite<L>(i);
        if constexpr (i < o) {
            real even = Aw, odd = real(0);
            static_for<0, D>([&](auto C) {
                constexpr int c = decltype(C)::value;
                constexpr int ec = e_comp<L>(i, c);
                add_signed<ec>(odd, Jw[c]);
                if constexpr (ec != 0) even += Tq[c][c];
                static_for<c + 1, D>([&](auto Dd) {
                    constexpr int d = decltype(Dd)::value;
                    add_signed<ec * e_comp<L>(i, d)>(even, Tq[c][d]);
                });
            });
            constexpr real wi = real(w_vel<L>(i));
            real ev = wi * even;
            if constexpr (!FORCING) {
                static_for<0, D>([&](auto C) {
                    constexpr int c = decltype(C)::value;
                    static_for<c, D>([&](auto Dd) {
                        constexpr int d = decltype(Dd)::value;
                        constexpr double wm = w_m<L>(i, c, d);
                        if constexpr (wm != 0.0) ev += real(wm) * Mw[c][d];
                    });
                });
            }
            sum += ev;
            out[i] = omw * f[i] + (ev + wi * odd);
            out[o] = omw * f[o] + (ev - wi * odd);
        }
    });
    out[0] = omw * f[0] + (omega * (rho - rsum) - real(2) * sum);  // Eq. 6 and sum_i F_i = 0
}

template <class L, bool FORCING, class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) step_kernel(const StepArgs args) {
    using real = typename S::real;
    using Lay = StepLayout<L, FORCING, TX, TY, real>;
    constexpr int Q = L::Q, D = L::D, H = Lay::H, NT = Lay::NT;
    constexpr int RX = Lay::RX, RN = Lay::RN, SX = Lay::SX, SN = Lay::SN;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    real* sm = reinterpret_cast<real*>(smem_raw);
    real* rho_s = sm + Lay::OFF_RHO;
    real* stash = sm + Lay::OFF_STASH;
    real* mp_s = sm + Lay::OFF_MP;
    real* g0_s = sm + Lay::OFF_G;
    real* l0_s = sm + Lay::OFF_L;

    const int nx = args.nx, ny = args.ny, nz = args.nz;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = Lay::D3 ? blockIdx.z * args.lz : 0;
    const int z1 = Lay::D3 ? min(z0 + args.lz, nz) : 1;
    const int plane = nx * ny;

    const real pa = real(args.a), pb = real(args.b), pT = real(args.T), pk = real(args.kappa);
    const real om = real(args.omega), nu = real(args.nu);
    const real pref = real(args.pref), rsum = real(args.rsum);

    // stage-A work items: wrapped in-plane index of each halo-region site
    int a_in[Lay::NA], a_st[Lay::NA];
#pragma unroll
    for (int m = 0; m < Lay::NA; ++m) {
        const int k = tid + m * NT;
        a_in[m] = -1;
        a_st[m] = -1;
        if (k < RN) {
            const int rx = k % RX, ry = k / RX;
            a_in[m] = wrapi(y0 - H + ry, ny) * nx + wrapi(x0 - H + rx, nx);
            if (rx >= H && rx < H + TX && ry >= H && ry < H + TY) a_st[m] = (ry - H) * TX + (rx - H);
        }
    }
    const int xs = x0 + tx, ys = y0 + ty;
    const bool own = xs < nx && ys < ny;
    const int xw[3] = {wrapi(xs - 1, nx), wrapi(xs, nx), wrapi(xs + 1, nx)};
    const int yr[3] = {wrapi(ys - 1, ny) * nx, wrapi(ys, ny) * nx, wrapi(ys + 1, ny) * nx};

    const int pstart = z0 - Lay::LAG_C;
    const int pend = z1 + Lay::LAG_C;

    // Populations of the halo region of one plane, held in registers.  In 3D
    // with 32-bit arithmetic the loads of plane p+1 are issued before stages
    // B and C of plane p, so their latency overlaps that work.
    constexpr bool PREFETCH = Lay::D3 && sizeof(real) == 4;
    typename S::raw0 r0[Lay::NA];
    typename S::rawi ri[Lay::NA][Q - 1];
    auto issue = [&](int p) {
        const int poff = Lay::D3 ? wrapi(p, nz) * plane : 0;
#pragma unroll
        for (int m = 0; m < Lay::NA; ++m) {
            if (a_in[m] >= 0) {
                const size_t q = size_t(poff + a_in[m]);
                r0[m] = S::ld0(args.src[0], q);
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    ri[m][i - 1] = S::ldi(args.src[i], q);
                });
            }
        }
    };
    if (PREFETCH) issue(pstart);

    for (int p = pstart; p < pend; ++p) {
        const int it = p - pstart;
        // ---------------- stage A: density of plane p on the halo region
        {
            if (!PREFETCH) issue(p);
            real* rho_w = rho_s + (it % Lay::NRHO) * RN;
            real* st_w = stash + (it % Lay::NSTASH) * Q * NT;
            const bool keep = p >= z0 && p < z1;
#pragma unroll
            for (int m = 0; m < Lay::NA; ++m) {
                if (a_in[m] >= 0) {
                    real f[Q];               // f_0 and the deviations d_i
                    f[0] = S::dec0(r0[m]);
                    static_for<1, Q>([&](auto I) {
                        constexpr int i = decltype(I)::value;
                        f[i] = S::devi(ri[m][i - 1]);
                    });
                    real r = rsum;
                    static_for<1, Q>([&](auto I) { r += f[decltype(I)::value]; });
                    r += f[0];
                    rho_w[tid + m * NT] = r;
                    if (keep && a_st[m] >= 0) {
                        static_for<0, Q>([&](auto I) {
                            constexpr int i = decltype(I)::value;
                            st_w[i * NT + a_st[m]] = f[i];
                        });
                    }
                }
            }
            if (PREFETCH && p + 1 < pend) issue(p + 1);
        }
        __syncthreads();

        // ---------------- stage B (forcing): G, M' on the tile + 1 ring of plane q
        if constexpr (FORCING) {
            const int q = p - Lay::LAG_B;
            const int iq = q - pstart;
            if (!Lay::D3 || q >= z0 - 1) {
                const real* rho_p[3] = {rho_s + ((iq + 2) % Lay::NRHO) * RN, rho_s + (iq % Lay::NRHO) * RN,
                                        rho_s + ((iq + 1) % Lay::NRHO) * RN};   // planes q-1, q, q+1
                real* mp_w = mp_s + (iq % Lay::NMP) * Lay::NMC * SN;
                const int gs = iq % Lay::NGL;
#pragma unroll
                for (int m = 0; m < Lay::NB; ++m) {
                    const int k = tid + m * NT;
                    if (k < SN) {
                        const int sx = k % SX, sy = k / SX;
                        const int rc = (sy + H - 1) * RX + (sx + H - 1);
                        const real r0 = rho_p[1][rc];
                        real G[3] = {real(0), real(0), real(0)};
                        real lap = real(0);
                        static_for<1, Q>([&](auto I) {
                            constexpr int i = decltype(I)::value;
                            const real rn = rho_p[1 + L::ez(i)][rc + L::ey(i) * RX + L::ex(i)];
                            constexpr real wi = real(w_vel<L>(i));
                            add_signed<L::ex(i)>(G[0], wi * rn);
                            add_signed<L::ey(i)>(G[1], wi * rn);
                            if constexpr (D == 3) add_signed<L::ez(i)>(G[2], wi * rn);
                            lap += wi * (rn - r0);
                        });
                        real g2 = real(0);
#pragma unroll
                        for (int c = 0; c < D; ++c) g2 += G[c] * G[c];
#pragma unroll
                        for (int c = 0; c < D; ++c)
#pragma unroll
                            for (int d = c; d < D; ++d) {
                                real v = pk * G[c] * G[d];
                                if (c == d) v -= real(0.5) * pk * g2;
                                mp_w[mcomp<D>(c, d) * SN + k] = v;
                            }
                        if (sx >= 1 && sx <= TX && sy >= 1 && sy <= TY) {
                            const int r0i = (sy - 1) * TX + (sx - 1);
#pragma unroll
                            for (int c = 0; c < D; ++c) g0_s[(gs * D + c) * NT + r0i] = G[c];
                            l0_s[gs * NT + r0i] = real(2) * lap;
                        }
                    }
                }
            }
            __syncthreads();
        }

        // ---------------- stage C: collide and push plane s
        const int s = p - Lay::LAG_C;
        if (s >= z0 && own) {
            const int is = s - pstart;
            const real* st_r = stash + (is % Lay::NSTASH) * Q * NT;
            real f[Q];
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                f[i] = st_r[i * NT + tid];
            });
            const int rc = (ty + H) * RX + (tx + H);
            const real rho = rho_s[(is % Lay::NRHO) * RN + rc];
            real G[3] = {real(0), real(0), real(0)};
            real g[3] = {real(0), real(0), real(0)};
            real lap = real(0);
            if constexpr (FORCING) {
                const int gs = is % Lay::NGL;
#pragma unroll
                for (int c = 0; c < D; ++c) G[c] = g0_s[(gs * D + c) * NT + tid];
                lap = l0_s[gs * NT + tid];
                // g_a = -sum_i w_i sum_b e_ib M'_ab(r + e_i)   (Eq. 28)
                const real* mp_p[3] = {mp_s + ((is + 2) % Lay::NMP) * Lay::NMC * SN,
                                       mp_s + (is % Lay::NMP) * Lay::NMC * SN,
                                       mp_s + ((is + 1) % Lay::NMP) * Lay::NMC * SN};   // planes s-1, s, s+1
                const int kc = (ty + 1) * SX + (tx + 1);
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    const real* mp = mp_p[1 + L::ez(i)] + kc + L::ey(i) * SX + L::ex(i);
                    constexpr real wi = real(w_vel<L>(i));
                    static_for<0, D>([&](auto C) {
                        constexpr int c = decltype(C)::value;
                        real acc = real(0);
                        bool any = false;
                        static_for<0, D>([&](auto Dd) {
                            constexpr int d = decltype(Dd)::value;
                            constexpr int ed = e_comp<L>(i, d);
                            if constexpr (ed != 0) {
                                add_signed<ed>(acc, mp[mcomp<D>(c, d) * SN]);
                                any = true;
                            }
                        });
                        if (any) g[c] -= wi * acc;
                    });
                });
            } else {
                const real* rho_p[3] = {rho_s + ((is + 2) % Lay::NRHO) * RN, rho_s + (is % Lay::NRHO) * RN,
                                        rho_s + ((is + 1) % Lay::NRHO) * RN};
                static_for<1, Q>([&](auto I) {
                    constexpr int i = decltype(I)::value;
                    const real rn = rho_p[1 + L::ez(i)][rc + L::ey(i) * RX + L::ex(i)];
                    constexpr real wi = real(w_vel<L>(i));
                    add_signed<L::ex(i)>(G[0], wi * rn);
                    add_signed<L::ey(i)>(G[1], wi * rn);
                    if constexpr (D == 3) add_signed<L::ez(i)>(G[2], wi * rn);
                    lap += wi * (rn - rho);
                });
                lap *= real(2);
            }
            if (!(rho > real(0)) || !(rho < real(1e30))) atomicOr(args.status, 1u);
            real out[Q];
            collide<L, FORCING, real>(f, rho, G, lap, g, pa, pb, pT, pk, om, nu, pref, rsum, out);
            const int zc = Lay::D3 ? wrapi(s, nz) : 0;
            const int zr[3] = {Lay::D3 ? wrapi(s - 1, nz) * plane : 0, zc * plane,
                               Lay::D3 ? wrapi(s + 1, nz) * plane : 0};
            static_for<0, Q>([&](auto I) {
                constexpr int i = decltype(I)::value;
                const int idx = zr[1 + L::ez(i)] + yr[1 + L::ey(i)] + xw[1 + L::ex(i)];
                if constexpr (i == 0) S::st0(args.dst[0], size_t(idx), out[0]);
                else S::sti(args.dst[i], size_t(idx), out[i]);
            });
        }
        if (Lay::D3) __syncthreads();
    }
}

}  // namespace lbk
