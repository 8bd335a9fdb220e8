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
// plane and no lag between the stages.
#pragma once
#include "lattice.cuh"
#include "storage.cuh"

namespace lbk {

constexpr int MAXQ = 19;

struct StepArgs {
    const char* src[MAXQ];
    char* dst[MAXQ];
    float fref[MAXQ];
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

// Tuned equilibrium (Eqs. 5, 6) and force populations (Eq. 27) of one site,
// from its density rho, momentum j = rho u, velocity u, gradient G and
// Laplacian lap of rho, and (forcing scheme) body force g.  feq[0] and F[0]
// close the sums: sum_i feq_i = rho, sum_i F_i = 0.
template <class L, bool FORCING, class real>
__device__ __forceinline__ void equilibrium(real rho, const real (&j)[3], const real (&u)[3],
                                            const real (&G)[3], real lap, const real (&g)[3],
                                            real a, real b, real T, real kappa, real nu,
                                            real (&feq)[L::Q], real (&F)[L::Q]) {
    constexpr int Q = L::Q, D = L::D;
    const real ib = real(1) / (real(1) - b * rho);
    const real p0 = rho * T * ib - a * rho * rho;            // Eq. 2
    const real cs2 = T * ib * ib - real(2) * a * rho;        // dp0/drho
    const real lam = nu * (real(1) - real(3) * cs2);         // Eq. 36
    real udg = real(0);
#pragma unroll
    for (int c = 0; c < D; ++c) udg += u[c] * G[c];
    real Qt[3][3];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d = c; d < D; ++d) {
            real v = rho * u[c] * u[d] + lam * (u[c] * G[d] + u[d] * G[c]);
            if (c == d) v += lam * udg;
            Qt[c][d] = v;
            Qt[d][c] = v;
        }
    real trQ = real(0);
#pragma unroll
    for (int c = 0; c < D; ++c) trQ += Qt[c][c];
    // w_i (e.j + 3/2 (e e - 1/3) : Q) + w_i (p0 - kappa rho lap), with w^p = w^t = w
    const real A0 = (p0 - kappa * rho * lap) - real(0.5) * trQ;
    real M[3][3];
    if (!FORCING) {
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int d = c; d < D; ++d) M[c][d] = kappa * G[c] * G[d];
    }
    real ug = real(0);
    if (FORCING) {
#pragma unroll
        for (int c = 0; c < D; ++c) ug += u[c] * g[c];
    }
    real sum_eq = real(0), sum_F = real(0);
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        real ej = real(0), eqe = real(0);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const int ec = e_comp<L>(i, c);
            if (ec == 1) ej += j[c];
            if (ec == -1) ej -= j[c];
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const int ed = e_comp<L>(i, d);
                if (ec * ed == 1) eqe += Qt[c][d];
                if (ec * ed == -1) eqe -= Qt[c][d];
            }
        }
        const real wi = real(w_vel<L>(i));
        real fe = wi * (ej + real(1.5) * eqe + A0);
        if (!FORCING) {
#pragma unroll
            for (int c = 0; c < D; ++c)
#pragma unroll
                for (int d = c; d < D; ++d) {
                    const double wm = w_m<L>(i, c, d);
                    if (wm != 0.0) fe += real(wm) * M[c][d];
                }
        }
        feq[i] = fe;
        sum_eq += fe;
        real Fi = real(0);
        if (FORCING) {
            real eg = real(0), eu = real(0);
#pragma unroll
            for (int c = 0; c < D; ++c) {
                const int ec = e_comp<L>(i, c);
                if (ec == 1) { eg += g[c]; eu += u[c]; }
                if (ec == -1) { eg -= g[c]; eu -= u[c]; }
            }
            Fi = wi * (eg + real(3) * eu * eg - ug);          // Eq. 27
            sum_F += Fi;
        }
        F[i] = Fi;
    }
    feq[0] = rho - sum_eq;                                    // Eq. 6
    F[0] = -sum_F;                                            // sum_i F_i = 0
}

// Momentum j = sum_i f_i e_i (Eq. 3).
template <class L, class real>
__device__ __forceinline__ void momentum(const real (&f)[L::Q], real (&j)[3]) {
    j[0] = j[1] = j[2] = real(0);
#pragma unroll
    for (int i = 1; i < L::Q; ++i) {
#pragma unroll
        for (int c = 0; c < L::D; ++c) {
            if (e_comp<L>(i, c) == 1) j[c] += f[i];
            if (e_comp<L>(i, c) == -1) j[c] -= f[i];
        }
    }
}

// BGK collision with force (Eq. 4): f*_i = f_i + omega (f^eq_i - f_i) + F_i.
template <class L, bool FORCING, class real>
__device__ __forceinline__ void collide(const real (&f)[L::Q], real rho, const real (&G)[3], real lap,
                                        const real (&g)[3], real a, real b, real T, real kappa,
                                        real omega, real nu, real (&out)[L::Q]) {
    constexpr int Q = L::Q, D = L::D;
    real j[3];
    momentum<L, real>(f, j);
    const real irho = real(1) / rho;
    real u[3] = {j[0] * irho, j[1] * irho, D == 3 ? j[2] * irho : real(0)};
    real feq[Q], F[Q];
    equilibrium<L, FORCING, real>(rho, j, u, G, lap, g, a, b, T, kappa, nu, feq, F);
#pragma unroll
    for (int i = 0; i < Q; ++i) out[i] = f[i] + omega * (feq[i] - f[i]) + F[i];
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
    const size_t plane = size_t(nx) * ny;

    const real pa = real(args.a), pb = real(args.b), pT = real(args.T), pk = real(args.kappa);
    const real om = real(args.omega), nu = real(args.nu);

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
    const int yw[3] = {wrapi(ys - 1, ny), wrapi(ys, ny), wrapi(ys + 1, ny)};

    const int pstart = z0 - Lay::LAG_C;
    const int pend = z1 + Lay::LAG_C;
    for (int p = pstart; p < pend; ++p) {
        // ---------------- stage A: density of plane p on the halo region
        {
            const size_t poff = Lay::D3 ? size_t(wrapi(p, nz)) * plane : 0;
            const int rs = (p - pstart) % Lay::NRHO;
            const int ss = (p - pstart) % Lay::NSTASH;
            const bool keep = p >= z0 && p < z1;
#pragma unroll
            for (int m = 0; m < Lay::NA; ++m) {
                if (a_in[m] >= 0) {
                    const size_t q = poff + size_t(a_in[m]);
                    real f[Q];
                    real r = real(0);
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        f[i] = S::load(i, args.src[i], q, args.fref[i]);
                        r += f[i];
                    }
                    rho_s[rs * RN + tid + m * NT] = r;
                    if (keep && a_st[m] >= 0) {
#pragma unroll
                        for (int i = 0; i < Q; ++i) stash[(ss * Q + i) * NT + a_st[m]] = f[i];
                    }
                }
            }
        }
        __syncthreads();

        // ---------------- stage B (forcing): G, M' on the tile + 1 ring of plane q
        if constexpr (FORCING) {
            const int q = p - Lay::LAG_B;
            if (!Lay::D3 || q >= z0 - 1) {
                const int ms = (q - pstart) % (Lay::NMP > 0 ? Lay::NMP : 1);
                const int gs = (q - pstart) % (Lay::NGL > 0 ? Lay::NGL : 1);
#pragma unroll
                for (int m = 0; m < Lay::NB; ++m) {
                    const int k = tid + m * NT;
                    if (k < SN) {
                        const int sx = k % SX, sy = k / SX;
                        const int rc = (sy + H - 1) * RX + (sx + H - 1);
                        const real r0 = rho_s[((q - pstart) % Lay::NRHO) * RN + rc];
                        real G[3] = {real(0), real(0), real(0)};
                        real lap = real(0);
#pragma unroll
                        for (int i = 1; i < Q; ++i) {
                            const int pl = (q + L::ez(i) - pstart) % Lay::NRHO;
                            const real rn = rho_s[pl * RN + rc + L::ey(i) * RX + L::ex(i)];
                            const real wi = real(w_vel<L>(i));
#pragma unroll
                            for (int c = 0; c < D; ++c) {
                                if (e_comp<L>(i, c) == 1) G[c] += wi * rn;
                                if (e_comp<L>(i, c) == -1) G[c] -= wi * rn;
                            }
                            lap += wi * (rn - r0);
                        }
                        real g2 = real(0);
#pragma unroll
                        for (int c = 0; c < D; ++c) g2 += G[c] * G[c];
#pragma unroll
                        for (int c = 0; c < D; ++c)
#pragma unroll
                            for (int d = c; d < D; ++d) {
                                real v = pk * G[c] * G[d];
                                if (c == d) v -= real(0.5) * pk * g2;
                                mp_s[(ms * Lay::NMC + mcomp<D>(c, d)) * SN + k] = v;
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
            const int ss = (s - pstart) % Lay::NSTASH;
            const int rsl = (s - pstart) % Lay::NRHO;
            real f[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = stash[(ss * Q + i) * NT + tid];
            const int rc = (ty + H) * RX + (tx + H);
            const real rho = rho_s[rsl * RN + rc];
            real G[3] = {real(0), real(0), real(0)};
            real g[3] = {real(0), real(0), real(0)};
            real lap = real(0);
            if constexpr (FORCING) {
                const int gs = (s - pstart) % Lay::NGL;
#pragma unroll
                for (int c = 0; c < D; ++c) G[c] = g0_s[(gs * D + c) * NT + tid];
                lap = l0_s[gs * NT + tid];
                // g_a = -sum_i w_i sum_b e_ib M'_ab(r + e_i)   (Eq. 28)
                const int kc = (ty + 1) * SX + (tx + 1);
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int pl = (s + L::ez(i) - pstart) % Lay::NMP;
                    const int kn = kc + L::ey(i) * SX + L::ex(i);
                    const real wi = real(w_vel<L>(i));
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        real acc = real(0);
                        bool any = false;
#pragma unroll
                        for (int d = 0; d < D; ++d) {
                            const int ed = e_comp<L>(i, d);
                            if (ed != 0) {
                                const real mv = mp_s[(pl * Lay::NMC + mcomp<D>(c, d)) * SN + kn];
                                if (ed == 1) acc += mv;
                                else acc -= mv;
                                any = true;
                            }
                        }
                        if (any) g[c] -= wi * acc;
                    }
                }
            } else {
                const real r0 = rho;
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int pl = (s + L::ez(i) - pstart) % Lay::NRHO;
                    const real rn = rho_s[pl * RN + rc + L::ey(i) * RX + L::ex(i)];
                    const real wi = real(w_vel<L>(i));
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        if (e_comp<L>(i, c) == 1) G[c] += wi * rn;
                        if (e_comp<L>(i, c) == -1) G[c] -= wi * rn;
                    }
                    lap += wi * (rn - r0);
                }
                lap *= real(2);
            }
            if (!(rho > real(0)) || !(rho < real(1e30))) atomicOr(args.status, 1u);
            real out[Q];
            collide<L, FORCING, real>(f, rho, G, lap, g, pa, pb, pT, pk, om, nu, out);
            const int zc = Lay::D3 ? wrapi(s, nz) : 0;
            const int zw[3] = {Lay::D3 ? wrapi(s - 1, nz) : 0, zc, Lay::D3 ? wrapi(s + 1, nz) : 0};
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const size_t idx = (size_t(zw[1 + L::ez(i)]) * ny + yw[1 + L::ey(i)]) * nx + xw[1 + L::ex(i)];
                S::store(i, args.dst[i], idx, out[i], args.fref[i]);
            }
        }
        if (Lay::D3) __syncthreads();
    }
}

}  // namespace lbk
