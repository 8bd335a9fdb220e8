// Host side of the C ABI declared in include/lb.h: parameter validation,
// the Maxwell construction, device buffers, and kernel launches.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "dispatch.h"
#include "param2d.h"

namespace {

thread_local std::string g_last_error;

lb_status fail(lb_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

lb_status cuda_fail(cudaError_t e, const char* where) {
    return fail(LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// ------------------------------------------------------------ thermodynamics
// van der Waals bulk pressure (Eq. 2), its derivative and the chemical potential.
double p0_vdw(double r, double a, double b, double T) { return r * T / (1.0 - b * r) - a * r * r; }
double cs2_vdw(double r, double a, double b, double T) {
    const double ib = 1.0 / (1.0 - b * r);
    return T * ib * ib - 2.0 * a * r;
}
double mu_vdw(double r, double a, double b, double T) {
    return T * std::log(r / (1.0 - b * r)) + T * b * r / (1.0 - b * r) - 2.0 * a * r;
}

// Safeguarded Newton for fn(x) = target on [lo, hi] with fn increasing.
template <class F, class DF>
double newton_bracketed(F fn, DF dfn, double target, double lo, double hi) {
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        const double r = fn(x) - target;
        if (r > 0) hi = x; else lo = x;
        const double d = dfn(x);
        double xn = (d > 0) ? x - r / d : 0.5 * (lo + hi);
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (std::fabs(xn - x) <= 1e-15 * std::fabs(x)) return xn;
        x = xn;
    }
    return x;
}

// Maxwell construction: pressure P such that mu(rho_l(P)) = mu(rho_g(P)),
// where rho_g(P), rho_l(P) solve p0 = P on the gas and liquid branches.  Newton
// on P with d(mu_l - mu_g)/dP = 1/rho_l - 1/rho_g (dmu = dp/rho on a branch).
lb_status maxwell(double a, double b, double T, double* rl_out, double* rg_out) {
    if (!(a > 0 && b > 0)) return fail(LB_EINVAL, "coexistence: a and b must be positive");
    const double Tc = 8.0 * a / (27.0 * b);
    if (!(T > 0 && T < Tc)) return fail(LB_EINVAL, "coexistence: T must lie in (0, 8a/27b)");
    // c_s^2 decreases up to rho* = (1 - (bT/a)^(1/3))/b and increases beyond;
    // the spinodals are its zeros on either side.
    const double rstar = (1.0 - std::cbrt(b * T / a)) / b;
    auto dcs2 = [&](double r) { return 2.0 * b * T / std::pow(1.0 - b * r, 3) - 2.0 * a; };
    auto neg_cs2 = [&](double r) { return -cs2_vdw(r, a, b, T); };
    auto neg_dcs2 = [&](double r) { return -dcs2(r); };
    const double sp_g = newton_bracketed(neg_cs2, neg_dcs2, 0.0, 1e-300, rstar);
    const double sp_l = newton_bracketed([&](double r) { return cs2_vdw(r, a, b, T); }, dcs2, 0.0, rstar,
                                         (1.0 - 1e-15) / b);
    auto p = [&](double r) { return p0_vdw(r, a, b, T); };
    auto dp = [&](double r) { return cs2_vdw(r, a, b, T); };
    double plo = std::max(p(sp_l), 1e-300), phi = p(sp_g);
    double P = 0.5 * (plo + phi);
    double rl = 0, rg = 0;
    for (int it = 0; it < 200; ++it) {
        rg = newton_bracketed(p, dp, P, 1e-300, sp_g);
        rl = newton_bracketed(p, dp, P, sp_l, (1.0 - 1e-15) / b);
        const double dmu = mu_vdw(rl, a, b, T) - mu_vdw(rg, a, b, T);
        // mu_l - mu_g decreases with P (slope 1/rho_l - 1/rho_g < 0): keep the bracket
        if (dmu > 0) plo = P; else phi = P;
        const double slope = 1.0 / rl - 1.0 / rg;
        double Pn = P - dmu / slope;
        if (!(Pn > plo && Pn < phi)) Pn = 0.5 * (plo + phi);
        if (std::fabs(Pn - P) <= 1e-16 * std::fabs(P)) { P = Pn; break; }
        P = Pn;
    }
    rg = newton_bracketed(p, dp, P, 1e-300, sp_g);
    rl = newton_bracketed(p, dp, P, sp_l, (1.0 - 1e-15) / b);
    *rl_out = rl;
    *rg_out = rg;
    return LB_OK;
}

}  // namespace

// Sets the thread-local message returned by lb_last_error; used by the other
// translation units of the library (not exported through the C ABI).
__attribute__((visibility("hidden"))) void lb_internal_set_error(const char* msg) { g_last_error = msg; }

// ------------------------------------------------------------------ context
struct lb_ctx {
    lb_params p{};
    int D = 2, Q = 9;
    size_t N = 0;
    size_t pitch = 0;        // elements per population array (padded)
    size_t buf_bytes = 0;    // bytes of one population buffer
    char* fbuf = nullptr;    // two buffers back to back
    bool own_fbuf = true;    // false: the caller's memory (lb_create_with_buffers), not freed here
    int cur = 0;
    bool aos = false;        // populations 1..Q-1 in the interleaved block layout (PopPtrs aos)
    double rho_l = 0, rho_g = 0;
    float fref[lbk::MAXQ] = {};
    float pref = 0.0f, rsum = 0.0f;
    cudaStream_t stream = nullptr;
    unsigned* d_status = nullptr;
    LbKernelSet ks;
    int lz = 1;
    dim3 grid;
    int4* d_work = nullptr;   // 3D: per-CTA (x0, y0, z0, z1)
    bool initialised = false;
    long long step = 0;
    lb_status sticky = LB_OK;
    // pressure probes of lb_stats dP (x, y, z of the inside and outside sites)
    int probe_in[3] = {0, 0, 0}, probe_out[3] = {0, 0, 0};
    // velocity field of the previous lb_stats_get (max_du) and its step
    double* w_uprev = nullptr;
    bool uprev_valid = false;
    long long uprev_step = 0;
    // lazily allocated work arrays (fields, reductions)
    double* w_rho = nullptr;
    double* w_u = nullptr;
    double* w_v = nullptr;
    double* w_mp = nullptr;
    double* w_part = nullptr;
    int stat_blocks = 0;
    double* w_io = nullptr;   // Q*N staging for population import/export
    // run-time free parameters (lb_set_free_params): D2Q9 float64 only
    bool free_params = false;
    lbk::Free2D fw{};
    double* p2_rho = nullptr;   // N
    double* p2_gl = nullptr;    // 3N: d_x rho, d_y rho, lap rho
    double* p2_mp = nullptr;    // 2N: M'_xx, M'_xy
    // CUDA graphs of GRAPH_STEPS fused steps, one per starting buffer, captured on
    // a private stream and launched on `stream` (lb_step with nsteps >= GRAPH_STEPS)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
    bool graph_failed = false;
};

namespace {

size_t pop_offset(const lb_ctx* c, int i, int buf) {
    // buffer layout: population 0 first, then 1..Q-1; each array padded to
    // `pitch`, or (aos) populations 1..Q-1 interleaved in blocks of
    // AOS_SITES sites, population i's row of block 0 at (i - 1) * 2 * AOS_SITES
    size_t off = 0;
    const int elem0 = (c->p.storage == LB_F64) ? 8 : 4;
    const int elemi = (c->p.storage == LB_F64) ? 8 : (c->p.storage == LB_F32 ? 4 : 2);
    if (i > 0)
        off = c->pitch * elem0 + (c->aos ? size_t(i - 1) * 2 * lbk::AOS_SITES : size_t(i - 1) * c->pitch * elemi);
    return size_t(buf) * c->buf_bytes + off;
}

lbk::PopPtrs pop_ptrs(const lb_ctx* c, int buf) {
    lbk::PopPtrs pp{};
    for (int i = 0; i < c->Q; ++i) {
        pp.p[i] = c->fbuf + pop_offset(c, i, buf);
        pp.fref[i] = c->fref[i];
    }
    pp.aos = c->aos ? 1 : 0;
    return pp;
}

lbk::Grid3 grid3(const lb_ctx* c) { return lbk::Grid3{c->p.nx, c->p.ny, c->p.nz}; }

lbk::Phys phys(const lb_ctx* c) {
    return lbk::Phys{c->p.a, c->p.b, c->p.T, c->p.kappa, (c->p.tau - 0.5) / 3.0};
}

lbk::Phys2 phys2(const lb_ctx* c) {
    return lbk::Phys2{c->p.a, c->p.b, c->p.T, c->p.kappa, 1.0 / c->p.tau, (c->p.tau - 0.5) / 3.0};
}

double* pop_base(lb_ctx* c, int buf) { return reinterpret_cast<double*>(c->fbuf + size_t(buf) * c->buf_bytes); }

lb_status check_ctx(lb_ctx* c) {
    if (!c) return fail(LB_EINVAL, "null context");
    if (c->sticky != LB_OK) return fail(c->sticky, "context is in an error state: " + g_last_error);
    return LB_OK;
}

lb_status record(lb_ctx* c, cudaError_t e, const char* where) {
    if (e == cudaSuccess) return LB_OK;
    c->sticky = LB_ECUDA;
    return cuda_fail(e, where);
}

// The D3Q19 step's work list: one (x0, y0, z0, z1) per CTA, a column tile of
// tx x ty sites and a chunk [z0, z1) of its planes, in launch order.  With at
// least two resident slots per tile (small lattices) the list fills exactly the
// resident slots: each tile gets slots / tiles chunks, the remainder one more (no
// chunk under 4 planes).  Otherwise every tile gets the same number c of chunks:
// the smallest c whose estimated efficiency (W / ceil(W)) * L / (L + 4) is within
// 0.02 of the best, W = waves of resident CTAs per SM (CTAs per SM / resident
// CTAs per SM), L = chunk length, 4 the halo planes a chunk
// loads in addition (measured on GB300: 224^3 c = 3, 256^3 c = 4, 320^3 c = 3 are
// 13-17% faster than one chunk per tile).  CTAs are listed longest chunk first so
// that the first wave puts one long CTA on every SM and the second wave pairs it
// with a short one.  CTAs resident together march at the same time, so the halo
// rows neighbouring tiles share are read close together (from L2).
std::vector<int4> build_work_list(long long sms, long long occ, int nx, int ny, int nz, int tx, int ty) {
    sms = std::max(sms, 1LL);
    occ = std::max(occ, 1LL);
    const int gx = (nx + tx - 1) / tx, gy = (ny + ty - 1) / ty;
    const long long slots = sms * occ;
    const long long tiles = (long long)gx * gy;
    const int maxc = std::max(1, nz / 4);
    long long uniform_c = 0;
    if (2 * tiles > slots) {
        const long long cmax = std::max(1, nz / 16);
        auto eff = [&](long long cc) {
            // waves of `occ` resident CTAs per SM, the last one partly filled
            const double W = double(cc * tiles) / double(sms * occ), L = double(nz) / double(cc);
            return W / std::ceil(W) * L / (L + 4.0);
        };
        double best = 0.0;
        for (long long cc = 1; cc <= cmax; ++cc) best = std::max(best, eff(cc));
        for (uniform_c = 1; uniform_c < cmax && eff(uniform_c) < best - 0.02; ++uniform_c) {
        }
    }
    std::vector<int4> work;
    for (long long t = 0; t < tiles; ++t) {
        long long ct = uniform_c ? uniform_c : slots / tiles + (t < slots % tiles ? 1 : 0);
        ct = std::max(1LL, std::min<long long>(ct, maxc));
        const int x0 = int(t % gx) * tx, y0 = int(t / gx) * ty;
        for (long long k = 0; k < ct; ++k)
            work.push_back(make_int4(x0, y0, int(k * nz / ct), int((k + 1) * nz / ct)));
    }
    std::stable_sort(work.begin(), work.end(), [](const int4& u, const int4& v) { return u.w - u.z > v.w - v.z; });
    return work;
}

constexpr int GRAPH_STEPS = 64;

// Captures GRAPH_STEPS launches of launch_one, starting from buffer c->cur, into
// an executable graph (on the context's private capture stream).
template <class F>
cudaError_t capture_steps(lb_ctx* c, F& launch_one, cudaGraphExec_t* exec) {
    cudaError_t e = cudaSuccess;
    if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return e;
    int cur = c->cur;
    cudaError_t le = cudaSuccess;
    for (int j = 0; j < GRAPH_STEPS && le == cudaSuccess; ++j) {
        le = launch_one(cur, c->cap_stream);
        cur = 1 - cur;
    }
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(c->cap_stream, &graph);
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    return e;
}

// The density staging array alone (the initialisation paths need no more).
lb_status ensure_rho(lb_ctx* c) {
    if (c->w_rho) return LB_OK;
    cudaError_t e = cudaMalloc(&c->w_rho, c->N * sizeof(double));
    if (e != cudaSuccess) {
        c->w_rho = nullptr;
        return fail(LB_ENOMEM, std::string("density array: ") + cudaGetErrorString(e));
    }
    return LB_OK;
}

// All float64 field and reduction arrays (lb_fields, lb_stats_get, velocity uploads).
lb_status ensure_work(lb_ctx* c) {
    lb_status s = ensure_rho(c);
    if (s != LB_OK) return s;
    if (c->w_part) return LB_OK;
    const size_t n = c->N;
    const int nmc = c->D == 3 ? 6 : 3;
    c->stat_blocks = int(std::min<size_t>(1024, (n + lbk::FR_THREADS - 1) / lbk::FR_THREADS));
    if (c->stat_blocks < 1) c->stat_blocks = 1;
    cudaError_t e = cudaSuccess;
    if ((!c->w_u && (e = cudaMalloc(&c->w_u, 3 * n * sizeof(double))) != cudaSuccess) ||
        (!c->w_v && (e = cudaMalloc(&c->w_v, 3 * n * sizeof(double))) != cudaSuccess) ||
        (!c->w_mp && (e = cudaMalloc(&c->w_mp, nmc * n * sizeof(double))) != cudaSuccess) ||
        (e = cudaMalloc(&c->w_part, (size_t(c->stat_blocks) + 1) * lbk::FR_NQ * sizeof(double))) != cudaSuccess) {
        c->w_part = nullptr;
        return fail(LB_ENOMEM, std::string("work arrays: ") + cudaGetErrorString(e));
    }
    return LB_OK;
}

lb_status ensure_io(lb_ctx* c) {
    if (c->w_io) return LB_OK;
    cudaError_t e = cudaMalloc(&c->w_io, size_t(c->Q) * c->N * sizeof(double));
    if (e != cudaSuccess) return fail(LB_ENOMEM, std::string("staging buffer: ") + cudaGetErrorString(e));
    return LB_OK;
}

lb_status sync_status(lb_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return record(c, e, "cudaStreamSynchronize");
    unsigned st = 0;
    e = cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return record(c, e, "status read");
    if (st) {
        c->sticky = LB_EUNSTABLE;
        return fail(LB_EUNSTABLE, "non-finite or non-positive density");
    }
    return LB_OK;
}

// rho, u (and v for the forcing scheme) of the current state in the work arrays.
lb_status compute_fields(lb_ctx* c, bool need_v) {
    lb_status s = ensure_work(c);
    if (s != LB_OK) return s;
    const lbk::PopPtrs src = pop_ptrs(c, c->cur);
    cudaError_t e = c->ks.moments(src, grid3(c), c->w_rho, c->w_u, c->stream);
    if (e != cudaSuccess) return record(c, e, "moments");
    if (need_v && c->p.scheme == LB_SCHEME_FORCING && c->free_params) {
        e = lbk::free2d_velocity_v(c->fw, c->p.kappa, c->w_rho, c->w_u, c->p.nx, c->p.ny, c->p2_gl, c->p2_mp,
                                   c->w_v, c->stream);
        if (e != cudaSuccess) return record(c, e, "body force");
    } else if (need_v && c->p.scheme == LB_SCHEME_FORCING) {
        e = c->ks.mprime(c->w_rho, grid3(c), c->p.kappa, c->w_mp, c->stream);
        if (e == cudaSuccess) e = c->ks.velocity_v(c->w_rho, c->w_u, c->w_mp, grid3(c), c->w_v, c->stream);
        if (e != cudaSuccess) return record(c, e, "body force");
    } else if (need_v) {
        e = cudaMemcpyAsync(c->w_v, c->w_u, size_t(c->D) * c->N * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream);
        if (e != cudaSuccess) return record(c, e, "copy u");
    }
    return LB_OK;
}

lb_status validate(const lb_params* p) {
    if (!p) return fail(LB_EINVAL, "null parameters");
    if (p->lattice != LB_D2Q9 && p->lattice != LB_D3Q19) return fail(LB_EINVAL, "unknown lattice");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(LB_EINVAL, "grid sizes must be >= 1");
    if (p->lattice == LB_D2Q9 && p->nz != 1) return fail(LB_EINVAL, "D2Q9 needs nz = 1");
    if (double(p->nx) * p->ny * p->nz > 2147483647.0)
        return fail(LB_EINVAL, "lattice too large: the kernels index sites with 32-bit integers (at most 2^31 - 1 sites)");
    if (!(p->tau > 0.5)) return fail(LB_EINVAL, "tau must exceed 1/2");
    if (!(p->kappa > 0)) return fail(LB_EINVAL, "kappa must be positive");
    if (!(p->a > 0 && p->b > 0)) return fail(LB_EINVAL, "a and b must be positive");
    const double Tc = 8.0 * p->a / (27.0 * p->b);
    if (!(p->T > 0 && p->T < Tc)) return fail(LB_EINVAL, "T must lie in (0, 8a/27b)");
    if (p->scheme != LB_SCHEME_EQUILIBRIUM && p->scheme != LB_SCHEME_FORCING) return fail(LB_EINVAL, "unknown scheme");
    if (p->storage < LB_F64 || p->storage > LB_BF16DEV) return fail(LB_EINVAL, "unknown storage");
    if (p->rho_ref < 0 || (p->rho_ref > 0 && p->rho_ref * p->b >= 1.0)) return fail(LB_EINVAL, "rho_ref out of range");
    return LB_OK;
}

// Pressure probes of a drop configuration: inside = the site nearest to the
// first drop's centre; outside = the site farthest (periodic minimum image)
// from every centre, searched on a grid of step ceil(n/64) per axis (every
// site when n <= 64), the first such site in x-fastest order.
void set_drop_probes(lb_ctx* c, int ndrops, const double* centres) {
    const int n[3] = {c->p.nx, c->p.ny, c->p.nz};
    const int D = c->D;
    for (int a = 0; a < 3; ++a) {
        long long v = a < D ? (long long)std::llround(centres[a]) : 0;
        v %= n[a];
        if (v < 0) v += n[a];
        c->probe_in[a] = int(v);
    }
    int step[3], best[3] = {0, 0, 0};
    for (int a = 0; a < 3; ++a) step[a] = std::max(1, (n[a] + 63) / 64);
    double best_d = -1.0;
    for (int z = 0; z < n[2]; z += step[2])
        for (int y = 0; y < n[1]; y += step[1])
            for (int x = 0; x < n[0]; x += step[0]) {
                const int xyz[3] = {x, y, z};
                double dmin = 1e300;
                for (int k = 0; k < ndrops; ++k) {
                    double d2 = 0.0;
                    for (int a = 0; a < D; ++a) {
                        double dd = std::fabs(xyz[a] - centres[k * D + a]);
                        dd = std::fmod(dd, double(n[a]));
                        dd = std::min(dd, n[a] - dd);
                        d2 += dd * dd;
                    }
                    dmin = std::min(dmin, d2);
                }
                if (dmin > best_d) {
                    best_d = dmin;
                    best[0] = x;
                    best[1] = y;
                    best[2] = z;
                }
            }
    for (int a = 0; a < 3; ++a) c->probe_out[a] = best[a];
}

// 64-bit FNV-1a over the bytes of the values that define a context's dynamics
// and its state layout.
struct Fnv {
    unsigned long long h = 1469598103934665603ULL;
    template <class T>
    void add(const T& v) {
        const unsigned char* b = reinterpret_cast<const unsigned char*>(&v);
        for (size_t i = 0; i < sizeof(T); ++i) {
            h ^= b[i];
            h *= 1099511628211ULL;
        }
    }
};

unsigned long long params_hash(const lb_params* p) {
    Fnv f;
    const int ints[6] = {p->lattice, p->nx, p->ny, p->nz, p->scheme, p->storage};
    const double dbl[6] = {p->a, p->b, p->T, p->kappa, p->tau, p->rho_ref};
    for (int v : ints) f.add(v);
    for (double v : dbl) f.add(v);
    return f.h;
}

// Header of an exported state (lb_get_state); the raw population buffer follows it.
struct StateHeader {
    char magic[8];                 // "LBGBSTA1"
    unsigned int version;          // 1
    unsigned int header_bytes;     // sizeof(StateHeader)
    int lattice, nx, ny, nz, scheme, storage, aos, pad;
    long long step;
    unsigned long long params_hash;
    unsigned long long payload_bytes;
};
constexpr char STATE_MAGIC[8] = {'L', 'B', 'G', 'B', 'S', 'T', 'A', '1'};

}  // namespace

// first recorded index violation of each kernel translation unit (bounds.cuh)
unsigned long long lbk_bounds_d3q19();
unsigned long long lbk_bounds_d3pk();
unsigned long long lbk_bounds_d2q9();
unsigned long long lbk_bounds_d2pk();
unsigned long long lbk_bounds_d3pke();
unsigned long long lbk_bounds_batch();

extern "C" {

const char* lb_version(void) { return "lbgb 0.1 (sm_103a)"; }

const char* lb_last_error(void) { return g_last_error.c_str(); }

lb_status lb_coexistence(double a, double b, double T, double* rho_l, double* rho_g) {
    if (!rho_l || !rho_g) return fail(LB_EINVAL, "null output");
    return maxwell(a, b, T, rho_l, rho_g);
}

}  // extern "C"

namespace {

// Bytes of the two population buffers of a context with parameters *p
// (validated): 2 x pitch x (size of f_0 + (Q - 1) x size of f_i).
size_t population_bytes(const lb_params* p) {
    const size_t Q = p->lattice == LB_D2Q9 ? 9 : 19;
    const size_t N = size_t(p->nx) * p->ny * p->nz;
    const size_t pitch = (N + 127) / 128 * 128;
    const size_t elem0 = p->storage == LB_F64 ? 8 : 4;
    const size_t elemi = p->storage == LB_F64 ? 8 : (p->storage == LB_F32 ? 4 : 2);
    return 2 * pitch * (elem0 + (Q - 1) * elemi);
}

lb_status create_impl(const lb_params* p, void* cuda_stream, void* pop_buf, size_t pop_bytes, lb_ctx** out);

}  // namespace

extern "C" {

lb_status lb_population_bytes(const lb_params* p, size_t* bytes) {
    if (!bytes) return fail(LB_EINVAL, "null output");
    lb_status s = validate(p);
    if (s != LB_OK) return s;
    *bytes = population_bytes(p);
    return LB_OK;
}

lb_status lb_create(const lb_params* p, void* cuda_stream, lb_ctx** out) {
    return create_impl(p, cuda_stream, nullptr, 0, out);
}

lb_status lb_create_with_buffers(const lb_params* p, void* cuda_stream, void* populations, size_t bytes,
                                 lb_ctx** out) {
    if (out) *out = nullptr;
    if (!populations) return fail(LB_EINVAL, "null population buffer");
    if (reinterpret_cast<uintptr_t>(populations) % 256 != 0)
        return fail(LB_EINVAL, "population buffer must be 256-byte aligned");
    lb_status s = validate(p);
    if (s != LB_OK) return s;
    if (bytes < population_bytes(p))
        return fail(LB_EINVAL, "population buffer too small: " + std::to_string(bytes) + " < " +
                                   std::to_string(population_bytes(p)) + " bytes (lb_population_bytes)");
    return create_impl(p, cuda_stream, populations, bytes, out);
}

}  // extern "C"

namespace {

lb_status create_impl(const lb_params* p, void* cuda_stream, void* pop_buf, size_t pop_bytes, lb_ctx** out) {
    (void)pop_bytes;
    if (!out) return fail(LB_EINVAL, "null output");
    *out = nullptr;
    lb_status s = validate(p);
    if (s != LB_OK) return s;
    lb_ctx* c = new (std::nothrow) lb_ctx();
    if (!c) return fail(LB_ENOMEM, "host allocation");
    c->p = *p;
    c->D = p->lattice == LB_D2Q9 ? 2 : 3;
    c->Q = p->lattice == LB_D2Q9 ? 9 : 19;
    c->N = size_t(p->nx) * p->ny * p->nz;
    c->pitch = (c->N + 127) / 128 * 128;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    s = maxwell(p->a, p->b, p->T, &c->rho_l, &c->rho_g);
    if (s != LB_OK) { delete c; return s; }
    const double rref = p->rho_ref > 0 ? p->rho_ref : c->rho_l;
    const double pref = p0_vdw(rref, p->a, p->b, p->T);
    for (int i = 0; i < lbk::MAXQ; ++i) c->fref[i] = 0.0f;
    if (p->storage == LB_F16DEV || p->storage == LB_BF16DEV) {
        double wsum = 0.0;
        for (int i = 1; i < c->Q; ++i) {
            const double w = c->D == 2 ? lbk::w_vel<lbk::D2Q9>(i) : lbk::w_vel<lbk::D3Q19>(i);
            c->fref[i] = float(w * pref);
            wsum += w;
        }
        c->pref = float(pref);
        c->rsum = float(pref * wsum);
    }
    const int elem0 = p->storage == LB_F64 ? 8 : 4;
    const int elemi = p->storage == LB_F64 ? 8 : (p->storage == LB_F32 ? 4 : 2);
    c->buf_bytes = c->pitch * (elem0 + size_t(c->Q - 1) * elemi);
    c->ks = c->D == 2 ? lbk_kernels_d2q9(p->scheme, p->storage) : lbk_kernels_d3q19(p->scheme, p->storage, p->nx);
    if (!c->ks.step) { delete c; return fail(LB_EINVAL, "no kernel for this combination"); }
    // two sites per halo load need an even nx; LB_NO_PAIR selects the
    // one-site form (same arithmetic) everywhere, for comparison
    if (c->ks.step_pair_needs_even_nx && (p->nx % 2 != 0 || std::getenv("LB_NO_PAIR"))) {
        c->ks.step = c->ks.step1;
        c->ks.step_fn = c->ks.step1_fn;
        c->ks.tx = c->ks.tx1;
        c->ks.ty = c->ks.ty1;
        c->ks.threads = c->ks.threads1;
        c->ks.smem = c->ks.smem1;
        c->ks.name = c->ks.name1;
        c->ks.aos = false;
    }
    // the interleaved layout holds whole blocks of sites (pitch is a multiple of 128)
    c->aos = c->ks.aos && c->p.storage >= LB_F16DEV && c->pitch % lbk::AOS_SITES == 0;

    cudaError_t e = cudaSuccess;
    if (pop_buf) {
        c->fbuf = static_cast<char*>(pop_buf);
        c->own_fbuf = false;
    } else {
        e = cudaMalloc(&c->fbuf, 2 * c->buf_bytes);
        if (e != cudaSuccess) { delete c; return fail(LB_ENOMEM, std::string("population buffers: ") + cudaGetErrorString(e)); }
    }
    e = cudaMalloc(&c->d_status, sizeof(unsigned));
    if (e != cudaSuccess) {
        if (c->own_fbuf) cudaFree(c->fbuf);
        delete c;
        return fail(LB_ENOMEM, "status word");
    }
    cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);

    // launch geometry of the fused step: one CTA per TX x TY column tile and z chunk;
    // the z chunk is sized so that all CTAs are resident at once where possible.
    int dev = 0, sms = 0, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(c->ks.step_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(c->ks.smem));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, c->ks.step_fn, c->ks.threads, c->ks.smem) !=
            cudaSuccess || occ < 1)
        occ = 1;
    cudaGetLastError();
    const int gx = (p->nx + c->ks.tx - 1) / c->ks.tx;
    const int gy = (p->ny + c->ks.ty - 1) / c->ks.ty;
    c->lz = 1;
    c->grid = dim3(gx, gy, 1);
    if (c->D == 3) {
        const std::vector<int4> work = build_work_list(sms, occ, p->nx, p->ny, p->nz, c->ks.tx, c->ks.ty);
        c->lz = work.front().w - work.front().z;
        if (cudaMalloc(&c->d_work, work.size() * sizeof(int4)) != cudaSuccess ||
            cudaMemcpy(c->d_work, work.data(), work.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess) {
            lb_destroy(c);
            return fail(LB_ENOMEM, "work list");
        }
        c->grid = dim3(unsigned(work.size()), 1, 1);
    }
    c->probe_in[0] = p->nx / 2;
    c->probe_in[1] = p->ny / 2;
    c->probe_in[2] = p->nz / 2;
    *out = c;
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_destroy(lb_ctx* c) {
    if (!c) return LB_OK;
    if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
    if (c->own_fbuf) cudaFree(c->fbuf);
    cudaFree(c->d_status);
    cudaFree(c->w_rho);
    cudaFree(c->w_u);
    cudaFree(c->w_v);
    cudaFree(c->w_mp);
    cudaFree(c->w_part);
    cudaFree(c->w_io);
    cudaFree(c->w_uprev);
    cudaFree(c->d_work);
    cudaFree(c->p2_rho);
    cudaFree(c->p2_gl);
    cudaFree(c->p2_mp);
    for (cudaGraphExec_t g : c->step_graph)
        if (g) cudaGraphExecDestroy(g);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
    return LB_OK;
}

lb_status lb_set_free_params(lb_ctx* c, const lb_free_params* fp) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!fp) {
        c->free_params = false;
        return LB_OK;
    }
    if (c->p.lattice != LB_D2Q9 || c->p.storage != LB_F64)
        return fail(LB_EINVAL, "free parameters need a D2Q9 context with float64 storage");
    const double v[6] = {fp->wp58, fp->wt58, fp->wxx58, fp->B, fp->D, fp->F};
    for (double x : v)
        if (!std::isfinite(x)) return fail(LB_EINVAL, "free parameters must be finite");
    if (!c->p2_rho) {
        cudaError_t e;
        if ((e = cudaMalloc(&c->p2_rho, c->N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&c->p2_gl, 3 * c->N * sizeof(double))) != cudaSuccess ||
            (e = cudaMalloc(&c->p2_mp, 2 * c->N * sizeof(double))) != cudaSuccess)
            return fail(LB_ENOMEM, std::string("free-parameter work arrays: ") + cudaGetErrorString(e));
    }
    c->fw = lbk::free2d_weights(fp->wp58, fp->wt58, fp->wxx58, fp->B, fp->D, fp->F);
    c->free_params = true;
    return LB_OK;
}

lb_status lb_get_coexistence(const lb_ctx* c, double* rho_l, double* rho_g) {
    if (!c || !rho_l || !rho_g) return fail(LB_EINVAL, "null argument");
    *rho_l = c->rho_l;
    *rho_g = c->rho_g;
    return LB_OK;
}

lb_status lb_shape(const lb_ctx* c, long long* n_sites, int* q) {
    if (!c) return fail(LB_EINVAL, "null context");
    if (n_sites) *n_sites = (long long)c->N;
    if (q) *q = c->Q;
    return LB_OK;
}

lb_status lb_kernel_info(const lb_ctx* c, char* name, size_t cap, int* tile_x, int* tile_y, int* threads,
                         size_t* smem, int* ctas) {
    if (!c) return fail(LB_EINVAL, "null context");
    if (name && cap > 0) {
        std::snprintf(name, cap, "%s", c->free_params ? "run-time free parameters (three float64 kernels)"
                                                       : c->ks.name);
    }
    if (tile_x) *tile_x = c->ks.tx;
    if (tile_y) *tile_y = c->ks.ty;
    if (threads) *threads = c->ks.threads;
    if (smem) *smem = c->ks.smem;
    if (ctas) *ctas = int(c->grid.x * c->grid.y * c->grid.z);
    return LB_OK;
}

lb_status lb_device_state(lb_ctx* c, void** dptr, size_t* bytes) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (dptr) *dptr = c->fbuf + size_t(c->cur) * c->buf_bytes;
    if (bytes) *bytes = c->buf_bytes;
    return LB_OK;
}

static lb_status init_from_device_rho(lb_ctx* c, const double* d_rho, const double* d_u) {
    const lbk::PopPtrs dst = pop_ptrs(c, c->cur);
    cudaError_t e = c->free_params
                        ? lbk::free2d_init(c->fw, phys2(c), c->p.scheme == LB_SCHEME_FORCING, pop_base(c, c->cur),
                                           (long long)c->pitch, c->p.nx, c->p.ny, d_rho, d_u, c->p2_gl, c->p2_mp,
                                           c->stream)
                        : c->ks.init_feq(d_rho, d_u, dst, grid3(c), phys(c), c->stream);
    if (e != cudaSuccess) return record(c, e, "init_feq");
    e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return record(c, e, "status reset");
    c->initialised = true;
    c->step = 0;
    c->uprev_valid = false;
    return sync_status(c);
}

lb_status lb_init_drops(lb_ctx* c, int ndrops, const double* centres, const double* radii, double width) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (ndrops < 0 || (ndrops > 0 && (!centres || !radii))) return fail(LB_EINVAL, "bad drop list");
    if (!(width > 0)) return fail(LB_EINVAL, "width must be positive");
    for (int k = 0; k < ndrops; ++k)
        if (!(radii[k] > 0)) return fail(LB_EINVAL, "drop radii must be positive");
    if ((s = ensure_rho(c)) != LB_OK) return s;
    double* d_drops = nullptr;
    const size_t nd = size_t(ndrops) * (c->D + 1);
    cudaError_t e = cudaSuccess;
    if (ndrops > 0) {
        e = cudaMalloc(&d_drops, nd * sizeof(double));
        if (e != cudaSuccess) return fail(LB_ENOMEM, "drop list");
        std::vector<double> h(nd);
        std::memcpy(h.data(), centres, size_t(ndrops) * c->D * sizeof(double));
        std::memcpy(h.data() + size_t(ndrops) * c->D, radii, size_t(ndrops) * sizeof(double));
        e = cudaMemcpyAsync(d_drops, h.data(), nd * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e == cudaSuccess) {
        lbk::drop_density_kernel<<<lbk_aux_blocks(c->N), 256, 0, c->stream>>>(
            c->w_rho, grid3(c), c->D, ndrops, d_drops, d_drops ? d_drops + size_t(ndrops) * c->D : nullptr,
            width, c->rho_l, c->rho_g);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) { cudaFree(d_drops); return record(c, e, "drop density"); }
    if (ndrops > 0) set_drop_probes(c, ndrops, centres);
    s = init_from_device_rho(c, c->w_rho, nullptr);
    cudaFree(d_drops);
    return s;
}

lb_status lb_init_fields(lb_ctx* c, const double* rho, const double* u) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!rho) return fail(LB_EINVAL, "null density");
    if ((s = (u ? ensure_work(c) : ensure_rho(c))) != LB_OK) return s;
    cudaError_t e = cudaMemcpyAsync(c->w_rho, rho, c->N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && u)
        e = cudaMemcpyAsync(c->w_u, u, size_t(c->D) * c->N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return record(c, e, "field upload");
    return init_from_device_rho(c, c->w_rho, u ? c->w_u : nullptr);
}

lb_status lb_set_populations(lb_ctx* c, const double* f) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!f) return fail(LB_EINVAL, "null populations");
    if ((s = ensure_io(c)) != LB_OK) return s;
    cudaError_t e = cudaMemcpyAsync(c->w_io, f, size_t(c->Q) * c->N * sizeof(double), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e == cudaSuccess) e = c->ks.set_pops(pop_ptrs(c, c->cur), c->N, c->w_io, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return record(c, e, "set populations");
    c->initialised = true;
    c->step = 0;
    c->uprev_valid = false;
    return sync_status(c);
}

lb_status lb_get_populations(lb_ctx* c, double* f) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!f) return fail(LB_EINVAL, "null output");
    if (!c->initialised) return fail(LB_ESTATE, "state not initialised");
    if ((s = ensure_io(c)) != LB_OK) return s;
    cudaError_t e = c->ks.get_pops(pop_ptrs(c, c->cur), c->N, c->w_io, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(f, c->w_io, size_t(c->Q) * c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return record(c, e, "get populations");
    return sync_status(c);
}

lb_status lb_work_list(int sms, int ctas_per_sm, int nx, int ny, int nz, int tile_x, int tile_y, int* out,
                       int capacity, int* count) {
    if (!count) return fail(LB_EINVAL, "null count");
    if (sms < 1 || ctas_per_sm < 1 || nx < 1 || ny < 1 || nz < 1 || tile_x < 1 || tile_y < 1 ||
        (long long)nx * ny * nz > 0x7fffffffLL)
        return fail(LB_EINVAL, "sizes must be positive (at most 2^31 - 1 sites)");
    const std::vector<int4> w = build_work_list(sms, ctas_per_sm, nx, ny, nz, tile_x, tile_y);
    if (w.size() > size_t(0x7fffffff)) return fail(LB_EINVAL, "work list too long");
    *count = int(w.size());
    if (out)
        for (size_t k = 0; k < w.size() && k < size_t(std::max(capacity, 0)); ++k) {
            out[4 * k] = w[k].x;
            out[4 * k + 1] = w[k].y;
            out[4 * k + 2] = w[k].z;
            out[4 * k + 3] = w[k].w;
        }
    return LB_OK;
}

lb_status lb_get_populations_box(lb_ctx* c, int x0, int y0, int z0, int bx, int by, int bz, double* f) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!f) return fail(LB_EINVAL, "null output");
    if (bx < 1 || by < 1 || bz < 1 || bx > c->p.nx || by > c->p.ny || bz > c->p.nz)
        return fail(LB_EINVAL, "box sizes must be in [1, lattice size]");
    if (x0 < 0 || y0 < 0 || z0 < 0 || x0 >= c->p.nx || y0 >= c->p.ny || z0 >= c->p.nz)
        return fail(LB_EINVAL, "box origin must lie in the lattice");
    const size_t n = size_t(bx) * by * bz;
    if (n > (size_t(1) << LB_BOX_MAX_LOG2_SITES)) return fail(LB_EINVAL, "box larger than LB_BOX_MAX_LOG2_SITES");
    if (!c->initialised) return fail(LB_ESTATE, "state not initialised");
    double* d = nullptr;
    const size_t bytes = size_t(c->Q) * n * sizeof(double);
    cudaError_t e = cudaMalloc(&d, bytes);
    if (e != cudaSuccess) return fail(LB_ENOMEM, std::string("box staging: ") + cudaGetErrorString(e));
    const int o[3] = {x0, y0, z0}, b[3] = {bx, by, bz};
    e = c->ks.get_box(pop_ptrs(c, c->cur), grid3(c), o, b, d, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return record(c, e, "get population box");
    return sync_status(c);
}

lb_status lb_step(lb_ctx* c, int nsteps) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (nsteps < 0) return fail(LB_EINVAL, "nsteps must be >= 0");
    if (!c->initialised) return fail(LB_ESTATE, "step before init");
    lbk::StepArgs a{};
    a.nx = c->p.nx;
    a.ny = c->p.ny;
    a.nz = c->p.nz;
    a.lz = c->lz;
    a.work = c->d_work;
    a.pair2d = (c->D == 2 && c->p.nx % 2 == 0 && !std::getenv("LB_NO_PAIR")) ? 1 : 0;
    a.a = c->p.a;
    a.b = c->p.b;
    a.T = c->p.T;
    a.kappa = c->p.kappa;
    a.omega = 1.0 / c->p.tau;
    a.nu = (c->p.tau - 0.5) / 3.0;
    a.fa = float(a.a);
    a.fb = float(a.b);
    a.fT = float(a.T);
    a.fkappa = float(a.kappa);
    a.fomega = float(a.omega);
    a.fnu = float(a.nu);
    a.status = c->d_status;
    for (int i = 0; i < lbk::MAXQ; ++i) a.fref[i] = c->fref[i];
    a.pref = c->pref;
    a.rsum = c->rsum;
    // one fused step from buffer `cur` into the other, on stream st
    auto launch_one = [&](int cur, cudaStream_t st) -> cudaError_t {
        for (int i = 0; i < c->Q; ++i) {
            a.src[i] = c->fbuf + pop_offset(c, i, cur);
            a.dst[i] = c->fbuf + pop_offset(c, i, 1 - cur);
        }
        a.src_base = a.src[0];
        a.dst_base = a.dst[0];
        a.pitch = (long long)c->pitch;
        return c->free_params
                   ? lbk::free2d_step(c->fw, phys2(c), c->p.scheme == LB_SCHEME_FORCING, pop_base(c, cur),
                                      pop_base(c, 1 - cur), (long long)c->pitch, c->p.nx, c->p.ny, c->p2_rho,
                                      c->p2_gl, c->p2_mp, c->d_status, st)
                   : c->ks.step(a, c->grid, st);
    };
    int k = 0;
    // long runs: replay a captured graph of GRAPH_STEPS steps (an even count, so a
    // replay ends in the buffer it started from).  The graph is captured after one
    // ordinary launch (which sets the kernel's attributes) and kept for the
    // context's lifetime: the buffers, work list and parameters it holds are fixed.
    // If the capture fails the steps run as ordinary launches (the same kernels).
    if (!c->free_params && !c->graph_failed && nsteps > GRAPH_STEPS) {
        if (!c->step_graph[c->cur]) {
            cudaError_t e = launch_one(c->cur, c->stream);
            if (e != cudaSuccess) return record(c, e, "step kernel");
            c->cur = 1 - c->cur;
            ++c->step;
            ++k;
            if (!c->step_graph[c->cur]) {
                cudaGraphExec_t exec = nullptr;
                if (capture_steps(c, launch_one, &exec) == cudaSuccess) {
                    c->step_graph[c->cur] = exec;
                } else {
                    cudaGetLastError();
                    c->graph_failed = true;
                }
            }
        }
        cudaGraphExec_t g = c->step_graph[c->cur];
        for (; g && k + GRAPH_STEPS <= nsteps; k += GRAPH_STEPS) {
            cudaError_t e = cudaGraphLaunch(g, c->stream);
            if (e != cudaSuccess) return record(c, e, "step graph launch");
            c->step += GRAPH_STEPS;
        }
    }
    for (; k < nsteps; ++k) {
        cudaError_t e = launch_one(c->cur, c->stream);
        if (e != cudaSuccess) return record(c, e, "step kernel");
        c->cur = 1 - c->cur;
        ++c->step;
    }
    return LB_OK;
}

lb_status lb_synchronize(lb_ctx* c) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    return sync_status(c);
}

lb_status lb_fields(lb_ctx* c, double* rho, double* u, double* v) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!c->initialised) return fail(LB_ESTATE, "state not initialised");
    if ((s = compute_fields(c, v != nullptr)) != LB_OK) return s;
    cudaError_t e = cudaSuccess;
    const size_t dn = size_t(c->D) * c->N * sizeof(double);
    if (rho) e = cudaMemcpyAsync(rho, c->w_rho, c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, c->w_u, dn, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && v) e = cudaMemcpyAsync(v, c->w_v, dn, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return record(c, e, "field download");
    return sync_status(c);
}

lb_status lb_stats_get(lb_ctx* c, lb_stats* out) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!out) return fail(LB_EINVAL, "null output");
    if (!c->initialised) return fail(LB_ESTATE, "state not initialised");
    if ((s = compute_fields(c, true)) != LB_OK) return s;
    const size_t du = size_t(c->D) * c->N;
    if (!c->w_uprev) {
        cudaError_t e = cudaMalloc(&c->w_uprev, du * sizeof(double));
        if (e != cudaSuccess) {
            c->w_uprev = nullptr;
            return fail(LB_ENOMEM, std::string("previous velocity field: ") + cudaGetErrorString(e));
        }
        c->uprev_valid = false;
    }
    double* part = c->w_part;
    double* res = c->w_part + size_t(c->stat_blocks) * lbk::FR_NQ;
    lbk::fr_partial_kernel<lbk::FR_NQ><<<c->stat_blocks, lbk::FR_THREADS, 0, c->stream>>>(
        c->w_rho, c->w_u, c->w_v, c->uprev_valid ? c->w_uprev : nullptr, c->D, (long long)c->N, 0, part);
    lbk::fr_final_kernel<lbk::FR_NQ><<<1, lbk::FR_THREADS, 0, c->stream>>>(part, c->stat_blocks, res);
    double h[lbk::FR_NQ], rp[2];
    const size_t in = (size_t(c->probe_in[2]) * c->p.ny + c->probe_in[1]) * c->p.nx + c->probe_in[0];
    const size_t ou = (size_t(c->probe_out[2]) * c->p.ny + c->probe_out[1]) * c->p.nx + c->probe_out[0];
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, res, sizeof(h), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rp[0], c->w_rho + in, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rp[1], c->w_rho + ou, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    // this state's velocity becomes the reference of the next call's max_du
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->w_uprev, c->w_u, du * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return record(c, e, "stats");
    s = sync_status(c);
    std::memset(out, 0, sizeof(*out));
    out->mass = h[0];
    out->momentum[0] = h[1];
    out->momentum[1] = h[2];
    out->momentum[2] = h[3];
    out->max_u = h[4];
    out->max_v = h[5];
    out->min_rho = h[6];
    out->max_rho = h[7];
    out->step = c->step;
    out->status = int(c->sticky);
    out->dP = p0_vdw(rp[0], c->p.a, c->p.b, c->p.T) - p0_vdw(rp[1], c->p.a, c->p.b, c->p.T);
    out->max_du = c->uprev_valid ? h[8] : -1.0;
    out->du_steps = c->uprev_valid ? c->step - c->uprev_step : 0;
    c->uprev_valid = true;
    c->uprev_step = c->step;
    return s;
}

lb_status lb_set_probes(lb_ctx* c, const int* inside, const int* outside) {
    if (!c) return fail(LB_EINVAL, "null context");
    if (!inside || !outside) return fail(LB_EINVAL, "null probe");
    const int n[3] = {c->p.nx, c->p.ny, c->p.nz};
    for (int a = 0; a < 3; ++a)
        if (inside[a] < 0 || inside[a] >= n[a] || outside[a] < 0 || outside[a] >= n[a])
            return fail(LB_EINVAL, "probe sites must lie in the lattice");
    for (int a = 0; a < 3; ++a) {
        c->probe_in[a] = inside[a];
        c->probe_out[a] = outside[a];
    }
    return LB_OK;
}

lb_status lb_get_probes(const lb_ctx* c, int* inside, int* outside) {
    if (!c || !inside || !outside) return fail(LB_EINVAL, "null argument");
    for (int a = 0; a < 3; ++a) {
        inside[a] = c->probe_in[a];
        outside[a] = c->probe_out[a];
    }
    return LB_OK;
}

lb_status lb_debug_bounds(int* checked, unsigned long long* violation) {
    if (checked) *checked = lbk::kBoundsChecked ? 1 : 0;
    unsigned long long v = 0;
    for (unsigned long long w : {lbk_bounds_d3pk(), lbk_bounds_d3pke(), lbk_bounds_d3q19(), lbk_bounds_d2q9(), lbk_bounds_d2pk(),
                                 lbk_bounds_batch()})
        if (!v) v = w;
    if (violation) *violation = v;
    return LB_OK;
}

lb_status lb_params_hash(const lb_params* p, unsigned long long* hash) {
    if (!p || !hash) return fail(LB_EINVAL, "null argument");
    lb_status s = validate(p);
    if (s != LB_OK) return s;
    *hash = params_hash(p);
    return LB_OK;
}

lb_status lb_get_state(lb_ctx* c, void* buf, size_t* bytes) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!bytes) return fail(LB_EINVAL, "null size");
    const size_t need = sizeof(StateHeader) + c->buf_bytes;
    if (!buf) {
        *bytes = need;
        return LB_OK;
    }
    if (!c->initialised) return fail(LB_ESTATE, "state not initialised");
    if (*bytes < need) return fail(LB_EINVAL, "buffer smaller than the state (" + std::to_string(need) + " bytes)");
    if ((s = sync_status(c)) != LB_OK) return s;
    StateHeader h{};
    std::memcpy(h.magic, STATE_MAGIC, 8);
    h.version = 1;
    h.header_bytes = sizeof(StateHeader);
    h.lattice = c->p.lattice;
    h.nx = c->p.nx;
    h.ny = c->p.ny;
    h.nz = c->p.nz;
    h.scheme = c->p.scheme;
    h.storage = c->p.storage;
    h.aos = c->aos ? 1 : 0;
    h.step = c->step;
    h.params_hash = params_hash(&c->p);
    h.payload_bytes = c->buf_bytes;
    std::memcpy(buf, &h, sizeof(h));
    cudaError_t e = cudaMemcpyAsync(static_cast<char*>(buf) + sizeof(h), c->fbuf + size_t(c->cur) * c->buf_bytes,
                                    c->buf_bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return record(c, e, "state export");
    *bytes = need;
    return LB_OK;
}

lb_status lb_set_state(lb_ctx* c, const void* buf, size_t bytes) {
    lb_status s = check_ctx(c);
    if (s != LB_OK) return s;
    if (!buf) return fail(LB_EINVAL, "null state");
    if (bytes < sizeof(StateHeader)) return fail(LB_EINVAL, "state shorter than its header");
    StateHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, STATE_MAGIC, 8) != 0 || h.version != 1 || h.header_bytes != sizeof(StateHeader))
        return fail(LB_EINVAL, "not a state exported by lb_get_state (magic, version or header size)");
    if (h.lattice != c->p.lattice || h.nx != c->p.nx || h.ny != c->p.ny || h.nz != c->p.nz ||
        h.scheme != c->p.scheme || h.storage != c->p.storage || h.aos != (c->aos ? 1 : 0))
        return fail(LB_EINVAL, "state of another lattice, scheme, storage or layout");
    if (h.params_hash != params_hash(&c->p))
        return fail(LB_EINVAL, "state exported with other physical parameters (parameter hash differs)");
    if (h.payload_bytes != c->buf_bytes || bytes != sizeof(StateHeader) + c->buf_bytes)
        return fail(LB_EINVAL, "state size does not match the context");
    if (h.step < 0) return fail(LB_EINVAL, "negative step counter");
    cudaError_t e = cudaMemcpyAsync(c->fbuf + size_t(c->cur) * c->buf_bytes, static_cast<const char*>(buf) + sizeof(h),
                                    c->buf_bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream);
    if (e != cudaSuccess) return record(c, e, "state import");
    c->initialised = true;
    c->step = h.step;
    c->uprev_valid = false;
    return sync_status(c);
}

}  // extern "C"
