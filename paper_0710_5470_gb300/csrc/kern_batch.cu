// Batched D2Q9 sweeps: kernel instantiations and the lb_batch_* C ABI.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "batch.cuh"
#include "dispatch.h"

void lb_internal_set_error(const char* msg);

using namespace lbk;

namespace {

lb_status fail(lb_status s, const std::string& m) {
    lb_internal_set_error(m.c_str());
    return s;
}

// ------------------------------------------------------------ kernel table
struct BatchKernels {
    int tx = 0, ty = 0;
    int threads = 0, check_threads = 0;   // per CTA of the step and of the check kernel
    size_t smem = 0;
    const void* step_fn = nullptr;
    const void* check_fn = nullptr;
    void (*step)(const BatchState&, char*, int, int nblocks, cudaStream_t) = nullptr;
    void (*check)(const BatchState&, const char*, int, int nblocks, cudaStream_t) = nullptr;
    cudaError_t (*init_feq)(const double*, const double*, const PopPtrs&, Grid3, Phys, cudaStream_t) = nullptr;
    cudaError_t (*moments)(const PopPtrs&, Grid3, double*, double*, cudaStream_t) = nullptr;
    cudaError_t (*get_pops)(const PopPtrs&, size_t, double*, cudaStream_t) = nullptr;
};

template <bool F, class S, int TX, int TY>
struct BatchLaunch {
    using Lay = StepLayout<D2Q9, F, TX, TY, typename S::real>;
    static void step(const BatchState& bs, char* buf, int parity, int nblocks, cudaStream_t st) {
        batch_step_kernel<F, S, TX, TY><<<nblocks, TX * TY, Lay::BYTES, st>>>(bs, buf, parity);
    }
    static void check(const BatchState& bs, const char* buf, int parity, int nblocks, cudaStream_t st) {
        batch_check_kernel<S, TX, TY><<<nblocks, TX * TY, 0, st>>>(bs, buf, parity);
    }
    static cudaError_t init_feq(const double* rho, const double* u, const PopPtrs& p, Grid3 g, Phys ph,
                                cudaStream_t st) {
        const size_t n = size_t(g.nx) * g.ny * g.nz;
        init_feq_kernel<D2Q9, F, S><<<lbk_aux_blocks(n), 256, 0, st>>>(rho, u, p, g, ph);
        return cudaGetLastError();
    }
    static cudaError_t moments(const PopPtrs& p, Grid3 g, double* rho, double* u, cudaStream_t st) {
        const size_t n = size_t(g.nx) * g.ny * g.nz;
        moments_kernel<D2Q9, S><<<lbk_aux_blocks(n), 256, 0, st>>>(p, g, rho, u);
        return cudaGetLastError();
    }
    static cudaError_t get_pops(const PopPtrs& p, size_t n, double* out, cudaStream_t st) {
        get_pops_kernel<D2Q9, S><<<lbk_aux_blocks(n), 256, 0, st>>>(p, n, out);
        return cudaGetLastError();
    }
    static BatchKernels make() {
        BatchKernels k;
        k.tx = TX;
        k.ty = TY;
        k.threads = k.check_threads = TX * TY;
        k.smem = Lay::BYTES;
        k.step_fn = reinterpret_cast<const void*>(batch_step_kernel<F, S, TX, TY>);
        k.check_fn = reinterpret_cast<const void*>(batch_check_kernel<S, TX, TY>);
        k.step = &step;
        k.check = &check;
        k.init_feq = &init_feq;
        k.moments = &moments;
        k.get_pops = &get_pops;
        return k;
    }
};

// The pair kernel (32-bit arithmetic) on the same tiles: (TX / 2) * TY threads.
template <bool F, class S, int TX, int TY>
struct BatchLaunchPK : BatchLaunch<F, S, TX, TY> {
    using Lay = Layout2PK<F, TX, TY>;
    static void step(const BatchState& bs, char* buf, int parity, int nblocks, cudaStream_t st) {
        batch_step_kernel_pk<F, S, TX, TY><<<nblocks, Lay::NTH, Lay::BYTES, st>>>(bs, buf, parity);
    }
    static BatchKernels make() {
        BatchKernels k = BatchLaunch<F, S, TX, TY>::make();
        k.threads = Lay::NTH;
        k.smem = Lay::BYTES;
        k.step_fn = reinterpret_cast<const void*>(batch_step_kernel_pk<F, S, TX, TY>);
        k.step = &step;
        return k;
    }
};

constexpr int NTILES = 3;   // tile variants tried by the autotuner: 32x8, 32x16, 64x8

// Float64 runs the one-site tile kernel; 32-bit arithmetic the pair kernel
// (LB_D2_VARIANT=0: the tile kernel, for comparisons).
template <bool F, class S>
BatchKernels pick_tile(int t) {
    if constexpr (sizeof(typename S::real) == 4) {
        const char* env = std::getenv("LB_D2_VARIANT");
        if (!(env && std::atoi(env) == 0)) {
            switch (t) {
                case 0: return BatchLaunchPK<F, S, 32, 8>::make();
                case 1: return BatchLaunchPK<F, S, 32, 16>::make();
                default: return BatchLaunchPK<F, S, 64, 8>::make();
            }
        }
    }
    switch (t) {
        case 0: return BatchLaunch<F, S, 32, 8>::make();
        case 1: return BatchLaunch<F, S, 32, 16>::make();
        default: return BatchLaunch<F, S, 64, 8>::make();
    }
}

BatchKernels batch_kernels(int scheme, int storage, int tile) {
    const bool f = scheme == LB_SCHEME_FORCING;
    switch (storage) {
        case LB_F64: return f ? pick_tile<true, StF64>(tile) : pick_tile<false, StF64>(tile);
        case LB_F32: return f ? pick_tile<true, StF32>(tile) : pick_tile<false, StF32>(tile);
        case LB_F16DEV: return f ? pick_tile<true, StF16>(tile) : pick_tile<false, StF16>(tile);
        default: return f ? pick_tile<true, StBF16>(tile) : pick_tile<false, StBF16>(tile);
    }
}

int elem0(int storage) { return storage == LB_F64 ? 8 : 4; }
int elemi(int storage) { return storage == LB_F64 ? 8 : (storage == LB_F32 ? 4 : 2); }

}  // namespace

struct lb_batch {
    int scheme = 0, storage = 0, n = 0;
    double a = 0, b = 0;
    std::vector<lb_instance> inst;
    std::vector<BatchInst> di;        // host copy of the device table
    std::vector<double> rho_l, rho_g;
    std::vector<double> pref64;   // per instance: p0(rho_l) in float64 (fref_i = w_i pref, rounded once)
    long long sites = 0, max_sites = 0;
    size_t state_bytes = 0;           // bytes of one state (all instances, one buffer)
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int tile = 0;
    bool tuned = false;
    BatchKernels k;
    int max_items = 0;
    // launch sizes of the step and check kernels: the CTAs resident at once (at most max_items)
    int step_grid = 1, check_grid = 1;
    long long gstep = 0;              // host copy of the step counter
    int parity = 0;
    // device
    char* buf = nullptr;              // states: [instance][buffer][populations]
    BatchInst* d_inst = nullptr;
    unsigned* d_items = nullptr;
    int* d_count = nullptr;
    int* d_active = nullptr;
    unsigned* d_status = nullptr;
    unsigned long long* d_maxdu = nullptr;
    unsigned long long* d_maxu = nullptr;
    unsigned long long* d_maxrho = nullptr;
    unsigned long long* d_minrho = nullptr;
    double* d_last = nullptr;
    double* d_ref = nullptr;          // per instance: reference max |u|, max rho, min rho
    int* d_inband = nullptr;
    double band = 0.05, tol_rho = 1e-3;
    int hold = 10;
    double self_rtol = 0.0, self_tol_rho = 0.0;   // lb_batch_set_self_test (0: off)
    int self_hold = 10;
    long long* d_steps = nullptr;
    long long* d_gstep = nullptr;
    double* d_uprev = nullptr;
    double* w_rho = nullptr;          // scratch of the largest instance
    double* w_u = nullptr;
    double* w_io = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_every = 0;
    double graph_tol = 0;
    long long graph_min = 0;
    int graph_tile = -1;
    double graph_band = -1, graph_tol_rho = -1;
    int graph_hold = -1;
    double graph_self_rtol = -1, graph_self_tol_rho = -1;
    int graph_self_hold = -1;
};

namespace {

BatchState state_of(lb_batch* B) {
    return BatchState{B->d_inst,   B->d_items,  B->d_count,  B->d_active, B->d_status, B->d_maxdu,
                      B->d_maxu,   B->d_maxrho, B->d_minrho, B->d_last,   B->d_ref,    B->d_inband,
                      B->d_steps,  B->d_gstep,  B->d_uprev,  B->n};
}

PopPtrs pops_of(lb_batch* B, int k, int parity) {
    PopPtrs p{};
    const BatchInst& I = B->di[k];
    char* base = B->buf + I.off[parity];
    const double pref = B->pref64[k];
    for (int i = 0; i < 9; ++i) {
        const long long o = i == 0 ? 0 : I.pitch * elem0(B->storage) + (i - 1) * I.pitch * elemi(B->storage);
        p.p[i] = base + o;
        p.fref[i] = (B->storage == LB_F16DEV || B->storage == LB_BF16DEV) && i > 0 ? float(w_vel<D2Q9>(i) * pref) : 0.f;
    }
    return p;
}

lb_status cuda_err(cudaError_t e, const char* where) {
    return fail(LB_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Tile table of the current tile variant, and the full work list (all instances active).
lb_status set_tile(lb_batch* B, int tile) {
    B->tile = tile;
    B->k = batch_kernels(B->scheme, B->storage, tile);
    cudaFuncSetAttribute(B->k.step_fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(B->k.smem));
    {
        int dev = 0, sms = 1, occ = 1, occ_c = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, B->k.step_fn, B->k.threads, B->k.smem) != cudaSuccess ||
            occ < 1)
            occ = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, B->k.check_fn, B->k.check_threads, 0) != cudaSuccess ||
            occ_c < 1)
            occ_c = 1;
        cudaGetLastError();
        B->step_grid = std::max(1, std::min(B->max_items, std::max(sms, 1) * occ));
        B->check_grid = std::max(1, std::min(B->max_items, std::max(sms, 1) * occ_c));
    }
    std::vector<unsigned> items;
    for (int k = 0; k < B->n; ++k) {
        BatchInst& I = B->di[k];
        I.tiles_x = (I.nx + B->k.tx - 1) / B->k.tx;
        I.tiles_y = (I.ny + B->k.ty - 1) / B->k.ty;
        for (int t = 0; t < I.tiles_x * I.tiles_y; ++t) items.push_back((unsigned(k) << 20) | unsigned(t));
    }
    if (int(items.size()) > B->max_items) return fail(LB_EINVAL, "work list larger than allocated");
    cudaError_t e = cudaMemcpyAsync(B->d_inst, B->di.data(), B->di.size() * sizeof(BatchInst),
                                    cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_items, items.data(), items.size() * sizeof(unsigned), cudaMemcpyHostToDevice,
                            B->stream);
    int cnt = int(items.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(B->d_count, &cnt, sizeof(int), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch work list");
    if (B->graph) {
        cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
    }
    return LB_OK;
}

lb_status reset_run_state(lb_batch* B) {
    std::vector<int> ones(B->n, 1);
    std::vector<long long> minus(B->n, -1);
    cudaError_t e = cudaMemcpyAsync(B->d_active, ones.data(), B->n * sizeof(int), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_status, 0, B->n * sizeof(unsigned), B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_maxdu, 0, B->n * sizeof(unsigned long long), B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_maxu, 0, B->n * sizeof(unsigned long long), B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_maxrho, 0, B->n * sizeof(unsigned long long), B->stream);
    const double big = 1e300;
    std::vector<double> bigs(B->n, big);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_minrho, bigs.data(), B->n * sizeof(double), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_last, 0, B->n * 4 * sizeof(double), B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_inband, 0, B->n * sizeof(int), B->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->d_steps, minus.data(), B->n * sizeof(long long), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_gstep, 0, sizeof(long long), B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_uprev, 0, size_t(B->sites) * 2 * sizeof(double), B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch reset");
    B->gstep = 0;
    B->parity = 0;
    return set_tile(B, B->tile);
}

lb_status launch_steps(lb_batch* B, int nsteps) {
    const BatchState bs = state_of(B);
    for (int s = 0; s < nsteps; ++s) {
        B->k.step(bs, B->buf, B->parity, B->step_grid, B->stream);
        B->parity ^= 1;
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? LB_OK : cuda_err(e, "batch step");
}

}  // namespace

extern "C" {

lb_status lb_batch_create(int scheme, int storage, double a, double b, int n, const lb_instance* inst,
                          void* cuda_stream, lb_batch** out) {
    if (!out) return fail(LB_EINVAL, "null output");
    *out = nullptr;
    if (n < 1 || n > 4096 || !inst) return fail(LB_EINVAL, "need 1..4096 instances");
    if (scheme != LB_SCHEME_EQUILIBRIUM && scheme != LB_SCHEME_FORCING) return fail(LB_EINVAL, "unknown scheme");
    if (storage < LB_F64 || storage > LB_BF16DEV) return fail(LB_EINVAL, "unknown storage");
    lb_batch* B = new (std::nothrow) lb_batch();
    if (!B) return fail(LB_ENOMEM, "host allocation");
    B->scheme = scheme;
    B->storage = storage;
    B->a = a;
    B->b = b;
    B->n = n;
    B->inst.assign(inst, inst + n);
    B->di.resize(n);
    B->rho_l.resize(n);
    B->pref64.assign(n, 0.0);
    B->rho_g.resize(n);
    long long off = 0;
    long long max_items = 0;
    for (int k = 0; k < n; ++k) {
        const lb_instance& in = inst[k];
        // a work item holds the tile index in 20 bits: at most 2^20 tiles of the smallest variant (32 x 8)
        if (in.nx < 1 || in.ny < 1 || double((in.nx + 31) / 32) * ((in.ny + 7) / 8) > double(1 << 20)) {
            delete B;
            return fail(LB_EINVAL, "bad instance size (1 <= nx, ny; at most 2^20 tiles of 32 x 8)");
        }
        if (!(in.tau > 0.5) || !(in.kappa > 0)) { delete B; return fail(LB_EINVAL, "bad instance tau/kappa"); }
        lb_status s = lb_coexistence(a, b, in.T, &B->rho_l[k], &B->rho_g[k]);
        if (s != LB_OK) { delete B; return s; }
        BatchInst& I = B->di[k];
        const long long N = (long long)in.nx * in.ny;
        I.pitch = (N + 127) / 128 * 128;
        const long long bytes = I.pitch * (elem0(storage) + 8LL * elemi(storage));
        I.off[0] = off;
        I.off[1] = off + bytes;
        off += 2 * bytes;
        I.site0 = B->sites;
        B->sites += N;
        B->max_sites = std::max(B->max_sites, N);
        I.nx = in.nx;
        I.ny = in.ny;
        I.pair = (in.nx % 2 == 0 && !std::getenv("LB_NO_PAIR")) ? 1 : 0;
        I.a = a;
        I.b = b;
        I.T = in.T;
        I.kappa = in.kappa;
        I.omega = 1.0 / in.tau;
        I.nu = (in.tau - 0.5) / 3.0;
        I.fa = float(I.a);
        I.fb = float(I.b);
        I.fT = float(I.T);
        I.fkappa = float(I.kappa);
        I.fomega = float(I.omega);
        I.fnu = float(I.nu);
        const double rl = B->rho_l[k];
        const double pref = (storage == LB_F16DEV || storage == LB_BF16DEV) ? rl * in.T / (1 - b * rl) - a * rl * rl : 0.0;
        // sum_{i>=1} w_i (5/3 on D2Q9), summed in velocity order like a single
        // context does, so that the float32 rsum is the same bit for bit
        double wsum = 0.0;
        for (int i = 1; i < D2Q9::Q; ++i) wsum += w_vel<D2Q9>(i);
        B->pref64[k] = pref;
        I.pref = float(pref);
        I.rsum = float(pref * wsum);
        int most = 0;   // largest tile count over the tile variants (smallest tile: 32x8)
        most = int(((in.nx + 31) / 32) * ((in.ny + 7) / 8));
        max_items += most;
    }
    if (max_items > 0x7fffffffLL) { delete B; return fail(LB_EINVAL, "batch too large"); }
    B->max_items = int(max_items);
    B->state_bytes = size_t(off);
    if (cuda_stream) {
        B->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking);
        B->own_stream = true;
    }
    cudaError_t e;
    if ((e = cudaMalloc(&B->buf, B->state_bytes)) != cudaSuccess ||
        (e = cudaMalloc(&B->d_inst, n * sizeof(BatchInst))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_items, size_t(max_items) * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_count, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_active, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_status, n * sizeof(unsigned))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_maxdu, n * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_maxu, n * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_maxrho, n * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_minrho, n * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_last, n * 4 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_ref, n * 3 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_inband, n * sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_steps, n * sizeof(long long))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_gstep, sizeof(long long))) != cudaSuccess ||
        (e = cudaMalloc(&B->d_uprev, size_t(B->sites) * 2 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&B->w_rho, size_t(B->max_sites) * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&B->w_u, size_t(B->max_sites) * 2 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&B->w_io, size_t(B->max_sites) * 9 * sizeof(double))) != cudaSuccess) {
        lb_batch_destroy(B);
        return fail(LB_ENOMEM, std::string("batch buffers: ") + cudaGetErrorString(e));
    }
    if ((e = cudaMemsetAsync(B->d_ref, 0, n * 3 * sizeof(double), B->stream)) != cudaSuccess) {
        lb_batch_destroy(B);
        return cuda_err(e, "batch targets");
    }
    lb_status s = reset_run_state(B);
    if (s != LB_OK) { lb_batch_destroy(B); return s; }
    *out = B;
    return LB_OK;
}

lb_status lb_batch_destroy(lb_batch* B) {
    if (!B) return LB_OK;
    if (B->stream) cudaStreamSynchronize(B->stream);
    if (B->graph) cudaGraphExecDestroy(B->graph);
    cudaFree(B->buf);
    cudaFree(B->d_inst);
    cudaFree(B->d_items);
    cudaFree(B->d_count);
    cudaFree(B->d_active);
    cudaFree(B->d_status);
    cudaFree(B->d_maxdu);
    cudaFree(B->d_maxu);
    cudaFree(B->d_maxrho);
    cudaFree(B->d_minrho);
    cudaFree(B->d_last);
    cudaFree(B->d_ref);
    cudaFree(B->d_inband);
    cudaFree(B->d_steps);
    cudaFree(B->d_gstep);
    cudaFree(B->d_uprev);
    cudaFree(B->w_rho);
    cudaFree(B->w_u);
    cudaFree(B->w_io);
    if (B->own_stream) cudaStreamDestroy(B->stream);
    delete B;
    return LB_OK;
}

lb_status lb_batch_init_drops(lb_batch* B, double width) {
    if (!B) return fail(LB_EINVAL, "null batch");
    if (!(width > 0)) return fail(LB_EINVAL, "width must be positive");
    for (int k = 0; k < B->n; ++k) {
        const BatchInst& I = B->di[k];
        const Grid3 g{I.nx, I.ny, 1};
        const double c[2] = {I.nx / 2.0, I.ny / 2.0};
        const double r = B->inst[k].radius;
        double* d_c = B->w_u;            // centre and radius staged in the velocity scratch
        double h[3] = {c[0], c[1], r};
        cudaError_t e = cudaMemcpyAsync(d_c, h, sizeof(h), cudaMemcpyHostToDevice, B->stream);
        if (e != cudaSuccess) return cuda_err(e, "drop upload");
        drop_density_kernel<<<lbk_aux_blocks(size_t(I.nx) * I.ny), 256, 0, B->stream>>>(
            B->w_rho, g, 2, r > 0 ? 1 : 0, d_c, d_c + 2, width, B->rho_l[k], B->rho_g[k]);
        const Phys ph{B->a, B->b, I.T, I.kappa, I.nu};
        e = B->k.init_feq(B->w_rho, nullptr, pops_of(B, k, 0), g, ph, B->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
        if (e != cudaSuccess) return cuda_err(e, "batch init");
    }
    return reset_run_state(B);
}

lb_status lb_batch_init_fields(lb_batch* B, int k, const double* rho, const double* u) {
    if (!B || k < 0 || k >= B->n || !rho) return fail(LB_EINVAL, "bad arguments");
    const BatchInst& I = B->di[k];
    const size_t N = size_t(I.nx) * I.ny;
    cudaError_t e = cudaMemcpyAsync(B->w_rho, rho, N * sizeof(double), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(B->w_u, u, 2 * N * sizeof(double), cudaMemcpyHostToDevice, B->stream);
    if (e != cudaSuccess) return cuda_err(e, "field upload");
    const Phys ph{B->a, B->b, I.T, I.kappa, I.nu};
    e = B->k.init_feq(B->w_rho, u ? B->w_u : nullptr, pops_of(B, k, B->parity), Grid3{I.nx, I.ny, 1}, ph, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    return e == cudaSuccess ? LB_OK : cuda_err(e, "batch init fields");
}

lb_status lb_batch_step(lb_batch* B, int nsteps) {
    if (!B || nsteps < 0) return fail(LB_EINVAL, "bad arguments");
    lb_status s = launch_steps(B, nsteps);
    if (s != LB_OK) return s;
    B->gstep += nsteps;
    return LB_OK;
}

lb_status lb_batch_autotune(lb_batch* B, int steps, int* tile_x, int* tile_y) {
    if (!B || steps < 1) return fail(LB_EINVAL, "bad arguments");
    // time every tile variant on a copy of the state, keep the fastest, restore the state
    char* backup = nullptr;
    cudaError_t e = cudaMalloc(&backup, B->state_bytes);
    if (e != cudaSuccess) return fail(LB_ENOMEM, "autotune backup");
    e = cudaMemcpyAsync(backup, B->buf, B->state_bytes, cudaMemcpyDeviceToDevice, B->stream);
    const int parity0 = B->parity;
    float best = 1e30f;
    int best_t = B->tile;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int t = 0; t < NTILES && e == cudaSuccess; ++t) {
        lb_status s = set_tile(B, t);
        if (s != LB_OK) { cudaFree(backup); return s; }
        launch_steps(B, 2);
        cudaEventRecord(e0, B->stream);
        launch_steps(B, steps);
        cudaEventRecord(e1, B->stream);
        e = cudaEventSynchronize(e1);
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_t = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(B->buf, backup, B->state_bytes, cudaMemcpyDeviceToDevice, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    cudaFree(backup);
    if (e != cudaSuccess) return cuda_err(e, "autotune");
    B->parity = parity0;
    B->tuned = true;
    lb_status s = set_tile(B, best_t);
    if (s != LB_OK) return s;
    e = cudaMemsetAsync(B->d_status, 0, B->n * sizeof(unsigned), B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (tile_x) *tile_x = B->k.tx;
    if (tile_y) *tile_y = B->k.ty;
    return e == cudaSuccess ? LB_OK : cuda_err(e, "autotune");
}

lb_status lb_batch_run_to_steady(lb_batch* B, double tol, int every, long long min_steps, long long max_steps,
                                 long long* steps_out, int* status_out, long long* total_steps) {
    if (!B || every < 2 || (every & 1) || max_steps < every || !(tol > 0))
        return fail(LB_EINVAL, "need tol > 0, an even check interval >= 2 and max_steps >= it");
    if (B->parity != 0) {
        lb_status s = launch_steps(B, 1);   // align the buffers with the even-step graph
        if (s != LB_OK) return s;
        B->gstep += 1;
    }
    // one graph: `every` steps, the convergence check, retirement and work-list rebuild
    if (!B->graph || B->graph_every != every || B->graph_tol != tol || B->graph_min != min_steps ||
        B->graph_tile != B->tile || B->graph_band != B->band || B->graph_hold != B->hold ||
        B->graph_tol_rho != B->tol_rho || B->graph_self_rtol != B->self_rtol ||
        B->graph_self_tol_rho != B->self_tol_rho || B->graph_self_hold != B->self_hold) {
        if (B->graph) cudaGraphExecDestroy(B->graph);
        B->graph = nullptr;
        cudaGraph_t g;
        cudaError_t e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_err(e, "begin capture");
        const BatchState bs = state_of(B);
        for (int s = 0; s < every; ++s) B->k.step(bs, B->buf, s & 1, B->step_grid, B->stream);
        B->k.check(bs, B->buf, 0, B->check_grid, B->stream);
        batch_finalize_kernel<<<1, 1024, 0, B->stream>>>(bs, tol, every, min_steps, B->band, B->tol_rho, B->hold,
                                                         B->self_rtol, B->self_tol_rho, B->self_hold);
        e = cudaStreamEndCapture(B->stream, &g);
        if (e != cudaSuccess) return cuda_err(e, "end capture");
        e = cudaGraphInstantiate(&B->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_err(e, "graph instantiate");
        B->graph_every = every;
        B->graph_tol = tol;
        B->graph_min = min_steps;
        B->graph_tile = B->tile;
        B->graph_band = B->band;
        B->graph_tol_rho = B->tol_rho;
        B->graph_hold = B->hold;
        B->graph_self_rtol = B->self_rtol;
        B->graph_self_tol_rho = B->self_tol_rho;
        B->graph_self_hold = B->self_hold;
    }
    // the device step counter continues from the host one
    cudaError_t e = cudaMemcpyAsync(B->d_gstep, &B->gstep, sizeof(long long), cudaMemcpyHostToDevice, B->stream);
    if (e != cudaSuccess) return cuda_err(e, "step counter");
    long long done = 0;
    int count = 1;
    while (done < max_steps && count > 0) {
        e = cudaGraphLaunch(B->graph, B->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&count, B->d_count, sizeof(int), cudaMemcpyDeviceToHost, B->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
        if (e != cudaSuccess) return cuda_err(e, "batch run");
        done += every;
        B->gstep += every;
    }
    std::vector<long long> st(B->n);
    std::vector<unsigned> stat(B->n);
    e = cudaMemcpy(st.data(), B->d_steps, B->n * sizeof(long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(stat.data(), B->d_status, B->n * sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "batch results");
    for (int k = 0; k < B->n; ++k) {
        if (steps_out) steps_out[k] = st[k];
        if (status_out) status_out[k] = stat[k] ? LB_EUNSTABLE : (st[k] < 0 ? LB_ETIMEOUT : LB_OK);
    }
    if (total_steps) *total_steps = done;
    return LB_OK;
}

lb_status lb_batch_set_reference(lb_batch* B, int k, double umax_ref, double rho_max_ref, double rho_min_ref) {
    if (!B || k < 0 || k >= B->n) return fail(LB_EINVAL, "bad arguments");
    if (!(umax_ref >= 0.0) || !std::isfinite(umax_ref) || !std::isfinite(rho_max_ref) || !std::isfinite(rho_min_ref))
        return fail(LB_EINVAL, "references must be finite, umax_ref >= 0");
    const double r[3] = {umax_ref, rho_max_ref, rho_min_ref};
    cudaError_t e = cudaMemcpyAsync(B->d_ref + 3 * k, r, sizeof(r), cudaMemcpyHostToDevice, B->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_inband + k, 0, sizeof(int), B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch reference");
    return LB_OK;
}

lb_status lb_batch_set_band(lb_batch* B, double band, double tol_rho, int hold) {
    if (!B || !(band >= 0.0) || !(tol_rho >= 0.0) || hold < 1)
        return fail(LB_EINVAL, "need band >= 0, tol_rho >= 0 and hold >= 1");
    B->band = band;
    B->tol_rho = tol_rho;
    B->hold = hold;
    return LB_OK;
}

lb_status lb_batch_set_self_test(lb_batch* B, double rtol_u, double tol_rho, int hold) {
    if (!B || !(rtol_u >= 0.0) || !(tol_rho >= 0.0) || hold < 1 || !std::isfinite(rtol_u) || !std::isfinite(tol_rho))
        return fail(LB_EINVAL, "need finite rtol_u >= 0, tol_rho >= 0 and hold >= 1");
    B->self_rtol = rtol_u;
    B->self_tol_rho = tol_rho;
    B->self_hold = hold;
    cudaError_t e = cudaMemsetAsync(B->d_inband, 0, B->n * sizeof(int), B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch self test");
    return LB_OK;
}

lb_status lb_batch_last_check(lb_batch* B, double* du, double* umax, double* rho_max, double* rho_min) {
    if (!B) return fail(LB_EINVAL, "null batch");
    std::vector<double> last(size_t(B->n) * 4);
    cudaError_t e = cudaMemcpyAsync(last.data(), B->d_last, last.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                    B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e != cudaSuccess) return cuda_err(e, "batch last check");
    for (int k = 0; k < B->n; ++k) {
        if (du) du[k] = last[4 * k];
        if (umax) umax[k] = last[4 * k + 1];
        if (rho_max) rho_max[k] = last[4 * k + 2];
        if (rho_min) rho_min[k] = last[4 * k + 3];
    }
    return LB_OK;
}

lb_status lb_batch_fields(lb_batch* B, int k, double* rho, double* u) {
    if (!B || k < 0 || k >= B->n) return fail(LB_EINVAL, "bad arguments");
    const BatchInst& I = B->di[k];
    const size_t N = size_t(I.nx) * I.ny;
    // a retired instance keeps the buffer it was in when it stopped: even step counts end in buffer 0
    long long sd = 0;
    cudaError_t e = cudaMemcpy(&sd, B->d_steps + k, sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "steps");
    const int par = sd >= 0 ? 0 : B->parity;
    e = B->k.moments(pops_of(B, k, par), Grid3{I.nx, I.ny, 1}, B->w_rho, B->w_u, B->stream);
    if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho, B->w_rho, N * sizeof(double), cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, B->w_u, 2 * N * sizeof(double), cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    return e == cudaSuccess ? LB_OK : cuda_err(e, "batch fields");
}

lb_status lb_batch_populations(lb_batch* B, int k, double* f) {
    if (!B || k < 0 || k >= B->n || !f) return fail(LB_EINVAL, "bad arguments");
    const BatchInst& I = B->di[k];
    const size_t N = size_t(I.nx) * I.ny;
    long long sd = 0;
    cudaError_t e = cudaMemcpy(&sd, B->d_steps + k, sizeof(long long), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e, "steps");
    const int par = sd >= 0 ? 0 : B->parity;
    e = B->k.get_pops(pops_of(B, k, par), N, B->w_io, B->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(f, B->w_io, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, B->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    return e == cudaSuccess ? LB_OK : cuda_err(e, "batch populations");
}

lb_status lb_batch_info(const lb_batch* B, int* tile_x, int* tile_y, long long* sites, long long* steps) {
    if (!B) return fail(LB_EINVAL, "null batch");
    if (tile_x) *tile_x = B->k.tx;
    if (tile_y) *tile_y = B->k.ty;
    if (sites) *sites = B->sites;
    if (steps) *steps = B->gstep;
    return LB_OK;
}

}  // extern "C"

// First recorded index violation of this unit's kernels (checked builds; see bounds.cuh).
LB_BOUNDS_READER(lbk_bounds_batch)
