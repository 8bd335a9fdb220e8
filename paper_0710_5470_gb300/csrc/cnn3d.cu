// Warm-start network for D3Q19 drops: 4 layers of periodic 3x3x3 convolutions
// (5 -> 32 -> 32 -> 32 -> 4 channels, tanh between layers), trained and
// evaluated on the GPU by the kernels below.  Activations are float32
// [sample][channel][z][y][x]; the convolutions read fp16 copies of the
// weights (float32 accumulation); Adam updates float32 master weights.
//
// Inputs (5 volumes): normalised tanh-start density, T, kappa, tau, 10/R.
// Outputs (4 volumes): (rho_steady - rho_tanh) / (rho_l - rho_g), 1000 u_x, 1000 u_y, 1000 u_z.
//
// Each CTA computes a 16 x 16 (y, x) tile of one z plane for all output
// channels; the three z taps are taken in turn, each from a shared-memory
// tile of one input plane and the weight slice of that tap.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lb.h"
#include "cnn_common.cuh"

void lb_internal_set_error(const char* msg);

namespace {

constexpr int TILE = 16;
constexpr int TP = TILE + 2;             // tile with its periodic halo
constexpr int NL = 4;
constexpr int CH[NL + 1] = {LB_WS_IN, LB_WS_HIDDEN, LB_WS_HIDDEN, LB_WS_HIDDEN, LB_WS3_OUT};

lb_status fail(lb_status s, const std::string& m) {
    lb_internal_set_error(m.c_str());
    return s;
}

// Loads plane z of `a` (C channels, volume D x H x Wd, sample n) around the
// tile at (y0, x0) with a one-site periodic halo into t[C][TP][TP].
__device__ __forceinline__ void load_plane(const float* a, int C, int n, int z, int D, int H, int Wd, int y0, int x0,
                                           float* t) {
    for (int i = threadIdx.x; i < C * TP * TP; i += blockDim.x) {
        const int c = i / (TP * TP), r = i % (TP * TP);
        const int ty = r / TP, tx = r % TP;
        t[i] = a[(((size_t(n) * C + c) * D + z) * H + wrap(y0 + ty - 1, H)) * Wd + wrap(x0 + tx - 1, Wd)];
    }
}

// out[n,o,z,y,x] = act(b[o] + sum_{c,dz,dy,dx} W[o,c,dz+1,dy+1,dx+1] in[n,c,z+dz,y+dy,x+dx]), periodic.
template <int CIN, int COUT, bool TANH>
__global__ void __launch_bounds__(TILE* TILE) conv3_fwd(const float* in, const __half* W, const float* bias,
                                                        float* out, int D, int H, int Wd) {
    extern __shared__ float sm[];
    float* tile = sm;                   // [CIN][TP][TP]
    float* wsh = sm + CIN * TP * TP;    // [CIN][9][COUT] for one z tap
    const int n = blockIdx.z / D, z = blockIdx.z % D;
    const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
    for (int kz = 0; kz < 3; ++kz) {
        __syncthreads();
        load_plane(in, CIN, n, wrap(z + kz - 1, D), D, H, Wd, y0, x0, tile);
        for (int i = threadIdx.x; i < COUT * CIN * 9; i += blockDim.x) {
            const int o = i / (CIN * 9), r = i % (CIN * 9);          // r = c * 9 + ky * 3 + kx
            wsh[r * COUT + o] = __half2float(W[(size_t(o) * CIN + r / 9) * 27 + kz * 9 + r % 9]);
        }
        __syncthreads();
        for (int c = 0; c < CIN; ++c) {
            float v[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] = tile[(c * TP + ly + k / 3) * TP + lx + k % 3];
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const float* w = wsh + (c * 9 + k) * COUT;
#pragma unroll
                for (int o = 0; o < COUT; ++o) acc[o] += w[o] * v[k];
            }
        }
    }
    const int x = x0 + lx, y = y0 + ly;
    if (x < Wd && y < H) {
#pragma unroll
        for (int o = 0; o < COUT; ++o)
            out[(((size_t(n) * COUT + o) * D + z) * H + y) * Wd + x] = TANH ? tanhf(acc[o]) : acc[o];
    }
}

// din[n,c,z,y,x] = (sum_{o,dz,dy,dx} W[o,c,dz+1,dy+1,dx+1] dout[n,o,z-dz,y-dy,x-dx]) * (1 - h^2 if h).
template <int CIN, int COUT>
__global__ void __launch_bounds__(TILE* TILE) conv3_bwd_data(const float* dout, const __half* W, const float* h,
                                                             float* din, int D, int H, int Wd) {
    extern __shared__ float sm[];
    float* tile = sm;                    // [COUT][TP][TP] of dout
    float* wsh = sm + COUT * TP * TP;    // [COUT][9][CIN] for one z tap
    const int n = blockIdx.z / D, z = blockIdx.z % D;
    const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
    const int lx = threadIdx.x % TILE, ly = threadIdx.x / TILE;
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
    for (int kz = 0; kz < 3; ++kz) {
        __syncthreads();
        load_plane(dout, COUT, n, wrap(z - (kz - 1), D), D, H, Wd, y0, x0, tile);
        for (int i = threadIdx.x; i < COUT * CIN * 9; i += blockDim.x) {
            const int o = i / (CIN * 9), r = i % (CIN * 9);
            const int c = r / 9, k = r % 9;
            wsh[(o * 9 + k) * CIN + c] = __half2float(W[(size_t(o) * CIN + c) * 27 + kz * 9 + k]);
        }
        __syncthreads();
        for (int o = 0; o < COUT; ++o) {
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int dy = k / 3 - 1, dx = k % 3 - 1;
                const float g = tile[(o * TP + ly - dy + 1) * TP + lx - dx + 1];
                const float* w = wsh + (o * 9 + k) * CIN;
#pragma unroll
                for (int c = 0; c < CIN; ++c) acc[c] += w[c] * g;
            }
        }
    }
    const int x = x0 + lx, y = y0 + ly;
    if (x < Wd && y < H) {
#pragma unroll
        for (int c = 0; c < CIN; ++c) {
            const size_t idx = (((size_t(n) * CIN + c) * D + z) * H + y) * Wd + x;
            float v = acc[c];
            if (h) v *= 1.f - h[idx] * h[idx];
            din[idx] = v;
        }
    }
}

// dW[o,c,k] += sum over voxels of dout[o,p] h[c,p+k]; db[o] += sum dout[o,p].  One thread per
// (c, tap) pair; each CTA sweeps many (sample, z, 16 x 16) tiles and adds its partial sums once.
template <int CIN>
constexpr int bwd3_threads() {
    return CIN * 27 > TILE * TILE ? (CIN * 27 + 31) / 32 * 32 : TILE * TILE;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(bwd3_threads<CIN>()) conv3_bwd_weight(const float* h, const float* dout, float* dW,
                                                                         float* db, int N, int D, int H, int Wd) {
    extern __shared__ float sm[];
    float* tile = sm;                         // [3][CIN][TP][TP] of h (planes z-1, z, z+1)
    float* gt = sm + 3 * CIN * TP * TP;       // [COUT][TILE*TILE] of dout
    const int tid = threadIdx.x;
    const int tiles_x = (Wd + TILE - 1) / TILE, tiles_y = (H + TILE - 1) / TILE;
    const int per = tiles_x * tiles_y;
    const int ntiles = N * D * per;
    constexpr int NPAIR = CIN * 27;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
    float bacc = 0.f;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int nz = t / per, r0 = t % per;
        const int n = nz / D, z = nz % D;
        const int x0 = (r0 % tiles_x) * TILE, y0 = (r0 / tiles_x) * TILE;
        __syncthreads();
        for (int kz = 0; kz < 3; ++kz)
            load_plane(h, CIN, n, wrap(z + kz - 1, D), D, H, Wd, y0, x0, tile + kz * CIN * TP * TP);
        for (int i = tid; i < COUT * TILE * TILE; i += blockDim.x) {
            const int o = i / (TILE * TILE), p = i % (TILE * TILE);
            const int x = x0 + p % TILE, y = y0 + p / TILE;
            gt[i] = (x < Wd && y < H) ? dout[(((size_t(n) * COUT + o) * D + z) * H + y) * Wd + x] : 0.f;
        }
        __syncthreads();
        if (tid < NPAIR) {
            const int c = tid / 27, k = tid % 27;
            const int kz = k / 9, ky = (k / 3) % 3, kx = k % 3;
            const float* tc = tile + (kz * CIN + c) * TP * TP;
            for (int p = 0; p < TILE * TILE; ++p) {
                const float v = tc[(p / TILE + ky) * TP + p % TILE + kx];
#pragma unroll
                for (int o = 0; o < COUT; ++o) acc[o] += gt[o * TILE * TILE + p] * v;
            }
        }
        if (tid < COUT)
            for (int p = 0; p < TILE * TILE; ++p) bacc += gt[tid * TILE * TILE + p];
    }
    if (tid < NPAIR) {
        const int c = tid / 27, k = tid % 27;
#pragma unroll
        for (int o = 0; o < COUT; ++o) atomicAdd(dW + (size_t(o) * CIN + c) * 27 + k, acc[o]);
    }
    if (tid < COUT) atomicAdd(db + tid, bacc);
}

size_t smem_fwd3(int cin, int cout) { return size_t(cin * TP * TP + cin * 9 * cout) * 4; }
size_t smem_bwd3_w(int cin, int cout) { return size_t(3 * cin * TP * TP + cout * TILE * TILE) * 4; }

}  // namespace

struct lb_ws3 {
    int nparams = 0;
    int woff[NL], boff[NL];
    float* p = nullptr;
    __half* p16 = nullptr;
    float* g = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    double* loss = nullptr;
    int adam_t = 0;
    float* act[NL + 1] = {};
    float* dact[NL + 1] = {};
    size_t cap = 0;                 // voxels x batch capacity of the activation buffers
    cudaStream_t st = nullptr;
};

namespace {

lb_status ensure_acts3(lb_ws3* w, size_t vox) {
    if (vox <= w->cap) return LB_OK;
    for (int l = 0; l <= NL; ++l) {
        cudaFree(w->act[l]);
        cudaFree(w->dact[l]);
        w->act[l] = w->dact[l] = nullptr;
    }
    w->cap = 0;
    for (int l = 0; l <= NL; ++l) {
        if (cudaMalloc(&w->act[l], vox * CH[l] * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&w->dact[l], vox * CH[l] * sizeof(float)) != cudaSuccess)
            return fail(LB_ENOMEM, "3D warm-start activations");
    }
    w->cap = vox;
    return LB_OK;
}

template <int CIN, int COUT, bool T>
void launch_fwd3(const float* in, const __half* W, const float* b, float* out, int n, int D, int H, int Wd,
                 cudaStream_t st) {
    const size_t sm = smem_fwd3(CIN, COUT);
    cudaFuncSetAttribute(conv3_fwd<CIN, COUT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    dim3 grid((Wd + TILE - 1) / TILE, (H + TILE - 1) / TILE, n * D);
    conv3_fwd<CIN, COUT, T><<<grid, TILE * TILE, sm, st>>>(in, W, b, out, D, H, Wd);
}

template <int CIN, int COUT>
void launch_bwd3(lb_ws3* w, int l, int n, int D, int H, int Wd) {
    const size_t smw = smem_bwd3_w(CIN, COUT);
    cudaFuncSetAttribute(conv3_bwd_weight<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smw));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = n * D * ((Wd + TILE - 1) / TILE) * ((H + TILE - 1) / TILE);
    const int blocks = ntiles < 2 * sms ? ntiles : 2 * sms;
    conv3_bwd_weight<CIN, COUT><<<blocks, bwd3_threads<CIN>(), smw, w->st>>>(
        w->act[l], w->dact[l + 1], w->g + w->woff[l], w->g + w->boff[l], n, D, H, Wd);
    if (l > 0) {
        const size_t smd = smem_fwd3(COUT, CIN);
        cudaFuncSetAttribute(conv3_bwd_data<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smd));
        dim3 grid((Wd + TILE - 1) / TILE, (H + TILE - 1) / TILE, n * D);
        conv3_bwd_data<CIN, COUT><<<grid, TILE * TILE, smd, w->st>>>(w->dact[l + 1], w->p16 + w->woff[l], w->act[l],
                                                                     w->dact[l], D, H, Wd);
    }
}

cudaError_t forward3(lb_ws3* w, int n, int D, int H, int Wd) {
    launch_fwd3<LB_WS_IN, LB_WS_HIDDEN, true>(w->act[0], w->p16 + w->woff[0], w->p + w->boff[0], w->act[1], n, D, H, Wd, w->st);
    launch_fwd3<LB_WS_HIDDEN, LB_WS_HIDDEN, true>(w->act[1], w->p16 + w->woff[1], w->p + w->boff[1], w->act[2], n, D, H, Wd, w->st);
    launch_fwd3<LB_WS_HIDDEN, LB_WS_HIDDEN, true>(w->act[2], w->p16 + w->woff[2], w->p + w->boff[2], w->act[3], n, D, H, Wd, w->st);
    launch_fwd3<LB_WS_HIDDEN, LB_WS3_OUT, false>(w->act[3], w->p16 + w->woff[3], w->p + w->boff[3], w->act[4], n, D, H, Wd, w->st);
    return cudaGetLastError();
}

lb_status loss_grad3(lb_ws3* w, const float* t, int n, int D, int H, int Wd, double* loss_out) {
    forward3(w, n, D, H, Wd);
    cudaMemsetAsync(w->g, 0, size_t(w->nparams) * sizeof(float), w->st);
    cudaMemsetAsync(w->loss, 0, sizeof(double), w->st);
    const size_t nout = size_t(n) * LB_WS3_OUT * D * H * Wd;
    mse_grad<<<256, 256, 0, w->st>>>(w->act[4], t, w->dact[4], nout, w->loss);
    launch_bwd3<LB_WS_HIDDEN, LB_WS3_OUT>(w, 3, n, D, H, Wd);
    launch_bwd3<LB_WS_HIDDEN, LB_WS_HIDDEN>(w, 2, n, D, H, Wd);
    launch_bwd3<LB_WS_HIDDEN, LB_WS_HIDDEN>(w, 1, n, D, H, Wd);
    launch_bwd3<LB_WS_IN, LB_WS_HIDDEN>(w, 0, n, D, H, Wd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("3D warm-start backward: ") + cudaGetErrorString(e));
    if (loss_out) {
        e = cudaMemcpyAsync(loss_out, w->loss, sizeof(double), cudaMemcpyDeviceToHost, w->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
        if (e != cudaSuccess) return fail(LB_ECUDA, std::string("3D warm-start loss: ") + cudaGetErrorString(e));
    }
    return LB_OK;
}

// (sample, z plane) is the grid's z dimension: at most 65535 per launch.
bool dims_ok(int n, int D, int H, int Wd) {
    return n >= 1 && D >= 1 && H >= 1 && Wd >= 1 && (long long)n * D <= 65535;
}

}  // namespace

extern "C" {

lb_status lb_ws3_create(int seed, void* cuda_stream, lb_ws3** out) {
    if (!out) return fail(LB_EINVAL, "null output");
    lb_ws3* w = new (std::nothrow) lb_ws3();
    if (!w) return fail(LB_ENOMEM, "host allocation");
    w->st = static_cast<cudaStream_t>(cuda_stream);
    int off = 0;
    for (int l = 0; l < NL; ++l) {
        w->woff[l] = off;
        off += CH[l + 1] * CH[l] * 27;
        w->boff[l] = off;
        off += CH[l + 1];
    }
    w->nparams = off;
    // W ~ U(-s, s), s = 1/sqrt(27 C_in), from a SplitMix64 stream; b = 0
    std::vector<float> h(off, 0.f);
    unsigned long long st = (unsigned long long)seed;
    for (int l = 0; l < NL; ++l) {
        const double s = 1.0 / std::sqrt(27.0 * CH[l]);
        for (int i = 0; i < CH[l + 1] * CH[l] * 27; ++i) h[w->woff[l] + i] = float((2.0 * splitmix_u01(st) - 1.0) * s);
    }
    cudaError_t e;
    if ((e = cudaMalloc(&w->p, off * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&w->p16, off * sizeof(__half))) != cudaSuccess ||
        (e = cudaMalloc(&w->g, off * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&w->m, off * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&w->v, off * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&w->loss, sizeof(double))) != cudaSuccess) {
        lb_ws3_destroy(w);
        return fail(LB_ENOMEM, std::string("3D warm-start parameters: ") + cudaGetErrorString(e));
    }
    lb_status s = lb_ws3_set_params(w, h.data(), size_t(off));
    if (s != LB_OK) {
        lb_ws3_destroy(w);
        return s;
    }
    *out = w;
    return LB_OK;
}

lb_status lb_ws3_destroy(lb_ws3* w) {
    if (!w) return LB_OK;
    cudaStreamSynchronize(w->st);
    cudaFree(w->p);
    cudaFree(w->p16);
    cudaFree(w->g);
    cudaFree(w->m);
    cudaFree(w->v);
    cudaFree(w->loss);
    for (int l = 0; l <= NL; ++l) {
        cudaFree(w->act[l]);
        cudaFree(w->dact[l]);
    }
    delete w;
    return LB_OK;
}

lb_status lb_ws3_num_params(const lb_ws3* w, long long* n) {
    if (!w || !n) return fail(LB_EINVAL, "null argument");
    *n = w->nparams;
    return LB_OK;
}

lb_status lb_ws3_set_params(lb_ws3* w, const float* params, size_t count) {
    if (!w || !params || count != size_t(w->nparams)) return fail(LB_EINVAL, "parameter count mismatch");
    cudaError_t e = cudaMemcpyAsync(w->p, params, count * sizeof(float), cudaMemcpyHostToDevice, w->st);
    if (e == cudaSuccess) {
        to_half<<<64, 256, 0, w->st>>>(w->p, w->p16, int(count));
        e = cudaMemsetAsync(w->m, 0, count * sizeof(float), w->st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(w->v, 0, count * sizeof(float), w->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
    w->adam_t = 0;
    return e == cudaSuccess ? LB_OK : fail(LB_ECUDA, std::string("set params: ") + cudaGetErrorString(e));
}

lb_status lb_ws3_get_params(lb_ws3* w, float* params, size_t count) {
    if (!w || !params || count != size_t(w->nparams)) return fail(LB_EINVAL, "parameter count mismatch");
    cudaError_t e = cudaMemcpyAsync(params, w->p, count * sizeof(float), cudaMemcpyDeviceToHost, w->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
    return e == cudaSuccess ? LB_OK : fail(LB_ECUDA, std::string("get params: ") + cudaGetErrorString(e));
}

lb_status lb_ws3_forward(lb_ws3* w, const float* x, int n, int D, int H, int Wd, float* y) {
    if (!w || !x || !y || !dims_ok(n, D, H, Wd)) return fail(LB_EINVAL, "bad arguments");
    const size_t vox = size_t(n) * D * H * Wd;
    lb_status s = ensure_acts3(w, vox);
    if (s != LB_OK) return s;
    cudaError_t e = cudaMemcpyAsync(w->act[0], x, vox * LB_WS_IN * sizeof(float), cudaMemcpyHostToDevice, w->st);
    if (e != cudaSuccess) return fail(LB_ECUDA, "upload");
    if ((e = forward3(w, n, D, H, Wd)) != cudaSuccess)
        return fail(LB_ECUDA, std::string("3D warm-start forward launch: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(y, w->act[4], vox * LB_WS3_OUT * sizeof(float), cudaMemcpyDeviceToHost, w->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
    return e == cudaSuccess ? LB_OK : fail(LB_ECUDA, std::string("3D warm-start forward: ") + cudaGetErrorString(e));
}

lb_status lb_ws3_loss_grad(lb_ws3* w, const float* x, const float* t, int n, int D, int H, int Wd, double* loss,
                           float* grads) {
    if (!w || !x || !t || !dims_ok(n, D, H, Wd)) return fail(LB_EINVAL, "bad arguments");
    const size_t vox = size_t(n) * D * H * Wd;
    lb_status s = ensure_acts3(w, vox);
    if (s != LB_OK) return s;
    float* dt = nullptr;
    if (cudaMalloc(&dt, vox * LB_WS3_OUT * sizeof(float)) != cudaSuccess) return fail(LB_ENOMEM, "targets");
    cudaMemcpyAsync(w->act[0], x, vox * LB_WS_IN * sizeof(float), cudaMemcpyHostToDevice, w->st);
    cudaMemcpyAsync(dt, t, vox * LB_WS3_OUT * sizeof(float), cudaMemcpyHostToDevice, w->st);
    s = loss_grad3(w, dt, n, D, H, Wd, loss);
    if (s == LB_OK && grads) {
        cudaError_t e = cudaMemcpyAsync(grads, w->g, size_t(w->nparams) * sizeof(float), cudaMemcpyDeviceToHost, w->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
        if (e != cudaSuccess) s = fail(LB_ECUDA, "gradient download");
    }
    cudaFree(dt);
    return s;
}

lb_status lb_ws3_train(lb_ws3* w, const float* x, const float* t, int n, int D, int H, int Wd, int epochs, int batch,
                       float lr, int seed, double* loss_history) {
    if (!w || !x || !t || n < 1 || !dims_ok(1, D, H, Wd) || epochs < 1 || batch < 1)
        return fail(LB_EINVAL, "bad arguments");
    batch = batch < n ? batch : n;
    if (!dims_ok(batch, D, H, Wd)) return fail(LB_EINVAL, "batch * depth larger than 65535");
    const size_t vol = size_t(D) * H * Wd;
    lb_status s = ensure_acts3(w, size_t(batch) * vol);
    if (s != LB_OK) return s;
    float *dx = nullptr, *dt = nullptr, *bt = nullptr;
    if (cudaMalloc(&dx, size_t(n) * vol * LB_WS_IN * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dt, size_t(n) * vol * LB_WS3_OUT * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&bt, size_t(batch) * vol * LB_WS3_OUT * sizeof(float)) != cudaSuccess) {
        cudaFree(dx);
        cudaFree(dt);
        return fail(LB_ENOMEM, "training data");
    }
    cudaMemcpyAsync(dx, x, size_t(n) * vol * LB_WS_IN * sizeof(float), cudaMemcpyHostToDevice, w->st);
    cudaMemcpyAsync(dt, t, size_t(n) * vol * LB_WS3_OUT * sizeof(float), cudaMemcpyHostToDevice, w->st);
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    unsigned long long rs = (unsigned long long)seed * 0x9E3779B97F4A7C15ull + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < epochs && s == LB_OK; ++ep) {
        for (int i = n - 1; i > 0; --i) {   // shuffle (xorshift)
            rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17;
            std::swap(order[i], order[int(rs % (unsigned long long)(i + 1))]);
        }
        double ep_loss = 0.0;
        int nb = 0;
        for (int b0 = 0; b0 + batch <= n && s == LB_OK; b0 += batch, ++nb) {
            for (int k = 0; k < batch; ++k) {
                const int j = order[b0 + k];
                cudaMemcpyAsync(w->act[0] + size_t(k) * vol * LB_WS_IN, dx + size_t(j) * vol * LB_WS_IN,
                                vol * LB_WS_IN * sizeof(float), cudaMemcpyDeviceToDevice, w->st);
                cudaMemcpyAsync(bt + size_t(k) * vol * LB_WS3_OUT, dt + size_t(j) * vol * LB_WS3_OUT,
                                vol * LB_WS3_OUT * sizeof(float), cudaMemcpyDeviceToDevice, w->st);
            }
            double l = 0.0;
            s = loss_grad3(w, bt, batch, D, H, Wd, &l);
            ep_loss += l;
            ++w->adam_t;
            const float c1 = 1.f - std::pow(b1, float(w->adam_t)), c2 = 1.f - std::pow(b2, float(w->adam_t));
            adam_update<<<128, 256, 0, w->st>>>(w->p, w->p16, w->g, w->m, w->v, w->nparams, lr, b1, b2, eps, c1, c2);
        }
        if (loss_history) loss_history[ep] = nb ? ep_loss / nb : 0.0;
    }
    cudaError_t e = cudaStreamSynchronize(w->st);
    cudaFree(dx);
    cudaFree(dt);
    cudaFree(bt);
    if (s == LB_OK && e != cudaSuccess) s = fail(LB_ECUDA, std::string("3D training: ") + cudaGetErrorString(e));
    return s;
}

lb_status lb_ws3_predict_sym(lb_ws3* w, const float* x, int D, int H, int Wd, float* y) {
    if (!w || !x || !y || !dims_ok(1, D, H, Wd)) return fail(LB_EINVAL, "bad arguments");
    // the eight reflections a -> (n_a - a) mod n_a of the axes fix the point (W/2, H/2, D/2);
    // a reflected velocity component changes sign
    constexpr int NG = 8;
    const size_t N = size_t(D) * H * Wd;
    std::vector<float> xs(size_t(NG) * LB_WS_IN * N), ys(size_t(NG) * LB_WS3_OUT * N);
    std::vector<size_t> perm(N);
    std::fill(y, y + size_t(LB_WS3_OUT) * N, 0.f);
    auto build_perm = [&](int g) {
        const int fx = g & 1, fy = (g >> 1) & 1, fz = (g >> 2) & 1;
        for (int zz = 0; zz < D; ++zz)
            for (int yy = 0; yy < H; ++yy)
                for (int xx = 0; xx < Wd; ++xx) {
                    const int sx = fx ? (Wd - xx) % Wd : xx, sy = fy ? (H - yy) % H : yy, sz = fz ? (D - zz) % D : zz;
                    perm[(size_t(zz) * H + yy) * Wd + xx] = (size_t(sz) * H + sy) * Wd + sx;
                }
    };
    for (int g = 0; g < NG; ++g) {
        build_perm(g);
        for (int c = 0; c < LB_WS_IN; ++c)
            for (size_t p = 0; p < N; ++p) xs[(size_t(g) * LB_WS_IN + c) * N + p] = x[size_t(c) * N + perm[p]];
    }
    lb_status st = lb_ws3_forward(w, xs.data(), NG, D, H, Wd, ys.data());
    if (st != LB_OK) return st;
    for (int g = 0; g < NG; ++g) {
        build_perm(g);
        const float sgn[3] = {(g & 1) ? -1.f : 1.f, ((g >> 1) & 1) ? -1.f : 1.f, ((g >> 2) & 1) ? -1.f : 1.f};
        const float* yg = ys.data() + size_t(g) * LB_WS3_OUT * N;
        for (size_t p = 0; p < N; ++p) {
            const size_t q = perm[p];
            y[q] += yg[p] / NG;
            for (int a = 0; a < 3; ++a) y[size_t(a + 1) * N + q] += sgn[a] * yg[size_t(a + 1) * N + p] / NG;
        }
    }
    return LB_OK;
}

lb_status lb_ws3_decode(int nx, int ny, int nz, const double* rho_tanh, double rho_l, double rho_g, const float* y,
                        double* rho, double* u) {
    if (!rho_tanh || !y || nx < 1 || ny < 1 || nz < 1 || !(rho_l > rho_g)) return fail(LB_EINVAL, "bad arguments");
    const size_t N = size_t(nx) * ny * nz;
    const double span = rho_l - rho_g, mid = 0.5 * (rho_l + rho_g);
    // keep the tanh start's mass: remove the predicted correction's mass
    // residual with weight 1 - 4c^2 (c the normalised tanh density)
    double dm = 0.0, wsum = 0.0;
    for (size_t i = 0; i < N; ++i) {
        const double c = (rho_tanh[i] - mid) / span;
        dm += double(y[i]);
        wsum += std::max(0.0, 1.0 - 4.0 * c * c);
    }
    const double shift = wsum > 0 ? dm / wsum : 0.0;
    for (size_t i = 0; i < N; ++i) {
        const double c = (rho_tanh[i] - mid) / span;
        if (rho) rho[i] = rho_tanh[i] + span * (double(y[i]) - shift * std::max(0.0, 1.0 - 4.0 * c * c));
        if (u)
            for (int a = 0; a < 3; ++a) u[size_t(a) * N + i] = 1e-3 * double(y[size_t(a + 1) * N + i]);
    }
    return LB_OK;
}

}  // extern "C"
