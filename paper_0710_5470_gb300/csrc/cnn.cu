// Warm-start network: 4 layers of periodic 3x3 convolutions (5 -> 32 -> 32 ->
// 32 -> 3 channels, tanh between layers), trained and evaluated on the GPU
// by the kernels below.  Activations are float32 NCHW; the convolutions read
// fp16 copies of the weights (float32 accumulation); Adam updates float32
// master weights and refreshes the fp16 copies.
//
// Inputs (5 planes): normalised tanh-start density, T, kappa, tau, R.
// Outputs (3 planes): (rho_steady - rho_tanh) / (rho_l - rho_g), 1000 u_x, 1000 u_y.
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

constexpr int TILE = 16;                 // 16 x 16 output pixels per CTA
constexpr int NL = 4;
constexpr int CH[NL + 1] = {LB_WS_IN, LB_WS_HIDDEN, LB_WS_HIDDEN, LB_WS_HIDDEN, LB_WS_OUT};

lb_status fail(lb_status s, const std::string& m) {
    lb_internal_set_error(m.c_str());
    return s;
}

// out[n,o,y,x] = act(b[o] + sum_{c,dy,dx} W[o,c,dy+1,dx+1] in[n,c,y+dy,x+dx]), periodic.
template <int CIN, int COUT, bool TANH>
__global__ void __launch_bounds__(TILE* TILE) conv_fwd(const float* in, const __half* W, const float* bias,
                                                       float* out, int H, int Wd) {
    extern __shared__ float sm[];
    float* tile = sm;                                  // [CIN][18][18]
    float* wsh = sm + CIN * (TILE + 2) * (TILE + 2);   // [CIN][9][COUT]
    const int n = blockIdx.z;
    const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
    const int tid = threadIdx.x;
    const float* inn = in + size_t(n) * CIN * H * Wd;
    for (int i = tid; i < CIN * (TILE + 2) * (TILE + 2); i += TILE * TILE) {
        const int c = i / ((TILE + 2) * (TILE + 2)), r = i % ((TILE + 2) * (TILE + 2));
        const int ty = r / (TILE + 2), tx = r % (TILE + 2);
        tile[i] = inn[(size_t(c) * H + wrap(y0 + ty - 1, H)) * Wd + wrap(x0 + tx - 1, Wd)];
    }
    for (int i = tid; i < COUT * CIN * 9; i += TILE * TILE) {
        const int o = i / (CIN * 9), r = i % (CIN * 9);   // r = c*9 + k
        wsh[r * COUT + o] = __half2float(W[i]);
    }
    __syncthreads();
    const int lx = tid % TILE, ly = tid / TILE;
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = bias[o];
    for (int c = 0; c < CIN; ++c) {
        float v[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) v[k] = tile[(c * (TILE + 2) + ly + k / 3) * (TILE + 2) + lx + k % 3];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float* w = wsh + (c * 9 + k) * COUT;
#pragma unroll
            for (int o = 0; o < COUT; ++o) acc[o] += w[o] * v[k];
        }
    }
    const int x = x0 + lx, y = y0 + ly;
    if (x < Wd && y < H) {
#pragma unroll
        for (int o = 0; o < COUT; ++o)
            out[((size_t(n) * COUT + o) * H + y) * Wd + x] = TANH ? tanhf(acc[o]) : acc[o];
    }
}

// din[n,c,y,x] = (sum_{o,dy,dx} W[o,c,dy+1,dx+1] dout[n,o,y-dy,x-dx]) * (1 - h^2 if h), periodic.
template <int CIN, int COUT>
__global__ void __launch_bounds__(TILE* TILE) conv_bwd_data(const float* dout, const __half* W, const float* h,
                                                            float* din, int H, int Wd) {
    extern __shared__ float sm[];
    float* tile = sm;                                   // [COUT][18][18] of dout
    float* wsh = sm + COUT * (TILE + 2) * (TILE + 2);   // [COUT][9][CIN]
    const int n = blockIdx.z;
    const int x0 = blockIdx.x * TILE, y0 = blockIdx.y * TILE;
    const int tid = threadIdx.x;
    const float* dn = dout + size_t(n) * COUT * H * Wd;
    for (int i = tid; i < COUT * (TILE + 2) * (TILE + 2); i += TILE * TILE) {
        const int o = i / ((TILE + 2) * (TILE + 2)), r = i % ((TILE + 2) * (TILE + 2));
        const int ty = r / (TILE + 2), tx = r % (TILE + 2);
        tile[i] = dn[(size_t(o) * H + wrap(y0 + ty - 1, H)) * Wd + wrap(x0 + tx - 1, Wd)];
    }
    for (int i = tid; i < COUT * CIN * 9; i += TILE * TILE) {
        const int o = i / (CIN * 9), r = i % (CIN * 9);
        const int c = r / 9, k = r % 9;
        wsh[(o * 9 + k) * CIN + c] = __half2float(W[i]);
    }
    __syncthreads();
    const int lx = tid % TILE, ly = tid / TILE;
    float acc[CIN];
#pragma unroll
    for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
    for (int o = 0; o < COUT; ++o) {
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int dy = k / 3 - 1, dx = k % 3 - 1;
            const float g = tile[(o * (TILE + 2) + ly - dy + 1) * (TILE + 2) + lx - dx + 1];
            const float* w = wsh + (o * 9 + k) * CIN;
#pragma unroll
            for (int c = 0; c < CIN; ++c) acc[c] += w[c] * g;
        }
    }
    const int x = x0 + lx, y = y0 + ly;
    if (x < Wd && y < H) {
#pragma unroll
        for (int c = 0; c < CIN; ++c) {
            const size_t idx = ((size_t(n) * CIN + c) * H + y) * Wd + x;
            float v = acc[c];
            if (h) v *= 1.f - h[idx] * h[idx];
            din[idx] = v;
        }
    }
}

// dW[o,c,k] += sum over pixels of dout[o,p] h[c,p+k]; db[o] += sum dout[o,p].
// Each CTA sweeps many 16x16 tiles and adds its partial sums once.
template <int CIN>
constexpr int bwd_w_threads() {
    return CIN * 9 > TILE * TILE ? (CIN * 9 + 31) / 32 * 32 : TILE * TILE;
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(bwd_w_threads<CIN>()) conv_bwd_weight(const float* h, const float* dout, float* dW,
                                                                         float* db, int N, int H, int Wd) {
    extern __shared__ float sm[];
    float* tile = sm;                                   // [CIN][18][18] of h
    float* gt = sm + CIN * (TILE + 2) * (TILE + 2);     // [COUT][256] of dout
    const int tid = threadIdx.x;
    const int tiles_x = (Wd + TILE - 1) / TILE, tiles_y = (H + TILE - 1) / TILE;
    const int ntiles = N * tiles_x * tiles_y;
    constexpr int NPAIR = CIN * 9;                      // (c, k) pairs, one thread each
    float acc[COUT];
#pragma unroll
    for (int o = 0; o < COUT; ++o) acc[o] = 0.f;
    float bacc = 0.f;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int n = t / (tiles_x * tiles_y), r0 = t % (tiles_x * tiles_y);
        const int x0 = (r0 % tiles_x) * TILE, y0 = (r0 / tiles_x) * TILE;
        __syncthreads();
        for (int i = tid; i < CIN * (TILE + 2) * (TILE + 2); i += blockDim.x) {
            const int c = i / ((TILE + 2) * (TILE + 2)), r = i % ((TILE + 2) * (TILE + 2));
            const int ty = r / (TILE + 2), tx = r % (TILE + 2);
            tile[i] = h[((size_t(n) * CIN + c) * H + wrap(y0 + ty - 1, H)) * Wd + wrap(x0 + tx - 1, Wd)];
        }
        for (int i = tid; i < COUT * TILE * TILE; i += blockDim.x) {
            const int o = i / (TILE * TILE), p = i % (TILE * TILE);
            const int x = x0 + p % TILE, y = y0 + p / TILE;
            gt[i] = (x < Wd && y < H) ? dout[((size_t(n) * COUT + o) * H + y) * Wd + x] : 0.f;
        }
        __syncthreads();
        if (tid < NPAIR) {
            const int c = tid / 9, k = tid % 9;
            const int ky = k / 3, kx = k % 3;
            for (int p = 0; p < TILE * TILE; ++p) {
                const float v = tile[(c * (TILE + 2) + p / TILE + ky) * (TILE + 2) + p % TILE + kx];
#pragma unroll
                for (int o = 0; o < COUT; ++o) acc[o] += gt[o * TILE * TILE + p] * v;
            }
        }
        if (tid < COUT)
            for (int p = 0; p < TILE * TILE; ++p) bacc += gt[tid * TILE * TILE + p];
    }
    if (tid < NPAIR) {
        const int c = tid / 9, k = tid % 9;
#pragma unroll
        for (int o = 0; o < COUT; ++o) atomicAdd(dW + (o * CIN + c) * 9 + k, acc[o]);
    }
    if (tid < COUT) atomicAdd(db + tid, bacc);
}

size_t smem_fwd(int cin, int cout) { return size_t(cin * (TILE + 2) * (TILE + 2) + cin * 9 * cout) * 4; }
size_t smem_bwd_w(int cin, int cout) { return size_t(cin * (TILE + 2) * (TILE + 2) + cout * TILE * TILE) * 4; }

}  // namespace

struct lb_ws {
    int nparams = 0;
    int woff[NL], boff[NL];         // offsets of W_l and b_l in the packed parameter vector
    float* p = nullptr;             // float32 master parameters (packed)
    __half* p16 = nullptr;          // fp16 copies
    float* g = nullptr;             // gradients
    float* m = nullptr;
    float* v = nullptr;
    double* loss = nullptr;
    int adam_t = 0;
    // activations of the current batch
    float* act[NL + 1] = {};
    float* dact[NL + 1] = {};
    size_t cap = 0;                 // pixels x batch capacity of the activation buffers
    cudaStream_t st = nullptr;
};

namespace {

lb_status ensure_acts(lb_ws* w, size_t pix) {
    if (pix <= w->cap) return LB_OK;
    for (int l = 0; l <= NL; ++l) {
        cudaFree(w->act[l]);
        cudaFree(w->dact[l]);
        w->act[l] = w->dact[l] = nullptr;
    }
    for (int l = 0; l <= NL; ++l) {
        if (cudaMalloc(&w->act[l], pix * CH[l] * sizeof(float)) != cudaSuccess ||
            cudaMalloc(&w->dact[l], pix * CH[l] * sizeof(float)) != cudaSuccess)
            return fail(LB_ENOMEM, "warm-start activations");
    }
    w->cap = pix;
    return LB_OK;
}

template <int CIN, int COUT, bool T>
void launch_fwd(const float* in, const __half* W, const float* b, float* out, int n, int H, int Wd, cudaStream_t st) {
    const size_t sm = smem_fwd(CIN, COUT);
    cudaFuncSetAttribute(conv_fwd<CIN, COUT, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    dim3 grid((Wd + TILE - 1) / TILE, (H + TILE - 1) / TILE, n);
    conv_fwd<CIN, COUT, T><<<grid, TILE * TILE, sm, st>>>(in, W, b, out, H, Wd);
}

template <int CIN, int COUT>
void launch_bwd(lb_ws* w, int l, int n, int H, int Wd) {
    const float* hin = w->act[l];
    const size_t smw = smem_bwd_w(CIN, COUT);
    cudaFuncSetAttribute(conv_bwd_weight<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smw));
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = n * ((Wd + TILE - 1) / TILE) * ((H + TILE - 1) / TILE);
    const int blocks = ntiles < 2 * sms ? ntiles : 2 * sms;
    conv_bwd_weight<CIN, COUT><<<blocks, bwd_w_threads<CIN>(), smw, w->st>>>(hin, w->dact[l + 1], w->g + w->woff[l],
                                                                      w->g + w->boff[l], n, H, Wd);
    if (l > 0) {
        const size_t smd = smem_fwd(COUT, CIN);
        cudaFuncSetAttribute(conv_bwd_data<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smd));
        dim3 grid((Wd + TILE - 1) / TILE, (H + TILE - 1) / TILE, n);
        conv_bwd_data<CIN, COUT><<<grid, TILE * TILE, smd, w->st>>>(w->dact[l + 1], w->p16 + w->woff[l], w->act[l],
                                                                    w->dact[l], H, Wd);
    }
}

// The sample index is the grid's z dimension: at most 65535 samples per launch.
constexpr int MAX_SAMPLES = 65535;

cudaError_t forward(lb_ws* w, int n, int H, int Wd) {
    launch_fwd<LB_WS_IN, LB_WS_HIDDEN, true>(w->act[0], w->p16 + w->woff[0], w->p + w->boff[0], w->act[1], n, H, Wd, w->st);
    launch_fwd<LB_WS_HIDDEN, LB_WS_HIDDEN, true>(w->act[1], w->p16 + w->woff[1], w->p + w->boff[1], w->act[2], n, H, Wd, w->st);
    launch_fwd<LB_WS_HIDDEN, LB_WS_HIDDEN, true>(w->act[2], w->p16 + w->woff[2], w->p + w->boff[2], w->act[3], n, H, Wd, w->st);
    launch_fwd<LB_WS_HIDDEN, LB_WS_OUT, false>(w->act[3], w->p16 + w->woff[3], w->p + w->boff[3], w->act[4], n, H, Wd, w->st);
    return cudaGetLastError();
}

// loss and gradients of the batch whose inputs sit in act[0] and targets in dact[4]'s place (t)
lb_status loss_grad(lb_ws* w, const float* t, int n, int H, int Wd, double* loss_out) {
    forward(w, n, H, Wd);
    cudaMemsetAsync(w->g, 0, size_t(w->nparams) * sizeof(float), w->st);
    cudaMemsetAsync(w->loss, 0, sizeof(double), w->st);
    const size_t nout = size_t(n) * LB_WS_OUT * H * Wd;
    mse_grad<<<256, 256, 0, w->st>>>(w->act[4], t, w->dact[4], nout, w->loss);
    launch_bwd<LB_WS_HIDDEN, LB_WS_OUT>(w, 3, n, H, Wd);
    launch_bwd<LB_WS_HIDDEN, LB_WS_HIDDEN>(w, 2, n, H, Wd);
    launch_bwd<LB_WS_HIDDEN, LB_WS_HIDDEN>(w, 1, n, H, Wd);
    launch_bwd<LB_WS_IN, LB_WS_HIDDEN>(w, 0, n, H, Wd);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("warm-start backward: ") + cudaGetErrorString(e));
    if (loss_out) {
        e = cudaMemcpyAsync(loss_out, w->loss, sizeof(double), cudaMemcpyDeviceToHost, w->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
        if (e != cudaSuccess) return fail(LB_ECUDA, std::string("warm-start loss: ") + cudaGetErrorString(e));
    }
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_ws_create(int seed, void* cuda_stream, lb_ws** out) {
    if (!out) return fail(LB_EINVAL, "null output");
    lb_ws* w = new (std::nothrow) lb_ws();
    if (!w) return fail(LB_ENOMEM, "host allocation");
    w->st = static_cast<cudaStream_t>(cuda_stream);
    int off = 0;
    for (int l = 0; l < NL; ++l) {
        w->woff[l] = off;
        off += CH[l + 1] * CH[l] * 9;
        w->boff[l] = off;
        off += CH[l + 1];
    }
    w->nparams = off;
    // W ~ U(-s, s), s = 1/sqrt(9 C_in), from a SplitMix64 stream; b = 0
    std::vector<float> h(off, 0.f);
    unsigned long long st = (unsigned long long)seed;
    for (int l = 0; l < NL; ++l) {
        const double s = 1.0 / std::sqrt(9.0 * CH[l]);
        for (int i = 0; i < CH[l + 1] * CH[l] * 9; ++i) h[w->woff[l] + i] = float((2.0 * splitmix_u01(st) - 1.0) * s);
    }
    cudaError_t e;
    if ((e = cudaMalloc(&w->p, off * sizeof(float))) != cudaSuccess || (e = cudaMalloc(&w->p16, off * sizeof(__half))) != cudaSuccess ||
        (e = cudaMalloc(&w->g, off * sizeof(float))) != cudaSuccess || (e = cudaMalloc(&w->m, off * sizeof(float))) != cudaSuccess ||
        (e = cudaMalloc(&w->v, off * sizeof(float))) != cudaSuccess || (e = cudaMalloc(&w->loss, sizeof(double))) != cudaSuccess) {
        lb_ws_destroy(w);
        return fail(LB_ENOMEM, std::string("warm-start parameters: ") + cudaGetErrorString(e));
    }
    lb_status s = lb_ws_set_params(w, h.data(), size_t(off));
    if (s != LB_OK) { lb_ws_destroy(w); return s; }
    *out = w;
    return LB_OK;
}

lb_status lb_ws_destroy(lb_ws* w) {
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

lb_status lb_ws_num_params(const lb_ws* w, long long* n) {
    if (!w || !n) return fail(LB_EINVAL, "null argument");
    *n = w->nparams;
    return LB_OK;
}

lb_status lb_ws_set_params(lb_ws* w, const float* params, size_t count) {
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

lb_status lb_ws_get_params(lb_ws* w, float* params, size_t count) {
    if (!w || !params || count != size_t(w->nparams)) return fail(LB_EINVAL, "parameter count mismatch");
    cudaError_t e = cudaMemcpyAsync(params, w->p, count * sizeof(float), cudaMemcpyDeviceToHost, w->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
    return e == cudaSuccess ? LB_OK : fail(LB_ECUDA, std::string("get params: ") + cudaGetErrorString(e));
}

lb_status lb_ws_forward(lb_ws* w, const float* x, int n, int H, int Wd, float* y) {
    if (!w || !x || !y || n < 1 || n > MAX_SAMPLES || H < 1 || Wd < 1) return fail(LB_EINVAL, "bad arguments");
    const size_t pix = size_t(n) * H * Wd;
    lb_status s = ensure_acts(w, pix);
    if (s != LB_OK) return s;
    cudaError_t e = cudaMemcpyAsync(w->act[0], x, pix * LB_WS_IN * sizeof(float), cudaMemcpyHostToDevice, w->st);
    if (e != cudaSuccess) return fail(LB_ECUDA, "upload");
    if ((e = forward(w, n, H, Wd)) != cudaSuccess)
        return fail(LB_ECUDA, std::string("warm-start forward launch: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(y, w->act[4], pix * LB_WS_OUT * sizeof(float), cudaMemcpyDeviceToHost, w->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
    return e == cudaSuccess ? LB_OK : fail(LB_ECUDA, std::string("warm-start forward: ") + cudaGetErrorString(e));
}

lb_status lb_ws_loss_grad(lb_ws* w, const float* x, const float* t, int n, int H, int Wd, double* loss,
                          float* grads) {
    if (!w || !x || !t || n < 1 || n > MAX_SAMPLES || H < 1 || Wd < 1) return fail(LB_EINVAL, "bad arguments");
    const size_t pix = size_t(n) * H * Wd;
    lb_status s = ensure_acts(w, pix);
    if (s != LB_OK) return s;
    float* dt = nullptr;
    if (cudaMalloc(&dt, pix * LB_WS_OUT * sizeof(float)) != cudaSuccess) return fail(LB_ENOMEM, "targets");
    cudaMemcpyAsync(w->act[0], x, pix * LB_WS_IN * sizeof(float), cudaMemcpyHostToDevice, w->st);
    cudaMemcpyAsync(dt, t, pix * LB_WS_OUT * sizeof(float), cudaMemcpyHostToDevice, w->st);
    s = loss_grad(w, dt, n, H, Wd, loss);
    if (s == LB_OK && grads) {
        cudaError_t e = cudaMemcpyAsync(grads, w->g, size_t(w->nparams) * sizeof(float), cudaMemcpyDeviceToHost, w->st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
        if (e != cudaSuccess) s = fail(LB_ECUDA, "gradient download");
    }
    cudaFree(dt);
    return s;
}

lb_status lb_ws_train(lb_ws* w, const float* x, const float* t, int n, int H, int Wd, int epochs, int batch,
                      float lr, int seed, double* loss_history) {
    if (!w || !x || !t || n < 1 || H < 1 || Wd < 1 || epochs < 1 || batch < 1) return fail(LB_EINVAL, "bad arguments");
    batch = batch < n ? batch : n;
    if (batch > MAX_SAMPLES) return fail(LB_EINVAL, "batch larger than 65535 samples");
    const size_t img = size_t(H) * Wd;
    lb_status s = ensure_acts(w, size_t(batch) * img);
    if (s != LB_OK) return s;
    float *dx = nullptr, *dt = nullptr, *bt = nullptr;
    if (cudaMalloc(&dx, size_t(n) * img * LB_WS_IN * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&dt, size_t(n) * img * LB_WS_OUT * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&bt, size_t(batch) * img * LB_WS_OUT * sizeof(float)) != cudaSuccess) {
        cudaFree(dx);
        cudaFree(dt);
        return fail(LB_ENOMEM, "training data");
    }
    cudaMemcpyAsync(dx, x, size_t(n) * img * LB_WS_IN * sizeof(float), cudaMemcpyHostToDevice, w->st);
    cudaMemcpyAsync(dt, t, size_t(n) * img * LB_WS_OUT * sizeof(float), cudaMemcpyHostToDevice, w->st);
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
                cudaMemcpyAsync(w->act[0] + size_t(k) * img * LB_WS_IN, dx + size_t(j) * img * LB_WS_IN,
                                img * LB_WS_IN * sizeof(float), cudaMemcpyDeviceToDevice, w->st);
                cudaMemcpyAsync(bt + size_t(k) * img * LB_WS_OUT, dt + size_t(j) * img * LB_WS_OUT,
                                img * LB_WS_OUT * sizeof(float), cudaMemcpyDeviceToDevice, w->st);
            }
            double l = 0.0;
            s = loss_grad(w, bt, batch, H, Wd, &l);
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
    if (s == LB_OK && e != cudaSuccess) s = fail(LB_ECUDA, std::string("training: ") + cudaGetErrorString(e));
    return s;
}

lb_status lb_ws_predict_sym(lb_ws* w, const float* x, int H, int Wd, float* y) {
    if (!w || !x || !y || H < 1 || Wd < 1) return fail(LB_EINVAL, "bad arguments");
    // group of the periodic lattice fixing the point (W/2, H/2): reflections
    // x -> (W - x) mod W, y -> (H - y) mod H and, on square grids, the transpose.
    const int ng = (H == Wd) ? 8 : 4;
    const size_t N = size_t(H) * Wd;
    std::vector<float> xs(size_t(ng) * LB_WS_IN * N), ys(size_t(ng) * LB_WS_OUT * N);
    std::vector<int> perm(size_t(ng) * N);
    int A[8][2][2];
    for (int g = 0; g < ng; ++g) {
        const int fx = g & 1, fy = (g >> 1) & 1, tr = (g >> 2) & 1;
        // coordinate map p -> g(p): optional transpose, then the reflections
        int M[2][2] = {{1, 0}, {0, 1}};
        if (tr) { M[0][0] = 0; M[0][1] = 1; M[1][0] = 1; M[1][1] = 0; }
        for (int j = 0; j < 2; ++j) {
            if (fx) M[0][j] = -M[0][j];
            if (fy) M[1][j] = -M[1][j];
        }
        std::memcpy(A[g], M, sizeof(M));
        for (int yy = 0; yy < H; ++yy)
            for (int xx = 0; xx < Wd; ++xx) {
                int sx = tr ? yy : xx, sy = tr ? xx : yy;
                if (fx) sx = (Wd - sx) % Wd;
                if (fy) sy = (H - sy) % H;
                perm[size_t(g) * N + size_t(yy) * Wd + xx] = sy * Wd + sx;
            }
        for (int c = 0; c < LB_WS_IN; ++c)
            for (size_t p = 0; p < N; ++p)
                xs[(size_t(g) * LB_WS_IN + c) * N + p] = x[size_t(c) * N + perm[size_t(g) * N + p]];
    }
    lb_status st = lb_ws_forward(w, xs.data(), ng, H, Wd, ys.data());
    if (st != LB_OK) return st;
    std::fill(y, y + size_t(LB_WS_OUT) * N, 0.f);
    for (int g = 0; g < ng; ++g) {
        const float* yg = ys.data() + size_t(g) * LB_WS_OUT * N;
        for (size_t p = 0; p < N; ++p) {
            const size_t q = size_t(perm[size_t(g) * N + p]);
            const float ux = yg[N + p], uy = yg[2 * N + p];
            y[q] += yg[p] / ng;                                             // scalar channel
            y[N + q] += (A[g][0][0] * ux + A[g][0][1] * uy) / ng;           // u(g p) = A u_g(p)
            y[2 * N + q] += (A[g][1][0] * ux + A[g][1][1] * uy) / ng;
        }
    }
    return LB_OK;
}

lb_status lb_ws_features(int nx, int ny, const double* rho_tanh, double rho_l, double rho_g, double T, double kappa,
                         double tau, double R, float* x) {
    if (!rho_tanh || !x || nx < 1 || ny < 1 || !(rho_l > rho_g) || !(R > 0)) return fail(LB_EINVAL, "bad arguments");
    const size_t N = size_t(nx) * ny;
    const double mid = 0.5 * (rho_l + rho_g), span = rho_l - rho_g;
    const float planes[4] = {float((T - 0.53) / 0.03), float((kappa - 0.016) / 0.014), float((tau - 1.05) / 0.45),
                             float(10.0 / R)};
    for (size_t i = 0; i < N; ++i) {
        x[i] = float((rho_tanh[i] - mid) / span);
        for (int c = 0; c < 4; ++c) x[(c + 1) * N + i] = planes[c];
    }
    return LB_OK;
}

lb_status lb_ws_decode(int nx, int ny, const double* rho_tanh, double rho_l, double rho_g, const float* y, double* rho,
                       double* u) {
    if (!rho_tanh || !y || nx < 1 || ny < 1 || !(rho_l > rho_g)) return fail(LB_EINVAL, "bad arguments");
    const size_t N = size_t(nx) * ny;
    const double span = rho_l - rho_g, mid = 0.5 * (rho_l + rho_g);
    // The prediction must describe the same drop: its mass is the tanh start's.
    // The mass residual of the predicted correction is removed with weight
    // 1 - 4c^2 (c the normalised tanh density), i.e. inside the interface.
    double dm = 0.0, wsum = 0.0;
    for (size_t i = 0; i < N; ++i) {
        const double c = (rho_tanh[i] - mid) / span;
        dm += double(y[i]);
        wsum += std::max(0.0, 1.0 - 4.0 * c * c);
    }
    const double shift = wsum > 0 ? dm / wsum : 0.0;
    for (size_t i = 0; i < N; ++i) {
        const double c = (rho_tanh[i] - mid) / span;
        const double corr = double(y[i]) - shift * std::max(0.0, 1.0 - 4.0 * c * c);
        if (rho) rho[i] = rho_tanh[i] + span * corr;
        if (u) {
            u[i] = 1e-3 * double(y[N + i]);
            u[N + i] = 1e-3 * double(y[2 * N + i]);
        }
    }
    return LB_OK;
}

}  // extern "C"
