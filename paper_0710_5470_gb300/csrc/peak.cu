// lb_fma_peak: the fused multiply-add rate of this GPU in float64 or
// float32, the denominator of the ALU roofline of the step kernels (the
// float64 step is bound by the FP64 units, not by HBM).  A measurement
// helper with no counterpart in the paper.
//
// Every thread runs CHAINS independent chains x <- x * m + c, so the FMA
// latency is hidden by the chains and the resident warps; m < 1 and c > 0
// keep every value finite and positive.  The sum is stored only if it equals
// -1, which never happens, so nothing is written but no chain is dead code.
#include <string>

#include <cuda_runtime.h>

#include "../../include/lb.h"

void lb_internal_set_error(const char* msg);

namespace {

constexpr int CHAINS = 8;
constexpr int THREADS = 256;
constexpr int CTAS_PER_SM = 4;

lb_status fail(lb_status s, const std::string& m) {
    lb_internal_set_error(m.c_str());
    return s;
}

template <class T>
__global__ void __launch_bounds__(THREADS) fma_rate_kernel(T* out, int iters, T m, T c) {
    T x[CHAINS];
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < CHAINS; ++k) x[k] = fma(x[k], m, c);
    }
    T s = T(0);
#pragma unroll
    for (int k = 0; k < CHAINS; ++k) s += x[k];
    if (s == T(-1)) out[0] = s;
}

template <class T>
cudaError_t time_rate(int iters, int blocks, double* seconds) {
    T* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(T));
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        fma_rate_kernel<T><<<blocks, THREADS>>>(out, iters < 64 ? iters : 64, T(0.999), T(1e-3));   // warm-up
        cudaEventRecord(e0);
        fma_rate_kernel<T><<<blocks, THREADS>>>(out, iters, T(0.999), T(1e-3));
        cudaEventRecord(e1);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaGetLastError();
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        *seconds = double(ms) * 1e-3;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (out) cudaFree(out);
    return e;
}

}  // namespace

extern "C" lb_status lb_fma_peak(int precision, int iters, double* tflops) {
    if (!tflops) return fail(LB_EINVAL, "lb_fma_peak: tflops is NULL");
    if (precision != 0 && precision != 1) return fail(LB_EINVAL, "lb_fma_peak: precision must be 0 or 1");
    if (iters < 1 || iters > (1 << 24)) return fail(LB_EINVAL, "lb_fma_peak: iters must be in [1, 2^24]");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("lb_fma_peak: ") + cudaGetErrorString(e));
    const int blocks = sms * CTAS_PER_SM;
    double s = 0.0;
    e = precision == 0 ? time_rate<double>(iters, blocks, &s) : time_rate<float>(iters, blocks, &s);
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("lb_fma_peak: ") + cudaGetErrorString(e));
    if (!(s > 0.0)) return fail(LB_ECUDA, "lb_fma_peak: zero elapsed time");
    const double flops = 2.0 * CHAINS * double(iters) * double(blocks) * THREADS;
    *tflops = flops / s * 1e-12;
    return LB_OK;
}
