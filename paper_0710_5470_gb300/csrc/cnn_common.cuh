// Pieces shared by the 2D and 3D warm-start networks (cnn.cu, cnn3d.cu):
// periodic index wrap, the MSE loss gradient, the Adam update and the
// float32 -> fp16 weight copy.  Each including translation unit gets its own
// copies (anonymous namespace).
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ int wrap(int v, int n) {
    v %= n;
    return v < 0 ? v + n : v;
}

// dy = 2 (y - t) / count; loss += sum (y - t)^2 / count (float64 accumulation).
__global__ void mse_grad(const float* y, const float* t, float* dy, size_t n, double* loss) {
    __shared__ double red[256];
    double acc = 0.0;
    for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
        const float d = y[i] - t[i];
        dy[i] = 2.f * d / float(n);
        acc += double(d) * double(d);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (int(threadIdx.x) < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0] / double(n));
}

__global__ void adam_update(float* w, __half* w16, const float* g, float* m, float* v, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w16[i] = __float2half_rn(w[i]);
    }
}

__global__ void to_half(const float* w, __half* w16, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) w16[i] = __float2half_rn(w[i]);
}

// Uniform double in [0, 1) from a SplitMix64 stream (Steele, Lea, Flood 2014).
inline double splitmix_u01(unsigned long long& state) {
    state += 0x9E3779B97F4A7C15ull;
    unsigned long long z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return double(z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace
