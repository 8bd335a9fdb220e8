// float64 reductions of the density and velocity fields (the diagnostics of
// Sec. IV: mass, momentum, max|u|, max|v|, density range, and the largest
// change of u since an earlier state), shared by lb_stats_get (grid-stride
// blocks) and lb_field_stats_noalloc (one contiguous chunk per block).
//
// Quantities, in this order: mass, momentum x / y / z, max|u|, max|v|,
// min rho, max rho and, when a previous velocity field is given,
// max |u - u_prev|.  Every block reduces its sites into per-thread partials,
// folds them as a fixed binary tree and writes NQ partials; one more block
// folds those in a fixed order, so the sums are deterministic.
#pragma once
#include <cuda_runtime.h>

namespace lbk {

constexpr int FR_NQ = 9;          // quantities of the full reduction
constexpr int FR_THREADS = 256;   // threads per reducing block

template <int NQ>
__device__ __forceinline__ void fr_init(double (&acc)[NQ]) {
    static_assert(NQ == 8 || NQ == 9, "8 or 9 quantities");
#pragma unroll
    for (int k = 0; k < 6; ++k) acc[k] = 0.0;
    acc[6] = 1e300;
    acc[7] = -1e300;
    if constexpr (NQ == 9) acc[8] = 0.0;
}

// Adds site i of the fields to the partials.
template <int NQ>
__device__ __forceinline__ void fr_site(double (&acc)[NQ], const double* rho, const double* u, const double* v,
                                        const double* u_prev, int dim, long long n, long long i) {
    const double r = rho[i];
    double u2 = 0.0, v2 = 0.0, d2 = 0.0;
    acc[0] += r;
    for (int c = 0; c < dim; ++c) {
        const double uc = u[c * n + i], vc = v[c * n + i];
        acc[1 + c] += r * uc;
        u2 += uc * uc;
        v2 += vc * vc;
        if constexpr (NQ == 9) {
            if (u_prev) {
                const double dc = uc - u_prev[c * n + i];
                d2 += dc * dc;
            }
        }
    }
    acc[4] = fmax(acc[4], sqrt(u2));
    acc[5] = fmax(acc[5], sqrt(v2));
    acc[6] = fmin(acc[6], r);
    acc[7] = fmax(acc[7], r);
    if constexpr (NQ == 9) acc[8] = fmax(acc[8], sqrt(d2));
}

// b <- combine(b, a) for one quantity k
template <int NQ>
__device__ __forceinline__ void fr_merge(double* b, const double* a) {
#pragma unroll
    for (int k = 0; k < 4; ++k) b[k] += a[k];
    b[4] = fmax(b[4], a[4]);
    b[5] = fmax(b[5], a[5]);
    b[6] = fmin(b[6], a[6]);
    b[7] = fmax(b[7], a[7]);
    if constexpr (NQ == 9) b[8] = fmax(b[8], a[8]);
}

// Block fold of the per-thread partials (FR_THREADS threads) into out[0..NQ).
template <int NQ>
__device__ __forceinline__ void fr_block(double (&acc)[NQ], double* out) {
    __shared__ double sh[FR_THREADS][NQ];
#pragma unroll
    for (int k = 0; k < NQ; ++k) sh[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int s = FR_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) fr_merge<NQ>(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NQ; ++k) out[k] = sh[0][k];
}

// Partials of block b over the sites b*chunk ... (contiguous chunks; chunk = 0:
// grid-stride over all n sites).
template <int NQ>
__global__ void __launch_bounds__(FR_THREADS)
    fr_partial_kernel(const double* rho, const double* u, const double* v, const double* u_prev, int dim,
                      long long n, long long chunk, double* partial) {
    double acc[NQ];
    fr_init<NQ>(acc);
    if (chunk > 0) {
        const long long begin = (long long)blockIdx.x * chunk;
        const long long end = begin + chunk < n ? begin + chunk : n;
        for (long long i = begin + threadIdx.x; i < end; i += FR_THREADS) fr_site<NQ>(acc, rho, u, v, u_prev, dim, n, i);
    } else {
        for (long long i = (long long)blockIdx.x * FR_THREADS + threadIdx.x; i < n;
             i += (long long)gridDim.x * FR_THREADS)
            fr_site<NQ>(acc, rho, u, v, u_prev, dim, n, i);
    }
    fr_block<NQ>(acc, partial + (size_t)blockIdx.x * NQ);
}

// Folds nblocks partials into out[0..NQ): one block of FR_THREADS threads,
// thread t folding the blocks t*c ... (t+1)*c - 1 in order (c = nblocks /
// FR_THREADS rounded up), then the fixed tree of fr_block: the same order on
// every call, so the result is deterministic.
template <int NQ>
__global__ void __launch_bounds__(FR_THREADS) fr_final_kernel(const double* partial, int nblocks, double* out) {
    if (blockIdx.x != 0) return;
    double acc[NQ];
    fr_init<NQ>(acc);
    const int c = (nblocks + FR_THREADS - 1) / FR_THREADS;
    const int b0 = int(threadIdx.x) * c, b1 = b0 + c < nblocks ? b0 + c : nblocks;
    for (int b = b0; b < b1; ++b) fr_merge<NQ>(acc, partial + (size_t)b * NQ);
    fr_block<NQ>(acc, out);
}

}  // namespace lbk
