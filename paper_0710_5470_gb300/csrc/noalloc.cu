// lb_field_stats_noalloc: the float64 field reductions of lb_stats_get for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they want these
// numbers: an application whose own allocator has reserved the device memory
// it is allowed to use, or a time-stepping loop that must not pay for
// cudaMalloc / cudaFree (which can synchronise the device) or risk an
// allocation failure in the middle of a run.  This entry point takes the
// fields and the output buffer from the caller and keeps its per-block
// partial sums in a fixed file-scope device array instead of allocating.
//
// The array (LB_NOALLOC_MAX_BLOCKS x 8 doubles = 256 KiB) is created on
// every GPU that loads the library and stays there until the process exits.
// All calls share it: every call overwrites the partials it reads before
// reading them, so nothing has to start at zero, but two calls whose kernels
// overlap on the GPU (different streams, or different host threads) race on
// it and may return each other's numbers.
#include <cstdio>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lb.h"

// Sets the thread-local message returned by lb_last_error (defined in lb_api.cu).
void lb_internal_set_error(const char* msg);

namespace {

constexpr int NSTAT = 8;             // mass, momentum x/y/z, max|u|, max|v|, min rho, max rho
constexpr int THREADS = 256;
constexpr int SITES_PER_BLOCK = LB_NOALLOC_SITES_PER_BLOCK;
constexpr int MAX_DEVICES = 64;

static __device__ __align__(256) double g_partials[LB_NOALLOC_MAX_BLOCKS * NSTAT];

// Address of g_partials on each device, looked up once per device.
double* g_partials_addr[MAX_DEVICES] = {};

// One block reduces the sites [blockIdx.x * SITES_PER_BLOCK, ...) of its chunk
// in a fixed order and writes its 8 partials.
__global__ void __launch_bounds__(THREADS)
    noalloc_partial_kernel(const double* rho, const double* u, const double* v, int dim, long long n,
                           double* partial) {
    __shared__ double sh[NSTAT][THREADS];
    double acc[NSTAT] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1e300, -1e300};
    const long long begin = (long long)blockIdx.x * SITES_PER_BLOCK;
    const long long end = begin + SITES_PER_BLOCK < n ? begin + SITES_PER_BLOCK : n;
    for (long long i = begin + threadIdx.x; i < end; i += THREADS) {
        const double r = rho[i];
        double u2 = 0.0, v2 = 0.0;
        acc[0] += r;
        for (int c = 0; c < dim; ++c) {
            const double uc = u[c * n + i], vc = v[c * n + i];
            acc[1 + c] += r * uc;
            u2 += uc * uc;
            v2 += vc * vc;
        }
        acc[4] = fmax(acc[4], sqrt(u2));
        acc[5] = fmax(acc[5], sqrt(v2));
        acc[6] = fmin(acc[6], r);
        acc[7] = fmax(acc[7], r);
    }
    for (int k = 0; k < NSTAT; ++k) sh[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int s = THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
            sh[4][threadIdx.x] = fmax(sh[4][threadIdx.x], sh[4][threadIdx.x + s]);
            sh[5][threadIdx.x] = fmax(sh[5][threadIdx.x], sh[5][threadIdx.x + s]);
            sh[6][threadIdx.x] = fmin(sh[6][threadIdx.x], sh[6][threadIdx.x + s]);
            sh[7][threadIdx.x] = fmax(sh[7][threadIdx.x], sh[7][threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < NSTAT; ++k) partial[(size_t)blockIdx.x * NSTAT + k] = sh[k][0];
}

// Folds the partials of this call in block order into the caller's output.
__global__ void noalloc_final_kernel(const double* partial, int nblocks, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double acc[NSTAT] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 1e300, -1e300};
    for (int b = 0; b < nblocks; ++b) {
        const double* p = partial + (size_t)b * NSTAT;
        for (int k = 0; k < 4; ++k) acc[k] += p[k];
        acc[4] = fmax(acc[4], p[4]);
        acc[5] = fmax(acc[5], p[5]);
        acc[6] = fmin(acc[6], p[6]);
        acc[7] = fmax(acc[7], p[7]);
    }
    for (int k = 0; k < NSTAT; ++k) out[k] = acc[k];
}

lb_status fail(lb_status s, const std::string& m) {
    lb_internal_set_error(m.c_str());
    return s;
}

}  // namespace

extern "C" {

lb_status lb_field_stats_noalloc(const double* rho, const double* u, const double* v, int dim, long long n,
                                 double* out, void* cuda_stream) {
    if (!rho || !u || !v || !out) return fail(LB_EINVAL, "null pointer");
    if (dim < 1 || dim > 3) return fail(LB_EINVAL, "dim must be 1, 2 or 3");
    if (n < 1) return fail(LB_EINVAL, "n must be >= 1");
    const long long max_n = (long long)LB_NOALLOC_MAX_BLOCKS * SITES_PER_BLOCK;
    if (n > max_n)
        return fail(LB_EINVAL, "n = " + std::to_string(n) + " exceeds the maximum of " + std::to_string(max_n) +
                                   " sites of lb_field_stats_noalloc");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= MAX_DEVICES) return fail(LB_EINVAL, "device index out of range");
    if (!g_partials_addr[dev]) {
        // first call on this device (the current one): look up the array's device address
        double* ptr = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&ptr), g_partials);
        if (e != cudaSuccess) return fail(LB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_partials_addr[dev] = ptr;
    }
    double* partial = g_partials_addr[dev];
    const int nblocks = int((n + SITES_PER_BLOCK - 1) / SITES_PER_BLOCK);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    noalloc_partial_kernel<<<nblocks, THREADS, 0, st>>>(rho, u, v, dim, n, partial);
    noalloc_final_kernel<<<1, 32, 0, st>>>(partial, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return LB_OK;
}

}  // extern "C"
