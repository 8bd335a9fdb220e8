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
#include <atomic>
#include <cstdio>
#include <string>

#include <cuda_runtime.h>

#include "../../include/lb.h"
#include "field_reduce.cuh"

// Sets the thread-local message returned by lb_last_error (defined in lb_api.cu).
void lb_internal_set_error(const char* msg);

namespace {

constexpr int NSTAT = 8;             // mass, momentum x/y/z, max|u|, max|v|, min rho, max rho
constexpr int SITES_PER_BLOCK = LB_NOALLOC_SITES_PER_BLOCK;
constexpr int MAX_DEVICES = 64;
static_assert(lbk::FR_THREADS == 256, "block size of the shared reduction");

static __device__ __align__(256) double g_partials[LB_NOALLOC_MAX_BLOCKS * NSTAT];

// Address of g_partials on each device, looked up once per device (atomic:
// host threads may make their first call on a device at the same time; each
// stores the same address).
std::atomic<double*> g_partials_addr[MAX_DEVICES] = {};

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
    double* partial = g_partials_addr[dev].load();
    if (!partial) {
        // first call on this device (the current one): look up the array's device address
        e = cudaGetSymbolAddress(reinterpret_cast<void**>(&partial), g_partials);
        if (e != cudaSuccess) return fail(LB_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_partials_addr[dev].store(partial);
    }
    const int nblocks = int((n + SITES_PER_BLOCK - 1) / SITES_PER_BLOCK);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // one block per contiguous chunk of SITES_PER_BLOCK sites, folded in block order
    lbk::fr_partial_kernel<NSTAT><<<nblocks, lbk::FR_THREADS, 0, st>>>(rho, u, v, nullptr, dim, n, SITES_PER_BLOCK,
                                                                      partial);
    lbk::fr_final_kernel<NSTAT><<<1, lbk::FR_THREADS, 0, st>>>(partial, nblocks, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(LB_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return LB_OK;
}

}  // extern "C"
