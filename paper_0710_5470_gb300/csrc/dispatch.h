// Internal interface between the host API (lb_api.cu) and the kernel
// translation units (kern_d2q9.cu, kern_d3q19.cu).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "aux_kernels.cuh"

struct LbKernelSet {
    int tx = 0, ty = 0;           // CTA tile of the fused step
    int threads = 0;              // threads per CTA of the fused step
    size_t smem = 0;              // dynamic shared memory of the fused step
    const char* name = "";        // kernel form (reported by lb_kernel_info)
    bool aos = false;             // `step` needs the interleaved 16-bit layout (PopPtrs aos = 1)
    const void* step_fn = nullptr;
    cudaError_t (*step)(const lbk::StepArgs&, dim3 grid, cudaStream_t) = nullptr;
    // the same step with one site per load (any nx); `step` moves two sites
    // per load in its halo stage and needs an even nx when this flag is set
    const void* step1_fn = nullptr;
    cudaError_t (*step1)(const lbk::StepArgs&, dim3 grid, cudaStream_t) = nullptr;
    int tx1 = 0, ty1 = 0, threads1 = 0;   // tile, threads and shared memory of step1
    size_t smem1 = 0;
    const char* name1 = "";
    bool step_pair_needs_even_nx = false;
    cudaError_t (*init_feq)(const double* rho, const double* u, const lbk::PopPtrs&, lbk::Grid3, lbk::Phys,
                            cudaStream_t) = nullptr;
    cudaError_t (*moments)(const lbk::PopPtrs&, lbk::Grid3, double* rho, double* u, cudaStream_t) = nullptr;
    cudaError_t (*mprime)(const double* rho, lbk::Grid3, double kappa, double* mp, cudaStream_t) = nullptr;
    cudaError_t (*velocity_v)(const double* rho, const double* u, const double* mp, lbk::Grid3, double* v,
                              cudaStream_t) = nullptr;
    cudaError_t (*get_pops)(const lbk::PopPtrs&, size_t n, double* out, cudaStream_t) = nullptr;
    cudaError_t (*get_box)(const lbk::PopPtrs&, lbk::Grid3, const int (&origin)[3], const int (&box)[3], double* out,
                           cudaStream_t) = nullptr;
    cudaError_t (*set_pops)(const lbk::PopPtrs&, size_t n, const double* in, cudaStream_t) = nullptr;
};

// scheme: 0 equilibrium, 1 forcing; storage: lb_storage value.
LbKernelSet lbk_kernels_d2q9(int scheme, int storage);
LbKernelSet lbk_kernels_d3q19(int scheme, int storage, int nx);

// Grid size of the grid-stride auxiliary kernels.
inline unsigned lbk_aux_blocks(size_t n) {
    size_t b = (n + 255) / 256;
    if (b > 4096) b = 4096;
    return unsigned(b == 0 ? 1 : b);
}
