// Instantiations of the two-sites-per-thread D3Q19 equilibrium-scheme step
// (step3d_pk_eq.cuh).
#include <cstdlib>

#include "dispatch.h"
#include "step3d_pk_eq.cuh"

using namespace lbk;

namespace {

template <class S, int TX, int TY, int MINB, bool AOS>
struct PKELaunch {
    using Lay = LayoutPKE<TX, TY, PairIO<S>::RAW16>;
    static const void* fn() { return reinterpret_cast<const void*>(step_kernel3d_pk_eq<S, TX, TY, MINB, AOS>); }
    static cudaError_t step(const StepArgs& a, dim3 grid, cudaStream_t st) {
        static int attr_done = 0;
        if (!attr_done) {
            cudaError_t e = cudaFuncSetAttribute(fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(Lay::BYTES));
            if (e != cudaSuccess) return e;
            attr_done = 1;
        }
        step_kernel3d_pk_eq<S, TX, TY, MINB, AOS><<<grid, Lay::NTH, Lay::BYTES, st>>>(a);
        return cudaGetLastError();
    }
    static void apply(LbKernelSet& k, const char* name) {
        k.tx = TX;
        k.ty = TY;
        k.threads = Lay::NTH;
        k.smem = Lay::BYTES;
        k.step_fn = fn();
        k.step = &step;
        k.step_pair_needs_even_nx = true;
        k.name = name;
        k.aos = AOS;
    }
};

}  // namespace

// The pair kernel of the equilibrium scheme (step3d_pk_eq.cuh) for 32-bit
// arithmetic storage in place of `step` of `base` (an even nx is required;
// base.step1 stays the fallback; measured on GB300 at 128^3 / 512^3: fp16
// deviations 43.5 / 50.2 GLUPS against 37.7 / 43.1 for the tile kernel,
// float32 28.7 / 29.8 against 28.0 / 28.6).  LB_D3_VARIANT=0 keeps the tile kernel.
LbKernelSet lbk_pk_equilibrium(int storage, int nx, LbKernelSet k) {
    const char* env = std::getenv("LB_D3_VARIANT");
    const int v = env ? std::atoi(env) : -1;
    if (v == 0) return k;
    const bool aos = nx % AOS_SITES == 0;
    if (storage == 2) {
        if (aos) PKELaunch<StF16, 32, 8, 3, true>::apply(k, "pairs 32x8, equilibrium, interleaved blocks");
        else PKELaunch<StF16, 32, 8, 3, false>::apply(k, "pairs 32x8, equilibrium");
    } else if (storage == 3) {
        if (aos) PKELaunch<StBF16, 32, 8, 3, true>::apply(k, "pairs 32x8, equilibrium, interleaved blocks");
        else PKELaunch<StBF16, 32, 8, 3, false>::apply(k, "pairs 32x8, equilibrium");
    } else if (storage == 1) {
        PKELaunch<StF32, 32, 8, 2, false>::apply(k, "pairs 32x8, equilibrium");
    }
    return k;
}

// First recorded index violation of this unit's kernels (checked builds; see bounds.cuh).
LB_BOUNDS_READER(lbk_bounds_d3pke)
