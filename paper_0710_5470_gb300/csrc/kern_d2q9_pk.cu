// Instantiations of the two-sites-per-thread D2Q9 step (step2d_pk.cuh) for
// single lattices.
#include <cstdlib>

#include "dispatch.h"
#include "step2d_pk.cuh"

using namespace lbk;

namespace {

template <bool F, class S, int TX, int TY>
struct PK2Launch {
    using Lay = Layout2PK<F, TX, TY>;
    static const void* fn() { return reinterpret_cast<const void*>(step_kernel2d_pk<F, S, TX, TY>); }
    static cudaError_t step(const StepArgs& a, dim3 grid, cudaStream_t st) {
        static int attr_done = 0;
        if (!attr_done) {
            cudaError_t e = cudaFuncSetAttribute(fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(Lay::BYTES));
            if (e != cudaSuccess) return e;
            attr_done = 1;
        }
        Tile2DArgs t{a.src_base, a.dst_base, a.pitch, a.nx, a.ny, a.pair2d, a.a, a.b, a.T, a.kappa, a.omega,
                     a.nu, a.fa, a.fb, a.fT, a.fkappa, a.fomega, a.fnu, a.pref, a.rsum, a.status};
        step_kernel2d_pk<F, S, TX, TY><<<grid, Lay::NTH, Lay::BYTES, st>>>(t);
        return cudaGetLastError();
    }
    static void apply(LbKernelSet& k, const char* name) {
        k.tx = TX;
        k.ty = TY;
        k.threads = Lay::NTH;
        k.smem = Lay::BYTES;
        k.step_fn = fn();
        k.step = &step;
        k.step_pair_needs_even_nx = false;   // odd nx: every site of a pair loaded on its own
        k.name = name;
    }
};

template <bool F>
LbKernelSet pick(int storage, LbKernelSet k) {
    switch (storage) {
        case 1: PK2Launch<F, StF32, 32, 8>::apply(k, "pairs 32x8"); break;
        case 2: PK2Launch<F, StF16, 32, 8>::apply(k, "pairs 32x8, mixed adds"); break;
        case 3: PK2Launch<F, StBF16, 32, 8>::apply(k, "pairs 32x8, mixed adds"); break;
        default: break;
    }
    return k;
}

}  // namespace

// The pair kernel for D2Q9 with 32-bit arithmetic (storage 1, 2, 3) in place
// of `step` of `base` (float64 keeps the tile kernel: its arithmetic bounds
// it).  LB_D2_VARIANT=0 keeps the tile kernel for comparisons.
LbKernelSet lbk_pk2d(int scheme, int storage, LbKernelSet k) {
    const char* env = std::getenv("LB_D2_VARIANT");
    if (env && std::atoi(env) == 0) return k;
    return scheme == 1 ? pick<true>(storage, k) : pick<false>(storage, k);
}

// First recorded index violation of this unit's kernels (checked builds; see bounds.cuh).
LB_BOUNDS_READER(lbk_bounds_d2pk)
