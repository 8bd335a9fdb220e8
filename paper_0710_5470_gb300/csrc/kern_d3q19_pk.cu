// Instantiations of the two-sites-per-thread D3Q19 forcing step (step3d_pk.cuh).
#include <cstdlib>

#include "dispatch.h"
#include "step3d_pk.cuh"

using namespace lbk;

namespace {

template <class S, int TX, int TY, int MINB, int PF, bool MIXED, bool AOS = false, bool PB = false>
struct PKLaunch {
    using Lay = LayoutPK<TX, TY, PairIO<S>::RAW16>;
    static const void* fn() { return reinterpret_cast<const void*>(step_kernel3d_pk<S, TX, TY, MINB, PF, MIXED, AOS, PB>); }
    static cudaError_t step(const StepArgs& a, dim3 grid, cudaStream_t st) {
        static int attr_done = 0;
        if (!attr_done) {
            cudaError_t e = cudaFuncSetAttribute(fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(Lay::BYTES));
            if (e != cudaSuccess) return e;
            attr_done = 1;
        }
        step_kernel3d_pk<S, TX, TY, MINB, PF, MIXED, AOS, PB><<<grid, Lay::NTH, Lay::BYTES, st>>>(a);
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

// The pair kernel for the forcing scheme with 16-bit deviation storage
// (storage 2, 3), and with float32 storage at two CTAs per SM (its 82 KB of
// shared memory do not fit three; measured on GB300 at 128^3 / 256^3 / 512^3:
// 22.6 / 23.0 / 24.9 GLUPS against 19.9 / 21.2 / 22.5 for the tile kernel), in
// place of `step` of `base` (an even nx is required; base.step1, one site per
// thread, stays the fallback).  LB_D3_VARIANT selects another tile / prefetch
// form of the pair kernel for measurements; LB_D3_VARIANT=0 keeps the tile kernel.
LbKernelSet lbk_pk_forcing(int storage, int nx, LbKernelSet k) {
    const char* env = std::getenv("LB_D3_VARIANT");
    const int v = env ? std::atoi(env) : -1;
    if (v == 0) return k;
    // the interleaved 16-bit layout needs whole blocks in every row
    const bool aos = nx % AOS_SITES == 0;
    if (storage == 2) {
        switch (v) {
            case 1: PKLaunch<StF16, 64, 8, 2, 0, true>::apply(k, "pairs 64x8, mixed adds"); break;
            case 2: PKLaunch<StF16, 64, 8, 2, 2, true>::apply(k, "pairs 64x8, prefetch all, mixed adds"); break;
            case 4: PKLaunch<StF16, 64, 8, 1, 2, true>::apply(k, "pairs 64x8, one CTA per SM, prefetch all"); break;
            case 8: PKLaunch<StF16, 32, 8, 3, 2, true>::apply(k, "pairs 32x8, 3 CTAs per SM, prefetch all"); break;
            case 10: PKLaunch<StF16, 64, 12, 1, 2, true>::apply(k, "pairs 64x12, prefetch all"); break;
            case 9: PKLaunch<StF16, 32, 8, 3, 1, true>::apply(k, "pairs 32x8, 3 CTAs per SM, own pair prefetched"); break;
            case 14:
                if (aos) PKLaunch<StF16, 32, 8, 3, 2, true, true, true>::apply(k, "pairs 32x8, interleaved blocks, prefetch all");
                else PKLaunch<StF16, 32, 8, 3, 1, true>::apply(k, "pairs 32x8, 3 CTAs per SM, own pair prefetched");
                break;
            case 16:
                if (aos) PKLaunch<StF16, 64, 12, 1, 2, true, true>::apply(k, "pairs 64x12, interleaved blocks, prefetch all");
                else PKLaunch<StF16, 32, 8, 3, 1, true>::apply(k, "pairs 32x8, 3 CTAs per SM, own pair prefetched");
                break;
            case 15:
                if (aos) PKLaunch<StF16, 32, 8, 3, 1, true, true>::apply(k, "pairs 32x8, interleaved blocks, own pair prefetched");
                else PKLaunch<StF16, 32, 8, 3, 1, true>::apply(k, "pairs 32x8, 3 CTAs per SM, own pair prefetched");
                break;
            case 25:
                if (aos) PKLaunch<StF16, 32, 8, 3, 2, true, true>::apply(k, "pairs 32x8, interleaved blocks, prefetch all, stencils site by site");
                else PKLaunch<StF16, 32, 8, 3, 1, true>::apply(k, "pairs 32x8, 3 CTAs per SM, own pair prefetched");
                break;
            default:
                if (aos) PKLaunch<StF16, 32, 8, 3, 2, true, true, true>::apply(k, "pairs 32x8, interleaved blocks, prefetch all");
                else PKLaunch<StF16, 32, 8, 3, 1, true>::apply(k, "pairs 32x8, 3 CTAs per SM, own pair prefetched");
                break;
        }
    } else if (storage == 3) {
        if (aos) PKLaunch<StBF16, 32, 8, 3, 2, true, true, true>::apply(k, "pairs 32x8, interleaved blocks, prefetch all");
        else PKLaunch<StBF16, 32, 8, 3, 1, true>::apply(k, "pairs 32x8, 3 CTAs per SM, own pair prefetched");
    } else if (storage == 1) {
        if (v == 71) PKLaunch<StF32, 32, 8, 2, 1, false, false, true>::apply(k, "pairs 32x8, own pair prefetched");
        else if (v > 0 && v != 70) PKLaunch<StF32, 32, 8, 2, 0, false>::apply(k, "pairs 32x8");
        else PKLaunch<StF32, 32, 8, 2, 2, false, false, true>::apply(k, "pairs 32x8, prefetch all");
    }
    return k;
}

// First recorded index violation of this unit's kernels (checked builds; see bounds.cuh).
LB_BOUNDS_READER(lbk_bounds_d3pk)
