// Kernel instantiations for the D2Q9 lattice.
#include "kernels_impl.cuh"

using namespace lbk;

template <bool F>
static LbKernelSet pick(int storage) {
    switch (storage) {
        case 0: return Launchers<D2Q9, F, StF64, 32, 8>::make();
        case 1: return Launchers<D2Q9, F, StF32, 32, 8>::make();
        case 2: return Launchers<D2Q9, F, StF16, 32, 8>::make();
        case 3: return Launchers<D2Q9, F, StBF16, 32, 8>::make();
    }
    return LbKernelSet{};
}

LbKernelSet lbk_pk2d(int scheme, int storage, LbKernelSet k);

LbKernelSet lbk_kernels_d2q9(int scheme, int storage) {
    return lbk_pk2d(scheme, storage, scheme == 1 ? pick<true>(storage) : pick<false>(storage));
}

// First recorded index violation of this unit's kernels (checked builds; see bounds.cuh).
LB_BOUNDS_READER(lbk_bounds_d2q9)
