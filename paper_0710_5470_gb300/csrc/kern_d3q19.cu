// Kernel instantiations for the D3Q19 lattice.
#include "kernels_impl.cuh"

using namespace lbk;

template <bool F>
static LbKernelSet pick(int storage) {
    switch (storage) {
        case 0: return Launchers<D3Q19, F, StF64, 32, 4>::make();
        case 1: return Launchers<D3Q19, F, StF32, 32, 8>::make();
        case 2: return Launchers<D3Q19, F, StF16, 32, 8>::make();
        case 3: return Launchers<D3Q19, F, StBF16, 32, 8>::make();
    }
    return LbKernelSet{};
}

LbKernelSet lbk_pk_forcing(int storage, int nx, LbKernelSet base);       // kern_d3q19_pk.cu
LbKernelSet lbk_pk_equilibrium(int storage, int nx, LbKernelSet base);   // kern_d3q19_pk_eq.cu

LbKernelSet lbk_kernels_d3q19(int scheme, int storage, int nx) {
    if (scheme != 1) {
        LbKernelSet k = pick<false>(storage);
        return storage == 0 ? k : lbk_pk_equilibrium(storage, nx, k);
    }
    LbKernelSet k = pick<true>(storage);
    return storage == 0 ? k : lbk_pk_forcing(storage, nx, k);
}

// First recorded index violation of this unit's kernels (checked builds; see bounds.cuh).
LB_BOUNDS_READER(lbk_bounds_d3q19)
