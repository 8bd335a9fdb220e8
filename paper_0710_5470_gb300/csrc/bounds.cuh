// Optional index checks of the step kernels (compile with -DLB_DEBUG_BOUNDS).
//
// In a checked build every global population access of the fused step kernels
// tests its site index against the lattice before it happens.  A failed test
// skips the access (a load returns zero) and records the first violation of
// the translation unit in a device word: bit 63 set, the access kind in bits
// 48..55, the offending site index in bits 0..47.  Nothing traps: the host
// reads and clears the word with lb_debug_bounds.  In an ordinary build the
// test is the constant true and costs nothing.
#pragma once
#include <cuda_runtime.h>

namespace lbk {

// kinds of checked access
enum BoundsKind : unsigned {
    BK_PK_LOAD = 1,     // pair kernel: halo / own-pair population loads
    BK_PK_STORE = 2,    // pair kernel: push stores
    BK_PK_SHARED = 3,   // pair kernel: density / M' shared-memory writes
    BK_3D_LOAD = 4,     // D3Q19 tile kernel loads
    BK_3D_STORE = 5,    // D3Q19 tile kernel push stores
    BK_2D_LOAD = 6,     // D2Q9 tile (single lattice and batch) loads
    BK_2D_STORE = 7,    // D2Q9 tile push stores
    BK_2D_SHARED = 8,   // D2Q9 pair kernel: M' shared-memory writes
};

#ifdef LB_DEBUG_BOUNDS
constexpr bool kBoundsChecked = true;
// one word per translation unit (static): each unit reads and clears its own
static __device__ unsigned long long g_bounds_violation;

__device__ __forceinline__ bool in_bounds(bool ok, unsigned kind, unsigned long long index) {
    if (!ok)
        atomicCAS(&g_bounds_violation, 0ull,
                  (1ull << 63) | ((unsigned long long)(kind & 0xffu) << 48) | (index & 0xffffffffffffull));
    return ok;
}
#else
constexpr bool kBoundsChecked = false;
__device__ __forceinline__ constexpr bool in_bounds(bool, unsigned, unsigned long long) { return true; }
#endif

}  // namespace lbk

// LB_GUARD(cond, kind, index, on_fail): in a checked build, when cond is false
// record the violation and run on_fail (skip the access); in an ordinary build
// it expands to nothing, so the kernels compile exactly as without checks.
#ifdef LB_DEBUG_BOUNDS
#define LB_GUARD(cond, kind, index, ...) \
    if (!lbk::in_bounds((cond), (kind), (unsigned long long)(index))) { __VA_ARGS__; }
#else
#define LB_GUARD(cond, kind, index, ...)
#endif

// Defines `unsigned long long NAME()`: the first violation recorded by this
// translation unit's kernels (0 if none, always 0 in an unchecked build), and
// clears it.  Synchronises the device.
#ifdef LB_DEBUG_BOUNDS
#define LB_BOUNDS_READER(NAME)                                                                  \
    unsigned long long NAME() {                                                                 \
        unsigned long long v = 0, zero = 0;                                                     \
        if (cudaMemcpyFromSymbol(&v, lbk::g_bounds_violation, sizeof(v)) != cudaSuccess) return 0; \
        cudaMemcpyToSymbol(lbk::g_bounds_violation, &zero, sizeof(zero));                       \
        return v;                                                                               \
    }
#else
#define LB_BOUNDS_READER(NAME) \
    unsigned long long NAME() { return 0; }
#endif
