// Launchers of every kernel for one (lattice, scheme, storage, tile)
// combination; included by one translation unit per lattice.
#pragma once
#include "dispatch.h"
#include "step3d.cuh"

namespace lbk {

// Fused step kernel of a lattice: the z-split kernel for D3Q19 (PAIR: two
// sites per stage-A load, even nx only), the generic single-plane kernel for
// D2Q9 (PAIR ignored).
template <class L, bool FORCING, class S, int TX, int TY, bool PAIR = false>
struct StepKernelOf {
    using real = typename S::real;
    static constexpr bool D3 = L::D == 3;
    static constexpr size_t bytes() {
        if constexpr (D3) return Layout3D<FORCING, TX, TY, real, sizeof(typename S::rawi) == 2>::BYTES;
        else return StepLayout<L, FORCING, TX, TY, real>::BYTES;
    }
    static const void* fn() {
        if constexpr (D3) return reinterpret_cast<const void*>(step_kernel3d<FORCING, S, TX, TY, PAIR>);
        else return reinterpret_cast<const void*>(step_kernel<L, FORCING, S, TX, TY>);
    }
    static void launch(dim3 grid, cudaStream_t st, const StepArgs& a) {
        if constexpr (D3) {
            step_kernel3d<FORCING, S, TX, TY, PAIR><<<grid, TX * TY, bytes(), st>>>(a);
        } else {
            Tile2DArgs t{a.src_base, a.dst_base, a.pitch, a.nx, a.ny, a.pair2d, a.a, a.b, a.T, a.kappa, a.omega,
                         a.nu, a.fa, a.fb, a.fT, a.fkappa, a.fomega, a.fnu, a.pref, a.rsum, a.status};
            step_kernel<L, FORCING, S, TX, TY><<<grid, TX * TY, bytes(), st>>>(t);
        }
    }
};

template <class L, bool FORCING, class S, int TX, int TY>
struct Launchers {
    using real = typename S::real;
    // paired stage A for D3Q19 with 32-bit arithmetic (float64 is bound by its
    // arithmetic and would spill with twice the halo registers)
    static constexpr bool PAIRED = L::D == 3 && sizeof(real) == 4;
    using K = StepKernelOf<L, FORCING, S, TX, TY, PAIRED>;
    using K1 = StepKernelOf<L, FORCING, S, TX, TY, false>;       // one site per stage-A item

    template <class KK>
    static cudaError_t launch_step(const StepArgs& a, dim3 grid, cudaStream_t st) {
        static int attr_done = 0;
        if (!attr_done) {
            cudaError_t e = cudaFuncSetAttribute(KK::fn(), cudaFuncAttributeMaxDynamicSharedMemorySize, int(KK::bytes()));
            if (e != cudaSuccess) return e;
            attr_done = 1;
        }
        KK::launch(grid, st, a);
        return cudaGetLastError();
    }
    static cudaError_t step(const StepArgs& a, dim3 grid, cudaStream_t st) { return launch_step<K>(a, grid, st); }
    static cudaError_t step1(const StepArgs& a, dim3 grid, cudaStream_t st) { return launch_step<K1>(a, grid, st); }
    static cudaError_t init_feq(const double* rho, const double* u, const PopPtrs& p, Grid3 g, Phys ph,
                                cudaStream_t st) {
        const size_t n = size_t(g.nx) * g.ny * g.nz;
        init_feq_kernel<L, FORCING, S><<<lbk_aux_blocks(n), 256, 0, st>>>(rho, u, p, g, ph);
        return cudaGetLastError();
    }
    static cudaError_t moments(const PopPtrs& p, Grid3 g, double* rho, double* u, cudaStream_t st) {
        const size_t n = size_t(g.nx) * g.ny * g.nz;
        moments_kernel<L, S><<<lbk_aux_blocks(n), 256, 0, st>>>(p, g, rho, u);
        return cudaGetLastError();
    }
    static cudaError_t mprime(const double* rho, Grid3 g, double kappa, double* mp, cudaStream_t st) {
        const size_t n = size_t(g.nx) * g.ny * g.nz;
        mprime_kernel<L><<<lbk_aux_blocks(n), 256, 0, st>>>(rho, g, kappa, mp);
        return cudaGetLastError();
    }
    static cudaError_t velocity_v(const double* rho, const double* u, const double* mp, Grid3 g, double* v,
                                  cudaStream_t st) {
        const size_t n = size_t(g.nx) * g.ny * g.nz;
        velocity_v_kernel<L><<<lbk_aux_blocks(n), 256, 0, st>>>(rho, u, mp, g, v);
        return cudaGetLastError();
    }
    static cudaError_t get_box(const PopPtrs& p, Grid3 g, const int (&o)[3], const int (&b)[3], double* out,
                               cudaStream_t st) {
        const size_t n = size_t(b[0]) * b[1] * b[2];
        get_box_kernel<L, S><<<lbk_aux_blocks(n), 256, 0, st>>>(p, g, o[0], o[1], o[2], b[0], b[1], b[2], out);
        return cudaGetLastError();
    }
    static cudaError_t get_pops(const PopPtrs& p, size_t n, double* out, cudaStream_t st) {
        get_pops_kernel<L, S><<<lbk_aux_blocks(n), 256, 0, st>>>(p, n, out);
        return cudaGetLastError();
    }
    static cudaError_t set_pops(const PopPtrs& p, size_t n, const double* in, cudaStream_t st) {
        set_pops_kernel<L, S><<<lbk_aux_blocks(n), 256, 0, st>>>(p, n, in);
        return cudaGetLastError();
    }
    static LbKernelSet make() {
        LbKernelSet k;
        k.tx = k.tx1 = TX;
        k.ty = k.ty1 = TY;
        k.threads = k.threads1 = TX * TY;
        k.smem = K::bytes();
        k.smem1 = K1::bytes();
        k.name = PAIRED ? "tile, two sites per halo load" : "tile, one site per thread";
        k.name1 = "tile, one site per thread";
        k.step_fn = K::fn();
        k.step = &step;
        k.step1_fn = K1::fn();
        k.step1 = &step1;
        k.step_pair_needs_even_nx = PAIRED;
        k.init_feq = &init_feq;
        k.moments = &moments;
        k.mprime = &mprime;
        k.velocity_v = &velocity_v;
        k.get_pops = &get_pops;
        k.get_box = &get_box;
        k.set_pops = &set_pops;
        return k;
    }
};

}  // namespace lbk
