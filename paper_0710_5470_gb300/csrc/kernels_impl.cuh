// Launchers of every kernel for one (lattice, scheme, storage, tile)
// combination; included by one translation unit per lattice.
#pragma once
#include "dispatch.h"

namespace lbk {

template <class L, bool FORCING, class S, int TX, int TY>
struct Launchers {
    using real = typename S::real;
    using Lay = StepLayout<L, FORCING, TX, TY, real>;

    static cudaError_t step(const StepArgs& a, dim3 grid, cudaStream_t st) {
        static int attr_done = 0;
        if (!attr_done) {
            cudaError_t e = cudaFuncSetAttribute(step_kernel<L, FORCING, S, TX, TY>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(Lay::BYTES));
            if (e != cudaSuccess) return e;
            attr_done = 1;
        }
        step_kernel<L, FORCING, S, TX, TY><<<grid, TX * TY, Lay::BYTES, st>>>(a);
        return cudaGetLastError();
    }
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
        k.tx = TX;
        k.ty = TY;
        k.smem = Lay::BYTES;
        k.step_fn = reinterpret_cast<const void*>(step_kernel<L, FORCING, S, TX, TY>);
        k.step = &step;
        k.init_feq = &init_feq;
        k.moments = &moments;
        k.mprime = &mprime;
        k.velocity_v = &velocity_v;
        k.get_pops = &get_pops;
        k.set_pops = &set_pops;
        return k;
    }
};

}  // namespace lbk
