// Batched D2Q9 sweeps: many independent lattices (own size, T, kappa, tau)
// advanced together.  A device table describes every instance; a device list
// of work items (instance, tile) drives the launches, so one launch advances
// every active instance by one time step with the same per-tile code as the
// single-lattice kernel (step2d_tile).  Every `every` steps a check kernel
// computes max |u(t) - u(t - every)| and max |u| per instance (float64), a
// finalize kernel retires converged or unstable instances and rebuilds the
// work list on the device.  No kernel waits on another CTA.
#pragma once
#include "aux_kernels.cuh"
#include "step2d_pk.cuh"

namespace lbk {

struct BatchInst {
    long long off[2];      // byte offsets of the instance's two population buffers
    long long pitch;       // elements per population array
    long long site0;       // first site of the instance in the batch-wide site numbering
    int nx, ny, tiles_x, tiles_y;
    int pair;              // two sites per halo load (nx even)
    double a, b, T, kappa, omega, nu;
    float fa, fb, fT, fkappa, fomega, fnu;   // their float32 roundings
    float pref, rsum;
};

struct BatchState {
    const BatchInst* inst;
    unsigned* items;             // (instance << 20) | tile (12 + 20 bits), active instances only
    int* count;                  // number of valid items
    int* active;                 // per instance: 1 while stepping
    unsigned int* status;        // per instance: bit 0 = non-finite density seen
    unsigned long long* maxdu;   // per instance: max |du| of the current check (double bits)
    unsigned long long* maxu;    // per instance: max |u| of the current check (double bits)
    unsigned long long* maxrho;  // per instance: max rho of the current check (double bits)
    unsigned long long* minrho;  // per instance: min rho of the current check (double bits)
    double* last;                // per instance: max |du|, max |u|, max rho, min rho of its last check
    const double* ref;           // per instance: reference max |u|, max rho, min rho (max |u| <= 0: tol test;
                                 // max rho <= 0: no density condition)
    int* inband;                 // per instance: consecutive checks inside the band
    long long* steps_done;       // per instance: steps when retired (-1 while active)
    long long* gstep;            // steps taken by the batch (device copy)
    double* uprev;               // u at the previous check, 2 per site
    int n;                       // instances
};

// The launches of a batch are sized to the CTAs the GPU holds at once, not to
// the work list: every CTA takes the items blockIdx.x, blockIdx.x + gridDim.x,
// ... below the current count, so a batch whose instances have mostly retired
// launches no CTAs that only find nothing to do.
template <bool FORCING, class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) batch_step_kernel(BatchState bs, char* buf, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned count = unsigned(*bs.count);
    for (unsigned item = blockIdx.x; item < count; item += gridDim.x) {
        const unsigned it = bs.items[item];
        const int k = int(it >> 20), t = int(it & 0xFFFFFu);
        const BatchInst& I = bs.inst[k];
        Tile2DArgs a{buf + I.off[parity], buf + I.off[1 - parity], I.pitch, I.nx, I.ny, I.pair, I.a, I.b, I.T,
                     I.kappa, I.omega, I.nu, I.fa, I.fb, I.fT, I.fkappa, I.fomega, I.fnu, I.pref, I.rsum,
                     bs.status + k};
        const int tx = I.tiles_x;
        step2d_tile<D2Q9, FORCING, S, TX, TY>(a, (t % tx) * TX, (t / tx) * TY,
                                              reinterpret_cast<typename S::real*>(smem_raw));
        __syncthreads();   // shared memory is reused by the next item
    }
}

// The same step with the pair kernel of step2d_pk.cuh ((TX / 2) * TY threads per
// tile; 32-bit arithmetic): aligned pairs for instances with an even nx.
template <bool FORCING, class S, int TX, int TY>
__global__ void __launch_bounds__((TX / 2) * TY) batch_step_kernel_pk(BatchState bs, char* buf, int parity) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const unsigned count = unsigned(*bs.count);
    for (unsigned item = blockIdx.x; item < count; item += gridDim.x) {
        const unsigned it = bs.items[item];
        const int k = int(it >> 20), t = int(it & 0xFFFFFu);
        const BatchInst& I = bs.inst[k];
        Tile2DArgs a{buf + I.off[parity], buf + I.off[1 - parity], I.pitch, I.nx, I.ny, I.pair, I.a, I.b, I.T,
                     I.kappa, I.omega, I.nu, I.fa, I.fb, I.fT, I.fkappa, I.fomega, I.fnu, I.pref, I.rsum,
                     bs.status + k};
        const int tx = I.tiles_x;
        if (I.pair) step2d_pair_tile<FORCING, S, TX, TY, true>(a, (t % tx) * TX, (t / tx) * TY, smem_raw);
        else step2d_pair_tile<FORCING, S, TX, TY, false>(a, (t % tx) * TX, (t / tx) * TY, smem_raw);
        __syncthreads();   // shared memory is reused by the next item
    }
}

// max over the tile of |u - uprev| (u = j / rho, Eq. 3), folded into maxdu[k]; uprev <- u.
template <class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) batch_check_kernel(BatchState bs, const char* buf, int parity) {
    __shared__ double red[TX * TY], redu[TX * TY], rmax[TX * TY], rmin[TX * TY];
    const unsigned count = unsigned(*bs.count);
    for (unsigned item = blockIdx.x; item < count; item += gridDim.x) {
        const unsigned it = bs.items[item];
        const int k = int(it >> 20), t = int(it & 0xFFFFFu);
        const BatchInst& I = bs.inst[k];
        const int x = (t % I.tiles_x) * TX + int(threadIdx.x) % TX;
        const int y = (t / I.tiles_x) * TY + int(threadIdx.x) / TX;
        double du = 0.0, um = 0.0, rhi = 0.0, rlo = 1e300;
        if (x < I.nx && y < I.ny) {
            const size_t q = size_t(y) * I.nx + x;
            const char* src = buf + I.off[parity];
            using L = D2Q9;
            double f[L::Q];
            f[0] = double(S::dec0(S::ld0(src, q)));
            static_for<1, L::Q>([&](auto II) {
                constexpr int i = decltype(II)::value;
                f[i] = double(S::devi(S::ldi(src + S::pop_offset(i, I.pitch), q)));
            });
            double rho = double(I.rsum) + f[0];
            for (int i = 1; i < L::Q; ++i) rho += f[i];
            double j[3];
            momentum<L, double>(f, j);
            const double ux = j[0] / rho, uy = j[1] / rho;
            double* up = bs.uprev + 2 * (I.site0 + (long long)q);
            const double dx = ux - up[0], dy = uy - up[1];
            du = sqrt(dx * dx + dy * dy);
            if (!(du <= 1e300)) du = 1e300;   // non-finite -> huge
            um = sqrt(ux * ux + uy * uy);
            if (!(um <= 1e300)) um = 1e300;
            rhi = rho > 0.0 && rho <= 1e300 ? rho : 1e300;   // non-finite or non-positive -> out of any band
            rlo = rho > 0.0 && rho <= 1e300 ? rho : 0.0;
            up[0] = ux;
            up[1] = uy;
        }
        red[threadIdx.x] = du;
        redu[threadIdx.x] = um;
        rmax[threadIdx.x] = rhi;
        rmin[threadIdx.x] = rlo;
        __syncthreads();
        for (int s = TX * TY / 2; s > 0; s >>= 1) {
            if (int(threadIdx.x) < s) {
                red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
                redu[threadIdx.x] = fmax(redu[threadIdx.x], redu[threadIdx.x + s]);
                rmax[threadIdx.x] = fmax(rmax[threadIdx.x], rmax[threadIdx.x + s]);
                rmin[threadIdx.x] = fmin(rmin[threadIdx.x], rmin[threadIdx.x + s]);
            }
            __syncthreads();
        }
        // non-negative doubles order like their bit patterns
        if (threadIdx.x == 0) {
            atomicMax(bs.maxdu + k, (unsigned long long)__double_as_longlong(red[0]));
            atomicMax(bs.maxu + k, (unsigned long long)__double_as_longlong(redu[0]));
            atomicMax(bs.maxrho + k, (unsigned long long)__double_as_longlong(rmax[0]));
            atomicMin(bs.minrho + k, (unsigned long long)__double_as_longlong(rmin[0]));
        }
        __syncthreads();   // the reduction arrays are reused by the next item
    }
}

// Retire unstable and converged instances, advance the step counter by
// `every`, and rebuild the work list of the remaining instances.  Converged:
// max |du| < tol, or, for an instance with a reference, max |u| within
// band * (its reference) of the reference and (with reference densities) max
// rho and min rho within tol_rho of theirs, for `hold` consecutive checks.
// One block; instances are visited in order, so the list is deterministic.
// Convergence check after `every` steps, per active instance, in this order:
//  - a reference set (lb_batch_set_reference): max|u| within band of it and the
//    bulk densities within tol_rho of it for `hold` consecutive checks;
//  - else, with self_rtol > 0 (lb_batch_set_self_test): the instance's own
//    observables settled - max|u| changed by at most self_rtol of itself and
//    max rho, min rho by at most self_tol_rho since the previous check, for
//    self_hold consecutive checks (needs no steady values known in advance);
//  - else max|u(t) - u(t - every)| < tol.
__global__ void batch_finalize_kernel(BatchState bs, double tol, int every, long long min_steps, double band,
                                      double tol_rho, int hold, double self_rtol, double self_tol_rho,
                                      int self_hold) {
    __shared__ int offs[1025];
    __shared__ long long g;
    if (threadIdx.x == 0) {
        *bs.gstep += every;
        g = *bs.gstep;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < bs.n; k += blockDim.x) {
        if (bs.active[k]) {
            const double du = __longlong_as_double((long long)bs.maxdu[k]);
            const double um = __longlong_as_double((long long)bs.maxu[k]);
            const double hi = __longlong_as_double((long long)bs.maxrho[k]);
            const double lo = __longlong_as_double((long long)bs.minrho[k]);
            const double prev_um = bs.last[4 * k + 1], prev_hi = bs.last[4 * k + 2], prev_lo = bs.last[4 * k + 3];
            bs.last[4 * k] = du;
            bs.last[4 * k + 1] = um;
            bs.last[4 * k + 2] = hi;
            bs.last[4 * k + 3] = lo;
            bool done = false;
            const double* r = bs.ref + 3 * k;
            if (r[0] > 0.0) {
                const bool in = fabs(um - r[0]) <= band * r[0] &&
                                (!(r[1] > 0.0) || (fabs(hi - r[1]) <= tol_rho && fabs(lo - r[2]) <= tol_rho));
                const int c = in ? bs.inband[k] + 1 : 0;
                bs.inband[k] = c;
                done = c >= hold;
            } else if (self_rtol > 0.0) {
                const bool in = fabs(um - prev_um) <= self_rtol * um && fabs(hi - prev_hi) <= self_tol_rho &&
                                fabs(lo - prev_lo) <= self_tol_rho;
                const int c = in ? bs.inband[k] + 1 : 0;
                bs.inband[k] = c;
                done = c >= self_hold;
            } else {
                done = du < tol;
            }
            if (bs.status[k] || (done && g >= min_steps)) {
                bs.active[k] = 0;
                bs.steps_done[k] = g;
            }
        }
        bs.maxdu[k] = 0ull;
        bs.maxu[k] = 0ull;
        bs.maxrho[k] = 0ull;
        bs.minrho[k] = (unsigned long long)__double_as_longlong(1e300);
    }
    __syncthreads();
    // work list: prefix sum of active tile counts, in chunks of blockDim instances
    int base = 0;
    for (int k0 = 0; k0 < bs.n; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const int ntile = (k < bs.n && bs.active[k]) ? bs.inst[k].tiles_x * bs.inst[k].tiles_y : 0;
        if (threadIdx.x == 0) offs[0] = 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int m = 0; m < int(blockDim.x) && k0 + m < bs.n; ++m) {
                const int kk = k0 + m;
                acc += bs.active[kk] ? bs.inst[kk].tiles_x * bs.inst[kk].tiles_y : 0;
                offs[m + 1] = acc;
            }
        }
        __syncthreads();
        if (k < bs.n)
            for (int tt = 0; tt < ntile; ++tt) bs.items[base + offs[threadIdx.x] + tt] = (unsigned(k) << 20) | unsigned(tt);
        __syncthreads();
        const int chunk = offs[min(int(blockDim.x), bs.n - k0)];
        base += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) *bs.count = base;
}

}  // namespace lbk
