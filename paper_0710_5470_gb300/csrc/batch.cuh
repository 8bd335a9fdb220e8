// Batched D2Q9 sweeps: many independent lattices (own size, T, kappa, tau)
// advanced together.  A device table describes every instance; a device list
// of work items (instance, tile) drives the launches, so one launch advances
// every active instance by one time step with the same per-tile code as the
// single-lattice kernel (step2d_tile).  Every `every` steps a check kernel
// computes max |u(t) - u(t - every)| per instance (float64), a finalize
// kernel retires converged or unstable instances and rebuilds the work list
// on the device.  No kernel waits on another CTA.
#pragma once
#include "aux_kernels.cuh"

namespace lbk {

struct BatchInst {
    long long off[2];      // byte offsets of the instance's two population buffers
    long long pitch;       // elements per population array
    long long site0;       // first site of the instance in the batch-wide site numbering
    int nx, ny, tiles_x, tiles_y;
    double a, b, T, kappa, omega, nu;
    float pref, rsum;
};

struct BatchState {
    const BatchInst* inst;
    int* items;                  // (instance << 20) | tile, active instances only
    int* count;                  // number of valid items
    int* active;                 // per instance: 1 while stepping
    unsigned int* status;        // per instance: bit 0 = non-finite density seen
    unsigned long long* maxdu;   // per instance: max |du| of the current check (double bits)
    long long* steps_done;       // per instance: steps when retired (-1 while active)
    long long* gstep;            // steps taken by the batch (device copy)
    double* uprev;               // u at the previous check, 2 per site
    int n;                       // instances
};

template <bool FORCING, class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) batch_step_kernel(BatchState bs, char* buf, int parity) {
    if (blockIdx.x >= *bs.count) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int it = bs.items[blockIdx.x];
    const int k = it >> 20, t = it & 0xFFFFF;
    const BatchInst& I = bs.inst[k];
    Tile2DArgs a{buf + I.off[parity], buf + I.off[1 - parity], I.pitch, I.nx, I.ny, I.a, I.b, I.T, I.kappa,
                 I.omega, I.nu, I.pref, I.rsum, bs.status + k};
    const int tx = I.tiles_x;
    step2d_tile<D2Q9, FORCING, S, TX, TY>(a, (t % tx) * TX, (t / tx) * TY,
                                          reinterpret_cast<typename S::real*>(smem_raw));
}

// max over the tile of |u - uprev| (u = j / rho, Eq. 3), folded into maxdu[k]; uprev <- u.
template <class S, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) batch_check_kernel(BatchState bs, const char* buf, int parity) {
    if (blockIdx.x >= *bs.count) return;
    __shared__ double red[TX * TY];
    const int it = bs.items[blockIdx.x];
    const int k = it >> 20, t = it & 0xFFFFF;
    const BatchInst& I = bs.inst[k];
    const int x = (t % I.tiles_x) * TX + int(threadIdx.x) % TX;
    const int y = (t / I.tiles_x) * TY + int(threadIdx.x) / TX;
    double du = 0.0;
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
        up[0] = ux;
        up[1] = uy;
    }
    red[threadIdx.x] = du;
    __syncthreads();
    for (int s = TX * TY / 2; s > 0; s >>= 1) {
        if (int(threadIdx.x) < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(bs.maxdu + k, (unsigned long long)__double_as_longlong(red[0]));
}

// Retire converged (max |du| < tol) and unstable instances, advance the step
// counter by `every`, and rebuild the work list of the remaining instances.
// One block; instances are visited in order, so the list is deterministic.
__global__ void batch_finalize_kernel(BatchState bs, double tol, int every, long long min_steps) {
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
            if (bs.status[k]) {
                bs.active[k] = 0;
                bs.steps_done[k] = g;
            } else if (du < tol && g >= min_steps) {
                bs.active[k] = 0;
                bs.steps_done[k] = g;
            }
        }
        bs.maxdu[k] = 0ull;
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
            for (int tt = 0; tt < ntile; ++tt) bs.items[base + offs[threadIdx.x] + tt] = (k << 20) | tt;
        __syncthreads();
        const int chunk = offs[min(int(blockDim.x), bs.n - k0)];
        base += chunk;
        __syncthreads();
    }
    if (threadIdx.x == 0) *bs.count = base;
}

}  // namespace lbk
