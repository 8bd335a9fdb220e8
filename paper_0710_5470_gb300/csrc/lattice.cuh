// Lattice traits of the D2Q9 and D3Q19 velocity sets and the weights of the
// tuned equilibrium (Pooley & Furtado, Sec. II, Sec. III, Sec. VII).
//
// Velocity order follows the paper: D2Q9 e_0 = 0, e_{1,2} = (+-1,0),
// e_{3,4} = (0,+-1), e_{5,6} = (+-1,+-1), e_{7,8} = (-+1,+-1) (Sec. II);
// D3Q19 e_{1-6} along the axes, e_{7-18} the twelve diagonals in the column
// order printed in Sec. VII.
//
// Every weight is a function of the velocity vector, evaluated at compile
// time inside fully unrolled loops:
//   w_i          1/3 (2D) or 1/6 (3D) on axis directions, 1/12 on diagonals
//                (Eq. 5 text; Eq. 31 with w_{1-6} = 1/6, the value the second
//                moment of Eq. 34 requires);
//   w^p_i = w^t_i = w_i                 (optimum, Sec. III / Eq. 31);
//   w^aa_i  axis along a: 1/3 (2D) or 5/12 (3D; Eq. 34 needs
//                sum_i w^aa_i e_ia^2 = 1/2); other axis: -1/6 (2D) or -1/3 (3D);
//                diagonal touching a: -1/24; diagonal not touching a: 1/12 (3D);
//   w^ab_i  (a != b)  sign(e_ia e_ib)/4 on diagonals of the ab plane, else 0.
// With these weights sum_i w_i e_ia rho(r+e_i) and 2 sum_i w_i (rho(r+e_i) -
// rho(r)) are exactly the gradient and Laplacian stencils of Eq. 32 (2D) and
// Eq. 29 with A = 1/6, B = 1/12, C = 1/3, D = 1/6 (3D), so the kernels use
// that form for both.
#pragma once
#include <type_traits>

namespace lbk {

// Compile-time loop: calls f(std::integral_constant<int, k>) for k in [B, E),
// so that velocity components and weights are constant expressions inside f.
template <int B, int E, class F>
__host__ __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}


struct D2Q9 {
    static constexpr int D = 2;
    static constexpr int Q = 9;
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[9] = {0, 1, -1, 0, 0, 1, -1, -1, 1};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[9] = {0, 0, 0, 1, -1, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int) { return 0; }
};

struct D3Q19 {
    static constexpr int D = 3;
    static constexpr int Q = 19;
    __host__ __device__ static constexpr int ex(int i) {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int ey(int i) {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int ez(int i) {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
        return t[i];
    }
};

template <class L>
__host__ __device__ constexpr int e_comp(int i, int a) {
    return a == 0 ? L::ex(i) : (a == 1 ? L::ey(i) : L::ez(i));
}

template <class L>
__host__ __device__ constexpr int e_norm2(int i) {
    return L::ex(i) * L::ex(i) + L::ey(i) * L::ey(i) + L::ez(i) * L::ez(i);
}

// w_i of the velocity part (and w^p_i = w^t_i at the optimum).
template <class L>
__host__ __device__ constexpr double w_vel(int i) {
    return i == 0 ? 0.0 : (e_norm2<L>(i) == 1 ? (L::D == 2 ? 1.0 / 3.0 : 1.0 / 6.0) : 1.0 / 12.0);
}

// w^{ab}_i of the M_ab = kappa d_a rho d_b rho terms (a <= b).
template <class L>
__host__ __device__ constexpr double w_m(int i, int a, int b) {
    if (i == 0) return 0.0;
    const int ea = e_comp<L>(i, a), eb = e_comp<L>(i, b);
    if (a != b) return (e_norm2<L>(i) == 2) ? 0.25 * ea * eb : 0.0;
    if (e_norm2<L>(i) == 1) {                    // axis direction
        if (ea != 0) return L::D == 2 ? 1.0 / 3.0 : 5.0 / 12.0;
        return L::D == 2 ? -1.0 / 6.0 : -1.0 / 3.0;
    }
    return ea != 0 ? -1.0 / 24.0 : 1.0 / 12.0;  // diagonal
}

// First and second nonzero component of e_i (-1 if none).
template <class L>
__host__ __device__ constexpr int first_axis(int i) {
    return L::ex(i) != 0 ? 0 : (L::ey(i) != 0 ? 1 : (L::ez(i) != 0 ? 2 : -1));
}
template <class L>
__host__ __device__ constexpr int second_axis(int i) {
    const int a = first_axis<L>(i);
    for (int c = a + 1; c < 3; ++c)
        if (e_comp<L>(i, c) != 0) return c;
    return -1;
}

// Index of the opposite velocity -e_i.
template <class L>
__host__ __device__ constexpr int opposite(int i) {
    int r = 0;
    for (int k = 0; k < L::Q; ++k)
        if (L::ex(k) == -L::ex(i) && L::ey(k) == -L::ey(i) && L::ez(k) == -L::ez(i)) r = k;
    return r;
}

}  // namespace lbk
