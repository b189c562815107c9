// Per-pixel arithmetic of one Chambolle projection iteration (Chambolle 2004, as used for the
// ROF steps of Sec. 2.2 / Sec. 4.3). Every dual-iteration kernel calls these two functions,
// and each operation is an explicitly rounded intrinsic, so the compiler cannot contract or
// reorder differently in different kernels: the result of an iteration at a pixel does not
// depend on which kernel, tile shape or launch depth computed it.
//
// Both functions are symmetric under the transposition (i <-> j, p1 <-> p2): the two
// difference terms of the divergence and the two squares of |G| are added with a commutative
// rounded addition.
#pragma once

#include <cuda_runtime.h>

namespace tvspec {

// Hardware approximate square root / reciprocal (PTX sqrt.approx, rcp.approx).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// w_ij = (div p)_ij - g_ij / lambda with
//   (div p)_ij = (p1_ij - p1_{i-1,j}) + (p2_ij - p2_{i,j-1}),
// where p1_{-1,j} = p2_{i,-1} = 0 and p1 on the last row / p2 on the last column are zero
// (the kernels keep them zero), which makes div the negative adjoint of the forward gradient.
__device__ __forceinline__ float tv_w(float p1, float p1_up, float p2, float p2_left, float gl) {
    return __fsub_rn(__fadd_rn(__fsub_rn(p1, p1_up), __fsub_rn(p2, p2_left)), gl);
}

// p <- (p + tau G) / (1 + tau |G|), |G| = sqrt(G1^2 + G2^2)  (isotropic; Eq. TV's pointwise
// Euclidean norm). The division is a multiplication by the reciprocal of the denominator.
template <bool FAST>
__device__ __forceinline__ void tv_update(float &p1, float &p2, float G1, float G2, float tau) {
    float n2 = __fadd_rn(__fmul_rn(G1, G1), __fmul_rn(G2, G2));
    float nrm = FAST ? sqrt_approx(n2) : __fsqrt_rn(n2);
    float den = __fmaf_rn(tau, nrm, 1.0f);
    float s = FAST ? rcp_approx(den) : __frcp_rn(den);
    p1 = __fmul_rn(__fmaf_rn(tau, G1, p1), s);
    p2 = __fmul_rn(__fmaf_rn(tau, G2, p2), s);
}

}  // namespace tvspec
