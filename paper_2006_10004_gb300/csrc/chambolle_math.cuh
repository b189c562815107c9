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

// Programmatic dependent launch: wait until the preceding grid has completed and its memory
// is visible (a no-op when the launch has no programmatic dependency), and allow the next
// grid in the stream to be scheduled while this one runs.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

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
// The hardware reciprocal refined by one Newton-Raphson step, s1 = s0 + s0 (1 - x s0) (two
// fused multiply-adds). The raw approximation's error is not zero-mean, and over thousands of
// dual iterations it drifts p measurably; after the step the error is about an ulp.
__device__ __forceinline__ float rcp_fast(float x) {
    const float s0 = rcp_approx(x);
    return __fmaf_rn(s0, __fmaf_rn(-x, s0, 1.0f), s0);
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
    float s = FAST ? rcp_fast(den) : __frcp_rn(den);
    p1 = __fmul_rn(__fmaf_rn(tau, G1, p1), s);
    p2 = __fmul_rn(__fmaf_rn(tau, G2, p2), s);
}

// ---- the same arithmetic on two pixels at once (Blackwell packed f32x2 instructions) ----
// Each lane of a packed operation rounds exactly like the scalar intrinsic above: a - b is
// computed as fma(b, -1, a), which is the correctly rounded difference, and no packed product
// feeds a packed sum (see sq_norm2). So tv_w2 / tv_update2 give the same bits as
// tv_w / tv_update applied to .x and .y separately.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

__device__ __forceinline__ float2 tv_w2(float2 p1, float2 p1_up, float2 p2, float2 p2_left,
                                        float2 gl) {
    return sub2(__fadd2_rn(sub2(p1, p1_up), sub2(p2, p2_left)), gl);
}

// |G|^2 = G1*G1 + G2*G2 on a pixel pair: packed products, scalar sums. A product feeding a
// sum may be fused into one multiply-add by the compiler when both are packed; with the sums
// done by the scalar rounded addition each lane equals the scalar
// __fadd_rn(__fmul_rn(G1, G1), __fmul_rn(G2, G2)), which the tests check bit for bit.
__device__ __forceinline__ float2 sq_norm2(float2 G1, float2 G2) {
    const float2 a = __fmul2_rn(G1, G1);
    const float2 b = __fmul2_rn(G2, G2);
    return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}

template <bool FAST>
__device__ __forceinline__ void tv_update2(float2 &p1, float2 &p2, float2 G1, float2 G2,
                                           float tau) {
    const float2 n2 = sq_norm2(G1, G2);
    float2 nrm;
    nrm.x = FAST ? sqrt_approx(n2.x) : __fsqrt_rn(n2.x);
    nrm.y = FAST ? sqrt_approx(n2.y) : __fsqrt_rn(n2.y);
    const float2 t2 = make_float2(tau, tau);
    const float2 den = __ffma2_rn(t2, nrm, make_float2(1.0f, 1.0f));
    float2 s;
    s.x = FAST ? rcp_fast(den.x) : __frcp_rn(den.x);
    s.y = FAST ? rcp_fast(den.y) : __frcp_rn(den.y);
    p1 = __fmul2_rn(__ffma2_rn(t2, G1, p1), s);
    p2 = __fmul2_rn(__ffma2_rn(t2, G2, p2), s);
}

}  // namespace tvspec
