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
// The iteration works on wn = -tau w, where w_ij = (div p)_ij - g_ij / lambda and
//   (div p)_ij = (p1_ij - p1_{i-1,j}) + (p2_ij - p2_{i,j-1}),
// with p1_{-1,j} = p2_{i,-1} = 0 and p1 on the last row / p2 on the last column zero (the
// kernels keep them zero), which makes div the negative adjoint of the forward gradient. The
// forward differences of wn are then na = -tau G directly, the quantity the update needs, so
// no per-pixel product by tau remains in the loop. wn is formed with one rounding from the
// divergence and glt = tau g/lambda (each kernel multiplies g/lambda by tau once, when it loads
// it): wn = fma(div p, -tau, glt). For tau a power of two (1/8 by default) scaling by tau is
// exact, so wn = -tau w and na = -tau G to the bit, as if w and G were formed first.
__device__ __forceinline__ float tv_wn(float p1, float p1_up, float p2, float p2_left, float glt,
                                       float tau) {
    return __fmaf_rn(__fadd_rn(__fsub_rn(p1, p1_up), __fsub_rn(p2, p2_left)), -tau, glt);
}

// p <- (p + tau G) / (1 + tau |G|), |G| = sqrt(G1^2 + G2^2)  (isotropic; Eq. TV's pointwise
// Euclidean norm), evaluated in float32 as an increment from na = -tau G (the differences of
// wn above):
//   a = tau G,  x = |a| = tau |G|,  s = 1 / (1 + x),  p <- p + (a - p x) s.
// The result is the same real number; the order of the float32 roundings is what differs.
// Forming 1 + tau|G| and p + tau G first rounds away whatever of tau|G| and tau G lies below
// half an ulp of 1 and of p, and where |G| is small (flat regions, most of an image near
// convergence) that loss is always in the same direction: over the tens of thousands of dual
// iterations of a decomposition it drifts p, and the bands, far more than the rounding of p
// itself. In the increment form the small quantities x and a - p x are rounded relative to
// their own size, and the fixed point (a = p x) does not involve s at all: an error in the
// reciprocal only scales the step, so the hardware approximations of the square root and the
// reciprocal (about an ulp each) are used without refinement (a float32 model of this
// arithmetic gives the same errors against the float64 oracle with exact and with 2-ulp
// one-sided biased square root and reciprocal). Signs are arranged so that no negation is
// needed: na = -a, nden = -(1 + x), ns = 1 / nden, u = p x + na = -(a - p x), and u ns is the
// increment.
template <bool FAST>
__device__ __forceinline__ void tv_update(float &p1, float &p2, float na1, float na2) {
    const float n2 = __fadd_rn(__fmul_rn(na1, na1), __fmul_rn(na2, na2));
    const float x = FAST ? sqrt_approx(n2) : __fsqrt_rn(n2);
    const float nden = __fsub_rn(-1.0f, x);
    const float ns = FAST ? rcp_approx(nden) : __frcp_rn(nden);
    p1 = __fmaf_rn(__fmaf_rn(p1, x, na1), ns, p1);
    p2 = __fmaf_rn(__fmaf_rn(p2, x, na2), ns, p2);
}

// The same update with p held as an unevaluated sum hi + lo of two floats. hi stays fixed
// between fold points; lo accumulates the increments, lo <- lo + u ns in one fused operation;
// the iteration reads the working value p = fl(hi + lo) (tv_pval), for w and for the update
// alike. At the fold points, every kFold iterations of a step and after its last, hi <- p and
// lo <- 0, so p is stored as one float per component between launches. Increments of a slowly
// converging pixel are often smaller than half an ulp of p; rounded into p alone they vanish,
// always in the same direction, and over the 25 000 dual iterations of a 2048^2 decomposition
// (K = 50 steps of 500) that alone puts u at 1.5e-4 max|f| and the bands at 1.2e-3 max|f|
// from the float64 oracle, past the accuracy target. Here they are added to lo, whose ulp is
// far below p's, and reach p through the rounding of hi + lo, so only what is left below half
// an ulp of p at a fold point is lost. (Against carrying the remainder by Fast2Sum after each
// increment it needs one rounded addition per iteration instead of three: p = fl(hi + lo) is
// the rounded sum that Fast2Sum would also leave in hi.)
template <bool FAST>
__device__ __forceinline__ void tv_update_acc(float p1, float p2, float &l1, float &l2, float na1,
                                              float na2) {
    const float n2 = __fadd_rn(__fmul_rn(na1, na1), __fmul_rn(na2, na2));
    const float x = FAST ? sqrt_approx(n2) : __fsqrt_rn(n2);
    const float nden = __fsub_rn(-1.0f, x);
    const float ns = FAST ? rcp_approx(nden) : __frcp_rn(nden);
    l1 = __fmaf_rn(__fmaf_rn(p1, x, na1), ns, l1);
    l2 = __fmaf_rn(__fmaf_rn(p2, x, na2), ns, l2);
}
// The working value of a compensated component: p = fl(hi + lo).
__device__ __forceinline__ float tv_pval(float hi, float lo) { return __fadd_rn(hi, lo); }

// ---- the same arithmetic on two pixels at once (Blackwell packed f32x2 instructions) ----
// Each lane of a packed operation rounds exactly like the scalar intrinsic above: a - b is
// computed as fma(b, -1, a), which is the correctly rounded difference, and no packed product
// feeds a packed sum (see sq_norm2). So tv_wn2d / tv_update2 give the same bits as
// tv_wn / tv_update applied to .x and .y separately.
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}

// tv_wn on a pixel pair, with the column difference of p2 already formed (d2 = p2 - p2_left):
// wn = fma((p1 - p1_up) + d2, -tau, glt), ntau2 = (-tau, -tau).
__device__ __forceinline__ float2 tv_wn2d(float2 p1, float2 p1_up, float2 d2, float2 glt,
                                          float2 ntau2) {
    return __ffma2_rn(__fadd2_rn(sub2(p1, p1_up), d2), ntau2, glt);
}

// |a|^2 = a1*a1 + a2*a2 on a pixel pair: packed products, scalar sums. A product feeding a
// sum may be fused into one multiply-add by the compiler when both are packed; with the sums
// done by the scalar rounded addition each lane equals the scalar
// __fadd_rn(__fmul_rn(a1, a1), __fmul_rn(a2, a2)), which the tests check bit for bit.
__device__ __forceinline__ float2 sq_norm2(float2 a1, float2 a2) {
    const float2 a = __fmul2_rn(a1, a1);
    const float2 b = __fmul2_rn(a2, a2);
    return make_float2(__fadd_rn(a.x, b.x), __fadd_rn(a.y, b.y));
}

template <bool FAST>
__device__ __forceinline__ void tv_update2(float2 &p1, float2 &p2, float2 na1, float2 na2) {
    const float2 n2 = sq_norm2(na1, na2);
    float2 x;
    x.x = FAST ? sqrt_approx(n2.x) : __fsqrt_rn(n2.x);
    x.y = FAST ? sqrt_approx(n2.y) : __fsqrt_rn(n2.y);
    const float2 nden = sub2(make_float2(-1.0f, -1.0f), x);
    float2 ns;
    ns.x = FAST ? rcp_approx(nden.x) : __frcp_rn(nden.x);
    ns.y = FAST ? rcp_approx(nden.y) : __frcp_rn(nden.y);
    p1 = __ffma2_rn(__ffma2_rn(p1, x, na1), ns, p1);
    p2 = __ffma2_rn(__ffma2_rn(p2, x, na2), ns, p2);
}

// tv_update_acc on a pixel pair: only lo changes; the caller refreshes p = hi + lo (packed).
template <bool FAST>
__device__ __forceinline__ void tv_update2_acc(float2 p1, float2 p2, float2 &l1, float2 &l2,
                                               float2 na1, float2 na2) {
    const float2 n2 = sq_norm2(na1, na2);
    float2 x;
    x.x = FAST ? sqrt_approx(n2.x) : __fsqrt_rn(n2.x);
    x.y = FAST ? sqrt_approx(n2.y) : __fsqrt_rn(n2.y);
    const float2 nden = sub2(make_float2(-1.0f, -1.0f), x);
    float2 ns;
    ns.x = FAST ? rcp_approx(nden.x) : __frcp_rn(nden.x);
    ns.y = FAST ? rcp_approx(nden.y) : __frcp_rn(nden.y);
    l1 = __ffma2_rn(__ffma2_rn(p1, x, na1), ns, l1);
    l2 = __ffma2_rn(__ffma2_rn(p2, x, na2), ns, l2);
}

}  // namespace tvspec
