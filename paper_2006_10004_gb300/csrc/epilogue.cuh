// Per-pixel float64 part of one ROF step's epilogue, shared by every kernel that finishes a
// step (the multi-block epilogue and the resident small-image kernel). Every operation is an
// explicitly rounded intrinsic so all of them produce the same bits.
#pragma once

#include "ff_math.cuh"
#include "tvspec_internal.h"

namespace tvspec {

// The four values of p that the divergence at (i, j) combines, with the negative-adjoint
// boundary terms applied: (div p)_ij = (a1 - a0) + (b1 - b0), a1 = [i<H-1] p1_ij,
// a0 = [i>0] p1_{i-1,j}, b1 = [j<W-1] p2_ij, b0 = [j>0] p2_{i,j-1}.
struct DivTerms {
    float a1, a0, b1, b0;
};

__device__ __forceinline__ DivTerms div_terms(int i, int j, int H, int W, float p1_ij, float p1_up,
                                              float p2_ij, float p2_left) {
    return {i < H - 1 ? p1_ij : 0.0f, i > 0 ? p1_up : 0.0f, j < W - 1 ? p2_ij : 0.0f,
            j > 0 ? p2_left : 0.0f};
}

// Arithmetic of the epilogue in the two modes. acc_mode 0 is float64; acc_mode 1 float-float
// (about 48 bits, on the float32 pipes: GB300's float64 rate is a small fraction of its
// float32 rate). Values of u and of the running sums are stored in 8 bytes either way.
struct F64Ops {
    using T = double;
    static __device__ __forceinline__ T add(T a, T b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ T twice(T a) { return __dmul_rn(2.0, a); }
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T of_double(double a) { return a; }
    static __device__ __forceinline__ double to_double(T a) { return a; }
    static __device__ __forceinline__ float to_float(T a) { return (float)a; }
    static __device__ __forceinline__ bool finite(T a) { return isfinite(a); }
    static __device__ __forceinline__ T load(const double *p, size_t n) { return p[n]; }
    static __device__ __forceinline__ void store(double *p, size_t n, T v) { p[n] = v; }
    static __device__ __forceinline__ T divp(const DivTerms &v) {
        return __dadd_rn(__dsub_rn((double)v.a1, (double)v.a0), __dsub_rn((double)v.b1, (double)v.b0));
    }
    static __device__ __forceinline__ T dt(const ImgDesc &d) { return d.dt; }
    static __device__ __forceinline__ T inv_dt(const ImgDesc &d) { return d.inv_dt; }
    static __device__ __forceinline__ T coef(const ImgDesc &d) { return __dmul_rn(d.inv_dt, d.inv_dt); }
    static __device__ __forceinline__ T tk(const ImgDesc &d, int k) { return __dmul_rn((double)k, d.dt); }
};

struct FFOps {
    using T = ff;
    static __device__ __forceinline__ T add(T a, T b) { return ff_add(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return ff_sub(a, b); }
    static __device__ __forceinline__ T mul(T a, T b) { return ff_mul(a, b); }
    static __device__ __forceinline__ T twice(T a) { return ff_twice(a); }
    static __device__ __forceinline__ T zero() { return ff{0.0f, 0.0f}; }
    static __device__ __forceinline__ T of_double(double a) { return ff_from_double(a); }
    static __device__ __forceinline__ double to_double(T a) { return ff_to_double(a); }
    static __device__ __forceinline__ float to_float(T a) { return ff_to_float(a); }
    static __device__ __forceinline__ bool finite(T a) { return ff_isfinite(a); }
    static __device__ __forceinline__ T load(const double *p, size_t n) {
        return reinterpret_cast<const ff *>(p)[n];
    }
    static __device__ __forceinline__ void store(double *p, size_t n, T v) { reinterpret_cast<ff *>(p)[n] = v; }
    static __device__ __forceinline__ T divp(const DivTerms &v) {
        return ff_add(ff_two_sum(v.a1, -v.a0), ff_two_sum(v.b1, -v.b0));
    }
    static __device__ __forceinline__ T dt(const ImgDesc &d) { return {d.ff_dt[0], d.ff_dt[1]}; }
    static __device__ __forceinline__ T inv_dt(const ImgDesc &d) { return {d.ff_inv_dt[0], d.ff_inv_dt[1]}; }
    static __device__ __forceinline__ T coef(const ImgDesc &d) { return {d.ff_coef[0], d.ff_coef[1]}; }
    static __device__ __forceinline__ T tk(const ImgDesc &d, int k) { return ff_mul(ff_from_float((float)k), dt(d)); }
};

// First part of step k at pixel n (compact index), given u_k = uc and div p there:
//   u_{k+1} = u_k - dt div p      (primal recovery of the ROF step, Eq. ROF)
// writes g/dt of the next step to *gl_next and u_{k+1} to the trace; returns u_{k+1}.
template <class O>
__device__ __forceinline__ typename O::T epi_primal(const ImgDesc &d, int k, size_t n,
                                                    const DivTerms &dv, typename O::T uc,
                                                    float *gl_next) {
    const typename O::T un = O::sub(uc, O::mul(O::dt(d), O::divp(dv)));
    if (!O::finite(un)) atomicOr(d.status, kStatusNonFinite);
    *gl_next = O::to_float(O::mul(un, O::inv_dt(d)));
    if (d.u_trace) d.u_trace[(size_t)(k + 1) * ((size_t)d.H * d.W) + n] = O::to_double(un);
    return un;
}

// Second part of step k >= 1 at pixel n, given u_{k-1} = up, u_k = uc, u_{k+1} = un:
//   phi_k = t_k (u_{k+1} - 2 u_k + u_{k-1}) / dt^2       (Eq. TVtrafo)
// band accumulation and flush (Eq. spectral_bands), the residual at the last step
// (Eq. finite_inverse_trafo) and the spectral filters (Eq. filteredTVtrafo). Returns |phi_k|
// and, when the Parseval-type spectrum is requested, phi_k f in *phif.
template <class O>
__device__ __forceinline__ double epi_spectral(const ImgDesc &d, int k, size_t n,
                                               typename O::T up, typename O::T uc,
                                               typename O::T un, double *phif) {
    using T = typename O::T;
    const size_t N = (size_t)d.H * d.W;
    const T tk = O::tk(d, k);
    const T d2 = O::add(O::sub(un, O::twice(uc)), up);
    const T phi = O::mul(O::mul(tk, d2), O::coef(d));
    const double phid = O::to_double(phi);
    *phif = d.S_par ? __dmul_rn(phid, (double)d.f[n]) : 0.0;
    const int m = d.band_of_k[k];
    const int mp = (k >= 2) ? d.band_of_k[k - 1] : -1;
    T acc = O::zero();
    if (mp >= 0) {
        const T old = O::load(d.acc, n);
        if (mp == m) acc = old;
        else d.bands[(size_t)mp * N + n] = O::to_float(old);  // band mp is complete
    }
    if (m >= 0) acc = O::add(acc, O::mul(phi, O::dt(d)));
    const bool last = k == d.K - 1;
    T resid = O::zero();
    if (last) resid = O::sub(uc, O::mul(O::mul(tk, O::sub(un, uc)), O::inv_dt(d)));
    if (last) {
        if (m >= 0) d.bands[(size_t)m * N + n] = O::to_float(acc);
        d.residual[n] = O::to_float(resid);
    } else {
        O::store(d.acc, n, acc);
    }
    for (int q = 0; q < d.n_filters; ++q) {
        T fa = (k >= 2) ? O::load(d.facc, (size_t)q * N + n) : O::zero();
        const T hq = O::of_double(d.filt_H[(size_t)q * (d.K - 1) + (k - 1)]);
        fa = O::add(fa, O::mul(O::mul(hq, phi), O::dt(d)));
        if (last) d.filtered[(size_t)q * N + n] = O::to_float(O::add(fa, O::mul(O::of_double(d.filt_res[q]), resid)));
        else O::store(d.facc, (size_t)q * N + n, fa);
    }
    return fabs(phid);
}

// The whole of step k at pixel n with the u ping-pong of two buffers (u_k is ua for even k,
// ub for odd k; u_{k+1} replaces u_{k-1}). Returns |phi_k| (0 at k = 0), g/dt of the next step
// in *gl_next and phi_k f in *phif (0 at k = 0).
template <class O>
__device__ __forceinline__ double epilogue_pixel_t(const ImgDesc &d, int k, size_t n,
                                                   const DivTerms &dv, float *gl_next, double *phif) {
    double *ucur = (k & 1) ? d.ub : d.ua;
    double *uoth = (k & 1) ? d.ua : d.ub;  // u_{k-1} in, u_{k+1} out
    const typename O::T uc = O::load(ucur, n);
    const typename O::T un = epi_primal<O>(d, k, n, dv, uc, gl_next);
    double absphi = 0.0;
    *phif = 0.0;
    if (k >= 1) absphi = epi_spectral<O>(d, k, n, O::load(uoth, n), uc, un, phif);
    O::store(uoth, n, un);
    return absphi;
}

__device__ __forceinline__ double epilogue_pixel(const ImgDesc &d, int k, size_t n,
                                                 const DivTerms &dv, float *gl_next, double *phif) {
    return d.acc_mode ? epilogue_pixel_t<FFOps>(d, k, n, dv, gl_next, phif)
                      : epilogue_pixel_t<F64Ops>(d, k, n, dv, gl_next, phif);
}

// The u buffer of step k in the three-buffer rotation of the split epilogue (u_{k-1}, u_k and
// u_{k+1} live at once while the spectral part of step k overlaps the next step).
__device__ __forceinline__ double *u_buf3(const ImgDesc &d, int k) {
    const int r = k % 3;
    return r == 0 ? d.ua : (r == 1 ? d.ub : d.u3);
}

// u_0 = f at pixel n (Eq. TVflow) and g/dt of step 0; returns the latter.
__device__ __forceinline__ float init_pixel(const ImgDesc &d, size_t n, float fv) {
    if (d.acc_mode) {
        reinterpret_cast<ff *>(d.ua)[n] = ff_from_float(fv);
        return ff_to_float(ff_mul(ff_from_float(fv), ff{d.ff_inv_dt[0], d.ff_inv_dt[1]}));
    }
    const double u0 = (double)fv;
    d.ua[n] = u0;
    return (float)(u0 * d.inv_dt);
}

// Fixed-order sum of one double per thread over a block of kEpBlock threads: a shuffle tree
// in every warp, then the first warp over the warp sums (zero-padded to 32 lanes).
// The result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double *s_red) {
    constexpr unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(FULL, v, off);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? s_red[lane] : 0.0;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_down_sync(FULL, t, off);
    }
    __syncthreads();
    return t;
}

}  // namespace tvspec
