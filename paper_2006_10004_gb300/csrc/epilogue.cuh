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

// Step k at pixel n (compact index) given div p there:
//   u_{k+1} = u_k - dt div p                                    (primal recovery, Eq. ROF)
//   phi_k   = t_k (u_{k+1} - 2 u_k + u_{k-1}) / dt^2, k >= 1       (Eq. TVtrafo)
//   band accumulation, band flush and residual at the last step (Eq. spectral_bands,
//   Eq. finite_inverse_trafo), spectral filters (Eq. filteredTVtrafo); u_{k+1} replaces
//   u_{k-1} in the ping-pong buffer.
// Returns |phi_k| (0 at k = 0), g/dt of the next step in *gl_next and, when the Parseval-type
// spectrum is requested, phi_k f in *phif (0 at k = 0).
// acc_mode 0 computes in float64; acc_mode 1 in float-float (about 48 bits, on the float32
// pipes: GB300's float64 rate is a small fraction of its float32 rate). |phi| and phi f are
// returned as float64 either way; the S reductions are float64.
__device__ __forceinline__ double epilogue_pixel_f64(const ImgDesc &d, int k, size_t n,
                                                     const DivTerms &dv, float *gl_next,
                                                     double *phif) {
    const size_t N = (size_t)d.H * d.W;
    const double divp = __dadd_rn(__dsub_rn((double)dv.a1, (double)dv.a0),
                                  __dsub_rn((double)dv.b1, (double)dv.b0));
    double *ucur = (k & 1) ? d.ub : d.ua;
    double *uoth = (k & 1) ? d.ua : d.ub;  // u_{k-1} in, u_{k+1} out
    const double uc = ucur[n];
    const double un = __dsub_rn(uc, __dmul_rn(d.dt, divp));
    if (!isfinite(un)) atomicOr(d.status, kStatusNonFinite);
    *gl_next = (float)__dmul_rn(un, d.inv_dt);
    if (d.u_trace) d.u_trace[(size_t)(k + 1) * N + n] = un;
    double absphi = 0.0;
    *phif = 0.0;
    if (k >= 1) {
        const double up = uoth[n];
        const double tk = __dmul_rn((double)k, d.dt);
        const double d2 = __dadd_rn(__dsub_rn(un, __dmul_rn(2.0, uc)), up);
        const double phi = __dmul_rn(__dmul_rn(tk, d2), __dmul_rn(d.inv_dt, d.inv_dt));
        absphi = fabs(phi);
        if (d.S_par) *phif = __dmul_rn(phi, (double)d.f[n]);
        const int m = d.band_of_k[k];
        const int mp = (k >= 2) ? d.band_of_k[k - 1] : -1;
        double acc = 0.0;
        if (mp >= 0) {
            const double old = d.acc[n];
            if (mp == m) acc = old;
            else d.bands[(size_t)mp * N + n] = (float)old;  // band mp is complete
        }
        if (m >= 0) acc = __dadd_rn(acc, __dmul_rn(phi, d.dt));
        const bool last = k == d.K - 1;
        const double resid =
            last ? __dsub_rn(uc, __dmul_rn(__dmul_rn(tk, __dsub_rn(un, uc)), d.inv_dt)) : 0.0;
        if (last) {
            if (m >= 0) d.bands[(size_t)m * N + n] = (float)acc;
            d.residual[n] = (float)resid;
        } else {
            d.acc[n] = acc;
        }
        // spectral filters: sum_k H_q(t_k) phi_k dt + h_q f_r   (Eq. filteredTVtrafo)
        for (int q = 0; q < d.n_filters; ++q) {
            double fa = (k >= 2) ? d.facc[(size_t)q * N + n] : 0.0;
            fa = __dadd_rn(fa, __dmul_rn(__dmul_rn(d.filt_H[(size_t)q * (d.K - 1) + (k - 1)], phi), d.dt));
            if (last) d.filtered[(size_t)q * N + n] = (float)__dadd_rn(fa, __dmul_rn(d.filt_res[q], resid));
            else d.facc[(size_t)q * N + n] = fa;
        }
    }
    uoth[n] = un;
    return absphi;
}

__device__ __forceinline__ double epilogue_pixel_ff(const ImgDesc &d, int k, size_t n,
                                                    const DivTerms &dv, float *gl_next,
                                                    double *phif) {
    const size_t N = (size_t)d.H * d.W;
    const ff dt = {d.ff_dt[0], d.ff_dt[1]};
    const ff inv_dt = {d.ff_inv_dt[0], d.ff_inv_dt[1]};
    const ff coef = {d.ff_coef[0], d.ff_coef[1]};
    const ff divp = ff_add(ff_two_sum(dv.a1, -dv.a0), ff_two_sum(dv.b1, -dv.b0));
    ff *ucur = reinterpret_cast<ff *>((k & 1) ? d.ub : d.ua);
    ff *uoth = reinterpret_cast<ff *>((k & 1) ? d.ua : d.ub);
    ff *accv = reinterpret_cast<ff *>(d.acc);
    ff *faccv = reinterpret_cast<ff *>(d.facc);
    const ff uc = ucur[n];
    const ff un = ff_sub(uc, ff_mul(dt, divp));
    if (!ff_isfinite(un)) atomicOr(d.status, kStatusNonFinite);
    *gl_next = ff_to_float(ff_mul(un, inv_dt));
    if (d.u_trace) d.u_trace[(size_t)(k + 1) * N + n] = ff_to_double(un);
    double absphi = 0.0;
    *phif = 0.0;
    if (k >= 1) {
        const ff up = uoth[n];
        const ff tk = ff_mul(ff_from_float((float)k), dt);
        const ff d2 = ff_add(ff_sub(un, ff_twice(uc)), up);
        const ff phi = ff_mul(ff_mul(tk, d2), coef);
        const double phid = ff_to_double(phi);
        absphi = fabs(phid);
        if (d.S_par) *phif = __dmul_rn(phid, (double)d.f[n]);
        const int m = d.band_of_k[k];
        const int mp = (k >= 2) ? d.band_of_k[k - 1] : -1;
        ff acc = {0.0f, 0.0f};
        if (mp >= 0) {
            const ff old = accv[n];
            if (mp == m) acc = old;
            else d.bands[(size_t)mp * N + n] = ff_to_float(old);  // band mp is complete
        }
        if (m >= 0) acc = ff_add(acc, ff_mul(phi, dt));
        const bool last = k == d.K - 1;
        ff resid = {0.0f, 0.0f};
        if (last) resid = ff_sub(uc, ff_mul(ff_mul(tk, ff_sub(un, uc)), inv_dt));
        if (last) {
            if (m >= 0) d.bands[(size_t)m * N + n] = ff_to_float(acc);
            d.residual[n] = ff_to_float(resid);
        } else {
            accv[n] = acc;
        }
        for (int q = 0; q < d.n_filters; ++q) {
            ff fa = (k >= 2) ? faccv[(size_t)q * N + n] : ff{0.0f, 0.0f};
            const ff hq = ff_from_double(d.filt_H[(size_t)q * (d.K - 1) + (k - 1)]);
            fa = ff_add(fa, ff_mul(ff_mul(hq, phi), dt));
            if (last)
                d.filtered[(size_t)q * N + n] =
                    ff_to_float(ff_add(fa, ff_mul(ff_from_double(d.filt_res[q]), resid)));
            else
                faccv[(size_t)q * N + n] = fa;
        }
    }
    uoth[n] = un;
    return absphi;
}

__device__ __forceinline__ double epilogue_pixel(const ImgDesc &d, int k, size_t n,
                                                 const DivTerms &dv, float *gl_next, double *phif) {
    return d.acc_mode ? epilogue_pixel_ff(d, k, n, dv, gl_next, phif)
                      : epilogue_pixel_f64(d, k, n, dv, gl_next, phif);
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
