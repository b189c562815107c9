// Per-pixel float64 part of one ROF step's epilogue, shared by every kernel that finishes a
// step (the multi-block epilogue and the resident small-image kernel). Every operation is an
// explicitly rounded intrinsic so all of them produce the same bits.
#pragma once

#include "tvspec_internal.h"

namespace tvspec {

// Divergence at (i, j) from float values of p with the negative-adjoint boundary terms:
//   (div p)_ij = ([i<H-1] p1_ij - [i>0] p1_{i-1,j}) + ([j<W-1] p2_ij - [j>0] p2_{i,j-1}).
__device__ __forceinline__ double div_at(int i, int j, int H, int W, float p1_ij, float p1_up,
                                         float p2_ij, float p2_left) {
    const double a = __dsub_rn(i < H - 1 ? (double)p1_ij : 0.0, i > 0 ? (double)p1_up : 0.0);
    const double c = __dsub_rn(j < W - 1 ? (double)p2_ij : 0.0, j > 0 ? (double)p2_left : 0.0);
    return __dadd_rn(a, c);
}

// Step k at pixel n (compact index) given div p there:
//   u_{k+1} = u_k - dt div p                                    (primal recovery, Eq. ROF)
//   phi_k   = t_k (u_{k+1} - 2 u_k + u_{k-1}) / dt^2, k >= 1       (Eq. TVtrafo)
//   band accumulation, band flush and residual at the last step (Eq. spectral_bands,
//   Eq. finite_inverse_trafo), spectral filters (Eq. filteredTVtrafo); u_{k+1} replaces
//   u_{k-1} in the ping-pong buffer.
// Returns |phi_k| (0 at k = 0), g/dt of the next step in *gl_next and, when the Parseval-type
// spectrum is requested, phi_k f in *phif (0 at k = 0).
__device__ __forceinline__ double epilogue_pixel(const ImgDesc &d, int k, size_t n, double divp,
                                                 float *gl_next, double *phif) {
    const size_t N = (size_t)d.H * d.W;
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
