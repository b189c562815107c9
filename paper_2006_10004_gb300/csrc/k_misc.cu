// Kernels around the hot loop: the reference one-iteration kernel, the start of a
// decomposition, the per-step float64 epilogue and the standalone ROF helpers.
#include <algorithm>
#include <cstring>

#include "chambolle_math.cuh"
#include "epilogue.cuh"
#include "tvspec_internal.h"

namespace tvspec {

// ---------------------------------------------------------------------------------------------
// Reference dual-iteration kernel: one Chambolle iteration per launch, one thread per pixel,
// neighbours read from global memory, p_in -> p_out (Chambolle 2004 as used in Sec. 4.3).
// ---------------------------------------------------------------------------------------------
// Float32 storage: p is updated in the compensated form as hi + lo, with lo carried between
// launches in q1 / q2 (in -> out) and folded into hi at the fold points (kFold), exactly as the
// tiled kernels do in registers; `it` is the iteration's index within the step of n_total. hi
// (p1 / p2) changes only at the fold points.
template <typename P, bool FAST>
__global__ void __launch_bounds__(256)
    k_naive(const P *__restrict__ p1i, const P *__restrict__ p2i, P *__restrict__ p1o,
            P *__restrict__ p2o, const float *__restrict__ q1i, const float *__restrict__ q2i,
            float *__restrict__ q1o, float *__restrict__ q2o, const float *__restrict__ gl, int H,
            int W, int pitch, float tau, int it, int n_total) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= H || j >= W) return;
    auto P1 = [&](int y, int x) { return PStore<P>::load(p1i[(size_t)y * pitch + x]); };
    auto P2 = [&](int y, int x) { return PStore<P>::load(p2i[(size_t)y * pitch + x]); };
    // float32 storage: p1 / p2 hold hi, q1 / q2 lo (zero at a fold point, where the previous
    // launch folded it into hi); the iteration reads the working value fl(hi + lo)
    const bool carry = sizeof(P) == 4 && it % kFold != 0;
    auto V1 = [&](int y, int x) {
        const float h = P1(y, x);
        return carry ? tv_pval(h, q1i[(size_t)y * pitch + x]) : h;
    };
    auto V2 = [&](int y, int x) {
        const float h = P2(y, x);
        return carry ? tv_pval(h, q2i[(size_t)y * pitch + x]) : h;
    };
    // wn = -tau w at a pixel; its forward differences are na = -tau G
    auto wn_at = [&](int y, int x) {
        const float p1u = y > 0 ? V1(y - 1, x) : 0.0f;
        const float p2l = x > 0 ? V2(y, x - 1) : 0.0f;
        return tv_wn(V1(y, x), p1u, V2(y, x), p2l, __fmul_rn(tau, gl[(size_t)y * pitch + x]), tau);
    };
    const float wn = wn_at(i, j);
    const float na1 = (i < H - 1) ? __fsub_rn(wn_at(i + 1, j), wn) : 0.0f;
    const float na2 = (j < W - 1) ? __fsub_rn(wn_at(i, j + 1), wn) : 0.0f;
    float a = P1(i, j), b = P2(i, j);
    const size_t o = (size_t)i * pitch + j;
    if constexpr (sizeof(P) == 4) {
        float la = carry ? q1i[o] : 0.0f, lb = carry ? q2i[o] : 0.0f;
        tv_update_acc<FAST>(carry ? tv_pval(a, la) : a, carry ? tv_pval(b, lb) : b, la, lb, na1, na2);
        if ((it + 1) % kFold == 0 || it + 1 == n_total) {  // fold: hi <- fl(hi + lo), lo <- 0
            a = tv_pval(a, la);
            b = tv_pval(b, lb);
            la = lb = 0.0f;
        }
        q1o[o] = la;
        q2o[o] = lb;
    } else {
        tv_update<FAST>(a, b, na1, na2);
    }
    p1o[o] = PStore<P>::store(a);
    p2o[o] = PStore<P>::store(b);
}

template <typename P>
static cudaError_t naive_typed(bool fast, const void *p1i, const void *p2i, void *p1o,
                               void *p2o, const float *q1i, const float *q2i, float *q1o,
                               float *q2o, const float *gl, int H, int W, int pitch, float tau,
                               int it, int n_total, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((W + 31) / 32, (H + 7) / 8);
    if (fast)
        k_naive<P, true><<<grid, block, 0, st>>>((const P *)p1i, (const P *)p2i, (P *)p1o,
                                                 (P *)p2o, q1i, q2i, q1o, q2o, gl, H, W, pitch, tau, it, n_total);
    else
        k_naive<P, false><<<grid, block, 0, st>>>((const P *)p1i, (const P *)p2i, (P *)p1o,
                                                  (P *)p2o, q1i, q2i, q1o, q2o, gl, H, W, pitch, tau, it, n_total);
    return cudaGetLastError();
}

cudaError_t launch_naive(int p_storage, bool fast, const void *p1_in, const void *p2_in,
                         void *p1_out, void *p2_out, const float *q1_in, const float *q2_in,
                         float *q1_out, float *q2_out, const float *gl, int H, int W, int pitch,
                         float tau, int it, int n_total, cudaStream_t st) {
    switch (p_storage) {
        case 0:
            if (!q1_in || !q2_in || !q1_out || !q2_out) return cudaErrorInvalidValue;
            return naive_typed<float>(fast, p1_in, p2_in, p1_out, p2_out, q1_in, q2_in, q1_out, q2_out, gl, H, W, pitch, tau, it, n_total, st);
        case 1: return naive_typed<__half>(fast, p1_in, p2_in, p1_out, p2_out, nullptr, nullptr, nullptr, nullptr, gl, H, W, pitch, tau, it, n_total, st);
        case 2: return naive_typed<__nv_bfloat16>(fast, p1_in, p2_in, p1_out, p2_out, nullptr, nullptr, nullptr, nullptr, gl, H, W, pitch, tau, it, n_total, st);
        case 3: return naive_typed<short>(fast, p1_in, p2_in, p1_out, p2_out, nullptr, nullptr, nullptr, nullptr, gl, H, W, pitch, tau, it, n_total, st);
        default: return cudaErrorInvalidValue;
    }
}

// ---------------------------------------------------------------------------------------------
// Epilogue block mapping: block b of a launch belongs to image ep_img[b]; its local index is
// b - ep_base[img]; local block lb covers row lb / nbx, columns (lb % nbx) * kEpBlock + [0, 256).
// The partition depends only on (H, W), so a per-image reduction over it has the same order
// whether the image runs alone or in a batch.
// ---------------------------------------------------------------------------------------------

__global__ void __launch_bounds__(kEpBlock)
    k_init(ImgDesc *__restrict__ descs, const int *__restrict__ ep_img,
           const int *__restrict__ ep_base, int block_offset) {
    const int b = blockIdx.x + block_offset;
    const int img = ep_img[b];
    ImgDesc *d = descs + img;
    const int lb = b - ep_base[img];
    const int W = d->W;
    const int nbx = (W + kEpBlock - 1) / kEpBlock;
    const int i = lb / nbx;
    const int j = (lb % nbx) * kEpBlock + threadIdx.x;
    if (j >= W) return;
    const size_t n = (size_t)i * W + j;
    const float fv = d->f[n];
    if (!isfinite(fv)) atomicOr(d->status, kStatusNonFinite);
    d->gl[(size_t)i * d->pitch + j] = init_pixel(*d, n, fv);  // u_0 = f  (Eq. TVflow)
    if (d->u_trace) d->u_trace[n] = (double)fv;
}

cudaError_t launch_init(const ImgDesc *descs, const int *ep_img, const int *ep_base,
                        int n_blocks, cudaStream_t st, int block_offset) {
    if (n_blocks <= 0) return cudaSuccess;
    k_init<<<n_blocks, kEpBlock, 0, st>>>(const_cast<ImgDesc *>(descs), ep_img, ep_base,
                                          block_offset);
    return cudaGetLastError();
}

// One step's epilogue, per pixel, all in float64 (Sec. 2.1-2.2):
//   u_{k+1} = u_k - dt div p                 (Chambolle's primal recovery of the ROF step)
//   gl      = u_{k+1} / dt                    (data term of the next step's dual iterations)
//   phi_k   = t_k (u_{k+1} - 2 u_k + u_{k-1}) / dt^2, t_k = k dt, for k >= 1   (Eq. TVtrafo)
//   S(t_k)  = sum |phi_k|                     (deterministic two-level reduction)
//   b^m    += phi_k dt for the band m of t_k; a finished band is written out as float32
//   f_r     = u_{K-1} - t_{K-1} (u_K - u_{K-1}) / dt at the last step (Eq. finite_inverse_trafo)
// S(t_k) (and the Parseval-type spectrum) of one epilogue block's values: a fixed-order block
// tree into the block's partial, and in the image's last block the partials in block order.
__device__ __forceinline__ void s_reduce(const ImgDesc &dd, int lb, int k, double absphi,
                                         double phif, double *s_red, int &s_last) {
    const ImgDesc *d = &dd;
    const double bsum = block_sum(absphi, s_red);
    const double psum = d->S_par ? block_sum(phif, s_red) : 0.0;  // uniform per image
    if (threadIdx.x == 0) {
        d->partials[lb] = bsum;
        if (d->S_par) d->partials_par[lb] = psum;
        __threadfence();
        const unsigned prev = atomicAdd(d->counter, 1u);
        s_last = (prev == (unsigned)d->ep_blocks - 1u);
    }
    __syncthreads();
    if (!s_last) return;
    // last block of this image: sum the partials in block order (fixed) -> S(t_k)
    __threadfence();
    double t = 0.0;
    const volatile double *parts = d->partials;
    for (int q = threadIdx.x; q < d->ep_blocks; q += kEpBlock) t += parts[q];
    const double tot = block_sum(t, s_red);
    double ptot = 0.0;
    if (d->S_par) {
        double tp = 0.0;
        const volatile double *pp = d->partials_par;
        for (int q = threadIdx.x; q < d->ep_blocks; q += kEpBlock) tp += pp[q];
        ptot = block_sum(tp, s_red);
    }
    if (threadIdx.x == 0) {
        d->S[k - 1] = tot;
        if (d->S_par) d->S_par[k - 1] = ptot;
        *d->counter = 0u;
    }
}

// The divergence terms at pixel (i, j) from the copy of p the step's last launch wrote.
template <typename P>
__device__ __forceinline__ DivTerms step_div_terms(const ImgDesc &d, int k, int i, int j, int depth) {
    const int cp = p_copy(k + 1, launches_per_step(d.n_inner, depth), 0);
    const P *p1 = static_cast<const P *>(d.p1[cp]);
    const P *p2 = static_cast<const P *>(d.p2[cp]);
    const size_t o = (size_t)i * d.pitch + j;
    return div_terms(i, j, d.H, d.W, PStore<P>::load(p1[o]), i > 0 ? PStore<P>::load(p1[o - d.pitch]) : 0.0f,
                     PStore<P>::load(p2[o]), j > 0 ? PStore<P>::load(p2[o - 1]) : 0.0f);
}

template <typename P>
__device__ __forceinline__ void epilogue_block(const ImgDesc &dd, int lb, int gstep, int depth,
                                               double *s_red, int &s_last) {
    const ImgDesc *d = &dd;
    const int k = gstep - d->s0;
    if (k < 0 || k >= d->K) return;  // uniform over the block
    const int W = d->W;
    const int nbx = (W + kEpBlock - 1) / kEpBlock;
    const int i = lb / nbx;
    const int j = (lb % nbx) * kEpBlock + threadIdx.x;
    double absphi = 0.0, phif = 0.0;
    if (j < W) {
        const DivTerms dv = step_div_terms<P>(*d, k, i, j, depth);
        float gl_next;
        absphi = epilogue_pixel(*d, k, (size_t)i * W + j, dv, &gl_next, &phif);
        d->gl[(size_t)i * d->pitch + j] = gl_next;
    }
    if (k < 1) return;  // no phi at step 0
    s_reduce(*d, lb, k, absphi, phif, s_red, s_last);
}

// Split epilogue (u in the three-buffer rotation, u_k in u_buf3(k)). First part: u_{k+1} and
// g/dt of the next step; it is all the next step's dual iterations need.
// WAIT: the caller has not yet waited for the preceding grid (programmatic dependent launch).
// When the step ran dual iterations (which do not write u), u_k is then loaded before the wait
// and p after it; with n_inner = 0 the preceding grid is the previous step's epilogue, which
// writes u_k, so everything waits. The next grid is released after the wait.
template <typename P, bool WAIT = false>
__device__ __forceinline__ void epi_primal_block(const ImgDesc &d, int lb, int gstep, int depth) {
    const int k = gstep - d.s0;
    const int W = d.W;
    const int nbx = (W + kEpBlock - 1) / kEpBlock;
    const int i = lb / nbx;
    const int j = (lb % nbx) * kEpBlock + threadIdx.x;
    const bool live = k >= 0 && k < d.K && j < W;
    const size_t n = (size_t)i * W + j;
    double uc = 0.0;  // u_k: a float64 value, or a (hi, lo) float pair in the same 8 bytes
    const bool early = WAIT && d.n_inner > 0;
    if (live && early) uc = u_buf3(d, k)[n];
    if (WAIT) {
        pdl_wait();
        pdl_trigger();
    }
    if (!live) return;
    if (!early) uc = u_buf3(d, k)[n];
    const DivTerms dv = step_div_terms<P>(d, k, i, j, depth);
    float gl_next;
    if (d.acc_mode) {
        ff ucf;
        memcpy(&ucf, &uc, sizeof(ucf));
        const ff un = epi_primal<FFOps>(d, k, n, dv, ucf, &gl_next);
        FFOps::store(u_buf3(d, k + 1), n, un);
    } else {
        const double un = epi_primal<F64Ops>(d, k, n, dv, uc, &gl_next);
        F64Ops::store(u_buf3(d, k + 1), n, un);
    }
    d.gl[(size_t)i * d.pitch + j] = gl_next;
}

// Second part (k >= 1): phi_k, S, bands, filters and residual from u_{k-1}, u_k, u_{k+1}. It runs
// beside the next step's dual iterations, which do not read any of it.
__device__ __forceinline__ void epi_spectral_block(const ImgDesc &d, int lb, int gstep,
                                                   double *s_red, int &s_last) {
    const int k = gstep - d.s0;
    if (k < 1 || k >= d.K) return;  // uniform over the block
    const int W = d.W;
    const int nbx = (W + kEpBlock - 1) / kEpBlock;
    const int i = lb / nbx;
    const int j = (lb % nbx) * kEpBlock + threadIdx.x;
    double absphi = 0.0, phif = 0.0;
    if (j < W) {
        const size_t n = (size_t)i * W + j;
        const double *bp = u_buf3(d, k - 1), *bc = u_buf3(d, k), *bn = u_buf3(d, k + 1);
        absphi = d.acc_mode
                     ? epi_spectral<FFOps>(d, k, n, FFOps::load(bp, n), FFOps::load(bc, n), FFOps::load(bn, n), &phif)
                     : epi_spectral<F64Ops>(d, k, n, F64Ops::load(bp, n), F64Ops::load(bc, n), F64Ops::load(bn, n), &phif);
    }
    s_reduce(d, lb, k, absphi, phif, s_red, s_last);
}

template <typename P>
__global__ void __launch_bounds__(kEpBlock)
    k_epi_primal(const ImgDesc *__restrict__ descs, const int *__restrict__ ep_img,
                 const int *__restrict__ ep_base, int gstep, int depth) {
    pdl_wait();
    pdl_trigger();
    const int img = ep_img[blockIdx.x];
    epi_primal_block<P>(descs[img], blockIdx.x - ep_base[img], gstep, depth);
}

template <typename P>
__global__ void __launch_bounds__(kEpBlock)
    k_epi_primal_one(const __grid_constant__ ImgDesc d, int gstep, int depth) {
    epi_primal_block<P, true>(d, blockIdx.x, gstep, depth);
}

__global__ void __launch_bounds__(kEpBlock)
    k_epi_spectral(const ImgDesc *__restrict__ descs, const int *__restrict__ ep_img,
                   const int *__restrict__ ep_base, int gstep) {
    __shared__ double s_red[kEpBlock / 32];
    __shared__ int s_last;
    const int img = ep_img[blockIdx.x];
    epi_spectral_block(descs[img], blockIdx.x - ep_base[img], gstep, s_red, s_last);
}

__global__ void __launch_bounds__(kEpBlock)
    k_epi_spectral_one(const __grid_constant__ ImgDesc d, int gstep) {
    __shared__ double s_red[kEpBlock / 32];
    __shared__ int s_last;
    epi_spectral_block(d, blockIdx.x, gstep, s_red, s_last);
}

template <typename P>
__global__ void __launch_bounds__(kEpBlock)
    k_epilogue(ImgDesc *__restrict__ descs, const int *__restrict__ ep_img,
               const int *__restrict__ ep_base, int gstep, int depth) {
    __shared__ double s_red[kEpBlock / 32];
    __shared__ int s_last;
    pdl_wait();  // the step's last dual-iteration launch must be complete
    pdl_trigger();
    const int b = blockIdx.x;
    const int img = ep_img[b];
    epilogue_block<P>(descs[img], b - ep_base[img], gstep, depth, s_red, s_last);
}

// Single-image form: the descriptor is a kernel parameter, block b is local block b.
template <typename P>
__global__ void __launch_bounds__(kEpBlock)
    k_epilogue_one(const __grid_constant__ ImgDesc d, int gstep, int depth) {
    __shared__ double s_red[kEpBlock / 32];
    __shared__ int s_last;
    pdl_wait();
    pdl_trigger();
    epilogue_block<P>(d, blockIdx.x, gstep, depth, s_red, s_last);
}

cudaError_t launch_epilogue(int p_storage, const ImgDesc *descs, const int *ep_img,
                            const int *ep_base, int n_blocks, int gstep, int depth,
                            cudaStream_t st, bool pdl) {
    if (n_blocks <= 0) return cudaSuccess;
    ImgDesc *dd = const_cast<ImgDesc *>(descs);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_blocks);
    cfg.blockDim = dim3(kEpBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    switch (p_storage) {
        case 0: return cudaLaunchKernelEx(&cfg, k_epilogue<float>, dd, ep_img, ep_base, gstep, depth);
        case 1: return cudaLaunchKernelEx(&cfg, k_epilogue<__half>, dd, ep_img, ep_base, gstep, depth);
        case 2: return cudaLaunchKernelEx(&cfg, k_epilogue<__nv_bfloat16>, dd, ep_img, ep_base, gstep, depth);
        case 3: return cudaLaunchKernelEx(&cfg, k_epilogue<short>, dd, ep_img, ep_base, gstep, depth);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_epilogue_one(int p_storage, const ImgDesc &d, int gstep, int depth,
                                cudaStream_t st, bool pdl) {
    if (d.ep_blocks <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)d.ep_blocks);
    cfg.blockDim = dim3(kEpBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    switch (p_storage) {
        case 0: return cudaLaunchKernelEx(&cfg, k_epilogue_one<float>, d, gstep, depth);
        case 1: return cudaLaunchKernelEx(&cfg, k_epilogue_one<__half>, d, gstep, depth);
        case 2: return cudaLaunchKernelEx(&cfg, k_epilogue_one<__nv_bfloat16>, d, gstep, depth);
        case 3: return cudaLaunchKernelEx(&cfg, k_epilogue_one<short>, d, gstep, depth);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_epi_primal(int p_storage, const ImgDesc *descs, const int *ep_img,
                              const int *ep_base, int n_blocks, int gstep, int depth,
                              cudaStream_t st, bool pdl) {
    if (n_blocks <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_blocks);
    cfg.blockDim = dim3(kEpBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    switch (p_storage) {
        case 0: return cudaLaunchKernelEx(&cfg, k_epi_primal<float>, descs, ep_img, ep_base, gstep, depth);
        case 1: return cudaLaunchKernelEx(&cfg, k_epi_primal<__half>, descs, ep_img, ep_base, gstep, depth);
        case 2: return cudaLaunchKernelEx(&cfg, k_epi_primal<__nv_bfloat16>, descs, ep_img, ep_base, gstep, depth);
        case 3: return cudaLaunchKernelEx(&cfg, k_epi_primal<short>, descs, ep_img, ep_base, gstep, depth);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_epi_primal_one(int p_storage, const ImgDesc &d, int gstep, int depth,
                                  cudaStream_t st, bool pdl) {
    const int n_blocks = d.ep_blocks;
    if (n_blocks <= 0) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_blocks);
    cfg.blockDim = dim3(kEpBlock);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    switch (p_storage) {
        case 0: return cudaLaunchKernelEx(&cfg, k_epi_primal_one<float>, d, gstep, depth);
        case 1: return cudaLaunchKernelEx(&cfg, k_epi_primal_one<__half>, d, gstep, depth);
        case 2: return cudaLaunchKernelEx(&cfg, k_epi_primal_one<__nv_bfloat16>, d, gstep, depth);
        case 3: return cudaLaunchKernelEx(&cfg, k_epi_primal_one<short>, d, gstep, depth);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_epi_spectral(const ImgDesc *descs, const int *ep_img, const int *ep_base,
                                int n_blocks, int gstep, cudaStream_t st) {
    if (n_blocks <= 0) return cudaSuccess;
    k_epi_spectral<<<n_blocks, kEpBlock, 0, st>>>(descs, ep_img, ep_base, gstep);
    return cudaGetLastError();
}

cudaError_t launch_epi_spectral_one(const ImgDesc &d, int gstep, cudaStream_t st) {
    if (d.ep_blocks <= 0) return cudaSuccess;
    k_epi_spectral_one<<<d.ep_blocks, kEpBlock, 0, st>>>(d, gstep);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Standalone ROF step helpers.
// ---------------------------------------------------------------------------------------------
__global__ void k_gl_from_g(const float *__restrict__ g, float *__restrict__ gl, int H, int W,
                            int pitch, double inv_lam) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= W) return;
    gl[(size_t)i * pitch + j] = (float)((double)g[(size_t)i * W + j] * inv_lam);
}

cudaError_t launch_gl_from_g(const float *g, float *gl, int H, int W, int pitch, double lambda,
                             cudaStream_t st) {
    dim3 grid((W + 255) / 256, H);
    k_gl_from_g<<<grid, 256, 0, st>>>(g, gl, H, W, pitch, 1.0 / lambda);
    return cudaGetLastError();
}

__global__ void k_rof_primal(const float *__restrict__ p1, const float *__restrict__ p2,
                             int pitch, const float *__restrict__ g, float *__restrict__ u,
                             int H, int W, double lambda) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (j >= W) return;
    const size_t o = (size_t)i * pitch + j;
    const double a = (i < H - 1 ? (double)p1[o] : 0.0) - (i > 0 ? (double)p1[o - pitch] : 0.0);
    const double c = (j < W - 1 ? (double)p2[o] : 0.0) - (j > 0 ? (double)p2[o - 1] : 0.0);
    const size_t n = (size_t)i * W + j;
    u[n] = (float)((double)g[n] - lambda * (a + c));
}

cudaError_t launch_rof_primal(const float *p1, const float *p2, int pitch, const float *g,
                              float *u, int H, int W, double lambda, cudaStream_t st) {
    dim3 grid((W + 255) / 256, H);
    k_rof_primal<<<grid, 256, 0, st>>>(p1, p2, pitch, g, u, H, W, lambda);
    return cudaGetLastError();
}

}  // namespace tvspec

// ---------------------------------------------------------------------------------------------
// Copy list: many device-to-device copies in one launch. Block b copies chunk
// b - first[i] of item i (first[] = prefix sums of the items' chunk counts).
// ---------------------------------------------------------------------------------------------
namespace tvspec {

__global__ void __launch_bounds__(256)
    k_copy_list(const CopyItem *__restrict__ items, const unsigned *__restrict__ first, int n,
                unsigned n_chunks) {
    for (unsigned b = blockIdx.x; b < n_chunks; b += gridDim.x) {
        int lo = 0, hi = n - 1;  // last item with first[i] <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (first[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        const CopyItem it = items[lo];
        const size_t begin = (size_t)(b - first[lo]) * kCopyChunk;
        const size_t end = min(it.bytes, begin + kCopyChunk);
        const char *s = static_cast<const char *>(it.src);
        char *d = static_cast<char *>(it.dst);
        if ((((uintptr_t)s | (uintptr_t)d) & 15) == 0) {
            const size_t v_end = begin + ((end - begin) & ~(size_t)15);
            for (size_t o = begin + 16 * threadIdx.x; o < v_end; o += 16 * blockDim.x)
                *reinterpret_cast<int4 *>(d + o) = *reinterpret_cast<const int4 *>(s + o);
            for (size_t o = v_end + threadIdx.x; o < end; o += blockDim.x) d[o] = s[o];
        } else if ((((uintptr_t)s | (uintptr_t)d) & 3) == 0) {
            const size_t v_end = begin + ((end - begin) & ~(size_t)3);
            for (size_t o = begin + 4 * threadIdx.x; o < v_end; o += 4 * blockDim.x)
                *reinterpret_cast<unsigned *>(d + o) = *reinterpret_cast<const unsigned *>(s + o);
            for (size_t o = v_end + threadIdx.x; o < end; o += blockDim.x) d[o] = s[o];
        } else {
            for (size_t o = begin + threadIdx.x; o < end; o += blockDim.x) d[o] = s[o];
        }
    }
}

cudaError_t launch_copy_list(const CopyItem *items, const unsigned *first, int n,
                             unsigned n_chunks, cudaStream_t st) {
    if (n <= 0 || n_chunks == 0) return cudaSuccess;
    const unsigned grid = std::min<unsigned>(n_chunks, 152u * 16u);
    k_copy_list<<<grid, 256, 0, st>>>(items, first, n, n_chunks);
    return cudaGetLastError();
}

}  // namespace tvspec
