// Resident kernel for small images: one CTA runs a whole decomposition -- u_0 = f, then K
// steps of n_inner dual iterations and the float64 epilogue -- for an image that fits the
// CTA's register tile (W <= 32 V, H <= RW R), in one launch for a whole batch of such images.
//
// The tile is the image itself, so there is no halo and no exchange with other CTAs: the
// tiled kernel's iteration (tiled_iterate, with the border masks) runs n_inner times per step
// in registers. For the epilogue the CTA writes p to global memory (L2) once per step, reads
// the divergence neighbours back after a CTA barrier, and applies the shared per-pixel
// epilogue (epilogue_pixel). S(t_k) is reduced with the same partition (one 256-wide block per
// image row) and the same shuffle trees as the multi-block epilogue, so every output is
// bit-identical to the multi-launch path.
#include "epilogue.cuh"
#include "k_tiled.cuh"

namespace tvspec {

// Shuffle tree of one warp (lane 0 gets the sum), the order of block_sum's first level.
__device__ __forceinline__ double warp_tree(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    return v;
}

// block_sum's second level for 256 threads: lane j < 8 of warp 0 holds warp j's sum, the other
// 24 lanes zero, then the shuffle tree. Adding those zeros changes nothing but the sign of a
// zero, which the explicit (x + 0) + 0 reproduces: the result is
// ((w0 + w4) + (w2 + w6)) + ((w1 + w5) + (w3 + w7)) with w = (w + 0) + 0.
__device__ __forceinline__ double eight_tree(const double (&w)[8]) {
    double z[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) z[c] = __dadd_rn(__dadd_rn(w[c], 0.0), 0.0);
    return __dadd_rn(__dadd_rn(__dadd_rn(z[0], z[4]), __dadd_rn(z[2], z[6])),
                     __dadd_rn(__dadd_rn(z[1], z[5]), __dadd_rn(z[3], z[7])));
}

// The sum of vals (H x W) with exactly the operations of the multi-block epilogue: block_sum
// over one 256-wide block per image row (thread t holds column t, zero past W), then, in one
// block, block_sum of (0 + row sum) over the rows. A 256-wide tree is the warp trees of its 8
// chunks of 32 and eight_tree over them; chunks past the data are all-zero and sum to zero, so
// one warp per row computes only the chunks that hold data, with no CTA barrier per row.
// Valid in thread 0; every thread of the CTA must call it (two CTA barriers).
template <int RW>
__device__ __forceinline__ double resident_sum(const double *vals, int H, int W, double *s_part) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nch = (W + 31) >> 5;  // <= 8 (W <= 256)
    for (int i = warp; i < H; i += RW) {
        double w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            w[c] = 0.0;
            if (c < nch) {
                const int col = 32 * c + lane;
                w[c] = warp_tree(col < W ? vals[(size_t)i * W + col] : 0.0);
            }
        }
        if (lane == 0) s_part[i] = eight_tree(w);
    }
    __syncthreads();
    double x = 0.0;
    if (warp == 0) {
        const int nr = (H + 31) >> 5;  // <= 8 (H <= 256)
        double w[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            w[c] = 0.0;
            if (c < nr) {
                const int row = 32 * c + lane;
                w[c] = warp_tree(row < H ? __dadd_rn(0.0, s_part[row]) : 0.0);
            }
        }
        x = eight_tree(w);
    }
    __syncthreads();
    return x;
}

template <int V, int R, int RW, int MINB, bool FAST>
__global__ void __launch_bounds__(32 * RW, MINB)
    k_resident(const ImgDesc *__restrict__ descs, const int *__restrict__ idx, float tau,
               int warm_start) {
    constexpr int VP = V / 2;
    constexpr int TW = 32 * V;
    constexpr int TH = RW * R;
    __shared__ __align__(16) float s_p1b[RW][TW];
    __shared__ __align__(16) float s_wt[RW][TW];
    __shared__ double s_part[TH];
    // dynamic shared memory: tau g/dt of the tile (TH x TW floats; the registers stay free for p
    // and its low parts), then H * W values of |phi_k| [and H * W values of phi_k f]
    extern __shared__ double s_dyn[];
    float *s_gl = reinterpret_cast<float *>(s_dyn);
    double *s_phi = s_dyn + (size_t)TH * TW / 2;

    const ImgDesc &d = descs[idx[blockIdx.x]];
    const int H = d.H, W = d.W, pitch = d.pitch;
    double *s_phif = s_phi + (size_t)H * W;  // used only when the launch has room for it
    const int lane = threadIdx.x & 31;
    const int wy = threadIdx.x >> 5;
    const int cx = lane * V;
    const int ry = wy * R;
    float *gp1 = static_cast<float *>(d.p1[0]);
    float *gp2 = static_cast<float *>(d.p2[0]);

    // this kernel clears what it needs itself (the host skips the workspace memset): the
    // status word and the bands (a band without any t_k stays zero)
    if (threadIdx.x == 0) *d.status = 0u;
    for (size_t q = threadIdx.x; q < (size_t)d.n_bands * H * W; q += blockDim.x) d.bands[q] = 0.0f;
    __syncthreads();

    const bool exact = H == TH && W == TW;  // uniform over the CTA
    // border masks: the tile is the image, every tile pixel outside it stays zero
    unsigned m1 = 0u, m2 = 0u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = ry + r;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int c = cx + v;
            if (y < H - 1 && c < W) m1 |= 1u << (r * V + v);
            if (y < H && c < W - 1) m2 |= 1u << (r * V + v);
        }
    }

    // u_0 = f (Eq. TVflow), g/dt of step 0, p = 0
    float2 p1[R][VP], p2[R][VP];
    float2 l1[R][VP], l2[R][VP];  // low parts of p (zero between steps: a step ends at a fold point)
    float *my_gl = s_gl + (size_t)ry * TW + cx;  // this thread's pixels in s_gl (row stride TW)
    const GlShared gl{my_gl, TW};
#pragma unroll
    for (int r = 0; r < R; ++r) {
#pragma unroll
        for (int j = 0; j < VP; ++j) {
            p1[r][j] = p2[r][j] = make_float2(0.0f, 0.0f);
            l1[r][j] = l2[r][j] = make_float2(0.0f, 0.0f);
            float g2[2] = {0.0f, 0.0f};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int y = ry + r, c = cx + 2 * j + h;
                if (y < H && c < W) {
                    const size_t n = (size_t)y * W + c;
                    const float fv = d.f[n];
                    if (!isfinite(fv)) atomicOr(d.status, kStatusNonFinite);
                    g2[h] = init_pixel(d, n, fv);  // u_0 = f (Eq. TVflow)
                    if (d.u_trace) d.u_trace[n] = (double)fv;
                }
            }
            *reinterpret_cast<float2 *>(my_gl + r * TW + 2 * j) =
                make_float2(__fmul_rn(tau, g2[0]), __fmul_rn(tau, g2[1]));  // tau g/dt
        }
    }

    for (int k = 0; k < d.K; ++k) {
        if (!warm_start) {
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int j = 0; j < VP; ++j)
                    p1[r][j] = p2[r][j] = l1[r][j] = l2[r][j] = make_float2(0.0f, 0.0f);
        }
        __syncthreads();  // tau g/dt of the step in s_gl; the exchange rows free
        if (exact)  // the image fills the tile: masks only on its last row and column
            tiled_iterate_g<V, R, RW, FAST, kEdgeExact, true, true>(p1, p2, l1, l2, gl, d.n_inner, 0,
                                                                  d.n_inner, tau, 0u, 0u,
                                                            s_p1b, s_wt, lane, wy);
        else
            tiled_iterate_g<V, R, RW, FAST, kEdgeMasked, true, true>(p1, p2, l1, l2, gl, d.n_inner, 0,
                                                                   d.n_inner, tau, m1, m2,
                                                             s_p1b, s_wt, lane, wy);
        // p to global for the divergence's neighbours
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
            if (y < H && cx < W) {
                FPack<V> a, b;
#pragma unroll
                for (int j = 0; j < VP; ++j) {
                    a.v[2 * j] = p1[r][j].x;
                    a.v[2 * j + 1] = p1[r][j].y;
                    b.v[2 * j] = p2[r][j].x;
                    b.v[2 * j + 1] = p2[r][j].y;
                }
                *reinterpret_cast<FPack<V> *>(gp1 + (size_t)y * pitch + cx) = a;
                *reinterpret_cast<FPack<V> *>(gp2 + (size_t)y * pitch + cx) = b;
            }
        }
        __syncthreads();
        // the epilogue on every own pixel
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int j = 0; j < VP; ++j) {
                const float2 gcur = gl(r, j);
                float g2[2] = {gcur.x, gcur.y};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int y = ry + r, c = cx + 2 * j + h;
                    if (y < H && c < W) {
                        const size_t o = (size_t)y * pitch + c;
                        const float pv1 = h == 0 ? p1[r][j].x : p1[r][j].y;
                        const float pv2 = h == 0 ? p2[r][j].x : p2[r][j].y;
                        const DivTerms dv = div_terms(y, c, H, W, pv1, y > 0 ? gp1[o - pitch] : 0.0f,
                                                      pv2, c > 0 ? gp2[o - 1] : 0.0f);
                        double pf;
                        const double a = epilogue_pixel(d, k, (size_t)y * W + c, dv, &g2[h], &pf);
                        s_phi[(size_t)y * W + c] = a;
                        if (d.S_par) s_phif[(size_t)y * W + c] = pf;
                    }
                }
                *reinterpret_cast<float2 *>(my_gl + r * TW + 2 * j) =
                    make_float2(__fmul_rn(tau, g2[0]), __fmul_rn(tau, g2[1]));  // tau g/dt
            }
        }
        __syncthreads();
        if (k >= 1) {
            const double tot = resident_sum<RW>(s_phi, H, W, s_part);
            if (threadIdx.x == 0) d.S[k - 1] = tot;
            if (d.S_par) {
                const double ptot = resident_sum<RW>(s_phif, H, W, s_part);
                if (threadIdx.x == 0) d.S_par[k - 1] = ptot;
            }
            __syncthreads();
        }
    }
}

// Variants: (V, R, RW, MINB) -> image tile (32 V) x (RW R), CTAs per SM the registers are
// budgeted for. The automatic choice takes the first variant in kAutoOrder that holds the image.
using ResidentKernel = void (*)(const ImgDesc *, const int *, float, int);

struct ResidentVariant {
    int V, R, RW, MINB;
    ResidentKernel fast, ieee;
};

#define TVSPEC_RESIDENT(V, R, RW, MINB) \
    {V, R, RW, MINB, &k_resident<V, R, RW, MINB, true>, &k_resident<V, R, RW, MINB, false>}
static const ResidentVariant kResident[] = {
    TVSPEC_RESIDENT(2, 2, 32, 1),  // 0:  64 x  64, 1024 threads, 4 px each
    TVSPEC_RESIDENT(2, 4, 32, 1),  // 1: 128 x  64 (H x W)
    TVSPEC_RESIDENT(4, 2, 32, 1),  // 2:  64 x 128
    TVSPEC_RESIDENT(2, 8, 8, 2),   // 3:  64 x  64,  256 threads, 16 px each, 2 CTAs / SM
    TVSPEC_RESIDENT(2, 4, 16, 1),  // 4:  64 x  64,  512 threads, 8 px each
    TVSPEC_RESIDENT(2, 4, 16, 2),  // 5:  64 x  64,  512 threads, 2 CTAs / SM
    TVSPEC_RESIDENT(2, 8, 8, 3),   // 6:  64 x  64,  256 threads, 3 CTAs / SM
    TVSPEC_RESIDENT(2, 8, 8, 4),   // 7:  64 x  64,  256 threads, 4 CTAs / SM
};
#undef TVSPEC_RESIDENT
static constexpr int kNumResident = (int)(sizeof(kResident) / sizeof(kResident[0]));
// The compensated update keeps two more floats per pixel in registers, so g/dt lives in shared
// memory here. Measured on 3000 crops of 64^2 (K = 50, 300 iterations): the 256-thread,
// 16-pixel layout at 2 CTAs per SM 16.6 k crops/s, the 512-thread 8-pixel layouts 12.8 k (1 CTA
// per SM) and 15.4 k (2), the 16-pixel layouts budgeted for 3 or 4 CTAs per SM spill (4.7 k).
static const int kAutoOrder[] = {3, 1, 2};

static bool resident_holds(int i, int H, int W) {
    return W <= 32 * kResident[i].V && H <= kResident[i].RW * kResident[i].R;
}

int resident_variant_count() { return kNumResident; }

bool resident_variant_info(int i, int *max_h, int *max_w, int *threads, int *minb) {
    if (i < 0 || i >= kNumResident) return false;
    *max_h = kResident[i].RW * kResident[i].R;
    *max_w = 32 * kResident[i].V;
    *threads = 32 * kResident[i].RW;
    *minb = kResident[i].MINB;
    return true;
}

int resident_variant_for(int H, int W, int preferred) {
    if (preferred >= 0 && preferred < kNumResident && resident_holds(preferred, H, W)) return preferred;
    for (int i : kAutoOrder)
        if (resident_holds(i, H, W)) return i;
    return -1;
}

cudaError_t launch_resident(int variant, bool fast, const ImgDesc *descs, const int *idx, int n,
                            float tau, int warm_start, bool parseval, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (variant < 0 || variant >= kNumResident) return cudaErrorInvalidValue;
    const ResidentVariant &v = kResident[variant];
    const ResidentKernel k = fast ? v.fast : v.ieee;
    const size_t tile = (size_t)(32 * v.V) * (v.RW * v.R);
    const size_t smem = tile * sizeof(float) + tile * sizeof(double) * (parseval ? 2 : 1);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<n, 32 * v.RW, smem, st>>>(descs, idx, tau, warm_start);
    return cudaGetLastError();
}

}  // namespace tvspec
