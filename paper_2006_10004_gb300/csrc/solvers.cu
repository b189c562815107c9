// Inner solvers of one ROF step (Eq. ROF) for comparing accuracy per iteration and time:
// Chambolle's projection (the tiled kernel of the decomposition), Beck and Teboulle's fast
// gradient projection (FGP) on the same dual, and Chambolle and Pock's primal-dual hybrid
// gradient (PDHG), with the duality gap of the returned primal-dual pair.
//
// FGP runs temporally blocked in register tiles like the Chambolle kernel (a one-iteration-
// per-launch reference kernel gives the same bits); PDHG runs one iteration per launch (a dual
// and a primal launch) on pitched float32 arrays, one thread per pixel. The scalar step
// sequences (momentum, steps) are computed in float64 on the host. The gap is reduced in
// float64 over a fixed partition.
#include <algorithm>
#include <cmath>
#include <vector>

#include "epilogue.cuh"
#include "runtime.h"

namespace tvspec {

namespace {

constexpr int kSolverBlockX = 32, kSolverBlockY = 8;

__device__ __forceinline__ float divergence(const float *p1, const float *p2, int i, int j, int H,
                                            int W, int pitch) {
    const size_t o = (size_t)i * pitch + j;
    const float a = (i < H - 1 ? p1[o] : 0.0f) - (i > 0 ? p1[o - pitch] : 0.0f);
    const float b = (j < W - 1 ? p2[o] : 0.0f) - (j > 0 ? p2[o - 1] : 0.0f);
    return a + b;
}

// The FGP update of one pixel given w = div r - g/lambda there and its masked forward
// differences G: q = r + G / 8, p_new = q / max(1, |q|), r_new = p_new + beta (p_new - p).
// Explicitly rounded, so the one-iteration and the tiled kernels agree bit for bit.
__device__ __forceinline__ void fgp_pixel(float &p1, float &p2, float &r1, float &r2, float G1,
                                          float G2, float beta) {
    float q1 = __fadd_rn(r1, __fmul_rn(G1, 0.125f));
    float q2 = __fadd_rn(r2, __fmul_rn(G2, 0.125f));
    const float n2 = __fadd_rn(__fmul_rn(q1, q1), __fmul_rn(q2, q2));
    if (n2 > 1.0f) {
        // 1/|q| by the hardware reciprocal square root and one Newton-Raphson step,
        // y <- y (3/2 - n2 y^2 / 2)
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(n2));
        y = __fmul_rn(y, __fmaf_rn(__fmul_rn(-0.5f, n2), __fmul_rn(y, y), 1.5f));
        q1 = __fmul_rn(q1, y);
        q2 = __fmul_rn(q2, y);
    }
    r1 = __fadd_rn(q1, __fmul_rn(beta, __fsub_rn(q1, p1)));
    r2 = __fadd_rn(q2, __fmul_rn(beta, __fsub_rn(q2, p2)));
    p1 = q1;
    p2 = q2;
}

// w = (r1 - r1_up) + (r2 - r2_left) - g/lambda, explicitly rounded.
__device__ __forceinline__ float fgp_w(float r1, float r1u, float r2, float r2l, float gl) {
    return __fsub_rn(__fadd_rn(__fsub_rn(r1, r1u), __fsub_rn(r2, r2l)), gl);
}

// One FGP iteration per launch, one thread per pixel, neighbours from global memory.
__global__ void __launch_bounds__(kSolverBlockX * kSolverBlockY)
    k_fgp(float *__restrict__ p1, float *__restrict__ p2, const float *__restrict__ r1,
          const float *__restrict__ r2, float *__restrict__ r1o, float *__restrict__ r2o,
          const float *__restrict__ gl, int H, int W, int pitch, float beta) {
    const int j = blockIdx.x * kSolverBlockX + threadIdx.x;
    const int i = blockIdx.y * kSolverBlockY + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t o = (size_t)i * pitch + j;
    auto w_at = [&](int y, int x) {
        const size_t q = (size_t)y * pitch + x;
        return fgp_w(r1[q], y > 0 ? r1[q - pitch] : 0.0f, r2[q], x > 0 ? r2[q - 1] : 0.0f, gl[q]);
    };
    const float w = w_at(i, j);
    const float G1 = i < H - 1 ? __fsub_rn(w_at(i + 1, j), w) : 0.0f;
    const float G2 = j < W - 1 ? __fsub_rn(w_at(i, j + 1), w) : 0.0f;
    float a1 = p1[o], a2 = p2[o], b1 = r1[o], b2 = r2[o];
    fgp_pixel(a1, a2, b1, b2, G1, G2, beta);
    r1o[o] = b1;
    r2o[o] = b2;
    p1[o] = a1;
    p2[o] = a2;
}

// Temporally blocked FGP: a CTA holds a (RW R) x (32 V) tile of p, r and g/lambda in registers
// (lane l of warp wy: columns [lV, lV + V) of rows [wy R, wy R + R)), runs up to TB iterations
// and stores the centre (halo TB rows and roundup(TB, V) columns each side, recomputed by the
// neighbouring tiles: one iteration reads r at the offsets of the Chambolle iteration). Row
// neighbours come from registers or a warp shuffle, column neighbours across warps from two
// shared-memory rows (the bottom row of r1, the top row of w) with two CTA barriers per
// iteration. beta[k] is the momentum of iteration k of the launch. Pixels outside the image are
// zero and their differences masked, which realises the Neumann boundary.
struct FgpBetas {
    float v[16];
};

struct FgpDesc {
    const float *gl;
    float *p1[2], *p2[2], *r1[2], *r2[2];
    int H, W, pitch;
};

template <int V, int R, int RW, int TB>
__global__ void __launch_bounds__(32 * RW, 1)
    k_fgp_tiled(const __grid_constant__ FgpDesc d, int ntx, int src, int n_iter,
                const __grid_constant__ FgpBetas betas) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int TW = 32 * V, TH = RW * R;
    constexpr int HX = (TB + V - 1) / V * V;
    constexpr int OW = TW - 2 * HX, OH = TH - 2 * TB;
    static_assert(OW > 0 && OH > 0 && R * V <= 32, "tile");
    __shared__ float s_r1b[RW][TW];
    __shared__ float s_wt[RW][TW];
    const int H = d.H, W = d.W, pitch = d.pitch;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;
    const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int x0 = tx * OW, y0 = ty * OH;
    const int cx = x0 - HX + lane * V, ry = y0 - TB + wy * R;
    float p1[R][V], p2[R][V], r1[R][V], r2[R][V], gl[R][V];
    unsigned m1 = 0u, m2 = 0u;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = ry + r;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int c = cx + v;
            const bool in = y >= 0 && y < H && c >= 0 && c < W;
            const size_t o = (size_t)y * pitch + c;
            p1[r][v] = in ? d.p1[src][o] : 0.0f;
            p2[r][v] = in ? d.p2[src][o] : 0.0f;
            r1[r][v] = in ? d.r1[src][o] : 0.0f;
            r2[r][v] = in ? d.r2[src][o] : 0.0f;
            gl[r][v] = in ? d.gl[o] : 0.0f;
            if (in && y < H - 1) m1 |= 1u << (r * V + v);
            if (in && c < W - 1) m2 |= 1u << (r * V + v);
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) s_r1b[wy][lane * V + v] = r1[R - 1][v];
    __syncthreads();
    for (int it = 0; it < n_iter; ++it) {
        const float beta = betas.v[it];
        float w[R][V];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float left = __shfl_up_sync(FULL, r2[r][V - 1], 1);  // lane 0: halo, unused
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float up = r > 0 ? r1[r - 1][v] : (wy > 0 ? s_r1b[wy - 1][lane * V + v] : 0.0f);
                const float lf = v > 0 ? r2[r][v - 1] : left;
                w[r][v] = fgp_w(r1[r][v], up, r2[r][v], lf, gl[r][v]);
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) s_wt[wy][lane * V + v] = w[0][v];
        __syncthreads();
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float right = __shfl_down_sync(FULL, w[r][0], 1);  // lane 31: halo, unused
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const float wd = r < R - 1 ? w[r + 1][v] : (wy < RW - 1 ? s_wt[wy + 1][lane * V + v] : w[r][v]);
                const float wr = v < V - 1 ? w[r][v + 1] : right;
                const int b = r * V + v;
                const float G1 = ((m1 >> b) & 1u) ? __fsub_rn(wd, w[r][v]) : 0.0f;
                const float G2 = ((m2 >> b) & 1u) ? __fsub_rn(wr, w[r][v]) : 0.0f;
                fgp_pixel(p1[r][v], p2[r][v], r1[r][v], r2[r][v], G1, G2, beta);
            }
        }
#pragma unroll
        for (int v = 0; v < V; ++v) s_r1b[wy][lane * V + v] = r1[R - 1][v];
        __syncthreads();
    }
    // the exact centre into the other copy
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = ry + r;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            const int c = cx + v;
            if (y >= y0 && y < y0 + OH && y < H && c >= x0 && c < x0 + OW && c < W) {
                const size_t o = (size_t)y * pitch + c;
                d.p1[src ^ 1][o] = p1[r][v];
                d.p2[src ^ 1][o] = p2[r][v];
                d.r1[src ^ 1][o] = r1[r][v];
                d.r2[src ^ 1][o] = r2[r][v];
            }
        }
    }
}

// The tile shape of the blocked FGP kernel: 64 x 56 tiles, 8 iterations per launch.
constexpr int kFgpV = 2, kFgpR = 7, kFgpRW = 8, kFgpTB = 8;

// PDHG dual step: p = Pi(p - s grad ubar), s = sigma / lambda.
__global__ void __launch_bounds__(kSolverBlockX * kSolverBlockY)
    k_pdhg_dual(float *__restrict__ p1, float *__restrict__ p2, const float *__restrict__ ub, int H,
                int W, int pitch, float s) {
    const int j = blockIdx.x * kSolverBlockX + threadIdx.x;
    const int i = blockIdx.y * kSolverBlockY + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t o = (size_t)i * pitch + j;
    const float G1 = i < H - 1 ? ub[o + pitch] - ub[o] : 0.0f;
    const float G2 = j < W - 1 ? ub[o + 1] - ub[o] : 0.0f;
    float q1 = p1[o] - s * G1, q2 = p2[o] - s * G2;
    const float n = sqrtf(q1 * q1 + q2 * q2);
    if (n > 1.0f) {
        q1 = q1 / n;
        q2 = q2 / n;
    }
    p1[o] = q1;
    p2[o] = q2;
}

// PDHG primal step: u_new = (u - tl div p + t g) / (1 + t); ubar = u_new + theta (u_new - u).
__global__ void __launch_bounds__(kSolverBlockX * kSolverBlockY)
    k_pdhg_primal(float *__restrict__ u, float *__restrict__ ub, const float *__restrict__ p1,
                  const float *__restrict__ p2, const float *__restrict__ g, int H, int W, int pitch,
                  float tl, float t, float theta) {
    const int j = blockIdx.x * kSolverBlockX + threadIdx.x;
    const int i = blockIdx.y * kSolverBlockY + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t o = (size_t)i * pitch + j;
    const float uo = u[o];
    const float un = (uo - tl * divergence(p1, p2, i, j, H, W, pitch) + t * g[o]) / (1.0f + t);
    ub[o] = un + theta * (un - uo);
    u[o] = un;
}

// u = g - lambda div p (the primal point of a dual iterate), float64 arithmetic.
__global__ void __launch_bounds__(kSolverBlockX * kSolverBlockY)
    k_primal_of_dual(const float *__restrict__ p1, const float *__restrict__ p2,
                     const float *__restrict__ g, float *__restrict__ u, int H, int W, int pitch,
                     double lambda) {
    const int j = blockIdx.x * kSolverBlockX + threadIdx.x;
    const int i = blockIdx.y * kSolverBlockY + threadIdx.y;
    if (i >= H || j >= W) return;
    const size_t o = (size_t)i * pitch + j;
    const double a = (i < H - 1 ? (double)p1[o] : 0.0) - (i > 0 ? (double)p1[o - pitch] : 0.0);
    const double b = (j < W - 1 ? (double)p2[o] : 0.0) - (j > 0 ? (double)p2[o - 1] : 0.0);
    u[o] = (float)((double)g[o] - lambda * (a + b));
}

// Per block (256 pixels of one row): sum of 1/2(u-g)^2 + lambda |grad u| - 1/2 g^2
// + 1/2 (g - lambda div p)^2 in float64; the last block sums the partials in block order.
__global__ void __launch_bounds__(kEpBlock)
    k_gap(const float *__restrict__ u, const float *__restrict__ p1, const float *__restrict__ p2,
          const float *__restrict__ g, int H, int W, int pitch, double lambda,
          double *__restrict__ partials, unsigned *__restrict__ counter, double *__restrict__ gap) {
    __shared__ double s_red[kEpBlock / 32];
    __shared__ int s_last;
    const int nbx = (W + kEpBlock - 1) / kEpBlock;
    const int i = blockIdx.x / nbx;
    const int j = (blockIdx.x % nbx) * kEpBlock + threadIdx.x;
    double v = 0.0;
    if (j < W) {
        const size_t o = (size_t)i * pitch + j;
        const double uo = u[o], go = g[o];
        const double G1 = i < H - 1 ? (double)u[o + pitch] - uo : 0.0;
        const double G2 = j < W - 1 ? (double)u[o + 1] - uo : 0.0;
        const double a = (i < H - 1 ? (double)p1[o] : 0.0) - (i > 0 ? (double)p1[o - pitch] : 0.0);
        const double b = (j < W - 1 ? (double)p2[o] : 0.0) - (j > 0 ? (double)p2[o - 1] : 0.0);
        const double r = go - lambda * (a + b);
        v = 0.5 * (uo - go) * (uo - go) + lambda * sqrt(G1 * G1 + G2 * G2) - 0.5 * go * go + 0.5 * r * r;
    }
    const double bs = block_sum(v, s_red);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = bs;
        __threadfence();
        s_last = atomicAdd(counter, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    double t = 0.0;
    const volatile double *pp = partials;
    for (int q = threadIdx.x; q < (int)gridDim.x; q += kEpBlock) t += pp[q];
    const double tot = block_sum(t, s_red);
    if (threadIdx.x == 0) {
        *gap = tot;
        *counter = 0u;
    }
}

// dst = (float)(src * scale) in float64 on pitched rows (blockIdx.y = row).
__global__ void k_scale_pitched(const float *__restrict__ src, float *__restrict__ dst, int W,
                                int pitch, double scale) {
    const int j = blockIdx.x * 256 + threadIdx.x;
    const size_t o = (size_t)blockIdx.y * pitch + j;
    if (j < W) dst[o] = (float)((double)src[o] * scale);
}

struct SolverBuffers {
    float *g = nullptr, *gl = nullptr, *u = nullptr, *ub = nullptr;
    float *p1[2] = {nullptr, nullptr}, *p2[2] = {nullptr, nullptr};
    float *r1[2] = {nullptr, nullptr}, *r2[2] = {nullptr, nullptr};
    double *partials = nullptr, *gap = nullptr;
    unsigned *words = nullptr;  // [0] gap-reduction counter; [4..7] counter, status, barrier of the tiled path
};

}  // namespace

static tvspec_status check_rof_request(const tvspec_rof_request &q) {
    if (!q.g || !q.u) return fail(TVSPEC_EINVAL, "g and u are required");
    if (q.H < 1 || q.W < 1 || q.H > 65535 || (size_t)q.H * q.W > ((size_t)1 << 28))
        return fail(TVSPEC_EINVAL, "H, W must be >= 1 with H <= 65535 and H*W <= 2^28");
    if (!std::isfinite(q.lambda) || !(q.lambda > 0.0)) return fail(TVSPEC_EINVAL, "lambda must be > 0");
    if (q.solver < TVSPEC_SOLVER_CHAMBOLLE || q.solver > TVSPEC_SOLVER_FGP_REFERENCE)
        return fail(TVSPEC_EINVAL, "unknown solver");
    if (q.max_iter < 0 || q.max_iter > 10000000) return fail(TVSPEC_EINVAL, "max_iter out of range");
    if (q.check_every < 1) return fail(TVSPEC_EINVAL, "check_every must be >= 1");
    if (std::isnan(q.gap_tol)) return fail(TVSPEC_EINVAL, "gap_tol is NaN");
    if ((q.p1 == nullptr) != (q.p2 == nullptr) || (q.p1_in == nullptr) != (q.p2_in == nullptr))
        return fail(TVSPEC_EINVAL, "p1 and p2 must be given together");
    if (q.mem_kind != TVSPEC_MEM_HOST && q.mem_kind != TVSPEC_MEM_DEVICE) return fail(TVSPEC_EINVAL, "bad mem_kind");
    if (q.solver == TVSPEC_SOLVER_PDHG &&
        (!(q.pdhg_tau > 0.0f) || !(q.pdhg_sigma > 0.0f) || !(q.pdhg_gamma >= 0.0f) ||
         !std::isfinite(q.pdhg_tau) || !std::isfinite(q.pdhg_sigma) || !std::isfinite(q.pdhg_gamma) ||
         (double)q.pdhg_tau * q.pdhg_sigma * 8.0 > 1.0 + 1e-6))
        return fail(TVSPEC_EINVAL, "PDHG needs tau, sigma > 0, gamma >= 0 and 8 tau sigma <= 1");
    return TVSPEC_OK;
}

static tvspec_status rof_solve_locked(tvspec_plan *plan, tvspec_rof_request &q, cudaStream_t st) {
    const int H = q.H, W = q.W, pitch = (W + 3) / 4 * 4;
    const size_t pb = (size_t)H * pitch * sizeof(float);
    const int gap_blocks = H * ((W + kEpBlock - 1) / kEpBlock);
    const bool host = q.mem_kind == TVSPEC_MEM_HOST;
    // one allocation: g, gl, u, ub, p x2, p2 x2, r x2, r2 x2, partials, gap, words
    const size_t pa = (pb + 255) & ~(size_t)255;
    const size_t total = pa * 12 + (size_t)gap_blocks * 8 + 256 + 256;
    char *base = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&base, total, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TVSPEC_ENOMEM, "solver workspace");
    }
    SolverBuffers B;
    float **slots[12] = {&B.g, &B.gl, &B.u, &B.ub, &B.p1[0], &B.p1[1], &B.p2[0], &B.p2[1],
                         &B.r1[0], &B.r1[1], &B.r2[0], &B.r2[1]};
    for (int i = 0; i < 12; ++i) *slots[i] = reinterpret_cast<float *>(base + pa * i);
    B.partials = reinterpret_cast<double *>(base + pa * 12);
    B.gap = reinterpret_cast<double *>(base + pa * 12 + (((size_t)gap_blocks * 8 + 255) & ~(size_t)255));
    B.words = reinterpret_cast<unsigned *>(reinterpret_cast<char *>(B.gap) + 128);
    auto finish = [&](tvspec_status s) {
        cudaFreeAsync(base, st);
        cudaStreamSynchronize(st);
        return s;
    };
#define SV_CK(call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return finish(fail_cuda(e_, #call));   \
    } while (0)
    if (!plan->h_word) SV_CK(cudaMallocHost((void **)&plan->h_word, sizeof(double)));
    double *h_gap = plan->h_word;
    SV_CK(cudaMemsetAsync(base, 0, total, st));  // zero padding columns, p, r, words
    const cudaMemcpyKind in_kind = host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out_kind = host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const size_t row = (size_t)W * 4, prow = (size_t)pitch * 4;
    SV_CK(cudaMemcpy2DAsync(B.g, prow, q.g, row, row, H, in_kind, st));
    if (q.p1_in) {
        SV_CK(cudaMemcpy2DAsync(B.p1[0], prow, q.p1_in, row, row, H, in_kind, st));
        SV_CK(cudaMemcpy2DAsync(B.p2[0], prow, q.p2_in, row, row, H, in_kind, st));
    }
    const dim3 blk(kSolverBlockX, kSolverBlockY);
    const dim3 grid((W + kSolverBlockX - 1) / kSolverBlockX, (H + kSolverBlockY - 1) / kSolverBlockY);
    // gl = g / lambda for the dual methods (float64 quotient, as the decomposition forms it)
    k_scale_pitched<<<dim3((W + 255) / 256, H), 256, 0, st>>>(B.g, B.gl, W, pitch, 1.0 / q.lambda);
    SV_CK(cudaGetLastError());
    uint64_t nk = 1;
    if (q.solver == TVSPEC_SOLVER_PDHG) {  // u = ubar = g
        SV_CK(cudaMemcpyAsync(B.u, B.g, pb, cudaMemcpyDeviceToDevice, st));
        SV_CK(cudaMemcpyAsync(B.ub, B.g, pb, cudaMemcpyDeviceToDevice, st));
    }
    if (q.solver == TVSPEC_SOLVER_FGP || q.solver == TVSPEC_SOLVER_FGP_REFERENCE) {  // r = p
        SV_CK(cudaMemcpyAsync(B.r1[0], B.p1[0], pb, cudaMemcpyDeviceToDevice, st));
        SV_CK(cudaMemcpyAsync(B.r2[0], B.p2[0], pb, cudaMemcpyDeviceToDevice, st));
    }
    int cur_p = 0, cur_r = 0, it = 0;
    double t_fgp = 1.0, tau = q.pdhg_tau, sigma = q.pdhg_sigma, gap = NAN;
    bool gap_current = false;
    auto eval_gap = [&]() -> cudaError_t {
        const float *P1 = B.p1[cur_p], *P2 = B.p2[cur_p];
        if (q.solver != TVSPEC_SOLVER_PDHG) {
            k_primal_of_dual<<<grid, blk, 0, st>>>(P1, P2, B.g, B.u, H, W, pitch, q.lambda);
            ++nk;
        }
        k_gap<<<gap_blocks, kEpBlock, 0, st>>>(B.u, P1, P2, B.g, H, W, pitch, q.lambda, B.partials,
                                               B.words, B.gap);
        ++nk;
        cudaError_t e2 = cudaGetLastError();
        if (e2 == cudaSuccess) e2 = cudaMemcpyAsync(h_gap, B.gap, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
        if (e2 == cudaSuccess) gap = *h_gap;
        gap_current = true;
        return e2;
    };
    while (it < q.max_iter) {
        const int m = q.gap_tol > 0.0 ? std::min(q.check_every, q.max_iter - it) : q.max_iter - it;
        if (q.solver == TVSPEC_SOLVER_CHAMBOLLE) {
            ImgDesc d{};
            d.p1[0] = B.p1[cur_p];
            d.p1[1] = B.p1[cur_p ^ 1];
            d.p2[0] = B.p2[cur_p];
            d.p2[1] = B.p2[cur_p ^ 1];
            // the low parts of p (p = hi + lo) in FGP's momentum buffers, which Chambolle's
            // iteration does not use (zero from the workspace clear, carried across checks)
            d.q1[0] = B.r1[cur_p];
            d.q1[1] = B.r1[cur_p ^ 1];
            d.q2[0] = B.r2[cur_p];
            d.q2[1] = B.r2[cur_p ^ 1];
            d.gl = B.gl;
            d.counter = B.words + 4;
            d.status = B.words + 5;
            d.H = H;
            d.W = W;
            d.pitch = pitch;
            d.K = 1;
            d.n_inner = m;
            d.s0 = 0;
            d.dt = 1.0;
            d.inv_dt = 1.0;
            int fc = 0;
            tvspec_status s = run_iterations(plan, d, st, &fc);
            if (s != TVSPEC_OK) return finish(s);
            if (fc == 1) cur_p ^= 1;
        } else if (q.solver == TVSPEC_SOLVER_FGP_REFERENCE) {
            // one iteration per launch; p in place in copy 0, r ping-pong
            for (int k = 0; k < m; ++k) {
                const double t_new = (1.0 + std::sqrt(1.0 + 4.0 * t_fgp * t_fgp)) / 2.0;
                const double beta = (t_fgp - 1.0) / t_new;
                k_fgp<<<grid, blk, 0, st>>>(B.p1[0], B.p2[0], B.r1[cur_r], B.r2[cur_r], B.r1[cur_r ^ 1],
                                            B.r2[cur_r ^ 1], B.gl, H, W, pitch, (float)beta);
                cur_r ^= 1;
                t_fgp = t_new;
            }
            nk += m;
        } else if (q.solver == TVSPEC_SOLVER_FGP) {
            // temporally blocked: up to kFgpTB iterations per launch, p and r ping-pong together
            constexpr int OW = 32 * kFgpV - 2 * ((kFgpTB + kFgpV - 1) / kFgpV * kFgpV);
            constexpr int OH = kFgpRW * kFgpR - 2 * kFgpTB;
            const int ntx = (W + OW - 1) / OW, nty = (H + OH - 1) / OH;
            FgpDesc fd;
            fd.gl = B.gl;
            for (int c = 0; c < 2; ++c) {
                fd.p1[c] = B.p1[c];
                fd.p2[c] = B.p2[c];
                fd.r1[c] = B.r1[c];
                fd.r2[c] = B.r2[c];
            }
            fd.H = H;
            fd.W = W;
            fd.pitch = pitch;
            for (int done = 0; done < m;) {
                const int n = std::min(kFgpTB, m - done);
                FgpBetas bt{};
                for (int k = 0; k < n; ++k) {
                    const double t_new = (1.0 + std::sqrt(1.0 + 4.0 * t_fgp * t_fgp)) / 2.0;
                    bt.v[k] = (float)((t_fgp - 1.0) / t_new);
                    t_fgp = t_new;
                }
                k_fgp_tiled<kFgpV, kFgpR, kFgpRW, kFgpTB><<<ntx * nty, 32 * kFgpRW, 0, st>>>(fd, ntx, cur_p, n, bt);
                cur_p ^= 1;
                done += n;
                ++nk;
            }
        } else {
            for (int k = 0; k < m; ++k) {
                k_pdhg_dual<<<grid, blk, 0, st>>>(B.p1[0], B.p2[0], B.ub, H, W, pitch,
                                                  (float)(sigma / q.lambda));
                const double theta = q.pdhg_gamma > 0.0f ? 1.0 / std::sqrt(1.0 + 2.0 * q.pdhg_gamma * tau) : 1.0;
                k_pdhg_primal<<<grid, blk, 0, st>>>(B.u, B.ub, B.p1[0], B.p2[0], B.g, H, W, pitch,
                                                    (float)(tau * q.lambda), (float)tau, (float)theta);
                tau *= theta;
                sigma /= theta;
            }
            nk += 2 * (uint64_t)m;
        }
        SV_CK(cudaGetLastError());
        it += m;
        gap_current = false;
        if (q.gap_tol > 0.0) {
            SV_CK(eval_gap());
            if (gap <= q.gap_tol) break;
        }
    }
    if (!gap_current) SV_CK(eval_gap());
    plan->kernel_launches += nk;
    SV_CK(cudaMemcpy2DAsync(q.u, row, B.u, prow, row, H, out_kind, st));
    if (q.p1) {
        SV_CK(cudaMemcpy2DAsync(q.p1, row, B.p1[cur_p], prow, row, H, out_kind, st));
        SV_CK(cudaMemcpy2DAsync(q.p2, row, B.p2[cur_p], prow, row, H, out_kind, st));
    }
    q.iterations = it;
    q.gap = gap;
    return finish(TVSPEC_OK);
#undef SV_CK
}

}  // namespace tvspec

using namespace tvspec;

extern "C" tvspec_status tvspec_rof_solve(tvspec_plan *plan, tvspec_rof_request *req, void *stream) {
    NvtxRange range("tvspec rof_solve");
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    if (!req) return fail(TVSPEC_EINVAL, "request is NULL");
    tvspec_status s = check_rof_request(*req);
    if (s != TVSPEC_OK) return s;
    if (plan->cfg.p_storage != TVSPEC_P_FP32)
        return fail(TVSPEC_ENOTSUP, "tvspec_rof_solve needs p_storage = fp32");
    std::lock_guard<std::mutex> lock(plan->mu);
    TV_CK(cudaSetDevice(plan->device));
    cudaStream_t st = stream ? (cudaStream_t)stream : plan->stream;
    s = order_after(st, plan->stream);
    if (s != TVSPEC_OK) return s;
    s = rof_solve_locked(plan, *req, st);
    order_after(plan->stream, st);
    return s;
}
