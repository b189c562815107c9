// Tiled dual-iteration kernel with temporal blocking (the hot loop of every ROF step).
//
// One CTA owns a tile of TH = RW*R rows by TW = 32*V columns, held entirely in registers:
// lane l of warp wy owns columns [xs + lV, xs + lV + V) of rows [ys + wy R, ys + (wy+1) R).
// The CTA loads p1, p2 and g/lambda of its tile once, runs up to TB Chambolle iterations in
// registers, and stores the centre (the tile minus a halo of TB rows and roundup(TB, V)
// columns on each side). One iteration at a pixel reads p at the offsets (0,0), (+-1,0),
// (0,+-1), (+1,-1), (-1,+1), so after TB iterations exactly the centre is still exact; the
// halo is recomputed by the neighbouring tiles (overlapped tiling).
//
// Neighbour exchange inside an iteration:
//   - along a row (j +- 1): inside a lane's V columns in registers, across lanes by one warp
//     shuffle per row;
//   - along a column (i +- 1): inside a thread's R rows in registers, across warps through two
//     shared-memory rows per warp (the bottom row of p1, the top row of w), with two CTA
//     barriers per iteration.
//
// Image borders. Where the tiles are edge-aligned (tile_span: no tile reaches past the image),
// a tile on the left border sets p2_{i,-1} = 0 for its first column, one on the bottom border
// G1 = 0 on its last row and one on the right border G2 = 0 on its last column (the Neumann
// boundary); p1_{-1,j} = 0 holds for every tile's first row, whose upper neighbour is taken as
// zero. Otherwise pixels outside the image are loaded as zero and their gradient is masked to
// zero, so p stays zero there, which realises p1_{-1,j} = p2_{i,-1} = 0, and the gradient is
// masked on the last image row (G1) and column (G2). Tiles that touch none of the borders that
// need a condition skip all of them.
#pragma once

#include <cuda.h>  // CUtensorMap (a plain struct; no driver call in device code)

#include "chambolle_math.cuh"
#include "tvspec_internal.h"

namespace tvspec {

// Tensor maps of the tile loads by the tensor memory accelerator (option `tma`): the copy of
// p1 / p2 the launch reads, and g/lambda; 2-D float32 [H][W] with row stride pitch, box = the
// CTA's tile, zero fill outside the image.
struct TmaMaps {
    CUtensorMap p1, p2, gl;
};

template <typename P, int V>
struct alignas(sizeof(P) * V) PPack {
    P v[V];
};
template <int V>
struct alignas(sizeof(float) * V) FPack {
    float v[V];
};

// Border handling of tiled_iterate:
//   kEdgeNone   the tile touches no image border (no masks);
//   kEdgeMasked per-pixel masks m1bits / m2bits (bit r*V + v) for G1 / G2;
//   kEdgeExact  the tile is exactly the image (rows 0..RW*R-1, columns 0..32V-1): G1 is zero
//               on the last row and G2 on the last column, nothing else is masked. The same
//               values as kEdgeMasked with the masks of that image, with a select per row
//               instead of four per pixel pair.
//   kEdgeClamp  an edge-aligned tile on one or more image borders; m1bits holds this thread's
//               flags: kClampLeft (lane 0 of a tile on the left border: p2_{i,-1} = 0),
//               kClampRight (lane 31 on the right border: G2 = 0 on the last column),
//               kClampBottom (the last warp on the bottom border: G1 = 0 on the last row).
//               The same values as kEdgeMasked on the image's pixels.
constexpr int kEdgeNone = 0, kEdgeMasked = 1, kEdgeExact = 2, kEdgeClamp = 3;
constexpr unsigned kClampLeft = 1u, kClampRight = 2u, kClampBottom = 4u;

// The iterations of one launch on the registers of one thread. Pixels are processed in
// horizontal pairs (columns 2q, 2q+1 of the lane) with packed f32x2 arithmetic.
// ZERO_LEFT: the tile's first column is the image's first column (no halo), so lane 0's left
// neighbour p2_{i,-1} is 0 rather than a halo value.
// COMP (float32 storage): p is held as hi + lo (tv_update_acc): p1 / p2 carry the working
// value fl(hi + lo), l1 / l2 the low parts, and hi lives in this function; at the fold points
// (kFold) hi <- p, lo <- 0. The launch covers iterations [it0, it0 + n_iter) of a step of
// n_total, with it0 a fold point, so l1 / l2 start and end at zero and p = hi on entry and exit.
// Otherwise l1 / l2 are not touched.
// tau g/lambda of a thread's pixel pairs (glt of tv_wn), read by gl(r, j): held in registers
// (GlRegs), or in shared memory (GlShared: the thread's rows of a tile-sized array, for kernels
// that keep the registers for p). Kernels multiply g/lambda by tau as they load it.
template <int R, int VP>
struct GlRegs {
    const float2 (&a)[R][VP];
    __device__ __forceinline__ float2 operator()(int r, int j) const { return a[r][j]; }
};
struct GlShared {
    const float *base;  // the thread's first pixel: row ry, column lane * V of the tile
    int stride;         // floats per tile row
    __device__ __forceinline__ float2 operator()(int r, int j) const {
        return *reinterpret_cast<const float2 *>(base + r * stride + 2 * j);
    }
};

// Row exchange between the warps of a CTA. Warp wy needs p1 of the last row of warp wy - 1
// (for the divergence of its first row) and wn of the first row of warp wy + 1 (for the
// gradient of its last row); its other rows need only its own registers. So each iteration
// computes wn on rows 1..R-1 first, then on row 0 with p1 from above, and hands its wn row 0
// up; then, with wn from below read, it updates all rows and hands its p1 row R-1 down; two
// CTA barriers per iteration order the hand-offs. (Measured: this order is faster than rows in
// sequence in both phases and than putting the exchanged row last in both; faster too than
// pairwise named barriers between neighbouring warps, which let a warp wait for its neighbours
// only.) The function writes its first hand-off row itself; callers separate two calls by a CTA
// barrier (the exchange rows are reused). A call with n_iter <= 0 does nothing.
template <int V, int R, int RW, bool FAST, int EDGE, bool ZERO_LEFT = false, bool COMP = false,
          class GL>
__device__ __forceinline__ void tiled_iterate_g(float2 (&p1)[R][V / 2], float2 (&p2)[R][V / 2],
                                                float2 (&l1)[R][V / 2], float2 (&l2)[R][V / 2],
                                                const GL &gl, int n_iter, int it0, int n_total,
                                                float tau, unsigned m1bits, unsigned m2bits,
                                                float (*s_p1b)[32 * V], float (*s_wt)[32 * V],
                                                int lane, int wy) {
    constexpr unsigned FULL = 0xffffffffu;
    constexpr int VP = V / 2;
    if (n_iter <= 0) return;  // uniform over the CTA
    const float2 ntau2 = make_float2(-tau, -tau);
    float2 w[R][VP];  // wn = -tau (div p - g/lambda)
    float2 h1[R][VP], h2[R][VP];  // hi of the compensated form (COMP)
    if constexpr (COMP) {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < VP; ++j) {
                h1[r][j] = p1[r][j];
                h2[r][j] = p2[r][j];
            }
    }

    auto put_row = [&](float *dst, const float2 (&v)[VP]) {
        FPack<V> q;
#pragma unroll
        for (int j = 0; j < VP; ++j) {
            q.v[2 * j] = v[j].x;
            q.v[2 * j + 1] = v[j].y;
        }
        *reinterpret_cast<FPack<V> *>(dst + lane * V) = q;
    };
    auto get_row = [&](const float *src, float2 (&v)[VP]) {
        const FPack<V> q = *reinterpret_cast<const FPack<V> *>(src + lane * V);
#pragma unroll
        for (int j = 0; j < VP; ++j) v[j] = make_float2(q.v[2 * j], q.v[2 * j + 1]);
    };
    // wn = -tau w on row r, with p1 of the row above in upv
    auto wn_row = [&](int r, const float2 (&upv)[VP]) {
        float left0 = __shfl_up_sync(FULL, p2[r][VP - 1].y, 1);
        if (ZERO_LEFT && lane == 0) left0 = 0.0f;
        if (EDGE == kEdgeClamp && (m1bits & kClampLeft)) left0 = 0.0f;
#pragma unroll
        for (int j = 0; j < VP; ++j) {
            // the column differences of p2 as two scalar differences (the same roundings as a
            // packed difference with the left neighbours, without forming that pair)
            const float2 d2 = make_float2(__fsub_rn(p2[r][j].x, j == 0 ? left0 : p2[r][j - 1].y),
                                          __fsub_rn(p2[r][j].y, p2[r][j].x));
            w[r][j] = tv_wn2d(p1[r][j], upv[j], d2, gl(r, j), ntau2);
        }
    };
    // p <- (p + tau grad w) / (1 + tau |grad w|) on row r from na = grad wn = -tau grad w, with
    // wn of the row below in wdv
    auto update_row = [&](int r, const float2 (&wdv)[VP]) {
        const float right_last = __shfl_down_sync(FULL, w[r][0].x, 1);
#pragma unroll
        for (int j = 0; j < VP; ++j) {
            float2 na1 = sub2(wdv[j], w[r][j]);
            float2 na2 = make_float2(__fsub_rn(w[r][j].y, w[r][j].x),
                                     __fsub_rn(j < VP - 1 ? w[r][j + 1].x : right_last, w[r][j].y));
            if (EDGE == kEdgeMasked) {
                const int b0 = r * V + 2 * j;
                na1.x = ((m1bits >> b0) & 1u) ? na1.x : 0.0f;
                na1.y = ((m1bits >> (b0 + 1)) & 1u) ? na1.y : 0.0f;
                na2.x = ((m2bits >> b0) & 1u) ? na2.x : 0.0f;
                na2.y = ((m2bits >> (b0 + 1)) & 1u) ? na2.y : 0.0f;
            } else if (EDGE == kEdgeExact) {
                if (r == R - 1 && wy == RW - 1) na1 = make_float2(0.0f, 0.0f);  // last row
                if (j == VP - 1 && lane == 31) na2.y = 0.0f;                    // last column
            } else if (EDGE == kEdgeClamp) {
                if (r == R - 1 && (m1bits & kClampBottom)) na1 = make_float2(0.0f, 0.0f);
                if (j == VP - 1 && (m1bits & kClampRight)) na2.y = 0.0f;
            }
            if constexpr (COMP) {
                tv_update2_acc<FAST>(p1[r][j], p2[r][j], l1[r][j], l2[r][j], na1, na2);
                p1[r][j] = __fadd2_rn(h1[r][j], l1[r][j]);  // the row's new working value
                p2[r][j] = __fadd2_rn(h2[r][j], l2[r][j]);
            } else {
                tv_update2<FAST>(p1[r][j], p2[r][j], na1, na2);
            }
        }
    };

    // p1 of the last row for the warp below, as of the call's start
    if (RW > 1) {
        put_row(s_p1b[wy], p1[R - 1]);
        __syncthreads();
    }
    for (int it = 0; it < n_iter; ++it) {
        // ---- wn on rows 1..R-1, then on row 0 with p1 from the warp above (zero above the
        // tile's first row: a halo row, or the image's p1_{-1,j} = 0)
#pragma unroll
        for (int r = 1; r < R; ++r) wn_row(r, p1[r - 1]);
        float2 up[VP];
        if (RW > 1 && wy > 0) {
            get_row(s_p1b[wy - 1], up);
        } else {
#pragma unroll
            for (int j = 0; j < VP; ++j) up[j] = make_float2(0.0f, 0.0f);
        }
        wn_row(0, up);
        if (RW > 1) {
            put_row(s_wt[wy], w[0]);
            __syncthreads();
        }
        // ---- the update on every row, row R-1 with wn from the warp below (the tile's last
        // row: a halo row, or the image's last row, whose G1 is masked)
        float2 dn[VP];
        if (RW > 1 && wy < RW - 1) {
            get_row(s_wt[wy + 1], dn);
        } else {
#pragma unroll
            for (int j = 0; j < VP; ++j) dn[j] = w[R - 1][j];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) update_row(r, r < R - 1 ? w[r + 1] : dn);
        if constexpr (COMP) {
            const int done = it0 + it + 1;  // iterations of the step completed
            if (done % kFold == 0 || done == n_total) {  // uniform over the CTA
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int j = 0; j < VP; ++j) {  // hi <- fl(hi + lo) = p, lo <- 0
                        h1[r][j] = p1[r][j];
                        h2[r][j] = p2[r][j];
                        l1[r][j] = l2[r][j] = make_float2(0.0f, 0.0f);
                    }
            }
        }
        if (RW > 1 && it + 1 < n_iter) {  // (after the last iteration no one reads it)
            put_row(s_p1b[wy], p1[R - 1]);
            __syncthreads();
        }
    }
}

template <int V, int R, int RW, bool FAST, int EDGE, bool ZERO_LEFT = false, bool COMP = false>
__device__ __forceinline__ void tiled_iterate(float2 (&p1)[R][V / 2], float2 (&p2)[R][V / 2],
                                              float2 (&l1)[R][V / 2], float2 (&l2)[R][V / 2],
                                              const float2 (&gl)[R][V / 2], int n_iter, int it0,
                                              int n_total, float tau, unsigned m1bits, unsigned m2bits,
                                              float (*s_p1b)[32 * V], float (*s_wt)[32 * V],
                                              int lane, int wy) {
    tiled_iterate_g<V, R, RW, FAST, EDGE, ZERO_LEFT, COMP>(
        p1, p2, l1, l2, GlRegs<R, V / 2>{gl}, n_iter, it0, n_total, tau, m1bits, m2bits, s_p1b,
        s_wt, lane, wy);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// The tile of p1, p2 and g/lambda at (xs, ys) into shared memory by three TMA copies (issued by
// one thread, completing on one mbarrier), then each thread's own pixels into its registers:
// the values the per-thread loads give (the maps read zeros outside the image, as those loads
// substitute). The wait is bounded: if any thread runs out, the CTA sets kStatusCopyTimeout
// and returns false (uniformly), and the host reports the call as timed out.
constexpr long kTmaSpinLimit = 1l << 22;

template <int V, int R, int RW>
__device__ __forceinline__ bool tma_tile_load(const TmaMaps &tm, int xs, int ys, unsigned *status,
                                              float2 (&p1)[R][V / 2], float2 (&p2)[R][V / 2],
                                              float2 (&gl)[R][V / 2], int lane, int wy) {
    constexpr int VP = V / 2;
    constexpr int TW = 32 * V;
    constexpr int TH = RW * R;
    __shared__ __align__(128) float s_tile[3][TH][TW];
    __shared__ __align__(8) unsigned long long s_bar;
    const uint32_t bar = smem_addr(&s_bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                     "r"((unsigned)(3 * TH * TW * sizeof(float)))
                     : "memory");
        const CUtensorMap *maps[3] = {&tm.p1, &tm.p2, &tm.gl};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(&s_tile[a][0][0])),
                "l"(reinterpret_cast<uint64_t>(maps[a])), "r"(xs), "r"(ys), "r"(bar)
                : "memory");
    }
    uint32_t done = 0;
    for (long it = 0; it < kTmaSpinLimit && !done; ++it)
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(bar)
            : "memory");
    if (__syncthreads_or(!done)) {
        if (threadIdx.x == 0) atomicOr(status, kStatusCopyTimeout);
        return false;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int row = wy * R + r;
        const FPack<V> a = *reinterpret_cast<const FPack<V> *>(&s_tile[0][row][lane * V]);
        const FPack<V> b = *reinterpret_cast<const FPack<V> *>(&s_tile[1][row][lane * V]);
        const FPack<V> c = *reinterpret_cast<const FPack<V> *>(&s_tile[2][row][lane * V]);
#pragma unroll
        for (int j = 0; j < VP; ++j) {
            p1[r][j] = make_float2(a.v[2 * j], a.v[2 * j + 1]);
            p2[r][j] = make_float2(b.v[2 * j], b.v[2 * j + 1]);
            gl[r][j] = make_float2(c.v[2 * j], c.v[2 * j + 1]);
        }
    }
    return true;
}

// One CTA's work on tile (tx, ty) of image d: load, iterate, store the centre. TMA: the tile
// is loaded by tma_tile_load from the maps tm (float32 p only). Float32 storage updates p with
// the compensated form (hi + lo in registers, folded every kFold iterations); 16-bit storage
// rounds p between launches anyway and updates it directly.
// WAIT: the caller has neither waited for the preceding grid nor released the next one
// (programmatic dependent launch). g/lambda, which no launch of a step writes, is then loaded
// before the wait on every launch but a step's first (whose g/lambda the preceding epilogue
// writes), and p after it. The next grid is released only after the wait: a grid released
// earlier could start, and read g/lambda, while this one's predecessor still writes it.
template <int V, int R, int RW, int TB, typename P, bool FAST, bool TMA = false, bool WAIT = false>
__device__ __forceinline__ void tiled_tile(const ImgDesc &d, int tx, int ty, int gstep, int blk,
                                           int depth, float tau, const TmaMaps *tm = nullptr) {
    static_assert(R * V <= 32, "mask bits");
    static_assert(V % 2 == 0, "pixels are processed in pairs");
    constexpr int VP = V / 2;
    constexpr int TW = 32 * V;
    constexpr int TH = RW * R;
    constexpr int HX = (TB + V - 1) / V * V;
    constexpr int OW = TW - 2 * HX;
    constexpr int OH = TH - 2 * TB;
    static_assert(OW > 0 && OH > 0, "tile smaller than its halo");
    __shared__ __align__(16) float s_p1b[RW][TW];
    __shared__ __align__(16) float s_wt[RW][TW];

    const int H = d.H, W = d.W, pitch = d.pitch;
    // launch blk advances every tile by iterations [blk*depth, min((blk+1)*depth, n_inner));
    // depth <= TB keeps the centre exact
    const int k = gstep - d.s0;
    const int n_iter = min(min(depth, TB), d.n_inner - blk * depth);
    if (k < 0 || k >= d.K || n_iter <= 0) return;  // uniform over the CTA
    const int src = p_copy(k, launches_per_step(d.n_inner, depth), blk);
    const P *__restrict__ gp1 = static_cast<const P *>(d.p1[src]);
    const P *__restrict__ gp2 = static_cast<const P *>(d.p2[src]);
    P *__restrict__ op1 = static_cast<P *>(d.p1[src ^ 1]);
    P *__restrict__ op2 = static_cast<P *>(d.p2[src ^ 1]);
    const float *__restrict__ ggl = d.gl;

    const int lane = threadIdx.x & 31;
    const int wy = threadIdx.x >> 5;
    const bool aligned = tiles_edge_aligned(H, W, TH, TW, V);
    const TileSpan spx = tile_span(tx, tile_count(W, TW, OW, aligned), W, TW, HX, OW, aligned);
    const TileSpan spy = tile_span(ty, tile_count(H, TH, OH, aligned), H, TH, TB, OH, aligned);
    const int xs = spx.s, ys = spy.s;
    const int cx = xs + lane * V;
    const int ry = ys + wy * R;
    const bool col_ok = (cx >= 0) && (cx < pitch);

    constexpr bool COMP = sizeof(P) == 4;
    float2 p1[R][VP], p2[R][VP], gl[R][VP];
    float2 l1[R][VP], l2[R][VP];  // low parts of p: zero at a launch's start (a fold point)
    if constexpr (COMP) {
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < VP; ++j) l1[r][j] = l2[r][j] = make_float2(0.0f, 0.0f);
    }
    if constexpr (TMA) {
        static_assert(sizeof(P) == 4, "TMA tile loads read float32 p");
        if (!tma_tile_load<V, R, RW>(*tm, xs, ys, d.status, p1, p2, gl, lane, wy)) return;
    } else {
        if (WAIT && blk == 0) {
            pdl_wait();
            pdl_trigger();
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
            if (col_ok && y >= 0 && y < H) {
                const FPack<V> c = *reinterpret_cast<const FPack<V> *>(ggl + (size_t)y * pitch + cx);
#pragma unroll
                for (int j = 0; j < VP; ++j) gl[r][j] = make_float2(c.v[2 * j], c.v[2 * j + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < VP; ++j) gl[r][j] = make_float2(0.0f, 0.0f);
            }
        }
        if (WAIT && blk != 0) {
            pdl_wait();
            pdl_trigger();
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
            if (col_ok && y >= 0 && y < H) {
                const size_t off = (size_t)y * pitch + cx;
                PPack<P, V> a = *reinterpret_cast<const PPack<P, V> *>(gp1 + off);
                PPack<P, V> b = *reinterpret_cast<const PPack<P, V> *>(gp2 + off);
#pragma unroll
                for (int j = 0; j < VP; ++j) {
                    p1[r][j] = make_float2(PStore<P>::load(a.v[2 * j]), PStore<P>::load(a.v[2 * j + 1]));
                    p2[r][j] = make_float2(PStore<P>::load(b.v[2 * j]), PStore<P>::load(b.v[2 * j + 1]));
                }
            } else {
#pragma unroll
                for (int j = 0; j < VP; ++j) p1[r][j] = p2[r][j] = make_float2(0.0f, 0.0f);
            }
        }
    }
    {
        const float2 tau2 = make_float2(tau, tau);  // glt = tau g/lambda, once per launch
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int j = 0; j < VP; ++j) gl[r][j] = __fmul2_rn(tau2, gl[r][j]);
    }

    // (a tile on the top border needs no condition: its first row's upper neighbour is zero)
    const bool interior = aligned ? !(spx.first || spx.last || spy.last)
                                  : ys >= 0 && ys + TH <= H - 1 && xs >= 0 && xs + TW <= W - 1;
    if (interior) {
        tiled_iterate<V, R, RW, FAST, kEdgeNone, false, COMP>(p1, p2, l1, l2, gl, n_iter, blk * depth,
                                                              d.n_inner, tau, 0u, 0u, s_p1b, s_wt,
                                                              lane, wy);
    } else if (aligned) {
        const unsigned flags = (spx.first && lane == 0 ? kClampLeft : 0u) |
                               (spx.last && lane == 31 ? kClampRight : 0u) |
                               (spy.last && wy == RW - 1 ? kClampBottom : 0u);
        tiled_iterate<V, R, RW, FAST, kEdgeClamp, false, COMP>(p1, p2, l1, l2, gl, n_iter, blk * depth,
                                                               d.n_inner, tau, flags, 0u, s_p1b,
                                                               s_wt, lane, wy);
    } else {
        unsigned m1 = 0u, m2 = 0u;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int c = cx + v;
                const bool cin = c >= 0 && c < W;
                if (y >= 0 && y < H - 1 && cin) m1 |= 1u << (r * V + v);
                if (y >= 0 && y < H && c >= 0 && c < W - 1) m2 |= 1u << (r * V + v);
            }
        }
        tiled_iterate<V, R, RW, FAST, kEdgeMasked, false, COMP>(p1, p2, l1, l2, gl, n_iter, blk * depth,
                                                                d.n_inner, tau, m1, m2, s_p1b, s_wt,
                                                                lane, wy);
    }

    // store the exact centre into the other copy (the halo this CTA read belongs to other
    // tiles' centres, which they write into that copy too, never into the one being read)
    if (cx >= spx.a && cx < spx.b) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
            if (y >= spy.a && y < spy.b) {
                const size_t off = (size_t)y * pitch + cx;
                PPack<P, V> a, b;
#pragma unroll
                for (int j = 0; j < VP; ++j) {
                    a.v[2 * j] = PStore<P>::store(p1[r][j].x);
                    a.v[2 * j + 1] = PStore<P>::store(p1[r][j].y);
                    b.v[2 * j] = PStore<P>::store(p2[r][j].x);
                    b.v[2 * j + 1] = PStore<P>::store(p2[r][j].y);
                }
                *reinterpret_cast<PPack<P, V> *>(op1 + off) = a;
                *reinterpret_cast<PPack<P, V> *>(op2 + off) = b;
            }
        }
    }
}

// Table form: CTA b works on tiles[b] of image descs[tiles[b].img] (batches of images).
template <int V, int R, int RW, int TB, int MINB, typename P, bool FAST>
__global__ void __launch_bounds__(32 * RW, MINB)
    k_tiled(const TileRef *__restrict__ tiles, const ImgDesc *__restrict__ descs, int gstep,
            int blk, int depth, float tau) {
    // nothing below may read what the preceding launch wrote before this point
    pdl_wait();
    pdl_trigger();
    const TileRef t = tiles[blockIdx.x];
    tiled_tile<V, R, RW, TB, P, FAST>(descs[t.img], t.tx, t.ty, gstep, blk, depth, tau);
}

// Single-image form: the descriptor travels in the kernel parameters and the tile follows
// from the block index, so a CTA starts its loads without first reading any table.
template <int V, int R, int RW, int TB, int MINB, typename P, bool FAST>
__global__ void __launch_bounds__(32 * RW, MINB)
    k_tiled_one(const __grid_constant__ ImgDesc d, int ntx, int gstep, int blk, int depth,
                float tau) {
    const int b = blockIdx.x;
    tiled_tile<V, R, RW, TB, P, FAST, false, true>(d, b % ntx, b / ntx, gstep, blk, depth, tau);
}

// Single-image form with TMA tile loads (option `tma`; the shapes tma_shape_ok accepts).
template <int V, int R, int RW, int TB, int MINB, bool FAST>
__global__ void __launch_bounds__(32 * RW, MINB)
    k_tiled_one_tma(const __grid_constant__ ImgDesc d, int ntx, int gstep, int blk, int depth,
                    float tau, const __grid_constant__ TmaMaps tm) {
    pdl_wait();
    pdl_trigger();
    const int b = blockIdx.x;
    tiled_tile<V, R, RW, TB, float, FAST, true>(d, b % ntx, b / ntx, gstep, blk, depth, tau, &tm);
}

// Shape list: index (tile-shape id of the C ABI), columns per lane V, rows per thread R, warps
// RW, most iterations per launch TB, and the minimum CTAs per SM the register budget aims at
// (0: left to the compiler).
#define TVSPEC_TILE_SHAPES(X) \
    X(0, 4, 4, 16, 4, 0) \
    X(1, 4, 4, 16, 8, 0) \
    X(2, 4, 4, 8, 4, 0) \
    X(3, 4, 4, 8, 8, 0) \
    X(4, 2, 8, 8, 4, 0) \
    X(5, 2, 8, 8, 8, 0) \
    X(6, 2, 8, 16, 4, 0) \
    X(7, 2, 8, 16, 8, 0) \
    X(8, 2, 8, 4, 4, 0) \
    X(9, 4, 4, 16, 12, 0) \
    X(10, 2, 8, 16, 12, 0) \
    X(11, 2, 4, 8, 4, 0) \
    X(12, 2, 4, 16, 8, 0) \
    X(13, 2, 4, 32, 8, 0) \
    X(14, 2, 2, 32, 8, 0) \
    X(15, 4, 2, 32, 8, 0) \
    X(16, 2, 4, 16, 4, 0) \
    X(17, 2, 4, 32, 12, 0) \
    X(18, 2, 8, 8, 8, 3) \
    X(19, 2, 4, 16, 8, 2) \
    X(20, 2, 8, 8, 8, 4) \
    X(21, 2, 4, 8, 8, 4)         \
    X(22, 2, 8, 8, 8, 1)         \
    X(23, 4, 4, 8, 8, 1)         \
    X(24, 2, 7, 8, 8, 1)         \
    X(25, 2, 8, 7, 8, 1)         \
    X(26, 2, 6, 8, 6, 1)         \
    X(27, 2, 8, 6, 6, 1)         \
    X(28, 2, 4, 14, 8, 0)        \
    X(29, 2, 2, 28, 8, 0)

using TiledKernel = void (*)(const TileRef *, const ImgDesc *, int, int, int, float);
using TiledOneKernel = void (*)(const ImgDesc, int, int, int, int, float);
using TiledOneTmaKernel = void (*)(const ImgDesc, int, int, int, int, float, const TmaMaps);

}  // namespace tvspec
