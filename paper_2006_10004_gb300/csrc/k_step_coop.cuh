// Persistent form of one ROF step's dual iterations for one image (cooperative launch).
//
// Every CTA owns one tile for the whole step: it loads its tile and g/dt once, then runs the
// step's launches-worth of iterations ("blocks" of `depth` iterations) back to back. After a
// block it stores its exact centre into the other copy of p, waits at a grid-wide barrier,
// and reloads only the halo ring (which neighbouring tiles have just updated); the centre and
// g/dt stay in registers. The per-pixel arithmetic and the sequence of copies of p are those
// of the one-launch-per-block path, so the results are bit-identical to it.
//
// The barrier's wait is bounded: a CTA that has waited longer than timeout_ns sets
// kStatusBarrierTimeout in the image's status word and leaves the kernel, so a missing CTA
// ends the kernel with an error the host reports instead of hanging the device. All loads use
// the L2-coherent path (__ldcg): after a barrier, lines another SM wrote may be stale in L1.
#pragma once

#include "k_tiled.cuh"

namespace tvspec {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier of a cooperative launch. bar[0] counts arrivals, bar[1] is the generation.
// Returns false when this CTA gave up waiting (status bit set).
__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned nblocks,
                                             unsigned long long timeout_ns, unsigned *status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();  // this CTA's stores are visible before it arrives
        const unsigned gen = atomicAdd(bar + 1, 0u);
        const unsigned arrived = atomicAdd(bar, 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            volatile unsigned *vgen = bar + 1;
            const unsigned long long t0 = global_ns();
            while (*vgen == gen) {
                if (global_ns() - t0 > timeout_ns) {
                    ok = 0;
                    atomicOr(status, kStatusBarrierTimeout);
                    break;
                }
                __nanosleep(128);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <int V>
__device__ __forceinline__ FPack<V> ldcg_pack(const float *p) {
    FPack<V> q;
    if constexpr (V == 2) {
        const float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
        q.v[0] = v.x;
        q.v[1] = v.y;
    } else {
        static_assert(V == 4, "V");
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(p));
        q.v[0] = v.x;
        q.v[1] = v.y;
        q.v[2] = v.z;
        q.v[3] = v.w;
    }
    return q;
}

template <int V, int R, int RW, int TB, int MINB, bool FAST>
__global__ void __launch_bounds__(32 * RW, MINB)
    k_step_coop(const __grid_constant__ ImgDesc d, int ntx, int gstep, int depth, float tau,
                unsigned long long timeout_ns, int noshow_block) {
    constexpr int VP = V / 2;
    constexpr int TW = 32 * V;
    constexpr int TH = RW * R;
    constexpr int HX = (TB + V - 1) / V * V;
    constexpr int OW = TW - 2 * HX;
    constexpr int OH = TH - 2 * TB;
    __shared__ __align__(16) float s_p1b[RW][TW];
    __shared__ __align__(16) float s_wt[RW][TW];

    const int k = gstep - d.s0;
    if (k < 0 || k >= d.K || d.n_inner <= 0) return;  // uniform over the grid (one image)
    unsigned *bar = d.counter + 2;  // [count, generation] next to the epilogue's counter
    const int nb = launches_per_step(d.n_inner, depth);
    int src = p_copy(k, nb, 0);
    const int H = d.H, W = d.W, pitch = d.pitch;
    const int lane = threadIdx.x & 31;
    const int wy = threadIdx.x >> 5;
    const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int x0 = tx * OW, y0 = ty * OH;
    const int xs = x0 - HX, ys = y0 - TB;
    const int cx = xs + lane * V;
    const int ry = ys + wy * R;
    const bool col_ok = (cx >= 0) && (cx < pitch);
    const bool col_centre = cx >= x0 && cx < x0 + OW;

    float2 p1[R][VP], p2[R][VP], gl[R][VP];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = ry + r;
        if (col_ok && y >= 0 && y < H) {
            const size_t off = (size_t)y * pitch + cx;
            const FPack<V> a = ldcg_pack<V>(static_cast<const float *>(d.p1[src]) + off);
            const FPack<V> b = ldcg_pack<V>(static_cast<const float *>(d.p2[src]) + off);
            const FPack<V> c = ldcg_pack<V>(d.gl + off);
#pragma unroll
            for (int j = 0; j < VP; ++j) {
                p1[r][j] = make_float2(a.v[2 * j], a.v[2 * j + 1]);
                p2[r][j] = make_float2(b.v[2 * j], b.v[2 * j + 1]);
                gl[r][j] = __fmul2_rn(make_float2(tau, tau), make_float2(c.v[2 * j], c.v[2 * j + 1]));
            }
        } else {
#pragma unroll
            for (int j = 0; j < VP; ++j) p1[r][j] = p2[r][j] = gl[r][j] = make_float2(0.0f, 0.0f);
        }
    }
    float2 l1[R][VP], l2[R][VP];  // low parts of p: zero at every block's start (a fold point)
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < VP; ++j) l1[r][j] = l2[r][j] = make_float2(0.0f, 0.0f);
    const bool interior = ys >= 0 && ys + TH <= H - 1 && xs >= 0 && xs + TW <= W - 1;
    unsigned m1 = 0u, m2 = 0u;
    if (!interior) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int c = cx + v;
                if (y >= 0 && y < H - 1 && c >= 0 && c < W) m1 |= 1u << (r * V + v);
                if (y >= 0 && y < H && c >= 0 && c < W - 1) m2 |= 1u << (r * V + v);
            }
        }
    }

    for (int blk = 0; blk < nb; ++blk) {
        const int n_iter = min(min(depth, TB), d.n_inner - blk * depth);
        if (interior)
            tiled_iterate<V, R, RW, FAST, kEdgeNone, false, true>(p1, p2, l1, l2, gl, n_iter,
                                                              blk * depth, d.n_inner, tau, 0u, 0u,
                                                              s_p1b, s_wt, lane, wy);
        else
            tiled_iterate<V, R, RW, FAST, kEdgeMasked, false, true>(p1, p2, l1, l2, gl, n_iter,
                                                                blk * depth, d.n_inner, tau, m1, m2,
                                                                s_p1b, s_wt, lane, wy);
        // the exact centre into the other copy
        float *o1 = static_cast<float *>(d.p1[src ^ 1]);
        float *o2 = static_cast<float *>(d.p2[src ^ 1]);
        if (col_centre && cx < W) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int y = ry + r;
                if (y >= y0 && y < y0 + OH && y < H) {
                    const size_t off = (size_t)y * pitch + cx;
                    FPack<V> a, b;
#pragma unroll
                    for (int j = 0; j < VP; ++j) {
                        a.v[2 * j] = p1[r][j].x;
                        a.v[2 * j + 1] = p1[r][j].y;
                        b.v[2 * j] = p2[r][j].x;
                        b.v[2 * j + 1] = p2[r][j].y;
                    }
                    *reinterpret_cast<FPack<V> *>(o1 + off) = a;
                    *reinterpret_cast<FPack<V> *>(o2 + off) = b;
                }
            }
        }
        if (blk == nb - 1) break;
        // fault-injection hook for tests: this CTA never arrives at the barrier
        if ((int)blockIdx.x == noshow_block) return;
        if (!grid_barrier(bar, gridDim.x, timeout_ns, d.status)) return;
        src ^= 1;
        // reload the halo ring from the copy every tile has just written
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
            const bool in_centre = col_centre && y >= y0 && y < y0 + OH;
            if (!in_centre && col_ok && y >= 0 && y < H) {
                const size_t off = (size_t)y * pitch + cx;
                const FPack<V> a = ldcg_pack<V>(static_cast<const float *>(d.p1[src]) + off);
                const FPack<V> b = ldcg_pack<V>(static_cast<const float *>(d.p2[src]) + off);
#pragma unroll
                for (int j = 0; j < VP; ++j) {
                    p1[r][j] = make_float2(a.v[2 * j], a.v[2 * j + 1]);
                    p2[r][j] = make_float2(b.v[2 * j], b.v[2 * j + 1]);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------------------------
// Persistent form with neighbour-only synchronisation. The same per-CTA work as k_step_coop
// (tile and g/dt in registers for the whole step, the centre stored after every block of
// `depth` iterations, the halo ring reloaded from the copy the neighbours have just written),
// but instead of a grid-wide barrier each CTA publishes an epoch number for its tile
// (flags[tile] = k nb + blk + 1 after block blk of local step k, released after the centre's
// stores) and waits only until its up to eight neighbours (the tiles whose centres its halo
// ring covers, diagonals included) have published the same epoch. A CTA is therefore never
// more than one block ahead of a neighbour, which is what the two copies of p need: the copy a
// CTA writes in block b + 1 is the one its neighbours read their halos from after block b - 1,
// and they have finished those reads before publishing block b.
//
// The flags must be zero at the start of a decomposition (they lie in the region cleared per
// decomposition) and increase from step to step. Each wait is bounded: a CTA that has waited
// longer than timeout_ns for a neighbour sets kStatusBarrierTimeout and leaves the kernel; its
// neighbours then time out in turn, and the host reports the call as timed out. The kernel is
// launched cooperatively, which guarantees that every CTA is resident, so no wait depends on a
// CTA that cannot start.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned *p, unsigned v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits (threads 0..8 of the CTA, one neighbour each) until every neighbour of tile (tx, ty)
// has published at least `epoch`. Returns false on every thread if some wait ran out.
constexpr long kNbrSpinLimit = 1l << 30;  // polls per wait; the time limit normally ends it first

__device__ __forceinline__ bool wait_neighbours(const unsigned *flags, int tx, int ty, int ntx,
                                                int nty, unsigned epoch,
                                                unsigned long long timeout_ns, unsigned *status) {
    int ok = 1;
    const int t = threadIdx.x;
    if (t < 9 && t != 4) {
        const int nx = tx + t % 3 - 1, ny = ty + t / 3 - 1;
        if (nx >= 0 && nx < ntx && ny >= 0 && ny < nty) {
            const unsigned *f = flags + (size_t)ny * ntx + nx;
            // poll with relaxed loads; one acquire fence once the epoch is seen
            if (ld_relaxed_gpu(f) < epoch) {
                const unsigned long long t0 = global_ns();
                long polls = 0;
                while (ld_relaxed_gpu(f) < epoch) {
                    if (++polls >= kNbrSpinLimit || ((polls & 63) == 0 && global_ns() - t0 > timeout_ns)) {
                        ok = 0;
                        atomicOr(status, kStatusBarrierTimeout);
                        break;
                    }
                }
            }
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
        }
    }
    return !__syncthreads_or(!ok);
}

template <int V, int R, int RW, int TB, int MINB, bool FAST>
__global__ void __launch_bounds__(32 * RW, MINB)
    k_step_nbr(const __grid_constant__ ImgDesc d, int ntx, int nty, int gstep, int depth,
               float tau, unsigned long long timeout_ns, int noshow_block) {
    constexpr int VP = V / 2;
    constexpr int TW = 32 * V;
    constexpr int TH = RW * R;
    constexpr int HX = (TB + V - 1) / V * V;
    constexpr int OW = TW - 2 * HX;
    constexpr int OH = TH - 2 * TB;
    // the halo ring lies within the centres of the eight neighbouring tiles
    static_assert(HX <= OW && TB <= OH, "halo wider than a neighbour's centre");
    __shared__ __align__(16) float s_p1b[RW][TW];
    __shared__ __align__(16) float s_wt[RW][TW];

    const int k = gstep - d.s0;
    if (k < 0 || k >= d.K || d.n_inner <= 0) return;  // uniform over the grid (one image)
    const int nb = launches_per_step(d.n_inner, depth);
    int src = p_copy(k, nb, 0);
    const int H = d.H, W = d.W, pitch = d.pitch;
    const int lane = threadIdx.x & 31;
    const int wy = threadIdx.x >> 5;
    const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
    const int x0 = tx * OW, y0 = ty * OH;
    const int xs = x0 - HX, ys = y0 - TB;
    const int cx = xs + lane * V;
    const int ry = ys + wy * R;
    const bool col_ok = (cx >= 0) && (cx < pitch);
    const bool col_centre = cx >= x0 && cx < x0 + OW;
    unsigned *flags = d.tile_flags;
    const unsigned epoch0 = (unsigned)k * (unsigned)nb;

    float2 p1[R][VP], p2[R][VP], gl[R][VP];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = ry + r;
        if (col_ok && y >= 0 && y < H) {
            const size_t off = (size_t)y * pitch + cx;
            const FPack<V> a = ldcg_pack<V>(static_cast<const float *>(d.p1[src]) + off);
            const FPack<V> b = ldcg_pack<V>(static_cast<const float *>(d.p2[src]) + off);
            const FPack<V> c = ldcg_pack<V>(d.gl + off);
#pragma unroll
            for (int j = 0; j < VP; ++j) {
                p1[r][j] = make_float2(a.v[2 * j], a.v[2 * j + 1]);
                p2[r][j] = make_float2(b.v[2 * j], b.v[2 * j + 1]);
                gl[r][j] = __fmul2_rn(make_float2(tau, tau), make_float2(c.v[2 * j], c.v[2 * j + 1]));
            }
        } else {
#pragma unroll
            for (int j = 0; j < VP; ++j) p1[r][j] = p2[r][j] = gl[r][j] = make_float2(0.0f, 0.0f);
        }
    }
    float2 l1[R][VP], l2[R][VP];  // low parts of p: zero at every block's start (a fold point)
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int j = 0; j < VP; ++j) l1[r][j] = l2[r][j] = make_float2(0.0f, 0.0f);
    const bool interior = ys >= 0 && ys + TH <= H - 1 && xs >= 0 && xs + TW <= W - 1;
    unsigned m1 = 0u, m2 = 0u;
    if (!interior) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
#pragma unroll
            for (int v = 0; v < V; ++v) {
                const int c = cx + v;
                if (y >= 0 && y < H - 1 && c >= 0 && c < W) m1 |= 1u << (r * V + v);
                if (y >= 0 && y < H && c >= 0 && c < W - 1) m2 |= 1u << (r * V + v);
            }
        }
    }

    for (int blk = 0; blk < nb; ++blk) {
        const int n_iter = min(min(depth, TB), d.n_inner - blk * depth);
        if (interior)
            tiled_iterate<V, R, RW, FAST, kEdgeNone, false, true>(p1, p2, l1, l2, gl, n_iter,
                                                              blk * depth, d.n_inner, tau, 0u, 0u,
                                                              s_p1b, s_wt, lane, wy);
        else
            tiled_iterate<V, R, RW, FAST, kEdgeMasked, false, true>(p1, p2, l1, l2, gl, n_iter,
                                                                blk * depth, d.n_inner, tau, m1, m2,
                                                                s_p1b, s_wt, lane, wy);
        // the exact centre into the other copy
        float *o1 = static_cast<float *>(d.p1[src ^ 1]);
        float *o2 = static_cast<float *>(d.p2[src ^ 1]);
        if (col_centre && cx < W) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int y = ry + r;
                if (y >= y0 && y < y0 + OH && y < H) {
                    const size_t off = (size_t)y * pitch + cx;
                    FPack<V> a, b;
#pragma unroll
                    for (int j = 0; j < VP; ++j) {
                        a.v[2 * j] = p1[r][j].x;
                        a.v[2 * j + 1] = p1[r][j].y;
                        b.v[2 * j] = p2[r][j].x;
                        b.v[2 * j + 1] = p2[r][j].y;
                    }
                    *reinterpret_cast<FPack<V> *>(o1 + off) = a;
                    *reinterpret_cast<FPack<V> *>(o2 + off) = b;
                }
            }
        }
        if (blk == nb - 1) break;
        const unsigned epoch = epoch0 + (unsigned)blk + 1u;
        // publish: every thread's stores of the centre, then the tile's epoch
        __syncthreads();
        if (threadIdx.x == 0 && (int)blockIdx.x != noshow_block) {  // noshow: fault-injection hook
            __threadfence();  // the CTA's stores (ordered before by the barrier) before the flag
            st_relaxed_gpu(flags + blockIdx.x, epoch);
        }
        if (!wait_neighbours(flags, tx, ty, ntx, nty, epoch, timeout_ns, d.status)) return;
        src ^= 1;
        // reload the halo ring from the copy the neighbours have just written
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int y = ry + r;
            const bool in_centre = col_centre && y >= y0 && y < y0 + OH;
            if (!in_centre && col_ok && y >= 0 && y < H) {
                const size_t off = (size_t)y * pitch + cx;
                const FPack<V> a = ldcg_pack<V>(static_cast<const float *>(d.p1[src]) + off);
                const FPack<V> b = ldcg_pack<V>(static_cast<const float *>(d.p2[src]) + off);
#pragma unroll
                for (int j = 0; j < VP; ++j) {
                    p1[r][j] = make_float2(a.v[2 * j], a.v[2 * j + 1]);
                    p2[r][j] = make_float2(b.v[2 * j], b.v[2 * j + 1]);
                }
            }
        }
    }
}

using StepCoopKernel = void (*)(const ImgDesc, int, int, int, float, unsigned long long, int);
using StepNbrKernel = void (*)(const ImgDesc, int, int, int, int, float, unsigned long long, int);

}  // namespace tvspec
