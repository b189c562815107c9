// Shape table and launcher of the tiled dual-iteration kernel.
#include <atomic>

#include "k_tiled.cuh"

namespace tvspec {

TiledKernel tiled_kernel_f32(int shape, bool fast);
TiledKernel tiled_kernel_f16(int shape, bool fast);
TiledKernel tiled_kernel_bf16(int shape, bool fast);
TiledKernel tiled_kernel_s16(int shape, bool fast);
TiledOneKernel tiled_one_kernel_f32(int shape, bool fast);

#define TVSPEC_SHAPE_ROW(idx, V, R, RW, TB, MINB) {V, R, RW, TB},
static const TileShape kShapes[] = {TVSPEC_TILE_SHAPES(TVSPEC_SHAPE_ROW)};
#undef TVSPEC_SHAPE_ROW

int tiled_shape_count() { return (int)(sizeof(kShapes) / sizeof(kShapes[0])); }

TileShape tiled_shape(int index) { return kShapes[index]; }

void tiled_output_tile(const TileShape &s, int *ow, int *oh) {
    const int hx = (s.TB + s.V - 1) / s.V * s.V;
    *ow = 32 * s.V - 2 * hx;
    *oh = s.RW * s.R - 2 * s.TB;
}

static TiledKernel table_kernel(int shape, int p_storage, bool fast) {
    switch (p_storage) {
        case 0: return tiled_kernel_f32(shape, fast);
        case 1: return tiled_kernel_f16(shape, fast);
        case 2: return tiled_kernel_bf16(shape, fast);
        case 3: return tiled_kernel_s16(shape, fast);
        default: return nullptr;
    }
}

int tiled_ctas_per_sm(int shape, int p_storage, bool fast, bool one) {
    constexpr int kMaxShapes = 64;
    // 0 = not asked yet; plans on several threads may fill an entry at once (same value)
    static std::atomic<int> cache[kMaxShapes][4][2][2];
    if (shape < 0 || shape >= tiled_shape_count() || shape >= kMaxShapes || p_storage < 0 ||
        p_storage > 3)
        return 1;
    std::atomic<int> &c = cache[shape][p_storage][fast ? 1 : 0][one ? 1 : 0];
    int v = c.load(std::memory_order_relaxed);
    if (v == 0) {
        int n = 0;
        const int threads = 32 * kShapes[shape].RW;
        cudaError_t e = (one && p_storage == 0)
                            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, tiled_one_kernel_f32(shape, fast), threads, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, table_kernel(shape, p_storage, fast), threads, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            n = 1;
        }
        v = n > 0 ? n : 1;
        c.store(v, std::memory_order_relaxed);
    }
    return v;
}

cudaError_t launch_tiled(int shape, int p_storage, bool fast, const TileRef *tiles, int n_tiles,
                         const ImgDesc *descs, int gstep, int blk, int depth, float tau,
                         cudaStream_t st, bool pdl) {
    if (shape < 0 || shape >= tiled_shape_count()) return cudaErrorInvalidValue;
    if (n_tiles <= 0) return cudaSuccess;
    TiledKernel k = table_kernel(shape, p_storage, fast);
    if (!k) return cudaErrorInvalidValue;
    const int threads = 32 * kShapes[shape].RW;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_tiles);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, tiles, descs, gstep, blk, depth, tau);
}

bool tiled_one_available(int p_storage) { return p_storage == 0; }

cudaError_t launch_tiled_one(int shape, int p_storage, bool fast, const ImgDesc &d, int gstep,
                             int blk, int depth, float tau, cudaStream_t st, bool pdl) {
    if (shape < 0 || shape >= tiled_shape_count() || p_storage != 0) return cudaErrorInvalidValue;
    TiledOneKernel k = tiled_one_kernel_f32(shape, fast);
    if (!k) return cudaErrorInvalidValue;
    int ow, oh;
    tiled_output_tile(kShapes[shape], &ow, &oh);
    const int ntx = (d.W + ow - 1) / ow, nty = (d.H + oh - 1) / oh;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntx * nty));
    cfg.blockDim = dim3((unsigned)(32 * kShapes[shape].RW));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, d, ntx, gstep, blk, depth, tau);
}

}  // namespace tvspec
