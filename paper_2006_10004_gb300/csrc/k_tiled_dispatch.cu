// Shape table and launcher of the tiled dual-iteration kernel.
#include <atomic>
#include <mutex>

#include <cudaTypedefs.h>

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

// ---- TMA tile loads --------------------------------------------------------------------------
// Shapes with a TMA kernel: every tile's first column (tx * OW - HX, or tx * OW and W - TW for
// edge-aligned tiles) is a multiple of 4 floats (the 16-byte rule of a tiled TMA copy; OW and HX
// multiples of 4, and W for edge-aligned tiles, checked at launch), and the three
// TH x TW tiles plus the exchange rows fit the 48 KB of static shared memory.
#define TVSPEC_TMA_SHAPES(X) X(8, 2, 8, 4, 4, 0) X(24, 2, 7, 8, 8, 1) X(25, 2, 8, 7, 8, 1)

static TiledOneTmaKernel tma_kernel(int shape, bool fast) {
#define TVSPEC_TMA_CASE(idx, V, R, RW, TB, MINB) \
    case idx: return fast ? &k_tiled_one_tma<V, R, RW, TB, MINB, true> : &k_tiled_one_tma<V, R, RW, TB, MINB, false>;
    switch (shape) {
        TVSPEC_TMA_SHAPES(TVSPEC_TMA_CASE)
        default: return nullptr;
    }
#undef TVSPEC_TMA_CASE
}

bool tma_shape_ok(int shape, int p_storage) {
    if (p_storage != 0 || shape < 0 || shape >= tiled_shape_count() || !tma_kernel(shape, true))
        return false;
    const TileShape &s = kShapes[shape];
    int ow, oh;
    tiled_output_tile(s, &ow, &oh);
    const int hx = (s.TB + s.V - 1) / s.V * s.V;
    const size_t smem = 3u * (32u * s.V) * (s.RW * s.R) * 4u + 2u * s.RW * (32u * s.V) * 4u + 8u;
    return ow % 4 == 0 && hx % 4 == 0 && smem <= 48u * 1024u;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// A [H][W] float32 array with row stride pitch, read in TW x TH boxes, zeros outside.
static cudaError_t encode_map(CUtensorMap *m, const void *base, const ImgDesc &d, int tw, int th) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)d.W, (cuuint64_t)d.H};
    const cuuint64_t strides[1] = {(cuuint64_t)d.pitch * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)tw, (cuuint32_t)th};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides,
                           box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_tiled_one(int shape, int p_storage, bool fast, const ImgDesc &d, int gstep,
                             int blk, int depth, float tau, cudaStream_t st, bool pdl, bool tma) {
    if (shape < 0 || shape >= tiled_shape_count() || p_storage != 0) return cudaErrorInvalidValue;
    TiledOneKernel k = tiled_one_kernel_f32(shape, fast);
    if (!k) return cudaErrorInvalidValue;
    int ntx, nty;
    tiles_for(shape, d.H, d.W, &ntx, &nty);
    // edge-aligned tiles: the last column of tiles starts at W - TW, a multiple of 4 floats
    // only when W is
    const TileShape &s = kShapes[shape];
    const bool aligned = tiles_edge_aligned(d.H, d.W, s.RW * s.R, 32 * s.V, s.V);
    const bool use_tma = tma && tma_shape_ok(shape, p_storage) && (!aligned || d.W % 4 == 0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntx * nty));
    cfg.blockDim = dim3((unsigned)(32 * kShapes[shape].RW));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    if (!use_tma) return cudaLaunchKernelEx(&cfg, k, d, ntx, gstep, blk, depth, tau);
    // the copy of p this launch reads (as the kernel derives it); outside the image's steps
    // the kernel returns before loading, any copy will do
    const int kk = gstep - d.s0;
    const int src = (kk >= 0 && kk < d.K) ? p_copy(kk, launches_per_step(d.n_inner, depth), blk) : 0;
    const int tw = 32 * kShapes[shape].V, th = kShapes[shape].RW * kShapes[shape].R;
    TmaMaps tm;
    cudaError_t e = encode_map(&tm.p1, d.p1[src], d, tw, th);
    if (e == cudaSuccess) e = encode_map(&tm.p2, d.p2[src], d, tw, th);
    if (e == cudaSuccess) e = encode_map(&tm.gl, d.gl, d, tw, th);
    if (e != cudaSuccess) return e;
    return cudaLaunchKernelEx(&cfg, tma_kernel(shape, fast), d, ntx, gstep, blk, depth, tau, tm);
}

}  // namespace tvspec
