// Internal data structures shared by the kernels and the host runtime.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace tvspec {

// Float32 storage of p: each pixel's dual value is held in registers as hi + lo (the
// compensated update of chambolle_math.cuh: lo accumulates the increments, the iteration reads
// fl(hi + lo)), and lo is folded into hi after every iteration i (0-based within an ROF step)
// with (i + 1) % kFold == 0 and after the step's last iteration. Every launch therefore starts and ends at a fold point (iterations per launch are
// multiples of kFold), p is stored as one float32 per component, and the results do not depend
// on the tile shape or the iterations per launch.
constexpr int kFold = 4;

// Most band edges a request may carry (n_edges <= kMaxEdges).
constexpr int kMaxEdges = 65;
// Pixels of one row chunk handled by one epilogue block.
constexpr int kEpBlock = 256;
// Device status bits written by kernels into ImgDesc::status.
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusBarrierTimeout = 2u;  // a bounded grid-barrier wait ran out
constexpr unsigned kStatusCopyTimeout = 4u;     // a bounded wait for a tile's TMA copies ran out

// One image of a launch set. Lives in device memory; kernels read it, the epilogue updates
// the per-image counter and status word.
struct ImgDesc {
    const float *f;         // input image (compact H*W), device
    // dual field, storage type of the plan, pitched (pitch elements), two copies: every
    // launch of dual iterations reads one copy and writes the other (tiles read halo pixels
    // that neighbouring tiles of the same launch update)
    void *p1[2], *p2[2];
    // float32 storage, reference kernel only (one iteration per launch, so a launch may end
    // between fold points): the low parts of p, same layout and copies as p1 / p2; nullptr
    // elsewhere (the tiled kernels keep them in registers)
    float *q1[2], *q2[2];
    float *gl;              // g / lambda of the current ROF step, float32, pitched
    double *ua, *ub;        // u ping-pong (compact H*W): u_k is ua for even k, ub for odd k
    double *u3;             // third u buffer of the split epilogue: u_k in {ua, ub, u3}[k % 3]
    double *acc;            // running sum of the active band (compact H*W)
    float *bands;           // (n_bands) H W output (compact), device
    float *residual;        // H W output (compact), device
    double *S;              // K-1 output, device
    double *u_trace;        // optional (K+1) H W output, device, or nullptr
    double *partials;       // one partial |phi| sum per epilogue block
    unsigned *counter;      // epilogue blocks finished in the current step; counter[2..3]
                            // hold the persistent kernel's grid barrier (arrivals, generation)
    unsigned *status;       // device status bits (counter + 1)
    unsigned *tile_flags;   // one epoch word per tile of the neighbour-synchronised persistent
                            // kernel (zero at the start of a decomposition), or nullptr
    const signed char *band_of_k;  // K entries: band of t_k (host-decided in float64), -1 none
    int n_filters;          // spectral filters fused into the epilogue
    const double *filt_H;   // n_filters x (K-1): H_q(t_k) at q*(K-1) + k-1
    const double *filt_res; // n_filters residual weights
    double *facc;           // n_filters x H x W running filter sums (compact)
    float *filtered;        // n_filters x H x W output (compact), device
    int acc_mode;           // 0: float64 epilogue; 1: compensated float32 (float-float); the
                            // u, acc and facc arrays then hold (hi, lo) float pairs
    float ff_dt[2], ff_inv_dt[2], ff_coef[2];  // dt, 1/dt, 1/dt^2 as float-float (acc_mode 1)
    double *S_par;          // K-1 values <phi_k, f>, or nullptr (not requested)
    double *partials_par;   // per-epilogue-block partial sums of phi_k f
    int H, W, pitch;
    int K, n_inner;
    int s0;                 // global step at which this image's step 0 runs
    int n_bands;
    int ep_blocks;          // epilogue blocks of this image (H * ceil(W / kEpBlock))
    double dt;              // lambda of every step
    double inv_dt;          // 1 / dt (float64)
};

// Copy of the dual field read by launch blk (0-based) of local step k when every step runs
// nb = ceil(n_inner / depth) launches and step 0 starts from copy 0: the copy flips once per
// launch, so launch blk of step k reads copy (k nb + blk) mod 2 and the epilogue of step k
// reads copy ((k+1) nb) mod 2.
__host__ __device__ __forceinline__ int p_copy(int k, int nb, int blk) {
    return (((k & 1) & (nb & 1)) + blk) & 1;
}
__host__ __device__ __forceinline__ int launches_per_step(int n_inner, int depth) {
    return (n_inner + depth - 1) / depth;
}

// Placement of the tiled kernel's tiles along one image axis of n pixels, for a tile of T
// pixels with a halo of h on each side (centre c = T - 2h):
//  * edge-aligned, when the image is at least one tile long in both directions and its width a
//    multiple of the columns per lane V: tile t < m - 1 reads [t c, t c + T) and the last one
//    [n - T, n); tile 0 stores [0, c + h), tile t [t c + h, (t + 1) c + h), the last
//    [(m - 1) c + h, n). No tile reaches past the image, so the border conditions reduce to a
//    few selects on the tile's first column and last row and column, instead of per-pixel
//    masks; every stored pixel lies at least h from the edges of its tile that are not image
//    borders, so it is exact after up to h iterations;
//  * otherwise: tile t reads [t c - h, t c + c + h) and stores [t c, t c + c); the pixels
//    outside the image are masked.
__host__ __device__ __forceinline__ bool tiles_edge_aligned(int H, int W, int TH, int TW, int V) {
    return H >= TH && W >= TW && W % V == 0;
}
__host__ __device__ __forceinline__ int tile_count(int n, int T, int c, bool aligned) {
    return aligned ? 1 + (n - T + c - 1) / c : (n + c - 1) / c;
}
struct TileSpan {
    int s;       // first pixel the tile reads
    int a, b;    // pixels [a, b) the tile stores
    bool first;  // the tile starts at the image's first pixel (edge-aligned placement)
    bool last;   // the tile ends at the image's last pixel (edge-aligned placement)
};
__host__ __device__ __forceinline__ TileSpan tile_span(int t, int m, int n, int T, int h, int c,
                                                       bool aligned) {
    TileSpan sp;
    if (aligned) {
        sp.first = t == 0;
        sp.last = t == m - 1;
        sp.s = sp.last ? n - T : t * c;
        sp.a = sp.first ? 0 : t * c + h;
        sp.b = sp.last ? n : (t + 1) * c + h;
    } else {
        sp.first = sp.last = false;
        sp.s = t * c - h;
        sp.a = t * c;
        sp.b = t * c + c < n ? t * c + c : n;
    }
    return sp;
}

// One tile of the tiled dual-iteration kernel: image index and tile coordinates.
struct TileRef {
    int img;
    int tx, ty;
};

// Storage conversions for the dual field.
template <typename P> struct PStore;
template <> struct PStore<float> {
    static __device__ __forceinline__ float load(float x) { return x; }
    static __device__ __forceinline__ float store(float x) { return x; }
};
template <> struct PStore<__half> {
    static __device__ __forceinline__ float load(__half x) { return __half2float(x); }
    static __device__ __forceinline__ __half store(float x) { return __float2half_rn(x); }
};
template <> struct PStore<__nv_bfloat16> {
    static __device__ __forceinline__ float load(__nv_bfloat16 x) { return __bfloat162float(x); }
    static __device__ __forceinline__ __nv_bfloat16 store(float x) { return __float2bfloat16_rn(x); }
};
// SNORM16: the dual field lies in the unit ball (|p| <= 1), so a 16-bit signed fixed-point
// value q / 32767 covers it with a uniform step of 1/32767 (half a step of rounding error).
template <> struct PStore<short> {
    static __device__ __forceinline__ float load(short x) {
        return __fmul_rn(__int2float_rn((int)x), 1.0f / 32767.0f);
    }
    static __device__ __forceinline__ short store(float x) {
        const float c = fminf(fmaxf(x, -1.0f), 1.0f);
        return (short)__float2int_rn(__fmul_rn(c, 32767.0f));
    }
};

// ---- launchers (defined in the .cu files) -------------------------------------------------

// Tile shapes available to the tiled kernel.
struct TileShape {
    int V;      // columns per lane
    int R;      // rows per thread
    int RW;     // warps per block (stacked vertically)
    int TB;     // most iterations per launch (the halo width)
};
int tiled_shape_count();
TileShape tiled_shape(int index);
// Output tile (columns, rows) of a shape: (32 V - 2 roundup(TB, V), RW R - 2 TB).
void tiled_output_tile(const TileShape &s, int *ow, int *oh);
// Tiles of one image for a shape along x and y (tile_count, edge-aligned where
// tiles_edge_aligned allows).
void tiles_for(int shape, int H, int W, int *ntx, int *nty);

// Launch one tiled pass of global step gstep: every CTA advances its tile by
// min(depth, n_inner - blk depth) iterations (depth <= the shape's TB), reading copy
// p_copy(k, nb, blk) of the dual field and writing the other. p_storage: 0 fp32, 1 fp16, 2 bf16, 3 snorm16.
// With pdl, the launch may start while the preceding kernel in the stream drains
// (programmatic dependent launch); the kernels wait for it before touching any data.
cudaError_t launch_tiled(int shape, int p_storage, bool fast, const TileRef *tiles, int n_tiles,
                         const ImgDesc *descs, int gstep, int blk, int depth, float tau,
                         cudaStream_t st, bool pdl = false);

// The same pass over the tiles of one image whose descriptor is passed by value (no table
// reads before the tile loads). Available for p_storage 0 (tiled_one_available).
bool tiled_one_available(int p_storage);
// CTAs of the tiled kernel of a shape that fit on one SM (occupancy, asked once per kernel).
int tiled_ctas_per_sm(int shape, int p_storage, bool fast, bool one);
// tma: load the tile with the tensor memory accelerator where the shape allows it
// (tma_shape_ok: float32 p, the tile's first column 16-byte aligned for every tile, the tile in
// static shared memory); other shapes ignore it.
cudaError_t launch_tiled_one(int shape, int p_storage, bool fast, const ImgDesc &d, int gstep,
                             int blk, int depth, float tau, cudaStream_t st, bool pdl = false,
                             bool tma = false);
bool tma_shape_ok(int shape, int p_storage);

// Persistent form: all of a step's dual iterations for one image in one cooperative launch
// (fp32 storage). step_coop_fits says whether all tiles can be resident at once.
bool step_coop_fits(int shape, bool fast, int n_tiles);
cudaError_t launch_step_coop(int shape, bool fast, const ImgDesc &d, int gstep, int depth,
                             float tau, unsigned long long timeout_ns, int noshow_block,
                             cudaStream_t st);
// The same persistent step with neighbour-only synchronisation (epoch flags in d.tile_flags,
// one word per tile of the shape); step_nbr_fits says whether all tiles can be resident.
bool step_nbr_fits(int shape, bool fast, int n_tiles);
cudaError_t launch_step_nbr(int shape, bool fast, const ImgDesc &d, int gstep, int depth,
                            float tau, unsigned long long timeout_ns, int noshow_block,
                            cudaStream_t st);
// Most tiles any tile shape makes of an H x W image (the size of a tile-flag array).
int max_tiles_for(int H, int W);

// Resident small-image kernel: the whole decomposition of each image idx[0..n) of descs in
// one CTA (fp32). resident_variant_for gives the variant whose tile holds an H x W image, or -1.
int resident_variant_for(int H, int W, int preferred = -1);
int resident_variant_count();
bool resident_variant_info(int i, int *max_h, int *max_w, int *threads, int *minb);
// parseval: some image of the launch wants the Parseval-type spectrum (twice the shared memory).
cudaError_t launch_resident(int variant, bool fast, const ImgDesc *descs, const int *idx, int n,
                            float tau, int warm_start, bool parseval, cudaStream_t st);

// One iteration per launch over one image (reference GPU kernel): p_in -> p_out.
// Float32 storage needs the low-part arrays (q*_in of iteration `it` within a step of n_total).
cudaError_t launch_naive(int p_storage, bool fast, const void *p1_in, const void *p2_in,
                         void *p1_out, void *p2_out, const float *q1_in, const float *q2_in,
                         float *q1_out, float *q2_out, const float *gl, int H, int W, int pitch,
                         float tau, int it, int n_total, cudaStream_t st);

// Start of a decomposition for every image owning one of the epilogue blocks
// [block_offset, block_offset + n_blocks) of the ep_img/ep_base list:
// u_0 = f, gl = f / dt, trace[0] = f; non-finite f sets kStatusNonFinite. p, acc and the
// padding columns must already be zero.
cudaError_t launch_init(const ImgDesc *descs, const int *ep_img, const int *ep_base,
                        int n_blocks, cudaStream_t st, int block_offset = 0);

// Per-step epilogue over every epilogue block listed in ep_img/ep_base (one entry per block):
// u_{k+1} = u_k - dt div p, gl = u_{k+1}/dt, phi_k, S(t_k), band accumulation, residual.
// Each image's local step is gstep - s0; images outside [0, K) are skipped.
// `depth` is the iterations per launch of the step's dual iterations (1 for the reference
// kernel); it tells the epilogue which copy of p holds the step's result.
cudaError_t launch_epilogue(int p_storage, const ImgDesc *descs, const int *ep_img,
                            const int *ep_base, int n_blocks, int gstep, int depth,
                            cudaStream_t st, bool pdl = false);

// The epilogue of one image whose descriptor is passed by value (block b = local block b).
cudaError_t launch_epilogue_one(int p_storage, const ImgDesc &d, int gstep, int depth,
                                cudaStream_t st, bool pdl = false);

// The epilogue split in two (u in the three-buffer rotation ua / ub / u3, u_k in [k % 3]):
// the primal part (u_{k+1}, g/dt: all the next step's iterations need) and the spectral part
// (phi_k, S, bands, filters, residual), which may run beside the next step's iterations. The
// same per-pixel operations as the combined epilogue, so the same bits.
cudaError_t launch_epi_primal(int p_storage, const ImgDesc *descs, const int *ep_img,
                              const int *ep_base, int n_blocks, int gstep, int depth,
                              cudaStream_t st, bool pdl = false);
cudaError_t launch_epi_primal_one(int p_storage, const ImgDesc &d, int gstep, int depth,
                                  cudaStream_t st, bool pdl = false);
cudaError_t launch_epi_spectral(const ImgDesc *descs, const int *ep_img, const int *ep_base,
                                int n_blocks, int gstep, cudaStream_t st);
cudaError_t launch_epi_spectral_one(const ImgDesc &d, int gstep, cudaStream_t st);

// One ROF step's primal recovery for the standalone ROF entry: u = g - lambda div p (float32
// inputs, float32 output, compact layout for u and g, pitched p).
cudaError_t launch_rof_primal(const float *p1, const float *p2, int pitch, const float *g,
                              float *u, int H, int W, double lambda, cudaStream_t st);

// Many device-to-device copies in one launch: items[i] copies bytes from src to dst; first[i]
// is the index of item i's first chunk of kCopyChunk bytes (prefix sums), n_chunks the total.
struct CopyItem {
    const void *src;
    void *dst;
    size_t bytes;
};
constexpr size_t kCopyChunk = 16384;
cudaError_t launch_copy_list(const CopyItem *items, const unsigned *first, int n,
                             unsigned n_chunks, cudaStream_t st);

// Pitched copies between compact float images and pitched workspace arrays.
cudaError_t launch_gl_from_g(const float *g, float *gl, int H, int W, int pitch, double lambda,
                             cudaStream_t st);

}  // namespace tvspec
