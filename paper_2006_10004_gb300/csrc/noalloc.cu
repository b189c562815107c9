// tvspec_decompose_noalloc: the decomposition for callers that must not allocate device memory.
//
// Who needs it: code that may not call cudaMalloc/cudaFree at the point where it runs, e.g.
//   - a thread working while another thread captures a CUDA graph in global capture mode
//     (any cudaMalloc in the process is then an error that also invalidates the capture),
//   - real-time loops that cannot afford the implicit device synchronisation a cudaMalloc or
//     cudaFree may perform,
//   - frameworks that reserve the device memory up front for their own pool, so that a foreign
//     allocation fails or fragments it.
// Such callers pass device pointers for the image and the outputs; every other buffer the
// decomposition needs (the two copies of the dual field, g/dt, u_k and u_{k-1}, the band
// accumulator, the reduction partials and the launch tables) is carved out of one file-scope
// device array of fixed size, which every GPU that loads this library holds until the
// process exits.
//
// The arithmetic is the plan path's (same kernels, float32 dual iterations, float64 epilogue,
// tau = 1/8, warm start), so the results equal tvspec_decompose with a default plan.
#include <cmath>
#include <cstring>
#include <mutex>

#include "runtime.h"

namespace tvspec {
namespace {

constexpr size_t kNoAllocBytes = size_t(48) << 20;  // 48 MiB
constexpr int kNoAllocMaxSide = 2048;
constexpr int kNoAllocMaxK = 4096;
constexpr int kNoAllocMaxTiles = 4096;
constexpr int kNoAllocShape = 5;      // tile shape (V=2, R=8, 8 warps, 8 iterations)
constexpr int kNoAllocDepth = 8;
constexpr float kNoAllocTau = 0.125f;
constexpr int kMaxDevices = 64;

// The shared scratch array. Host code must not take its address directly (the host-side name
// is only a stand-in); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the scratch array on `dev` (which must be current), looked up once.
tvspec_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(TVSPEC_ENOTSUP, "device index above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail_cuda(e, "cudaGetSymbolAddress of the scratch array");
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_addr[dev]);
    return TVSPEC_OK;
}

}  // namespace
}  // namespace tvspec

using namespace tvspec;

extern "C" tvspec_status tvspec_decompose_noalloc(const float *f, int H, int W, double dt, int K,
                                                  int n_inner, const double *band_edges,
                                                  int n_edges, float *bands, float *residual,
                                                  double *S, void *stream) {
    // ---- argument checks (host only) ----
    if (!f || !bands || !residual || !S || !band_edges) return fail(TVSPEC_EINVAL, "NULL pointer");
    if (H < 1 || W < 1 || H > kNoAllocMaxSide || W > kNoAllocMaxSide)
        return fail(TVSPEC_EINVAL, "no-allocation entry point: H and W must be in [1, 2048]");
    if (K < 2 || K > kNoAllocMaxK)
        return fail(TVSPEC_EINVAL, "no-allocation entry point: K must be in [2, 4096]");
    if (n_inner < 0 || n_inner > 10000000) return fail(TVSPEC_EINVAL, "n_inner must be in [0, 1e7]");
    if (!std::isfinite(dt) || !(dt > 0.0)) return fail(TVSPEC_EINVAL, "dt must be finite and > 0");
    if (n_edges < 2 || n_edges > kMaxEdges) return fail(TVSPEC_EINVAL, "n_edges must be in [2, 65]");
    if (!std::isfinite(band_edges[0]) || band_edges[0] < 0.0)
        return fail(TVSPEC_EINVAL, "band_edges[0] must be finite and >= 0");
    for (int m = 1; m < n_edges; ++m) {
        if (std::isnan(band_edges[m]) || !(band_edges[m] > band_edges[m - 1]))
            return fail(TVSPEC_EINVAL, "band edges must be strictly increasing");
        if (!std::isfinite(band_edges[m]) && m != n_edges - 1)
            return fail(TVSPEC_EINVAL, "only the last band edge may be infinite");
    }

    // ---- carve the scratch array ----
    const int pitch = (W + 3) / 4 * 4;
    const size_t N = (size_t)H * W;
    const size_t pb = (size_t)H * pitch * sizeof(float);
    const int ep_blocks = H * ((W + kEpBlock - 1) / kEpBlock);
    int ntx = 0, nty = 0;
    tiles_for(kNoAllocShape, H, W, &ntx, &nty);
    const int n_tiles = ntx * nty;
    if (n_tiles > kNoAllocMaxTiles) return fail(TVSPEC_ENOTSUP, "too many tiles");
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + (bytes ? bytes : 1));
        return o;
    };
    const size_t o_desc = take(sizeof(ImgDesc));
    const size_t o_tiles = take((size_t)n_tiles * sizeof(TileRef));
    const size_t o_epimg = take((size_t)ep_blocks * sizeof(int));
    const size_t o_epbase = take(sizeof(int));
    const size_t o_band = take((size_t)K);
    const size_t o_part = take((size_t)ep_blocks * sizeof(double));
    const size_t zero_begin = off;
    const size_t o_ctr = take(16);
    const size_t o_p1a = take(pb), o_p2a = take(pb), o_p1b = take(pb), o_p2b = take(pb);
    const size_t o_gl = take(pb);
    const size_t o_acc = take(N * sizeof(double));
    const size_t zero_end = off;
    const size_t o_ua = take(N * sizeof(double));
    const size_t o_ub = take(N * sizeof(double));
    if (off > kNoAllocBytes) {
        return fail(TVSPEC_EINVAL, "image too large for the no-allocation entry point: needs " +
                                       std::to_string(off) + " bytes of scratch, the array holds " +
                                       std::to_string(kNoAllocBytes) + " (48 MiB)");
    }

    int dev = 0;
    TV_CK(cudaGetDevice(&dev));
    unsigned char *base = nullptr;
    tvspec_status s = scratch_address(dev, &base);
    if (s != TVSPEC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;

    // ---- host-side tables (stack memory; copied into the array in stream order) ----
    signed char band_of_k[kNoAllocMaxK];
    band_of_k[0] = -1;
    for (int k = 1; k < K; ++k) {
        const double t = (double)k * dt;
        band_of_k[k] = -1;
        for (int m = 0; m + 1 < n_edges; ++m)
            if (band_edges[m] <= t && t < band_edges[m + 1]) {
                band_of_k[k] = (signed char)m;
                break;
            }
    }
    TileRef tiles[kNoAllocMaxTiles];
    for (int ty = 0, i = 0; ty < nty; ++ty)
        for (int tx = 0; tx < ntx; ++tx, ++i) tiles[i] = TileRef{0, tx, ty};
    ImgDesc d{};
    d.f = f;
    d.p1[0] = base + o_p1a;
    d.p2[0] = base + o_p2a;
    d.p1[1] = base + o_p1b;
    d.p2[1] = base + o_p2b;
    d.gl = reinterpret_cast<float *>(base + o_gl);
    d.ua = reinterpret_cast<double *>(base + o_ua);
    d.ub = reinterpret_cast<double *>(base + o_ub);
    d.acc = reinterpret_cast<double *>(base + o_acc);
    d.bands = bands;
    d.residual = residual;
    d.S = S;
    d.u_trace = nullptr;
    d.partials = reinterpret_cast<double *>(base + o_part);
    d.counter = reinterpret_cast<unsigned *>(base + o_ctr);
    d.status = d.counter + 1;
    d.band_of_k = reinterpret_cast<const signed char *>(base + o_band);
    d.H = H;
    d.W = W;
    d.pitch = pitch;
    d.K = K;
    d.n_inner = n_inner;
    d.s0 = 0;
    d.n_bands = n_edges - 1;
    d.ep_blocks = ep_blocks;
    d.dt = dt;
    d.inv_dt = 1.0 / dt;

    // Every call shares the array and finds the previous call's contents in it: clear what
    // the kernels expect to start at zero (dual field and its padding, g/dt padding, band
    // accumulator, reduction counter, status) and the caller's band output.
    const ImgDesc *d_desc = reinterpret_cast<const ImgDesc *>(base + o_desc);
    const TileRef *d_tiles = reinterpret_cast<const TileRef *>(base + o_tiles);
    const int *d_epimg = reinterpret_cast<const int *>(base + o_epimg);
    const int *d_epbase = reinterpret_cast<const int *>(base + o_epbase);
    TV_CK(cudaMemsetAsync(base + zero_begin, 0, zero_end - zero_begin, st));
    TV_CK(cudaMemsetAsync(base + o_epimg, 0, (size_t)ep_blocks * sizeof(int), st));  // all image 0
    TV_CK(cudaMemsetAsync(base + o_epbase, 0, sizeof(int), st));
    TV_CK(cudaMemsetAsync(bands, 0, (size_t)(n_edges - 1) * N * sizeof(float), st));
    TV_CK(cudaMemcpyAsync(base + o_desc, &d, sizeof(d), cudaMemcpyHostToDevice, st));
    TV_CK(cudaMemcpyAsync(base + o_tiles, tiles, (size_t)n_tiles * sizeof(TileRef),
                          cudaMemcpyHostToDevice, st));
    TV_CK(cudaMemcpyAsync(base + o_band, band_of_k, (size_t)K, cudaMemcpyHostToDevice, st));

    // ---- the decomposition: u_0 = f, then K steps of dual iterations + epilogue ----
    cudaError_t e = launch_init(d_desc, d_epimg, d_epbase, ep_blocks, st);
    if (e != cudaSuccess) return fail_cuda(e, "init launch");
    const int nb = launches_per_step(n_inner, kNoAllocDepth);
    for (int k = 0; k < K; ++k) {
        for (int b = 0; b < nb; ++b) {
            e = launch_tiled(kNoAllocShape, TVSPEC_P_FP32, true, d_tiles, n_tiles, d_desc, k, b,
                             kNoAllocDepth, kNoAllocTau, st);
            if (e != cudaSuccess) return fail_cuda(e, "tiled kernel launch");
        }
        e = launch_epilogue(TVSPEC_P_FP32, d_desc, d_epimg, d_epbase, ep_blocks, k,
                            kNoAllocDepth, st);
        if (e != cudaSuccess) return fail_cuda(e, "epilogue launch");
    }
    return TVSPEC_OK;
}
