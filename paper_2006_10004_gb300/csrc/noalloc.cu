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
// The arithmetic is the plan path's (the same per-pixel operations in the tiled dual-iteration
// kernel and the per-step epilogue: float32 dual iterations, float64 epilogue, tau = 1/8, warm
// start), and a pixel's iterations do not depend on the tile shape, so the results are
// bit-identical to tvspec_decompose with a default plan.
//
// No host memory is read by the GPU work a call enqueues: the image descriptor travels in the
// kernels' parameters and the band of every t_k is written into the array by a kernel whose
// parameters carry it, so nothing on the stream refers to this function's stack.
#include <cmath>
#include <cstring>
#include <mutex>

#include <cudaTypedefs.h>

#include "runtime.h"

namespace tvspec {
namespace {

constexpr size_t kNoAllocBytes = size_t(48) << 20;  // 48 MiB
constexpr int kNoAllocMaxSide = 2048;
constexpr int kNoAllocMaxK = 4096;
constexpr int kNoAllocShape = 5;      // tile shape (V=2, R=8, 8 warps, 8 iterations)
constexpr int kNoAllocDepth = 8;
constexpr float kNoAllocTau = 0.125f;
constexpr int kMaxDevices = 64;

// The shared scratch array. Host code must not take its address directly (the host-side name
// is only a stand-in); the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The array's device address per device, with the context it was looked up in: a context
// torn down and created again (cudaDeviceReset) loads the module anew, possibly elsewhere.
struct ScratchAddr {
    unsigned long long ctx_id;
    void *addr;
};
std::mutex g_mu;
ScratchAddr g_addr[kMaxDevices] = {};

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Unique id of the calling thread's current context (0 when none is current or the driver
// entry points are unavailable); driver entry points found through the runtime, so the library
// does not link the driver library.
unsigned long long current_context_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        else
            cudaGetLastError();
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        else
            cudaGetLastError();
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    unsigned long long id = 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id + 1;  // never 0 for a real context
}

// Device address of the scratch array on `dev` (which must be current). Looked up by the first
// call in a context (that lookup may load the module, so it belongs before any stream capture)
// and again whenever the current context is not the one the cached address came from.
tvspec_status scratch_address(int dev, unsigned char **out) {
    if (dev < 0 || dev >= kMaxDevices) return fail(TVSPEC_ENOTSUP, "device index above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long ctx = current_context_id();
    ScratchAddr &c = g_addr[dev];
    if (!c.addr || ctx == 0 || c.ctx_id != ctx) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return fail_cuda(e, "cudaGetSymbolAddress of the scratch array");
        if (ctx == 0) ctx = current_context_id();  // the lookup made the context current
        c.addr = p;
        c.ctx_id = ctx;
    }
    *out = static_cast<unsigned char *>(c.addr);
    return TVSPEC_OK;
}

// A caller's buffer must be device (or managed) memory of the current device.
bool on_device(const void *ptr, int dev) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// The call's tables, carried into the array by a kernel's parameters (no host copy): the image
// descriptor the init kernel reads, and the band of every t_k (decided on the host in float64).
struct NoAllocTables {
    ImgDesc d;
    ImgDesc *d_dst;
    signed char *band_dst;
    int K;
    signed char band_of_k[kNoAllocMaxK];
};

__global__ void k_noalloc_tables(const __grid_constant__ NoAllocTables t) {
    for (int k = threadIdx.x; k < t.K; k += blockDim.x) t.band_dst[k] = t.band_of_k[k];
    if (threadIdx.x == 0) *t.d_dst = t.d;
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
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = up256(off + (bytes ? bytes : 1));
        return o;
    };
    const size_t o_desc = take(sizeof(ImgDesc));
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
    if (!on_device(f, dev) || !on_device(bands, dev) || !on_device(residual, dev) || !on_device(S, dev))
        return fail(TVSPEC_EINVAL, "no-allocation entry point: f, bands, residual and S must be "
                                   "device memory of the current device");
    unsigned char *base = nullptr;
    tvspec_status s = scratch_address(dev, &base);
    if (s != TVSPEC_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;

    // ---- the band of every t_k, decided on the host in float64 as the plan path does ----
    NoAllocTables tab;
    std::memset(&tab, 0, sizeof(tab));
    signed char *band_of_k = tab.band_of_k;
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
    ImgDesc *d_desc = reinterpret_cast<ImgDesc *>(base + o_desc);
    const int *d_epimg = reinterpret_cast<const int *>(base + o_epimg);
    const int *d_epbase = reinterpret_cast<const int *>(base + o_epbase);
    TV_CK(cudaMemsetAsync(base + zero_begin, 0, zero_end - zero_begin, st));
    TV_CK(cudaMemsetAsync(base + o_epimg, 0, (size_t)ep_blocks * sizeof(int), st));  // all image 0
    TV_CK(cudaMemsetAsync(base + o_epbase, 0, sizeof(int), st));
    TV_CK(cudaMemsetAsync(bands, 0, (size_t)(n_edges - 1) * N * sizeof(float), st));
    tab.d = d;
    tab.d_dst = d_desc;
    tab.band_dst = reinterpret_cast<signed char *>(base + o_band);
    tab.K = K;
    k_noalloc_tables<<<1, 256, 0, st>>>(tab);
    TV_CK(cudaGetLastError());

    // ---- the decomposition: u_0 = f, then K steps of dual iterations + epilogue ----
    cudaError_t e = launch_init(d_desc, d_epimg, d_epbase, ep_blocks, st);
    if (e != cudaSuccess) return fail_cuda(e, "init launch");
    const int nb = launches_per_step(n_inner, kNoAllocDepth);
    for (int k = 0; k < K; ++k) {
        for (int b = 0; b < nb; ++b) {
            e = launch_tiled_one(kNoAllocShape, TVSPEC_P_FP32, true, d, k, b, kNoAllocDepth,
                                 kNoAllocTau, st);
            if (e != cudaSuccess) return fail_cuda(e, "tiled kernel launch");
        }
        e = launch_epilogue_one(TVSPEC_P_FP32, d, k, kNoAllocDepth, st);
        if (e != cudaSuccess) return fail_cuda(e, "epilogue launch");
    }
    return TVSPEC_OK;
}
