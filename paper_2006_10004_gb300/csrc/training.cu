// Ground-truth generation for training (Sec. 4.1): crops of greyscale sources (some from
// windows twice as large, averaged over 2 x 2 blocks), standardisation to zero mean and unit
// standard deviation, the decompositions of all crops as one batch, and one gather of the
// outputs into crop-major arrays.
//
// The crops are written straight into the batch's per-image workspaces (no per-crop copies)
// and the outputs are gathered by one kernel, so a batch of thousands of crops costs a
// handful of launches besides the decomposition itself. Statistics are reduced in float64 in
// a fixed order (per-crop block trees, then one block over the crops), so they are
// deterministic; they match a sequential sum up to rounding.
#include <cmath>
#include <cstring>
#include <vector>

#include "epilogue.cuh"
#include "runtime.h"

namespace tvspec {

struct CropDev {
    int src, y, x, scale;
};

constexpr int kTrainBlock = 256;

__device__ __forceinline__ size_t grid_threads() { return (size_t)gridDim.x * blockDim.x; }
__device__ __forceinline__ size_t thread_index() {
    return (size_t)blockIdx.x * blockDim.x + threadIdx.x;
}

// raw[c][i][j] = (float)( sum_{a,b < s} src[y + s i + a][x + s j + b] / s^2 ), the block summed
// in row-major order in float64.
__global__ void __launch_bounds__(kTrainBlock)
    k_crop(const float *const *__restrict__ srcs, const int *__restrict__ src_w,
           const CropDev *__restrict__ crops, int n, int size, float *__restrict__ raw) {
    const size_t npx = (size_t)size * size, total = npx * n;
    for (size_t t = thread_index(); t < total; t += grid_threads()) {
        const int c = (int)(t / npx);
        const int p = (int)(t - (size_t)c * npx);
        const int i = p / size, j = p - (p / size) * size;
        const CropDev cr = crops[c];
        const float *src = srcs[cr.src];
        const size_t W = (size_t)src_w[cr.src];
        const int s = cr.scale;
        double sum = 0.0;
        for (int a = 0; a < s; ++a) {
            const float *row = src + (size_t)(cr.y + s * i + a) * W + (size_t)(cr.x + s * j);
            for (int b = 0; b < s; ++b) sum = __dadd_rn(sum, (double)row[b]);
        }
        raw[t] = __double2float_rn(__ddiv_rn(sum, (double)(s * s)));
    }
}

// out[c] = sum over crop c of x (centred == false) or of (x - mean)^2 with the crop's mean
// under `mode` (1: stats[0], 2: stats[2c]). One block per crop, fixed-order block tree.
template <bool CENTRED>
__global__ void __launch_bounds__(kTrainBlock)
    k_crop_moment(const float *__restrict__ raw, int n, int npx, int mode,
                  const double *__restrict__ stats, double *__restrict__ out) {
    __shared__ double s_red[kTrainBlock / 32];
    for (int c = blockIdx.x; c < n; c += gridDim.x) {
        const float *x = raw + (size_t)c * npx;
        const double m = CENTRED ? (mode == 1 ? stats[0] : stats[2 * c]) : 0.0;
        double v = 0.0;
        for (int p = threadIdx.x; p < npx; p += kTrainBlock) {
            const double d = __dsub_rn((double)x[p], m);
            v = CENTRED ? __dadd_rn(v, __dmul_rn(d, d)) : __dadd_rn(v, d);
        }
        const double t = block_sum(v, s_red);
        if (threadIdx.x == 0) out[c] = t;
    }
}

// Mode 1: one block sums the per-crop values in a fixed order; stats[which] = mean or
// deviation of the whole set. Mode 2: per crop. which = 0: mean = sum / npx; which = 1:
// deviation = sqrt(sum / npx).
__global__ void __launch_bounds__(kTrainBlock)
    k_crop_stats(const double *__restrict__ per_crop, int n, int npx, int mode, int which,
                 double *__restrict__ stats) {
    __shared__ double s_red[kTrainBlock / 32];
    if (mode == 1) {
        if (blockIdx.x != 0) return;
        double v = 0.0;
        for (int c = threadIdx.x; c < n; c += kTrainBlock) v = __dadd_rn(v, per_crop[c]);
        const double t = block_sum(v, s_red);
        if (threadIdx.x == 0) {
            const double q = __ddiv_rn(t, (double)n * (double)npx);
            stats[which] = which == 0 ? q : __dsqrt_rn(q);
        }
    } else {
        for (size_t c = thread_index(); c < (size_t)n; c += grid_threads()) {
            const double q = __ddiv_rn(per_crop[c], (double)npx);
            stats[2 * c + which] = which == 0 ? q : __dsqrt_rn(q);
        }
    }
}

// x' = (float)((x - mean) / sd) (sd == 0 -> 1), or x for mode 0; written into the image's
// workspace (the decomposition's f) and, if requested, into crops_out.
__global__ void __launch_bounds__(kTrainBlock)
    k_standardize(const float *__restrict__ raw, int n, int npx, int mode,
                  const double *__restrict__ stats, const ImgDesc *__restrict__ descs,
                  const int *__restrict__ slot_of, float *__restrict__ crops_out) {
    const size_t total = (size_t)npx * n;
    for (size_t t = thread_index(); t < total; t += grid_threads()) {
        const int c = (int)(t / npx);
        const int p = (int)(t - (size_t)c * npx);
        float v = raw[t];
        if (mode != 0) {
            const double m = (mode == 2) ? stats[2 * c] : stats[0];
            double sd = (mode == 2) ? stats[2 * c + 1] : stats[1];
            if (sd == 0.0) sd = 1.0;
            v = __double2float_rn(__ddiv_rn(__dsub_rn((double)v, m), sd));
        }
        const_cast<float *>(descs[slot_of[c]].f)[p] = v;
        if (crops_out) crops_out[t] = v;
    }
}

// bands / residual / S / status of every crop from its workspace into crop-major arrays.
__global__ void __launch_bounds__(kTrainBlock)
    k_gather(const ImgDesc *__restrict__ descs, const int *__restrict__ slot_of, int n, int npx,
             int nb, int km1, float *__restrict__ bands, float *__restrict__ residual,
             double *__restrict__ S, unsigned *__restrict__ status) {
    const size_t per = (size_t)(nb + 1) * npx;
    const size_t total = per * n;
    for (size_t t = thread_index(); t < total; t += grid_threads()) {
        const int c = (int)(t / per);
        const size_t r = t - (size_t)c * per;
        const ImgDesc &d = descs[slot_of[c]];
        if (r < (size_t)nb * npx) bands[(size_t)c * nb * npx + r] = d.bands[r];
        else residual[(size_t)c * npx + (r - (size_t)nb * npx)] = d.residual[r - (size_t)nb * npx];
    }
    const size_t ts = (size_t)km1 * n;
    for (size_t t = thread_index(); t < ts; t += grid_threads()) {
        const int c = (int)(t / km1);
        S[t] = descs[slot_of[c]].S[t - (size_t)c * km1];
    }
    for (size_t c = thread_index(); c < (size_t)n; c += grid_threads())
        status[c] = *descs[slot_of[c]].status;
}

static int grid_for(size_t work) {
    const size_t b = (work + kTrainBlock - 1) / kTrainBlock;
    return (int)std::max<size_t>(1, std::min<size_t>(b, (size_t)152 * 8));
}

// Stream-ordered scratch carved from one allocation.
struct Carve {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off = (off + std::max<size_t>(bytes, 1) + 255) & ~(size_t)255;
        return o;
    }
};

static tvspec_status check_training(const tvspec_training_request &q) {
    if (q.n_sources < 1 || !q.sources || !q.source_H || !q.source_W)
        return fail(TVSPEC_EINVAL, "sources, source_H and source_W are required (n_sources >= 1)");
    if (q.n_crops < 1 || !q.crops) return fail(TVSPEC_EINVAL, "n_crops must be >= 1 with crops");
    if (q.size < 1 || q.size > 4096) return fail(TVSPEC_EINVAL, "size must be in [1, 4096]");
    if ((size_t)q.n_crops * (size_t)q.size * (size_t)q.size > ((size_t)1 << 31))
        return fail(TVSPEC_EINVAL, "n_crops * size^2 exceeds 2^31");
    if (q.standardize < 0 || q.standardize > 3)
        return fail(TVSPEC_EINVAL, "standardize must be 0, 1, 2 or 3");
    if (q.standardize == 3 && (!std::isfinite(q.mean_std[0]) || !std::isfinite(q.mean_std[1]) ||
                               q.mean_std[1] < 0.0))
        return fail(TVSPEC_EINVAL, "mean_std must be finite with a deviation >= 0");
    if (!q.bands || !q.residual || !q.S) return fail(TVSPEC_EINVAL, "bands, residual and S are required");
    if (q.mem_kind != TVSPEC_MEM_HOST && q.mem_kind != TVSPEC_MEM_DEVICE)
        return fail(TVSPEC_EINVAL, "mem_kind must be TVSPEC_MEM_HOST or TVSPEC_MEM_DEVICE");
    for (int i = 0; i < q.n_sources; ++i) {
        if (!q.sources[i]) return fail(TVSPEC_EINVAL, "a source pointer is NULL");
        if (q.source_H[i] < 1 || q.source_W[i] < 1 ||
            (size_t)q.source_H[i] * (size_t)q.source_W[i] > ((size_t)1 << 30))
            return fail(TVSPEC_EINVAL, "source sizes must be >= 1 and at most 2^30 pixels");
    }
    for (int c = 0; c < q.n_crops; ++c) {
        const tvspec_crop &k = q.crops[c];
        if (k.src < 0 || k.src >= q.n_sources) return fail(TVSPEC_EINVAL, "crop source index out of range");
        if (k.scale < 1 || k.scale > 16) return fail(TVSPEC_EINVAL, "crop scale must be in [1, 16]");
        const long long side = (long long)k.scale * q.size;
        if (k.y < 0 || k.x < 0 || k.y + side > q.source_H[k.src] || k.x + side > q.source_W[k.src])
            return fail(TVSPEC_EINVAL, "crop window outside its source image");
    }
    return TVSPEC_OK;
}

static tvspec_status training_locked(tvspec_plan *plan, const tvspec_training_request &q,
                                     cudaStream_t user_st) {
    TV_CK(cudaSetDevice(plan->device));
    const int n = q.n_crops, size = q.size;
    const int npx = size * size;
    const bool host = q.mem_kind == TVSPEC_MEM_HOST;

    // one decomposition job per crop, all with the same schedule; f and the outputs live in
    // the workspaces and are filled / gathered by the kernels below
    static const float dummy = 0.0f;
    tvspec_request r{};
    r.f = &dummy;
    r.H = size;
    r.W = size;
    r.dt = q.dt;
    r.K = q.K;
    r.n_inner = q.n_inner;
    r.band_edges = q.band_edges;
    r.n_edges = q.n_edges;
    r.bands = q.bands;
    r.residual = q.residual;
    r.S = q.S;
    r.mem_kind = TVSPEC_MEM_DEVICE;
    Job j0;
    tvspec_status s = make_job(r, &j0);
    if (s != TVSPEC_OK) return s;
    const int nb = q.n_edges - 1, km1 = q.K - 1;
    std::vector<Job> jobs(n, j0);
    CacheEntry *E = nullptr;
    s = get_entry(plan, jobs, &E);
    if (s != TVSPEC_OK) return s;

    cudaStream_t st = user_st ? user_st : plan->stream;
    s = order_after(st, plan->stream);
    if (s != TVSPEC_OK) return s;

    // scratch: tables, raw crops, statistics, status words and (host mode) staging
    size_t src_px = 0;
    for (int i = 0; i < q.n_sources; ++i) src_px += (size_t)q.source_H[i] * q.source_W[i];
    Carve cv;
    const size_t o_crops = cv.take(sizeof(CropDev) * n);
    const size_t o_slot = cv.take(sizeof(int) * n);
    const size_t o_srcp = cv.take(sizeof(float *) * q.n_sources);
    const size_t o_srcw = cv.take(sizeof(int) * q.n_sources);
    const size_t o_raw = cv.take(sizeof(float) * (size_t)n * npx);
    const size_t o_sum = cv.take(sizeof(double) * n);
    const size_t o_stats = cv.take(sizeof(double) * std::max(2, 2 * n));
    const size_t o_status = cv.take(sizeof(unsigned) * n);
    const size_t o_src = host ? cv.take(sizeof(float) * src_px) : 0;
    const size_t o_bands = host ? cv.take(sizeof(float) * (size_t)n * nb * npx) : 0;
    const size_t o_res = host ? cv.take(sizeof(float) * (size_t)n * npx) : 0;
    const size_t o_S = host ? cv.take(sizeof(double) * (size_t)n * km1) : 0;
    const size_t o_cout = (host && q.crops_out) ? cv.take(sizeof(float) * (size_t)n * npx) : 0;
    char *base = nullptr;
    {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, plan->device) == cudaSuccess) {
            uint64_t keep = plan_budget(plan);
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    cudaError_t e = cudaMallocAsync((void **)&base, cv.off, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TVSPEC_ENOMEM, std::string("training scratch: ") + cudaGetErrorString(e));
    }
    auto done = [&](tvspec_status rs) {
        cudaFreeAsync(base, st);
        order_after(plan->stream, st);
        return rs;
    };
#define TR_CK(call)                                                      \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return done(fail_cuda(e_, #call));        \
    } while (0)

    std::vector<CropDev> hc(n);
    for (int c = 0; c < n; ++c) hc[c] = {q.crops[c].src, q.crops[c].y, q.crops[c].x, q.crops[c].scale};
    std::vector<int> slot_of(n);
    for (int i = 0; i < n; ++i) slot_of[E->order[i]] = i;
    std::vector<const float *> srcp(q.n_sources);
    std::vector<int> srcw(q.n_sources);
    size_t soff = 0;
    for (int i = 0; i < q.n_sources; ++i) {
        const size_t bytes = sizeof(float) * (size_t)q.source_H[i] * q.source_W[i];
        srcw[i] = q.source_W[i];
        if (host) {
            float *dst = reinterpret_cast<float *>(base + o_src) + soff;
            TR_CK(cudaMemcpyAsync(dst, q.sources[i], bytes, cudaMemcpyHostToDevice, st));
            srcp[i] = dst;
            soff += (size_t)q.source_H[i] * q.source_W[i];
        } else {
            srcp[i] = q.sources[i];
        }
    }
    TR_CK(cudaMemcpyAsync(base + o_crops, hc.data(), sizeof(CropDev) * n, cudaMemcpyHostToDevice, st));
    TR_CK(cudaMemcpyAsync(base + o_slot, slot_of.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    TR_CK(cudaMemcpyAsync(base + o_srcp, srcp.data(), sizeof(float *) * q.n_sources,
                          cudaMemcpyHostToDevice, st));
    TR_CK(cudaMemcpyAsync(base + o_srcw, srcw.data(), sizeof(int) * q.n_sources, cudaMemcpyHostToDevice, st));
    double *d_stats = reinterpret_cast<double *>(base + o_stats);
    if (q.standardize == 3)
        TR_CK(cudaMemcpyAsync(d_stats, q.mean_std, 2 * sizeof(double), cudaMemcpyHostToDevice, st));

    float *raw = reinterpret_cast<float *>(base + o_raw);
    const int *d_slot = reinterpret_cast<const int *>(base + o_slot);
    uint64_t nk = 0;
    k_crop<<<grid_for((size_t)n * npx), kTrainBlock, 0, st>>>(
        reinterpret_cast<const float *const *>(base + o_srcp), reinterpret_cast<const int *>(base + o_srcw),
        reinterpret_cast<const CropDev *>(base + o_crops), n, size, raw);
    TR_CK(cudaGetLastError());
    ++nk;
    const int mode = q.standardize;
    if (mode == 1 || mode == 2) {
        double *sums = reinterpret_cast<double *>(base + o_sum);
        const int mb = std::min(n, 152 * 8);
        k_crop_moment<false><<<mb, kTrainBlock, 0, st>>>(raw, n, npx, mode, d_stats, sums);
        k_crop_stats<<<mode == 1 ? 1 : grid_for(n), kTrainBlock, 0, st>>>(sums, n, npx, mode, 0, d_stats);
        k_crop_moment<true><<<mb, kTrainBlock, 0, st>>>(raw, n, npx, mode, d_stats, sums);
        k_crop_stats<<<mode == 1 ? 1 : grid_for(n), kTrainBlock, 0, st>>>(sums, n, npx, mode, 1, d_stats);
        TR_CK(cudaGetLastError());
        nk += 4;
    }
    float *cout = q.crops_out ? (host ? reinterpret_cast<float *>(base + o_cout) : q.crops_out) : nullptr;
    k_standardize<<<grid_for((size_t)n * npx), kTrainBlock, 0, st>>>(raw, n, npx, mode, d_stats,
                                                                     E->ls.d_descs, d_slot, cout);
    TR_CK(cudaGetLastError());
    ++nk;
    plan->kernel_launches += nk;
    s = launch_entry(plan, *E, st);
    if (s != TVSPEC_OK) return done(s);

    float *ob = host ? reinterpret_cast<float *>(base + o_bands) : q.bands;
    float *orr = host ? reinterpret_cast<float *>(base + o_res) : q.residual;
    double *oS = host ? reinterpret_cast<double *>(base + o_S) : q.S;
    unsigned *d_status = reinterpret_cast<unsigned *>(base + o_status);
    k_gather<<<grid_for((size_t)n * (nb + 1) * npx), kTrainBlock, 0, st>>>(
        E->ls.d_descs, d_slot, n, npx, nb, km1, ob, orr, oS, d_status);
    TR_CK(cudaGetLastError());
    plan->kernel_launches += 1;

    std::vector<unsigned> hstatus;
    const bool sync = host || q.stats;
    if (host) {
        TR_CK(cudaMemcpyAsync(q.bands, ob, sizeof(float) * (size_t)n * nb * npx, cudaMemcpyDeviceToHost, st));
        TR_CK(cudaMemcpyAsync(q.residual, orr, sizeof(float) * (size_t)n * npx, cudaMemcpyDeviceToHost, st));
        TR_CK(cudaMemcpyAsync(q.S, oS, sizeof(double) * (size_t)n * km1, cudaMemcpyDeviceToHost, st));
        if (q.crops_out)
            TR_CK(cudaMemcpyAsync(q.crops_out, cout, sizeof(float) * (size_t)n * npx, cudaMemcpyDeviceToHost, st));
        hstatus.resize(n);
        TR_CK(cudaMemcpyAsync(hstatus.data(), d_status, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, st));
    }
    if (q.stats) {
        const int ns = mode == 2 ? 2 * n : 2;
        if (mode == 0) {
            for (int i = 0; i < ns; ++i) q.stats[i] = 0.0;
        } else {
            TR_CK(cudaMemcpyAsync(q.stats, d_stats, sizeof(double) * ns, cudaMemcpyDeviceToHost, st));
        }
    }
    tvspec_status rs = done(TVSPEC_OK);
    if (sync) TV_CK(cudaStreamSynchronize(st));
#undef TR_CK
    if (rs != TVSPEC_OK) return rs;
    for (unsigned w : hstatus) {
        if (w & kStatusBarrierTimeout) return fail(TVSPEC_ETIMEOUT, "a grid barrier wait ran out");
        if (w & kStatusCopyTimeout) return fail(TVSPEC_ETIMEOUT, "a wait for a tile's TMA copies ran out");
        if (w & kStatusNonFinite) return fail(TVSPEC_ECUDA, "non-finite value in the flow");
    }
    plan->decompositions += n;
    return TVSPEC_OK;
}

}  // namespace tvspec

using namespace tvspec;

extern "C" tvspec_status tvspec_training_set(tvspec_plan *plan, const tvspec_training_request *req,
                                             void *stream) {
    NvtxRange range("tvspec training_set");
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    if (!req) return fail(TVSPEC_EINVAL, "request is NULL");
    tvspec_status s = check_training(*req);
    if (s != TVSPEC_OK) return s;
    std::lock_guard<std::mutex> lock(plan->mu);
    return training_locked(plan, *req, (cudaStream_t)stream);
}
