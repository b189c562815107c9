// Host runtime: validation, device workspace, launch tables, autotuning, CUDA graphs and the
// plain / batched entry points of the C ABI.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <sstream>

#include "runtime.h"

namespace tvspec {

static thread_local std::string g_last_error;

tvspec_status fail(tvspec_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

tvspec_status fail_cuda(cudaError_t e, const char *what) {
    const tvspec_status s = (e == cudaErrorMemoryAllocation) ? TVSPEC_ENOMEM : TVSPEC_ECUDA;
    return fail(s, std::string(what) + ": " + cudaGetErrorString(e));
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }
// resident = 1 uses the one-CTA-per-image kernel from this many eligible images on
constexpr int kResidentMinBatch = 32;
static int storage_bytes(int s) { return s == 0 ? 4 : 2; }
static int pitch_for(int W) { return (W + 3) / 4 * 4; }
static int ep_blocks_for(int H, int W) { return H * ((W + kEpBlock - 1) / kEpBlock); }

// ---------------------------------------------------------------------------------------------
// Validation. Band membership of t_k = k dt is decided here in float64 with the left-closed
// reading of Eq. spectral_bands: band m collects the phi_k with e_m <= t_k < e_{m+1}.
// ---------------------------------------------------------------------------------------------
tvspec_status make_job(const tvspec_request &req, Job *out) {
    if (req.H < 1 || req.W < 1) return fail(TVSPEC_EINVAL, "H and W must be >= 1");
    if ((size_t)req.H * (size_t)req.W > ((size_t)1 << 28))
        return fail(TVSPEC_EINVAL, "H*W exceeds 2^28");
    if (!std::isfinite(req.dt) || !(req.dt > 0.0)) return fail(TVSPEC_EINVAL, "dt must be finite and > 0");
    if (req.K < 2 || req.K > 100000) return fail(TVSPEC_EINVAL, "K must be in [2, 100000]");
    if (req.n_inner < 0 || req.n_inner > 10000000)
        return fail(TVSPEC_EINVAL, "n_inner must be in [0, 1e7]");
    if (req.n_edges < 2 || req.n_edges > kMaxEdges)
        return fail(TVSPEC_EINVAL, "n_edges must be in [2, 65]");
    if (!req.band_edges) return fail(TVSPEC_EINVAL, "band_edges is NULL");
    if (!req.f || !req.bands || !req.residual || !req.S)
        return fail(TVSPEC_EINVAL, "f, bands, residual and S must be non-NULL");
    if (req.mem_kind != TVSPEC_MEM_HOST && req.mem_kind != TVSPEC_MEM_DEVICE)
        return fail(TVSPEC_EINVAL, "mem_kind must be TVSPEC_MEM_HOST or TVSPEC_MEM_DEVICE");
    std::vector<double> e(req.band_edges, req.band_edges + req.n_edges);
    if (std::isnan(e[0]) || !std::isfinite(e[0]) || e[0] < 0.0)
        return fail(TVSPEC_EINVAL, "band_edges[0] must be finite and >= 0");
    for (int m = 1; m < req.n_edges; ++m) {
        if (std::isnan(e[m])) return fail(TVSPEC_EINVAL, "band edge is NaN");
        if (!(e[m] > e[m - 1])) return fail(TVSPEC_EINVAL, "band edges must be strictly increasing");
        if (!std::isfinite(e[m]) && m != req.n_edges - 1)
            return fail(TVSPEC_EINVAL, "only the last band edge may be infinite");
    }
    if (req.n_filters < 0 || req.n_filters > 64) return fail(TVSPEC_EINVAL, "n_filters must be in [0, 64]");
    if (req.n_filters > 0) {
        if (!req.filter_H || !req.filter_residual || !req.filtered)
            return fail(TVSPEC_EINVAL, "filter_H, filter_residual and filtered must be non-NULL");
        for (size_t q = 0; q < (size_t)req.n_filters * (req.K - 1); ++q)
            if (!std::isfinite(req.filter_H[q])) return fail(TVSPEC_EINVAL, "filter value is not finite");
        for (int q = 0; q < req.n_filters; ++q)
            if (!std::isfinite(req.filter_residual[q]))
                return fail(TVSPEC_EINVAL, "filter residual weight is not finite");
    }
    if (req.mem_kind == TVSPEC_MEM_HOST) {
        const size_t N = (size_t)req.H * (size_t)req.W;
        for (size_t n = 0; n < N; ++n)
            if (!std::isfinite(req.f[n])) return fail(TVSPEC_EINVAL, "f contains a non-finite value");
    }
    out->r = req;
    out->edges = e;
    out->band_of_k.assign(req.K, -1);
    for (int k = 1; k < req.K; ++k) {
        const double t = (double)k * req.dt;
        for (int m = 0; m + 1 < req.n_edges; ++m)
            if (e[m] <= t && t < e[m + 1]) {
                out->band_of_k[k] = (signed char)m;
                break;
            }
    }
    out->r.band_edges = out->edges.data();
    if (req.n_filters > 0) {
        out->filt_H.assign(req.filter_H, req.filter_H + (size_t)req.n_filters * (req.K - 1));
        out->filt_res.assign(req.filter_residual, req.filter_residual + req.n_filters);
        out->r.filter_H = out->filt_H.data();
        out->r.filter_residual = out->filt_res.data();
    } else {
        out->r.filter_H = nullptr;
        out->r.filter_residual = nullptr;
    }
    return TVSPEC_OK;
}

// ---------------------------------------------------------------------------------------------
// Workspace of one image. Layout of the single allocation:
//   band_of_k | f | p1 p2 p1' p2' gl acc bands partials counter,status | ua ub residual S [trace]
// The part from p1 to the status word is cleared at the start of every decomposition.
// ---------------------------------------------------------------------------------------------
struct SlotLayout {
    size_t band, fH, fres, f, p1, p2, q1, q2, l1a, l2a, l1b, l2b, gl, acc, facc, filt, bands, partials, ctr, flags, ua, ub,
        u3, res, S, tr, spar, ppar, zero_begin, zero_end, total;
    std::vector<std::pair<size_t, size_t>> guards;  // (offset, bytes) between and around arrays
};

// guard > 0 (test_guard_bytes, a multiple of 256): a guard region before the first array and
// after every array (its alignment slack plus `guard` bytes), for the write checks of
// slot_check_guards.
static SlotLayout layout_for(int H, int W, int K, int nb, int storage, bool naive, bool trace, int nf = 0,
                             bool par = false, size_t guard = 0) {
    SlotLayout L{};
    const size_t N = (size_t)H * W;
    const int pitch = pitch_for(W);
    const size_t pb = (size_t)H * pitch * storage_bytes(storage);
    size_t off = guard;
    if (guard) L.guards.push_back({0, guard});
    auto take = [&](size_t bytes) {
        const size_t o = off;
        const size_t end = o + std::max<size_t>(bytes, 1);
        off = a256(end) + guard;
        if (guard) L.guards.push_back({end, off - end});
        return o;
    };
    L.band = take(K);
    L.fH = take((size_t)nf * (K - 1) * 8);
    L.fres = take((size_t)nf * 8);
    L.f = take(N * 4);
    L.zero_begin = off;
    L.p1 = take(pb);
    L.p2 = take(pb);
    L.q1 = take(pb);
    L.q2 = take(pb);
    // float32 storage with the one-iteration reference kernel: the low parts of p (p = hi + lo)
    // of both copies, carried between its launches (the tiled kernels keep them in registers)
    const size_t lb = (storage == 0 && naive) ? (size_t)H * pitch * 4 : 0;
    L.l1a = take(lb);
    L.l2a = take(lb);
    L.l1b = take(lb);
    L.l2b = take(lb);
    L.gl = take((size_t)H * pitch * 4);
    L.acc = take(N * 8);
    L.bands = take((size_t)nb * N * 4);
    L.partials = take((size_t)ep_blocks_for(H, W) * 8);
    L.ctr = take(16);
    L.flags = take((size_t)max_tiles_for(H, W) * 4);  // persistent kernel's tile epochs
    L.zero_end = off;
    L.facc = take((size_t)nf * N * 8);  // written at k = 1 before any read
    L.filt = take((size_t)nf * N * 4);
    L.ua = take(N * 8);
    L.ub = take(N * 8);
    L.u3 = take(N * 8);
    L.res = take(N * 4);
    L.S = take((size_t)std::max(K - 1, 1) * 8);
    L.tr = trace ? take((size_t)(K + 1) * N * 8) : 0;
    L.spar = par ? take((size_t)std::max(K - 1, 1) * 8) : 0;
    L.ppar = par ? take((size_t)ep_blocks_for(H, W) * 8) : 0;
    L.total = off;
    return L;
}

static size_t guard_bytes(int g) { return g > 0 ? ((size_t)g + 255) / 256 * 256 : 0; }

size_t slot_bytes_for(const Job &j, int storage, bool naive, int guard) {
    return layout_for(j.r.H, j.r.W, j.r.K, j.r.n_edges - 1, storage, naive, j.r.u_trace != nullptr,
                      j.r.n_filters, j.r.S_parseval != nullptr, guard_bytes(guard))
        .total;
}

tvspec_status slot_alloc(Slot *s, const Job &j, int storage, bool naive, cudaStream_t st,
                         bool async_alloc, int acc_mode, int guard) {
    const tvspec_request &r = j.r;
    const bool trace = r.u_trace != nullptr;
    const int nb = r.n_edges - 1;
    const bool par = r.S_parseval != nullptr;
    const SlotLayout L = layout_for(r.H, r.W, r.K, nb, storage, naive, trace, r.n_filters, par,
                                    guard_bytes(guard));
    char *base = nullptr;
    cudaError_t e = async_alloc ? cudaMallocAsync((void **)&base, L.total, st)
                                : cudaMalloc((void **)&base, L.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(TVSPEC_ENOMEM, std::string("workspace allocation: ") + cudaGetErrorString(e));
    }
    Slot x;
    x.H = r.H;
    x.W = r.W;
    x.pitch = pitch_for(r.W);
    x.K = r.K;
    x.n_inner = r.n_inner;
    x.n_bands = nb;
    x.storage = storage;
    x.trace = trace;
    x.naive = naive;
    x.async_alloc = async_alloc;
    x.dt = r.dt;
    x.base = base;
    x.bytes = L.total;
    x.zero_off = L.zero_begin;
    x.zero_bytes = L.zero_end - L.zero_begin;
    x.band_of_k = (signed char *)(base + L.band);
    x.f = (float *)(base + L.f);
    x.p1[0] = base + L.p1;
    x.p2[0] = base + L.p2;
    x.p1[1] = base + L.q1;
    x.p2[1] = base + L.q2;
    if (storage == 0 && naive) {
        x.lo1[0] = (float *)(base + L.l1a);
        x.lo2[0] = (float *)(base + L.l2a);
        x.lo1[1] = (float *)(base + L.l1b);
        x.lo2[1] = (float *)(base + L.l2b);
    }
    x.gl = (float *)(base + L.gl);
    x.acc = (double *)(base + L.acc);
    x.bands = (float *)(base + L.bands);
    x.partials = (double *)(base + L.partials);
    x.counter = (unsigned *)(base + L.ctr);
    x.status = x.counter + 1;
    x.tile_flags = (unsigned *)(base + L.flags);
    x.ua = (double *)(base + L.ua);
    x.ub = (double *)(base + L.ub);
    x.u3 = (double *)(base + L.u3);
    x.residual = (float *)(base + L.res);
    x.S = (double *)(base + L.S);
    x.utrace = trace ? (double *)(base + L.tr) : nullptr;
    x.n_filters = r.n_filters;
    x.filt_H = (double *)(base + L.fH);
    x.filt_res = (double *)(base + L.fres);
    x.facc = (double *)(base + L.facc);
    x.filtered = (float *)(base + L.filt);
    x.acc_mode = acc_mode;
    x.S_par = par ? (double *)(base + L.spar) : nullptr;
    x.partials_par = par ? (double *)(base + L.ppar) : nullptr;
    x.ep_blocks = ep_blocks_for(r.H, r.W);
    x.p_bytes = (size_t)r.H * x.pitch * storage_bytes(storage);
    x.guards = L.guards;
    e = cudaSuccess;
    if (!L.guards.empty()) {
        // guards inside the region cleared per decomposition must stay zero, the others keep
        // kGuardByte; the whole cleared region starts at zero (the resident kernel clears
        // only what it uses)
        for (const auto &g : L.guards)
            if (e == cudaSuccess && !(g.first >= L.zero_begin && g.first < L.zero_end))
                e = cudaMemsetAsync(base + g.first, kGuardByte, g.second, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(base + L.zero_begin, 0, L.zero_end - L.zero_begin, st);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(x.band_of_k, j.band_of_k.data(), r.K, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && r.n_filters > 0)
        e = cudaMemcpyAsync(x.filt_H, j.filt_H.data(), j.filt_H.size() * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && r.n_filters > 0)
        e = cudaMemcpyAsync(x.filt_res, j.filt_res.data(), j.filt_res.size() * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        if (async_alloc) cudaFreeAsync(base, st); else cudaFree(base);
        return fail_cuda(e, "band table upload");
    }
    *s = x;
    return TVSPEC_OK;
}

tvspec_status slot_check_guards(const Slot &s, cudaStream_t st) {
    if (s.guards.empty() || !s.base) return TVSPEC_OK;
    size_t total = 0;
    for (const auto &g : s.guards) total += g.second;
    std::vector<unsigned char> h(total);
    size_t o = 0;
    for (const auto &g : s.guards) {
        TV_CK(cudaMemcpyAsync(h.data() + o, s.base + g.first, g.second, cudaMemcpyDeviceToHost, st));
        o += g.second;
    }
    TV_CK(cudaStreamSynchronize(st));
    o = 0;
    for (const auto &g : s.guards) {
        const bool zeroed = g.first >= s.zero_off && g.first < s.zero_off + s.zero_bytes;
        const unsigned char want = zeroed ? 0 : kGuardByte;
        for (size_t i = 0; i < g.second; ++i)
            if (h[o + i] != want)
                return fail(TVSPEC_ECUDA, "workspace guard overwritten at byte " +
                                              std::to_string(g.first + i) + " of an image's workspace");
        o += g.second;
    }
    return TVSPEC_OK;
}

void slot_free(Slot *s, cudaStream_t st) {
    if (s->base) {
        if (s->async_alloc) cudaFreeAsync(s->base, st);
        else cudaFree(s->base);
    }
    s->base = nullptr;
}

ImgDesc slot_desc(const Slot &s, int s0) {
    ImgDesc d{};
    d.f = s.f;
    d.p1[0] = s.p1[0];
    d.p1[1] = s.p1[1];
    d.p2[0] = s.p2[0];
    d.p2[1] = s.p2[1];
    for (int c = 0; c < 2; ++c) {
        d.q1[c] = s.lo1[c];
        d.q2[c] = s.lo2[c];
    }
    d.gl = s.gl;
    d.ua = s.ua;
    d.ub = s.ub;
    d.u3 = s.u3;
    d.acc = s.acc;
    d.bands = s.bands;
    d.residual = s.residual;
    d.S = s.S;
    d.u_trace = s.utrace;
    d.partials = s.partials;
    d.counter = s.counter;
    d.status = s.status;
    d.tile_flags = s.tile_flags;
    d.band_of_k = s.band_of_k;
    d.n_filters = s.n_filters;
    d.filt_H = s.filt_H;
    d.filt_res = s.filt_res;
    d.facc = s.facc;
    d.filtered = s.filtered;
    d.S_par = s.S_par;
    d.partials_par = s.partials_par;
    d.acc_mode = s.acc_mode;
    {
        // float-float forms of dt, 1/dt, 1/dt^2 (hi = nearest float, lo = nearest float of the rest)
        auto split = [](double v, float *out) {
            out[0] = (float)v;
            out[1] = (float)(v - (double)out[0]);
        };
        const double inv = 1.0 / s.dt;
        split(s.dt, d.ff_dt);
        split(inv, d.ff_inv_dt);
        split(inv * inv, d.ff_coef);
    }
    d.H = s.H;
    d.W = s.W;
    d.pitch = s.pitch;
    d.K = s.K;
    d.n_inner = s.n_inner;
    d.s0 = s0;
    d.n_bands = s.n_bands;
    d.ep_blocks = s.ep_blocks;
    d.dt = s.dt;
    d.inv_dt = 1.0 / s.dt;
    return d;
}

// ---------------------------------------------------------------------------------------------
// Launch tables.
// ---------------------------------------------------------------------------------------------
void LaunchSet::release() {
    cudaFree(d_descs);
    cudaFree(d_tiles);
    cudaFree(d_ep_img);
    cudaFree(d_ep_base);
    d_descs = nullptr;
    d_tiles = nullptr;
    d_ep_img = d_ep_base = nullptr;
    cap_descs = cap_tiles = cap_ep = cap_base = 0;
}

void tiles_for(int shape, int H, int W, int *ntx, int *nty) {
    const TileShape s = tiled_shape(shape);
    int ow, oh;
    tiled_output_tile(s, &ow, &oh);
    const bool aligned = tiles_edge_aligned(H, W, s.RW * s.R, 32 * s.V, s.V);
    *ntx = tile_count(W, 32 * s.V, ow, aligned);
    *nty = tile_count(H, s.RW * s.R, oh, aligned);
}

template <typename T>
static tvspec_status grow_upload(T **dptr, size_t *cap, const std::vector<T> &h) {
    const size_t need = std::max<size_t>(h.size(), 1);
    if (need > *cap) {
        // cudaFree / cudaMalloc wait for the device: grow geometrically so that a table that
        // is rebuilt often (the serving loop's) reallocates only a few times
        const size_t grow = std::max(need, 2 * *cap);
        cudaFree(*dptr);
        *dptr = nullptr;
        *cap = 0;
        TV_CK(cudaMalloc((void **)dptr, grow * sizeof(T)));
        *cap = grow;
    }
    if (!h.empty()) TV_CK(cudaMemcpy(*dptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return TVSPEC_OK;
}

tvspec_status launchset_build(LaunchSet *ls, const std::vector<ImgDesc> &descs, int shape,
                              int depth) {
    const int n = (int)descs.size();
    std::vector<TileRef> tiles;
    std::vector<int> ep_img, ep_base(n);
    ls->tile_prefix.assign(n + 1, 0);
    ls->ep_prefix.assign(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const ImgDesc &d = descs[i];
        if (shape >= 0) {
            int ntx, nty;
            tiles_for(shape, d.H, d.W, &ntx, &nty);
            for (int ty = 0; ty < nty; ++ty)
                for (int tx = 0; tx < ntx; ++tx) tiles.push_back({i, tx, ty});
        }
        ls->tile_prefix[i + 1] = (int)tiles.size();
        ep_base[i] = (int)ep_img.size();
        for (int b = 0; b < d.ep_blocks; ++b) ep_img.push_back(i);
        ls->ep_prefix[i + 1] = (int)ep_img.size();
    }
    tvspec_status s;
    if ((s = grow_upload(&ls->d_descs, &ls->cap_descs, descs)) != TVSPEC_OK) return s;
    if ((s = grow_upload(&ls->d_tiles, &ls->cap_tiles, tiles)) != TVSPEC_OK) return s;
    if ((s = grow_upload(&ls->d_ep_img, &ls->cap_ep, ep_img)) != TVSPEC_OK) return s;
    if ((s = grow_upload(&ls->d_ep_base, &ls->cap_base, ep_base)) != TVSPEC_OK) return s;
    ls->n = n;
    ls->shape = shape;
    ls->depth = depth;
    ls->h_descs = descs;
    return TVSPEC_OK;
}

// ---------------------------------------------------------------------------------------------
// Tile choice. Every shape gives bit-identical float32 results (the per-pixel arithmetic does
// not depend on the tiling), so the autotuner may pick freely; with 16-bit storage of p the
// rounding points depend on the iterations per launch, so there the depth is fixed.
// ---------------------------------------------------------------------------------------------
// With float32 storage the iterations per launch are a multiple of kFold (every launch starts
// and ends at a fold point of the compensated update): a shape's most, or the configured
// temporal block, rounded down to one (at least kFold; every shape allows kFold).
static int default_depth(const tvspec_config &c, int shape) {
    const int TB = tiled_shape(shape).TB;
    if (c.p_storage != TVSPEC_P_FP32) return c.temporal_block > 0 ? std::min(c.temporal_block, TB) : std::min(8, TB);
    const int want = c.temporal_block > 0 ? std::min(c.temporal_block, TB) : TB;
    return std::max(kFold, want / kFold * kFold);
}

// ---------------------------------------------------------------------------------------------
// Tune cache file: lines "<prefix> <key> <shape> <depth> <pdl>", prefix = GPU model, SM count and a
// checksum of the tile-shape table, so that choices of another GPU or build are skipped.
// ---------------------------------------------------------------------------------------------
static std::string tune_prefix_for(int device) {
    cudaDeviceProp prop{};
    std::string name = "unknown";
    int sms = 0;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
        name = prop.name;
        sms = prop.multiProcessorCount;
    } else {
        cudaGetLastError();
    }
    for (char &ch : name)
        if (ch == ' ' || ch == '\t') ch = '_';
    uint64_t h = 1469598103934665603ull;  // FNV-1a over the shape table
    for (int i = 0; i < tiled_shape_count(); ++i) {
        const TileShape t = tiled_shape(i);
        for (int v : {t.V, t.R, t.RW, t.TB}) {
            h ^= (uint64_t)(v + 1);
            h *= 1099511628211ull;
        }
    }
    std::ostringstream o;
    o << name << "/sm" << sms << "/shapes" << tiled_shape_count() << "-" << std::hex << h;
    return o.str();
}

static void tune_cache_load(tvspec_plan *plan) {
    if (plan->tune_cache.empty()) return;
    FILE *fp = std::fopen(plan->tune_cache.c_str(), "r");
    if (!fp) return;
    char line[4096];
    while (std::fgets(line, sizeof(line), fp)) {
        std::istringstream in(line);
        std::string prefix, key;
        int shape = -1, depth = 0, pdl = 0;
        if (!(in >> prefix >> key >> shape >> depth)) continue;
        if (!(in >> pdl)) pdl = 0;
        if (prefix != plan->tune_prefix) continue;
        if (shape < 0 || shape >= tiled_shape_count() || depth < 1 || depth > tiled_shape(shape).TB ||
            (plan->cfg.p_storage == TVSPEC_P_FP32 && depth % kFold != 0))
            continue;
        plan->tune[key] = {shape, depth, pdl != 0};
    }
    std::fclose(fp);
}

static void tune_cache_append(tvspec_plan *plan, const std::string &key, int shape, int depth,
                              bool pdl) {
    if (plan->tune_cache.empty() || key.size() > 3500) return;  // lines stay below 4 KB
    static std::mutex file_mu;  // plans of one process append whole lines
    std::lock_guard<std::mutex> lk(file_mu);
    FILE *fp = std::fopen(plan->tune_cache.c_str(), "a");
    if (!fp) return;  // the cache is an optimisation: an unwritable file is not an error
    std::fprintf(fp, "%s %s %d %d %d\n", plan->tune_prefix.c_str(), key.c_str(), shape, depth,
                 pdl ? 1 : 0);
    std::fclose(fp);
}

tvspec_status choose_tiles(tvspec_plan *plan, const std::vector<Slot *> &slots, cudaStream_t st,
                           int *shape, int *depth, bool table_form, bool *pdl_out) {
    const tvspec_config &c = plan->cfg;
    bool pdl_dummy = false;
    bool *pdl = pdl_out ? pdl_out : &pdl_dummy;
    *pdl = false;
    if (c.kernel == TVSPEC_KERNEL_NAIVE) {
        *shape = -1;
        *depth = 1;
        return TVSPEC_OK;
    }
    std::vector<int> shapes;
    if (c.tile >= 0) {
        shapes.push_back(c.tile);
    } else {
        for (int s = 0; s < tiled_shape_count(); ++s) {
            if (c.p_storage != TVSPEC_P_FP32 && c.temporal_block == 0 && tiled_shape(s).TB < 8)
                continue;
            shapes.push_back(s);
        }
    }
    // time the form the run will launch: the descriptor-in-parameters kernel for one image,
    // the tile-table kernel for a batch (and for serving, which always uses tables)
    const bool one = !table_form && slots.size() == 1 && tiled_one_available(c.p_storage);
    // Programmatic dependent launch, measured on whole decompositions: it pays where the tiled
    // kernel runs one CTA per SM (512^2, tile 24: 12.3 vs 13.0 ms) or its grid spans more than
    // one wave (1024^2 and 2048^2, tile 26: -4 % / -1 %), and costs up to 40 % where a shape with
    // room for a second CTA per SM runs a grid below one wave (512^2, tile 26: 17.7 vs 13.0 ms),
    // the next grid's CTAs then settling beside the running ones. Timing short graphs of
    // iteration launches alone did not reproduce either effect, so it is a rule, not a timing.
    auto pdl_rule = [&](int sh) {
        if (!c.pdl || sh < 0) return false;
        const int per_sm = tiled_ctas_per_sm(sh, c.p_storage, c.fast_math != 0, one);
        int n_tiles = 0;
        for (Slot *s : slots) {
            int ntx, nty;
            tiles_for(sh, s->H, s->W, &ntx, &nty);
            n_tiles += ntx * nty;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, plan->device) != cudaSuccess) {
            cudaGetLastError();
            sms = 1;
        }
        return per_sm == 1 || n_tiles > per_sm * sms;
    };
    std::vector<std::pair<int, bool>> cands;
    for (int sh : shapes) cands.push_back({sh, false});
    if (cands.size() == 1 || slots.empty()) {
        *shape = cands[0].first;
        *depth = default_depth(c, cands[0].first);
        *pdl = slots.empty() ? c.pdl != 0 : pdl_rule(*shape);
        return TVSPEC_OK;
    }
    std::vector<std::pair<int, int>> dims;
    for (Slot *s : slots) dims.push_back({s->H, s->W});
    std::sort(dims.begin(), dims.end());
    std::ostringstream key;
    key << c.p_storage << '/' << c.fast_math << '/' << c.temporal_block << '/' << (one ? 1 : 0)
        << '/' << c.pdl << '/' << c.tile << '/' << (one && c.tma ? 1 : 0);
    for (auto &d : dims) key << ';' << d.first << 'x' << d.second;
    auto it = plan->tune.find(key.str());
    if (it != plan->tune.end()) {
        *shape = it->second.shape;
        *depth = it->second.depth;
        *pdl = it->second.pdl;
        return TVSPEC_OK;
    }
    NvtxRange range("tvspec autotune");
    double total_px = 0.0;
    for (Slot *s : slots) total_px += (double)s->H * s->W;
    struct Cand {
        int shape, depth;
        bool pdl;
        LaunchSet ls;
        double cost = 1e300;
    };
    std::vector<Cand> cs(cands.size());
    auto release_all = [&]() {
        for (Cand &x : cs) x.ls.release();
    };
    const bool large = total_px > (double)(1 << 22);
    const int kReps = large ? 2 : 8;
    const int rounds = large ? 1 : 2;
    for (size_t i = 0; i < cands.size(); ++i) {
        cs[i].shape = cands[i].first;
        cs[i].pdl = cands[i].second;
        cs[i].depth = default_depth(c, cs[i].shape);
        std::vector<ImgDesc> descs;
        for (Slot *s : slots) {
            ImgDesc d = slot_desc(*s, 0);
            // kReps full launches of `depth` iterations, each reading what the previous one
            // wrote (the chain a step runs)
            d.n_inner = cs[i].depth * kReps;
            descs.push_back(d);
        }
        tvspec_status s = launchset_build(&cs[i].ls, descs, cs[i].shape, cs[i].depth);
        if (s != TVSPEC_OK) {
            release_all();
            return s;
        }
    }
    // Each candidate is timed as the run executes it: a CUDA graph of back-to-back launches
    // (direct launches would add a launch gap that graph replay does not have, and change the
    // ranking). Two rounds over all candidates, each candidate's cost the faster of its two:
    // the first round also brings the GPU to its working clock. A large set (several waves of
    // tiles per launch) times well with fewer launches: one round of graphs of 2 launches, so
    // that tuning stays a few launches per candidate.
    std::vector<cudaGraphExec_t> execs(cs.size(), nullptr);
    cudaError_t e = cudaSuccess;
    for (size_t i = 0; i < cs.size() && e == cudaSuccess; ++i) {
        Cand &x = cs[i];
        const int nt = x.ls.tile_prefix[x.ls.n];
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        cudaError_t le = cudaSuccess;
        for (int r = 0; r < kReps && le == cudaSuccess; ++r)
            le = one ? launch_tiled_one(x.shape, c.p_storage, c.fast_math != 0, x.ls.h_descs[0], 0, r,
                                        x.depth, c.tau, st, x.pdl, c.tma != 0)
                     : launch_tiled(x.shape, c.p_storage, c.fast_math != 0, x.ls.d_tiles, nt,
                                    x.ls.d_descs, 0, r, x.depth, c.tau, st, x.pdl);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (e == cudaSuccess) e = le;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&execs[i], g, 0);
        if (g) cudaGraphDestroy(g);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int round = 0; round < rounds && e == cudaSuccess; ++round) {
        for (size_t i = 0; i < cs.size() && e == cudaSuccess; ++i) {
            e = cudaGraphLaunch(execs[i], st);  // warm
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) e = cudaGraphLaunch(execs[i], st);
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess)
                cs[i].cost = std::min(cs[i].cost, (double)ms / (kReps * cs[i].depth * total_px));
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (cudaGraphExec_t x : execs)
        if (x) cudaGraphExecDestroy(x);
    release_all();
    if (e != cudaSuccess) return fail_cuda(e, "autotune launch");
    const Cand *best = &cs[0];
    for (const Cand &x : cs)
        if (x.cost < best->cost) best = &x;
    const bool use_pdl = pdl_rule(best->shape);
    plan->tune[key.str()] = {best->shape, best->depth, use_pdl};
    tune_cache_append(plan, key.str(), best->shape, best->depth, use_pdl);
    *shape = best->shape;
    *depth = best->depth;
    *pdl = use_pdl;
    return TVSPEC_OK;
}

// ---------------------------------------------------------------------------------------------
// Device work of one ROF step.
// ---------------------------------------------------------------------------------------------
static tvspec_status enqueue_iterations(tvspec_plan *plan, LaunchSet &ls,
                                        std::vector<Slot *> &slots, int n_active, int gstep,
                                        cudaStream_t st, uint64_t *nk) {
    const tvspec_config &c = plan->cfg;
    if (ls.shape < 0) {
        // reference kernel: single image, one launch per iteration between the two copies
        Slot &s = *slots[0];
        const ImgDesc &d = ls.h_descs[0];
        const int k = gstep - d.s0;
        if (k < 0 || k >= d.K) return TVSPEC_OK;
        const int n_it = d.n_inner;
        for (int it = 0; it < n_it; ++it) {
            const int src = p_copy(k, n_it, it);
            cudaError_t e = launch_naive(c.p_storage, c.fast_math != 0, d.p1[src], d.p2[src],
                                         d.p1[src ^ 1], d.p2[src ^ 1], d.q1[src], d.q2[src],
                                         d.q1[src ^ 1], d.q2[src ^ 1], s.gl, s.H, s.W, s.pitch,
                                         c.tau, it, n_it, st);
            if (e != cudaSuccess) return fail_cuda(e, "reference kernel launch");
            ++*nk;
        }
        return TVSPEC_OK;
    }
    int nblk = 0;
    for (int i = 0; i < n_active; ++i) {
        const ImgDesc &d = ls.h_descs[i];
        const int k = gstep - d.s0;
        if (k < 0 || k >= d.K) continue;
        nblk = std::max(nblk, launches_per_step(d.n_inner, ls.depth));
    }
    const int nt = ls.tile_prefix[n_active];
    // one image: its descriptor goes by value, no table reads before the tile loads
    const bool one = ls.n == 1 && n_active == 1 && tiled_one_available(c.p_storage);
    if (one && c.persistent == 2 && ls.h_descs[0].tile_flags != nullptr && nblk > 1 &&
        step_nbr_fits(ls.shape, c.fast_math != 0, nt)) {
        // the whole step in one cooperative launch, each tile waiting only on its neighbours
        cudaError_t e = launch_step_nbr(ls.shape, c.fast_math != 0, ls.h_descs[0], gstep,
                                        ls.depth, c.tau,
                                        (unsigned long long)c.barrier_timeout_ms * 1000000ull,
                                        c.test_barrier_noshow, st);
        if (e != cudaSuccess) return fail_cuda(e, "persistent kernel launch");
        ++*nk;
        return TVSPEC_OK;
    }
    if (one && c.persistent == 1 && ls.h_descs[0].counter != nullptr && nblk > 1 &&
        step_coop_fits(ls.shape, c.fast_math != 0, nt)) {
        // the whole step in one cooperative launch (tiles resident, bounded-wait barriers)
        cudaError_t e = launch_step_coop(ls.shape, c.fast_math != 0, ls.h_descs[0], gstep,
                                         ls.depth, c.tau,
                                         (unsigned long long)c.barrier_timeout_ms * 1000000ull,
                                         c.test_barrier_noshow, st);
        if (e != cudaSuccess) return fail_cuda(e, "persistent kernel launch");
        ++*nk;
        return TVSPEC_OK;
    }
    for (int b = 0; b < nblk; ++b) {
        cudaError_t e = one ? launch_tiled_one(ls.shape, c.p_storage, c.fast_math != 0,
                                               ls.h_descs[0], gstep, b, ls.depth, c.tau, st,
                                               ls.pdl, c.tma != 0)
                            : launch_tiled(ls.shape, c.p_storage, c.fast_math != 0, ls.d_tiles,
                                           nt, ls.d_descs, gstep, b, ls.depth, c.tau, st,
                                           ls.pdl);
        if (e != cudaSuccess) return fail_cuda(e, "tiled kernel launch");
        ++*nk;
    }
    return TVSPEC_OK;
}

tvspec_status enqueue_step(tvspec_plan *plan, LaunchSet &ls, std::vector<Slot *> &slots,
                           int n_active, int gstep, cudaStream_t st, uint64_t *nk) {
    const tvspec_config &c = plan->cfg;
    if (!c.warm_start) {
        for (int i = 0; i < n_active; ++i) {
            const int k = gstep - ls.h_descs[i].s0;
            if (k < 0 || k >= slots[i]->K) continue;
            for (int cpy = 0; cpy < 2; ++cpy) {
                TV_CK(cudaMemsetAsync(slots[i]->p1[cpy], 0, slots[i]->p_bytes, st));
                TV_CK(cudaMemsetAsync(slots[i]->p2[cpy], 0, slots[i]->p_bytes, st));
                if (slots[i]->lo1[cpy]) {
                    TV_CK(cudaMemsetAsync(slots[i]->lo1[cpy], 0, slots[i]->p_bytes, st));
                    TV_CK(cudaMemsetAsync(slots[i]->lo2[cpy], 0, slots[i]->p_bytes, st));
                }
            }
        }
    }
    tvspec_status s = enqueue_iterations(plan, ls, slots, n_active, gstep, st, nk);
    if (s != TVSPEC_OK) return s;
    const int ep_depth = ls.shape < 0 ? 1 : ls.depth;
    const bool one_ep = ls.n == 1 && n_active == 1;
    const bool pdl = ls.pdl;
    cudaError_t e = one_ep
                        ? launch_epilogue_one(c.p_storage, ls.h_descs[0], gstep, ep_depth, st, pdl)
                        : launch_epilogue(c.p_storage, ls.d_descs, ls.d_ep_img, ls.d_ep_base,
                                          ls.ep_prefix[n_active], gstep, ep_depth, st, pdl);
    if (e != cudaSuccess) return fail_cuda(e, "epilogue launch");
    if (ls.ep_prefix[n_active] > 0) ++*nk;
    return TVSPEC_OK;
}

// One ROF step with the split epilogue: cold-start clears, the dual iterations, then (after the
// previous step's spectral part, whose u_{k-2} buffer this step's primal part overwrites) the
// primal part on `st`, and the spectral part forked onto the plan's side stream.
static tvspec_status enqueue_step_split(tvspec_plan *plan, LaunchSet &ls, std::vector<Slot *> &slots,
                                        int n_active, int gstep, cudaStream_t st, bool *pending,
                                        uint64_t *nk) {
    const tvspec_config &c = plan->cfg;
    if (!c.warm_start) {
        for (int i = 0; i < n_active; ++i) {
            const int k = gstep - ls.h_descs[i].s0;
            if (k < 0 || k >= slots[i]->K) continue;
            for (int cpy = 0; cpy < 2; ++cpy) {
                TV_CK(cudaMemsetAsync(slots[i]->p1[cpy], 0, slots[i]->p_bytes, st));
                TV_CK(cudaMemsetAsync(slots[i]->p2[cpy], 0, slots[i]->p_bytes, st));
                if (slots[i]->lo1[cpy]) {
                    TV_CK(cudaMemsetAsync(slots[i]->lo1[cpy], 0, slots[i]->p_bytes, st));
                    TV_CK(cudaMemsetAsync(slots[i]->lo2[cpy], 0, slots[i]->p_bytes, st));
                }
            }
        }
    }
    tvspec_status s = enqueue_iterations(plan, ls, slots, n_active, gstep, st, nk);
    if (s != TVSPEC_OK) return s;
    if (*pending) TV_CK(cudaStreamWaitEvent(st, plan->ev_join, 0));
    const int ep_depth = ls.shape < 0 ? 1 : ls.depth;
    const bool one = ls.n == 1 && n_active == 1;
    const int nblk = ls.ep_prefix[n_active];
    const bool pdl = ls.pdl;
    cudaError_t e = one ? launch_epi_primal_one(c.p_storage, ls.h_descs[0], gstep, ep_depth, st, pdl)
                        : launch_epi_primal(c.p_storage, ls.d_descs, ls.d_ep_img, ls.d_ep_base, nblk,
                                            gstep, ep_depth, st, pdl);
    if (e != cudaSuccess) return fail_cuda(e, "epilogue launch");
    if (nblk > 0) ++*nk;
    if (gstep >= 1 && nblk > 0) {  // phi from the second step on (every image here has s0 = 0)
        TV_CK(cudaEventRecord(plan->ev_fork, st));
        TV_CK(cudaStreamWaitEvent(plan->side, plan->ev_fork, 0));
        e = one ? launch_epi_spectral_one(ls.h_descs[0], gstep, plan->side)
                : launch_epi_spectral(ls.d_descs, ls.d_ep_img, ls.d_ep_base, nblk, gstep, plan->side);
        if (e != cudaSuccess) return fail_cuda(e, "epilogue launch");
        TV_CK(cudaEventRecord(plan->ev_join, plan->side));
        *pending = true;
        ++*nk;
    }
    return TVSPEC_OK;
}

// The whole decomposition of a cached batch, from cleared workspace to the last epilogue.
static tvspec_status enqueue_decomposition(tvspec_plan *plan, CacheEntry &E, cudaStream_t st,
                                           uint64_t *nk) {
    std::vector<Slot *> sp;
    for (Slot &s : E.slots) sp.push_back(&s);
    // the resident kernel clears its own images' status and bands
    for (int i = 0; i < E.n_tiled; ++i)
        TV_CK(cudaMemsetAsync(E.slots[i].base + E.slots[i].zero_off, 0, E.slots[i].zero_bytes, st));
    // resident images: their whole decomposition, one launch per variant
    int off = 0;
    for (auto &g : E.res_groups) {
        bool par = false;
        for (int i = 0; i < g.second; ++i) par |= E.slots[E.n_tiled + off + i].S_par != nullptr;
        cudaError_t e = launch_resident(g.first, plan->cfg.fast_math != 0, E.ls.d_descs,
                                        E.d_res_idx + off, g.second, plan->cfg.tau,
                                        plan->cfg.warm_start, par, st);
        if (e != cudaSuccess) return fail_cuda(e, "resident kernel launch");
        ++*nk;
        off += g.second;
    }
    if (E.n_tiled == 0) return TVSPEC_OK;
    const bool split = true;  // the split epilogue (the serving loop uses the combined one)
    cudaError_t e = launch_init(E.ls.d_descs, E.ls.d_ep_img, E.ls.d_ep_base,
                                E.ls.ep_prefix[E.n_tiled], st);
    if (e != cudaSuccess) return fail_cuda(e, "init launch");
    ++*nk;
    bool pending = false;  // a spectral part on the side stream not yet joined
    for (int g = 0; g < E.maxK; ++g) {
        int n_active = 0;
        while (n_active < E.n_tiled && E.slots[n_active].K > g) ++n_active;
        if (n_active == 0) break;
        tvspec_status s = split ? enqueue_step_split(plan, E.ls, sp, n_active, g, st, &pending, nk)
                                : enqueue_step(plan, E.ls, sp, n_active, g, st, nk);
        if (s != TVSPEC_OK) {
            if (pending) cudaStreamWaitEvent(st, plan->ev_join, 0);  // rejoin before returning
            return s;
        }
    }
    if (pending) TV_CK(cudaStreamWaitEvent(st, plan->ev_join, 0));
    return TVSPEC_OK;
}

static void free_entry(CacheEntry &E, cudaStream_t st) {
    if (E.exec) cudaGraphExecDestroy(E.exec);
    if (E.graph) cudaGraphDestroy(E.graph);
    E.exec = nullptr;
    E.graph = nullptr;
    for (Slot &s : E.slots) slot_free(&s, st);
    E.slots.clear();
    E.ls.release();
    cudaFree(E.d_res_idx);
    E.d_res_idx = nullptr;
    if (E.h_status) cudaFreeHost(E.h_status);
    E.h_status = nullptr;
}

static std::string job_key(const tvspec_config &c, const std::vector<Job> &jobs) {
    std::ostringstream k;
    k << c.p_storage << '/' << c.warm_start << '/' << c.tau << '/' << c.kernel << '/' << c.tile
      << '/' << c.temporal_block << '/' << c.fast_math << '/' << c.use_graphs << '/' << c.acc_mode;
    k.precision(17);
    for (const Job &j : jobs) {
        k << ';' << j.r.H << 'x' << j.r.W << ',' << j.r.K << ',' << j.r.n_inner << ',' << j.r.dt
          << ',' << (j.r.u_trace ? 1 : 0);
        for (double e : j.edges) k << ',' << e;
        k << ",f" << j.r.n_filters << ",p" << (j.r.S_parseval ? 1 : 0);
        for (double v : j.filt_H) k << ',' << v;
        for (double v : j.filt_res) k << ',' << v;
    }
    return k.str();
}

tvspec_status get_entry(tvspec_plan *plan, const std::vector<Job> &jobs, CacheEntry **out) {
    const std::string key = job_key(plan->cfg, jobs);
    for (auto it = plan->cache.begin(); it != plan->cache.end(); ++it) {
        if ((*it)->key == key) {
            plan->cache.splice(plan->cache.begin(), plan->cache, it);
            *out = plan->cache.front().get();
            return TVSPEC_OK;
        }
    }
    // new entry: workspace, tile choice, tables, optionally a captured graph
    TV_CK(cudaStreamSynchronize(plan->stream));
    // least recently used entries leave while there are four, or while the cached workspaces
    // and the new one together exceed the memory budget (an entry larger than the budget on its
    // own still runs, alone)
    const bool naive_cfg = plan->cfg.kernel == TVSPEC_KERNEL_NAIVE;
    size_t need = 0;
    for (const Job &j : jobs) need += slot_bytes_for(j, plan->cfg.p_storage, naive_cfg, plan->cfg.test_guard_bytes);
    auto cached_bytes = [&]() {
        size_t b = 0;
        for (auto &e : plan->cache)
            for (const Slot &x : e->slots) b += x.bytes;
        return b;
    };
    while (!plan->cache.empty() &&
           (plan->cache.size() >= 4 || cached_bytes() + need > plan_budget(plan))) {
        free_entry(*plan->cache.back(), plan->stream);
        plan->cache.pop_back();
    }
    auto E = std::make_unique<CacheEntry>();
    E->key = key;
    const int n = (int)jobs.size();
    const tvspec_config &cf = plan->cfg;
    const bool resident_ok = cf.resident && cf.p_storage == TVSPEC_P_FP32 &&
                             (cf.kernel == TVSPEC_KERNEL_AUTO ||
                              (cf.kernel == TVSPEC_KERNEL_TILED && cf.tile < 0 && cf.temporal_block == 0));
    std::vector<int> variant(n, -1);
    if (resident_ok) {
        int eligible = 0;
        for (int i = 0; i < n; ++i) {
            variant[i] = resident_variant_for(jobs[i].r.H, jobs[i].r.W, cf.resident_variant);
            eligible += variant[i] >= 0;
        }
        // one CTA per image only pays off when there are enough images to fill the GPU
        if (cf.resident == 1 && eligible < kResidentMinBatch) variant.assign(n, -1);
    }
    // tiled images first, by K descending (the images still running at a step are a prefix),
    // then the resident ones grouped by variant
    E->order.resize(n);
    for (int i = 0; i < n; ++i) E->order[i] = i;
    std::stable_sort(E->order.begin(), E->order.end(), [&](int a, int b) {
        if ((variant[a] >= 0) != (variant[b] >= 0)) return variant[a] < 0;
        if (variant[a] >= 0) return variant[a] < variant[b];
        return jobs[a].r.K > jobs[b].r.K;
    });
    E->n_tiled = 0;
    while (E->n_tiled < n && variant[E->order[E->n_tiled]] < 0) ++E->n_tiled;
    const bool naive = plan->cfg.kernel == TVSPEC_KERNEL_NAIVE;
    if (naive && n != 1) return fail(TVSPEC_ENOTSUP, "the reference kernel runs one image at a time");
    for (int i = 0; i < n; ++i) {
        Slot s;
        tvspec_status st;
        if (plan->cfg.test_fail_alloc > 0 && ++plan->alloc_count == (uint64_t)plan->cfg.test_fail_alloc)
            st = fail(TVSPEC_ENOMEM, "injected workspace allocation failure (test_fail_alloc)");
        else
            st = slot_alloc(&s, jobs[E->order[i]], plan->cfg.p_storage, naive, plan->stream, false,
                            plan->cfg.acc_mode, plan->cfg.test_guard_bytes);
        if (st == TVSPEC_ENOMEM && !plan->cache.empty()) {
            // out of device memory with other workspaces cached: drop them all, start over
            free_entry(*E, plan->stream);
            E->slots.clear();
            E->maxK = 0;
            while (!plan->cache.empty()) {
                free_entry(*plan->cache.back(), plan->stream);
                plan->cache.pop_back();
            }
            cudaGetLastError();
            i = -1;
            continue;
        }
        if (st != TVSPEC_OK) {
            free_entry(*E, plan->stream);
            return st;
        }
        E->slots.push_back(s);
        E->maxK = std::max(E->maxK, s.K);
    }
    TV_CK(cudaStreamSynchronize(plan->stream));
    std::vector<Slot *> sp;
    for (int i = 0; i < E->n_tiled; ++i) sp.push_back(&E->slots[i]);
    int shape = -1, depth = 1;
    bool pdl = false;
    tvspec_status st = TVSPEC_OK;
    if (!sp.empty()) st = choose_tiles(plan, sp, plan->stream, &shape, &depth, false, &pdl);
    else if (plan->cfg.kernel != TVSPEC_KERNEL_NAIVE) shape = 0, depth = 1;
    if (st != TVSPEC_OK) {
        free_entry(*E, plan->stream);
        return st;
    }
    if (E->n_tiled < n) {
        std::vector<int> idx;
        for (int i = E->n_tiled; i < n; ++i) {
            const int v = variant[E->order[i]];
            if (E->res_groups.empty() || E->res_groups.back().first != v) E->res_groups.push_back({v, 0});
            E->res_groups.back().second++;
            idx.push_back(i);
        }
        size_t cap = 0;
        st = grow_upload(&E->d_res_idx, &cap, idx);
        if (st != TVSPEC_OK) {
            free_entry(*E, plan->stream);
            return st;
        }
    }
    std::vector<ImgDesc> descs;
    for (Slot &s : E->slots) descs.push_back(slot_desc(s, 0));
    st = launchset_build(&E->ls, descs, shape, depth);
    if (st != TVSPEC_OK) {
        free_entry(*E, plan->stream);
        return st;
    }
    E->ls.pdl = pdl;
    if (cudaMallocHost((void **)&E->h_status, sizeof(unsigned) * n) != cudaSuccess) {
        free_entry(*E, plan->stream);
        return fail(TVSPEC_ENOMEM, "pinned status words");
    }
    plan->last_tile = shape;
    plan->last_depth = depth;
    plan->cache.push_front(std::move(E));
    *out = plan->cache.front().get();
    return TVSPEC_OK;
}

tvspec_status enqueue_copy_list(const std::vector<CopyItem> &items, cudaStream_t st) {
    std::vector<CopyItem> it;
    for (const CopyItem &c : items)
        if (c.bytes > 0) it.push_back(c);
    if (it.empty()) return TVSPEC_OK;
    const int n = (int)it.size();
    std::vector<unsigned> first(n);
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        first[i] = (unsigned)total;
        total += (it[i].bytes + kCopyChunk - 1) / kCopyChunk;
    }
    if (total >= (size_t)UINT32_MAX) return fail(TVSPEC_EINVAL, "copy list too large");
    const size_t o_first = ((sizeof(CopyItem) * n) + 255) & ~(size_t)255;
    const size_t bytes = o_first + sizeof(unsigned) * n;
    std::vector<char> host(bytes);
    std::memcpy(host.data(), it.data(), sizeof(CopyItem) * n);
    std::memcpy(host.data() + o_first, first.data(), sizeof(unsigned) * n);
    char *d = nullptr;
    TV_CK(cudaMallocAsync((void **)&d, bytes, st));
    cudaError_t e = cudaMemcpyAsync(d, host.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_copy_list(reinterpret_cast<const CopyItem *>(d),
                             reinterpret_cast<const unsigned *>(d + o_first), n, (unsigned)total, st);
    cudaFreeAsync(d, st);
    if (e != cudaSuccess) return fail_cuda(e, "copy list");
    return TVSPEC_OK;
}

// Captures the entry's whole decomposition into a CUDA graph (on the plan stream).
static tvspec_status capture_entry(tvspec_plan *plan, CacheEntry &E) {
    uint64_t nk = 0;
    TV_CK(cudaStreamBeginCapture(plan->stream, cudaStreamCaptureModeThreadLocal));
    tvspec_status st = enqueue_decomposition(plan, E, plan->stream, &nk);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(plan->stream, &g);
    if (st != TVSPEC_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != TVSPEC_OK ? st : fail_cuda(e, "graph capture");
    }
    e = cudaGraphInstantiate(&E.exec, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        E.exec = nullptr;
        return fail_cuda(e, "graph instantiation");
    }
    E.graph = g;
    E.graph_kernels = nk;
    plan->graphs_built++;
    return TVSPEC_OK;
}

tvspec_status launch_entry(tvspec_plan *plan, CacheEntry &E, cudaStream_t st) {
    // a problem signature is captured into a graph on its second use: a one-off image (a batch
    // of many different sizes decomposed one at a time) does not pay for a capture it never
    // replays
    if (plan->cfg.use_graphs && !E.exec && E.uses >= 1) {
        tvspec_status s = capture_entry(plan, E);
        if (s != TVSPEC_OK) return s;
    }
    ++E.uses;
    uint64_t nk = 0;
    if (E.exec) {
        TV_CK(cudaGraphLaunch(E.exec, st));
        nk = E.graph_kernels;
        plan->graph_launches++;
    } else {
        tvspec_status s = enqueue_decomposition(plan, E, st, &nk);
        if (s != TVSPEC_OK) return s;
    }
    plan->kernel_launches += nk;
    return TVSPEC_OK;
}

tvspec_status order_after(cudaStream_t later, cudaStream_t earlier) {
    if (later == earlier) return TVSPEC_OK;
    cudaEvent_t ev;
    TV_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, earlier);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(later, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return fail_cuda(e, "stream ordering");
    return TVSPEC_OK;
}

static tvspec_status run_jobs(tvspec_plan *plan, std::vector<Job> &jobs, cudaStream_t user_st) {
    NvtxRange range(jobs.size() == 1 ? "tvspec decompose" : "tvspec decompose_batch");
    std::lock_guard<std::mutex> lock(plan->mu);
    TV_CK(cudaSetDevice(plan->device));
    const int mk = jobs[0].r.mem_kind;
    for (const Job &j : jobs)
        if (j.r.mem_kind != mk) return fail(TVSPEC_EINVAL, "all requests must share one mem_kind");
    CacheEntry *E = nullptr;
    tvspec_status s = get_entry(plan, jobs, &E);
    if (s != TVSPEC_OK) return s;
    cudaStream_t st = user_st ? user_st : plan->stream;
    if (user_st) {
        // order the (possibly different) user stream after anything still on the plan stream
        cudaEvent_t ev;
        TV_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        TV_CK(cudaEventRecord(ev, plan->stream));
        TV_CK(cudaStreamWaitEvent(st, ev, 0));
        cudaEventDestroy(ev);
    }
    const cudaMemcpyKind in_kind = mk == TVSPEC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out_kind = mk == TVSPEC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    const int n = (int)jobs.size();
    // device-memory batches move their inputs and outputs with one copy-list launch each
    const bool listed = mk == TVSPEC_MEM_DEVICE && n >= 2;
    std::vector<CopyItem> cin, cout;
    for (int i = 0; i < n; ++i) {
        const tvspec_request &r = jobs[E->order[i]].r;
        const size_t bytes = (size_t)r.H * r.W * 4;
        if (listed) cin.push_back({r.f, E->slots[i].f, bytes});
        else TV_CK(cudaMemcpyAsync(E->slots[i].f, r.f, bytes, in_kind, st));
    }
    s = enqueue_copy_list(cin, st);
    if (s != TVSPEC_OK) return s;
    s = launch_entry(plan, *E, st);
    if (s != TVSPEC_OK) return s;
    for (int i = 0; i < n; ++i) {
        const tvspec_request &r = jobs[E->order[i]].r;
        const Slot &sl = E->slots[i];
        const size_t N = (size_t)r.H * r.W;
        const CopyItem out[] = {{sl.bands, r.bands, (size_t)sl.n_bands * N * 4},
                                {sl.residual, r.residual, N * 4},
                                {sl.S, r.S, (size_t)(r.K - 1) * 8},
                                {sl.utrace, r.u_trace, r.u_trace ? (size_t)(r.K + 1) * N * 8 : 0},
                                {sl.filtered, r.filtered, (size_t)r.n_filters * N * 4},
                                {sl.S_par, r.S_parseval, r.S_parseval ? (size_t)(r.K - 1) * 8 : 0}};
        for (const CopyItem &c : out) {
            if (c.bytes == 0) continue;
            if (listed) cout.push_back(c);
            else TV_CK(cudaMemcpyAsync(c.dst, c.src, c.bytes, out_kind, st));
        }
        if (mk == TVSPEC_MEM_HOST)
            TV_CK(cudaMemcpyAsync(E->h_status + i, sl.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    }
    s = enqueue_copy_list(cout, st);
    if (s != TVSPEC_OK) return s;
    if (user_st) {
        // later work on the plan stream must see this call's use of the workspace
        cudaEvent_t ev;
        TV_CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        TV_CK(cudaEventRecord(ev, st));
        TV_CK(cudaStreamWaitEvent(plan->stream, ev, 0));
        cudaEventDestroy(ev);
    }
    if (plan->cfg.test_guard_bytes > 0)
        for (const Slot &sl : E->slots) {
            s = slot_check_guards(sl, st);
            if (s != TVSPEC_OK) return s;
        }
    if (mk == TVSPEC_MEM_HOST) {
        TV_CK(cudaStreamSynchronize(st));
        for (int i = 0; i < n; ++i) {
            if (E->h_status[i] & kStatusBarrierTimeout)
                return fail(TVSPEC_ETIMEOUT, "a grid barrier wait ran out (a CTA did not arrive)");
            if (E->h_status[i] & kStatusCopyTimeout)
                return fail(TVSPEC_ETIMEOUT, "a wait for a tile's TMA copies ran out");
            if (E->h_status[i] & kStatusNonFinite)
                return fail(TVSPEC_ECUDA, "non-finite value in the flow");
        }
    }
    plan->decompositions += n;
    return TVSPEC_OK;
}

size_t plan_budget(const tvspec_plan *plan) {
    return plan->cfg.mem_budget_bytes ? plan->cfg.mem_budget_bytes : ((size_t)60 << 30);
}

// ---------------------------------------------------------------------------------------------
// Standalone dual iterations (ROF step, hot-kernel timing).
// ---------------------------------------------------------------------------------------------
static tvspec_status scratch_slot(tvspec_plan *plan, int H, int W, Slot **out) {
    for (Slot &s : plan->scratch)
        if (s.H == H && s.W == W) {
            *out = &s;
            return TVSPEC_OK;
        }
    if (plan->scratch.size() >= 4) {
        TV_CK(cudaStreamSynchronize(plan->stream));
        slot_free(&plan->scratch.front(), plan->stream);
        plan->scratch.pop_front();
    }
    const double edges[2] = {0.0, INFINITY};
    tvspec_request r{};
    r.H = H;
    r.W = W;
    r.dt = 1.0;
    r.K = 2;
    r.n_inner = 0;
    r.n_edges = 2;
    r.band_edges = edges;
    Job j;
    j.r = r;
    j.edges.assign(edges, edges + 2);
    j.band_of_k.assign(2, -1);
    Slot s;
    tvspec_status st = slot_alloc(&s, j, plan->cfg.p_storage, true, plan->stream, false);
    if (st != TVSPEC_OK) return st;
    TV_CK(cudaMemsetAsync(s.base + s.zero_off, 0, s.zero_bytes, plan->stream));
    plan->scratch.push_back(s);
    *out = &plan->scratch.back();
    return TVSPEC_OK;
}

tvspec_status tune_for_size(tvspec_plan *plan, int H, int W, int *shape, int *depth, bool *pdl) {
    std::lock_guard<std::mutex> lock(plan->mu);
    TV_CK(cudaSetDevice(plan->device));
    Slot *sl = nullptr;
    tvspec_status s = scratch_slot(plan, H, W, &sl);
    if (s != TVSPEC_OK) return s;
    std::vector<Slot *> sp{sl};
    s = choose_tiles(plan, sp, plan->stream, shape, depth, /*table_form=*/true, pdl);
    if (s != TVSPEC_OK) return s;
    TV_CK(cudaStreamSynchronize(plan->stream));
    return TVSPEC_OK;
}

// Runs d.n_inner dual iterations as local step 0 of the image described by d (two copies of
// p, copy 0 holding the start); *final_copy receives the copy holding the result.
tvspec_status run_iterations(tvspec_plan *plan, ImgDesc d, cudaStream_t st, int *final_copy) {
    Slot *tune_slot = nullptr;
    tvspec_status s = scratch_slot(plan, d.H, d.W, &tune_slot);
    if (s != TVSPEC_OK) return s;
    int shape = -1, depth = 1;
    bool pdl = false;
    std::vector<Slot *> sp{tune_slot};
    s = choose_tiles(plan, sp, plan->stream, &shape, &depth, false, &pdl);
    if (s != TVSPEC_OK) return s;
    d.s0 = 0;
    d.K = std::max(d.K, 1);
    std::ostringstream key;
    key << d.p1[0] << '/' << d.p1[1] << '/' << d.p2[0] << '/' << d.p2[1] << '/' << d.gl << '/'
        << d.H << 'x' << d.W << '/' << d.pitch << '/' << d.n_inner << '/' << shape << '/' << depth
        << '/' << pdl;
    auto it = plan->iter_sets.find(key.str());
    LaunchSet *ls = nullptr;
    if (it == plan->iter_sets.end()) {
        if (plan->iter_sets.size() >= 16) {
            TV_CK(cudaDeviceSynchronize());
            for (auto &kv : plan->iter_sets) kv.second->release();
            plan->iter_sets.clear();
        }
        auto nls = std::make_unique<LaunchSet>();
        s = launchset_build(nls.get(), std::vector<ImgDesc>{d}, shape, depth);
        if (s != TVSPEC_OK) {
            nls->release();
            return s;
        }
        nls->pdl = pdl;
        ls = nls.get();
        plan->iter_sets[key.str()] = std::move(nls);
    } else {
        ls = it->second.get();
    }
    uint64_t nk = 0;
    Slot tmp;
    tmp.H = d.H;
    tmp.W = d.W;
    tmp.pitch = d.pitch;
    tmp.K = d.K;
    tmp.gl = d.gl;
    std::vector<Slot *> one{&tmp};
    s = enqueue_iterations(plan, *ls, one, 1, 0, st, &nk);
    plan->kernel_launches += nk;
    plan->last_tile = shape;
    plan->last_depth = depth;
    *final_copy = p_copy(1, shape < 0 ? d.n_inner : launches_per_step(d.n_inner, depth), 0);
    return s;
}

}  // namespace tvspec

using namespace tvspec;

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

void tvspec_config_init(tvspec_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->p_storage = TVSPEC_P_FP32;
    cfg->warm_start = 1;
    cfg->tau = 0.125f;
    cfg->kernel = TVSPEC_KERNEL_AUTO;
    cfg->tile = -1;
    cfg->temporal_block = 0;
    cfg->use_graphs = 1;
    cfg->fast_math = 1;
    cfg->mem_budget_bytes = 0;
    cfg->max_batch = 0;
    cfg->pdl = 1;
    cfg->persistent = 0;
    cfg->barrier_timeout_ms = 2000;
    cfg->test_barrier_noshow = -1;
    cfg->test_fail_alloc = 0;
    cfg->test_guard_bytes = 0;
    cfg->tma = 0;
    cfg->resident = 1;
    cfg->resident_variant = -1;
}

tvspec_status tvspec_plan_create(const tvspec_config *cfg, int device, tvspec_plan **out) {
    if (!out) return fail(TVSPEC_EINVAL, "out is NULL");
    *out = nullptr;
    tvspec_config c;
    if (cfg) c = *cfg; else tvspec_config_init(&c);
    if (c.p_storage < 0 || c.p_storage > 3) return fail(TVSPEC_EINVAL, "p_storage out of range");
    if (!(c.tau > 0.0f) || !(c.tau <= 0.25f)) return fail(TVSPEC_EINVAL, "tau must be in (0, 0.25]");
    if (c.kernel < 0 || c.kernel > 2) return fail(TVSPEC_EINVAL, "kernel out of range");
    if (c.tile < -1 || c.tile >= tiled_shape_count()) return fail(TVSPEC_EINVAL, "tile out of range");
    if (c.temporal_block < 0 || c.temporal_block > 16)
        return fail(TVSPEC_EINVAL, "temporal_block must be in [0, 16]");
    if (c.max_batch < 0) return fail(TVSPEC_EINVAL, "max_batch must be >= 0");
    if (c.barrier_timeout_ms < 1) return fail(TVSPEC_EINVAL, "barrier_timeout_ms must be >= 1");
    if (c.resident < 0 || c.resident > 2) return fail(TVSPEC_EINVAL, "resident must be 0, 1 or 2");
    if (c.persistent < 0 || c.persistent > 2) return fail(TVSPEC_EINVAL, "persistent must be 0, 1 or 2");
    if (c.acc_mode < 0 || c.acc_mode > 1) return fail(TVSPEC_EINVAL, "acc_mode must be 0 or 1");
    if (c.resident_variant < -1 || c.resident_variant >= resident_variant_count())
        return fail(TVSPEC_EINVAL, "resident_variant out of range");
    int n_dev = 0;
    cudaError_t e = cudaGetDeviceCount(&n_dev);
    if (e != cudaSuccess || n_dev == 0) {
        cudaGetLastError();
        return fail(TVSPEC_ECUDA, "no CUDA device available");
    }
    if (device < 0 || device >= n_dev) return fail(TVSPEC_EINVAL, "device index out of range");
    TV_CK(cudaSetDevice(device));
    auto *p = new (std::nothrow) tvspec_plan();
    if (!p) return fail(TVSPEC_ENOMEM, "plan allocation");
    p->device = device;
    p->cfg = c;
    if (c.tune_cache) p->tune_cache = c.tune_cache;
    p->cfg.tune_cache = nullptr;  // the plan keeps its own copy of the path
    p->tune_prefix = tune_prefix_for(device);
    tune_cache_load(p);
    // the spectral part of the split epilogue runs on a low-priority stream beside the next
    // step's dual iterations (the critical path), which keep the higher priority
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_low = prio_high = 0;
    }
    e = cudaStreamCreateWithPriority(&p->stream, cudaStreamNonBlocking, prio_high);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, prio_low);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        if (p->ev_fork) cudaEventDestroy(p->ev_fork);
        if (p->side) cudaStreamDestroy(p->side);
        if (p->stream) cudaStreamDestroy(p->stream);
        delete p;
        return fail_cuda(e, "stream creation");
    }
    *out = p;
    return TVSPEC_OK;
}

// serving.cu
void tvspec_server_stop(tvspec_plan *plan);

tvspec_status tvspec_plan_destroy(tvspec_plan *plan) {
    if (!plan) return TVSPEC_OK;
    tvspec_server_stop(plan);
    cudaSetDevice(plan->device);
    cudaStreamSynchronize(plan->stream);
    if (plan->h_word) cudaFreeHost(plan->h_word);
    plan->h_word = nullptr;
    for (auto &E : plan->cache) free_entry(*E, plan->stream);
    plan->cache.clear();
    for (auto &kv : plan->iter_sets) kv.second->release();
    plan->iter_sets.clear();
    for (Slot &s : plan->scratch) slot_free(&s, plan->stream);
    plan->scratch.clear();
    cudaFree(plan->ping);
    plan->ping = nullptr;
    cudaStreamSynchronize(plan->stream);
    cudaStreamSynchronize(plan->side);
    if (plan->ev_fork) cudaEventDestroy(plan->ev_fork);
    if (plan->ev_join) cudaEventDestroy(plan->ev_join);
    cudaStreamDestroy(plan->side);
    cudaStreamDestroy(plan->stream);
    delete plan;
    return TVSPEC_OK;
}

tvspec_status tvspec_validate(const tvspec_request *req) {
    if (!req) return fail(TVSPEC_EINVAL, "request is NULL");
    Job j;
    return make_job(*req, &j);
}

tvspec_status tvspec_decompose_ex(tvspec_plan *plan, const tvspec_request *req, void *stream) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    if (!req) return fail(TVSPEC_EINVAL, "request is NULL");
    std::vector<Job> jobs(1);
    tvspec_status s = make_job(*req, &jobs[0]);
    if (s != TVSPEC_OK) return s;
    return run_jobs(plan, jobs, (cudaStream_t)stream);
}

tvspec_status tvspec_decompose(tvspec_plan *plan, const float *f, int H, int W, double dt, int K,
                               int n_inner, const double *band_edges, int n_edges, float *bands,
                               float *residual, double *S, int mem_kind, void *stream) {
    tvspec_request r{};
    r.f = f;
    r.H = H;
    r.W = W;
    r.dt = dt;
    r.K = K;
    r.n_inner = n_inner;
    r.band_edges = band_edges;
    r.n_edges = n_edges;
    r.bands = bands;
    r.residual = residual;
    r.S = S;
    r.u_trace = nullptr;
    r.mem_kind = mem_kind;
    return tvspec_decompose_ex(plan, &r, stream);
}

tvspec_status tvspec_decompose_batch(tvspec_plan *plan, int n, const tvspec_request *reqs,
                                     void *stream) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    if (n < 1 || !reqs) return fail(TVSPEC_EINVAL, "need n >= 1 requests");
    if (n > 4096) return fail(TVSPEC_EINVAL, "at most 4096 requests per batch");
    std::vector<Job> jobs(n);
    for (int i = 0; i < n; ++i) {
        tvspec_status s = make_job(reqs[i], &jobs[i]);
        if (s != TVSPEC_OK) return s;
    }
    return run_jobs(plan, jobs, (cudaStream_t)stream);
}

// ---- checkpoint / resume ----------------------------------------------------------------
// The state between two ROF steps is the image's whole workspace (u_{k-1}, u_k, both copies of
// p, g/dt, the band and filter accumulators, the outputs written so far, S so far), saved
// byte for byte after a header that ties it to the request, the configuration and the step.

namespace {

struct CheckpointHeader {
    char magic[8];        // "TVSPCKP1"
    uint64_t key_hash;    // FNV-1a of the job key (configuration + request signature)
    uint64_t slot_bytes;  // workspace bytes that follow
    int32_t k_next;       // the ROF step the state resumes at
    int32_t launches;     // dual-iteration launches per step of the run that saved it
    int32_t reserved[4];
};

const char kCheckpointMagic[8] = {'T', 'V', 'S', 'P', 'C', 'K', 'P', '1'};

uint64_t fnv1a(const std::string &x) {
    uint64_t h = 1469598103934665603ull;
    for (unsigned char c : x) {
        h ^= c;
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

size_t tvspec_checkpoint_bytes(tvspec_plan *plan, const tvspec_request *req) {
    if (!plan || !req) return 0;
    Job j;
    if (make_job(*req, &j) != TVSPEC_OK) return 0;
    return sizeof(CheckpointHeader) +
           slot_bytes_for(j, plan->cfg.p_storage, plan->cfg.kernel == TVSPEC_KERNEL_NAIVE,
                          plan->cfg.test_guard_bytes);
}

tvspec_status tvspec_decompose_steps(tvspec_plan *plan, const tvspec_request *req, int k_begin,
                                     int k_end, const void *state_in, void *state_out) {
    NvtxRange range("tvspec decompose_steps");
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    if (!req) return fail(TVSPEC_EINVAL, "request is NULL");
    std::vector<Job> jobs(1);
    tvspec_status s = make_job(*req, &jobs[0]);
    if (s != TVSPEC_OK) return s;
    const tvspec_request &r = jobs[0].r;
    if (k_begin < 0 || k_end <= k_begin || k_end > r.K)
        return fail(TVSPEC_EINVAL, "need 0 <= k_begin < k_end <= K");
    if (k_begin > 0 && !state_in) return fail(TVSPEC_EINVAL, "resuming needs state_in");
    if (k_end < r.K && !state_out) return fail(TVSPEC_EINVAL, "stopping before K needs state_out");
    std::lock_guard<std::mutex> lock(plan->mu);
    TV_CK(cudaSetDevice(plan->device));
    CacheEntry *E = nullptr;
    s = get_entry(plan, jobs, &E);
    if (s != TVSPEC_OK) return s;
    if (E->n_tiled != 1)
        return fail(TVSPEC_ENOTSUP, "the resident kernel runs whole decompositions (resident = 2)");
    Slot &sl = E->slots[0];
    // the key covers what decides the state's layout and bits, not the launch choices (tile
    // shape, depth, graphs), which leave both unchanged
    tvspec_config kc = plan->cfg;
    kc.kernel = kc.kernel == TVSPEC_KERNEL_NAIVE ? TVSPEC_KERNEL_NAIVE : TVSPEC_KERNEL_AUTO;
    kc.tile = -1;
    kc.temporal_block = 0;
    kc.use_graphs = 1;
    const uint64_t key = fnv1a(job_key(kc, jobs));
    const int launches = launches_per_step(r.n_inner, E->ls.shape < 0 ? 1 : E->ls.depth);
    cudaStream_t st = plan->stream;
    std::vector<Slot *> sp{&sl};
    const cudaMemcpyKind in_kind = r.mem_kind == TVSPEC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out_kind = r.mem_kind == TVSPEC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (k_begin == 0) {
        TV_CK(cudaMemsetAsync(sl.base + sl.zero_off, 0, sl.zero_bytes, st));
        TV_CK(cudaMemcpyAsync(sl.f, r.f, (size_t)r.H * r.W * 4, in_kind, st));
        cudaError_t e = launch_init(E->ls.d_descs, E->ls.d_ep_img, E->ls.d_ep_base, E->ls.ep_prefix[1], st);
        if (e != cudaSuccess) return fail_cuda(e, "init launch");
        ++plan->kernel_launches;
    } else {
        CheckpointHeader h;
        std::memcpy(&h, state_in, sizeof h);
        if (std::memcmp(h.magic, kCheckpointMagic, 8) != 0 || h.key_hash != key ||
            h.slot_bytes != sl.bytes || h.launches < 1)
            return fail(TVSPEC_EINVAL, "state_in belongs to another request or configuration");
        if (h.k_next != k_begin) return fail(TVSPEC_EINVAL, "state_in was saved at another step");
        TV_CK(cudaMemcpyAsync(sl.base, static_cast<const char *>(state_in) + sizeof h, sl.bytes,
                              cudaMemcpyHostToDevice, st));
        // the copy of p that step k_begin reads depends on the launches per step (p_copy): if
        // this plan's tile choice differs in their parity, move p to the copy it will read
        const int was = p_copy(k_begin, h.launches, 0), now = p_copy(k_begin, launches, 0);
        if (was != now) {
            TV_CK(cudaMemcpyAsync(sl.p1[now], sl.p1[was], sl.p_bytes, cudaMemcpyDeviceToDevice, st));
            TV_CK(cudaMemcpyAsync(sl.p2[now], sl.p2[was], sl.p_bytes, cudaMemcpyDeviceToDevice, st));
            if (sl.lo1[now]) {
                TV_CK(cudaMemcpyAsync(sl.lo1[now], sl.lo1[was], sl.p_bytes, cudaMemcpyDeviceToDevice, st));
                TV_CK(cudaMemcpyAsync(sl.lo2[now], sl.lo2[was], sl.p_bytes, cudaMemcpyDeviceToDevice, st));
            }
        }
    }
    bool pending = false;
    for (int g = k_begin; g < k_end; ++g) {
        uint64_t nk = 0;
        s = enqueue_step_split(plan, E->ls, sp, 1, g, st, &pending, &nk);
        plan->kernel_launches += nk;
        if (s != TVSPEC_OK) {
            if (pending) cudaStreamWaitEvent(st, plan->ev_join, 0);
            return s;
        }
    }
    if (pending) TV_CK(cudaStreamWaitEvent(st, plan->ev_join, 0));
    if (k_end < r.K) {
        CheckpointHeader h{};
        std::memcpy(h.magic, kCheckpointMagic, 8);
        h.key_hash = key;
        h.slot_bytes = sl.bytes;
        h.k_next = k_end;
        h.launches = launches;
        std::memcpy(state_out, &h, sizeof h);
        TV_CK(cudaMemcpyAsync(static_cast<char *>(state_out) + sizeof h, sl.base, sl.bytes,
                              cudaMemcpyDeviceToHost, st));
    } else {
        const size_t N = (size_t)r.H * r.W;
        const CopyItem out[] = {{sl.bands, r.bands, (size_t)sl.n_bands * N * 4},
                                {sl.residual, r.residual, N * 4},
                                {sl.S, r.S, (size_t)(r.K - 1) * 8},
                                {sl.utrace, r.u_trace, r.u_trace ? (size_t)(r.K + 1) * N * 8 : 0},
                                {sl.filtered, r.filtered, (size_t)r.n_filters * N * 4},
                                {sl.S_par, r.S_parseval, r.S_parseval ? (size_t)(r.K - 1) * 8 : 0}};
        for (const CopyItem &c : out)
            if (c.bytes) TV_CK(cudaMemcpyAsync(c.dst, c.src, c.bytes, out_kind, st));
    }
    if (plan->cfg.test_guard_bytes > 0) {
        s = slot_check_guards(sl, st);
        if (s != TVSPEC_OK) return s;
    }
    if (!plan->h_word) TV_CK(cudaMallocHost((void **)&plan->h_word, sizeof(double)));
    TV_CK(cudaMemcpyAsync(plan->h_word, sl.status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    TV_CK(cudaStreamSynchronize(st));
    unsigned status;
    std::memcpy(&status, plan->h_word, sizeof status);
    if (status & kStatusBarrierTimeout)
        return fail(TVSPEC_ETIMEOUT, "a grid barrier wait ran out (a CTA did not arrive)");
    if (status & kStatusCopyTimeout) return fail(TVSPEC_ETIMEOUT, "a wait for a tile's TMA copies ran out");
    if (status & kStatusNonFinite) return fail(TVSPEC_ECUDA, "non-finite value in the flow");
    if (k_end == r.K) plan->decompositions++;
    return TVSPEC_OK;
}

tvspec_status tvspec_rof_step(tvspec_plan *plan, const float *g, int H, int W, double lambda,
                              int n_iter, float *p1, float *p2, float *u, int mem_kind,
                              void *stream) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    if (!g || !p1 || !p2 || !u) return fail(TVSPEC_EINVAL, "NULL buffer");
    if (H < 1 || W < 1 || (size_t)H * W > ((size_t)1 << 28)) return fail(TVSPEC_EINVAL, "bad H, W");
    if (!std::isfinite(lambda) || !(lambda > 0.0)) return fail(TVSPEC_EINVAL, "lambda must be > 0");
    if (n_iter < 0 || n_iter > 10000000) return fail(TVSPEC_EINVAL, "n_iter out of range");
    if (mem_kind != TVSPEC_MEM_HOST && mem_kind != TVSPEC_MEM_DEVICE)
        return fail(TVSPEC_EINVAL, "bad mem_kind");
    if (plan->cfg.p_storage != TVSPEC_P_FP32)
        return fail(TVSPEC_ENOTSUP, "tvspec_rof_step needs p_storage = fp32");
    std::lock_guard<std::mutex> lock(plan->mu);
    TV_CK(cudaSetDevice(plan->device));
    cudaStream_t st = stream ? (cudaStream_t)stream : plan->stream;
    if (stream) TV_CK(cudaStreamSynchronize(plan->stream));
    Slot *sl = nullptr;
    tvspec_status s = scratch_slot(plan, H, W, &sl);
    if (s != TVSPEC_OK) return s;
    {
        // tune first: the autotuner times kernels on these very buffers
        int shape, depth;
        std::vector<Slot *> sp{sl};
        s = choose_tiles(plan, sp, plan->stream, &shape, &depth);
        if (s != TVSPEC_OK) return s;
        TV_CK(cudaStreamSynchronize(plan->stream));
    }
    const cudaMemcpyKind in_kind = mem_kind == TVSPEC_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    const cudaMemcpyKind out_kind = mem_kind == TVSPEC_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    TV_CK(cudaMemsetAsync(sl->base + sl->zero_off, 0, sl->zero_bytes, st));
    const size_t row = (size_t)W * 4, prow = (size_t)sl->pitch * 4;
    TV_CK(cudaMemcpy2DAsync(sl->p1[0], prow, p1, row, row, H, in_kind, st));
    TV_CK(cudaMemcpy2DAsync(sl->p2[0], prow, p2, row, row, H, in_kind, st));
    TV_CK(cudaMemcpyAsync(sl->f, g, (size_t)H * W * 4, in_kind, st));
    cudaError_t e = launch_gl_from_g(sl->f, sl->gl, H, W, sl->pitch, lambda, st);
    if (e != cudaSuccess) return fail_cuda(e, "gl kernel");
    ImgDesc d = slot_desc(*sl, 0);
    d.n_inner = n_iter;
    int fc = 0;
    s = run_iterations(plan, d, st, &fc);
    if (s != TVSPEC_OK) return s;
    e = launch_rof_primal((const float *)sl->p1[fc], (const float *)sl->p2[fc], sl->pitch, sl->f,
                          sl->residual, H, W, lambda, st);
    if (e != cudaSuccess) return fail_cuda(e, "primal kernel");
    TV_CK(cudaMemcpy2DAsync(p1, row, sl->p1[fc], prow, row, H, out_kind, st));
    TV_CK(cudaMemcpy2DAsync(p2, row, sl->p2[fc], prow, row, H, out_kind, st));
    TV_CK(cudaMemcpyAsync(u, sl->residual, (size_t)H * W * 4, out_kind, st));
    TV_CK(cudaStreamSynchronize(st));
    return TVSPEC_OK;
}

tvspec_status tvspec_chambolle_iterate(tvspec_plan *plan, const float *gl, float *p1, float *p2,
                                       int H, int W, int pitch, int n_iter, void *stream) {
    if (!plan) return fail(TVSPEC_EINVAL, "plan is NULL");
    if (!gl || !p1 || !p2) return fail(TVSPEC_EINVAL, "NULL buffer");
    if (H < 1 || W < 1 || pitch < W || pitch % 4 != 0) return fail(TVSPEC_EINVAL, "bad H, W or pitch");
    if (((uintptr_t)gl | (uintptr_t)p1 | (uintptr_t)p2) & 15u)
        return fail(TVSPEC_EINVAL, "buffers must be 16-byte aligned");
    if (n_iter < 0) return fail(TVSPEC_EINVAL, "n_iter < 0");
    if (plan->cfg.p_storage != TVSPEC_P_FP32)
        return fail(TVSPEC_ENOTSUP, "tvspec_chambolle_iterate needs p_storage = fp32");
    std::lock_guard<std::mutex> lock(plan->mu);
    TV_CK(cudaSetDevice(plan->device));
    cudaStream_t st = stream ? (cudaStream_t)stream : plan->stream;
    // copy 1 of the dual field: a plan-owned buffer of the caller's pitched size
    const size_t pb = (size_t)H * pitch * 4;
    const size_t flag_bytes = ((size_t)max_tiles_for(H, W) * 4 + 255) / 256 * 256;
    // + counter, status, barrier and tile words, + the low parts of p of both copies (zero at
    // the start of every call: the caller's p is taken as exact)
    const size_t lb = (pb + 255) / 256 * 256;
    const size_t need = 2 * pb + 256 + flag_bytes + 4 * lb;
    if (plan->ping_bytes < need) {
        TV_CK(cudaStreamSynchronize(st));
        cudaFree(plan->ping);
        plan->ping = nullptr;
        plan->ping_bytes = 0;
        TV_CK(cudaMalloc(&plan->ping, need));
        plan->ping_bytes = need;
    }
    unsigned *words = reinterpret_cast<unsigned *>((char *)plan->ping + 2 * pb);
    char *lo = (char *)plan->ping + 2 * pb + 256 + flag_bytes;
    TV_CK(cudaMemsetAsync(words, 0, 256 + flag_bytes + 4 * lb, st));
    ImgDesc d{};
    d.p1[0] = p1;
    d.p2[0] = p2;
    d.p1[1] = plan->ping;
    d.p2[1] = (char *)plan->ping + pb;
    d.counter = words;
    d.status = words + 1;
    d.tile_flags = words + 64;
    for (int c = 0; c < 2; ++c) {
        d.q1[c] = reinterpret_cast<float *>(lo + (2 * c) * lb);
        d.q2[c] = reinterpret_cast<float *>(lo + (2 * c + 1) * lb);
    }
    d.gl = const_cast<float *>(gl);
    d.H = H;
    d.W = W;
    d.pitch = pitch;
    d.K = 1;
    d.n_inner = n_iter;
    d.s0 = 0;
    d.dt = 1.0;
    d.inv_dt = 1.0;
    int fc = 0;
    tvspec_status s = run_iterations(plan, d, st, &fc);
    if (s != TVSPEC_OK) return s;
    if (fc == 1) {
        TV_CK(cudaMemcpyAsync(p1, d.p1[1], pb, cudaMemcpyDeviceToDevice, st));
        TV_CK(cudaMemcpyAsync(p2, d.p2[1], pb, cudaMemcpyDeviceToDevice, st));
    }
    return TVSPEC_OK;
}

int tvspec_resident_variant_count(void) { return resident_variant_count(); }

tvspec_status tvspec_resident_variant_info(int index, int *max_H, int *max_W, int *threads,
                                           int *min_ctas_per_sm) {
    int h, w, t, m;
    if (!resident_variant_info(index, &h, &w, &t, &m))
        return fail(TVSPEC_EINVAL, "resident variant index out of range");
    if (max_H) *max_H = h;
    if (max_W) *max_W = w;
    if (threads) *threads = t;
    if (min_ctas_per_sm) *min_ctas_per_sm = m;
    return TVSPEC_OK;
}

int tvspec_tile_count(void) { return tiled_shape_count(); }

tvspec_status tvspec_tile_info(int index, int *cols_per_lane, int *rows_per_thread, int *warps,
                               int *max_temporal_block) {
    if (index < 0 || index >= tiled_shape_count()) return fail(TVSPEC_EINVAL, "tile index out of range");
    const TileShape s = tiled_shape(index);
    if (cols_per_lane) *cols_per_lane = s.V;
    if (rows_per_thread) *rows_per_thread = s.R;
    if (warps) *warps = s.RW;
    if (max_temporal_block) *max_temporal_block = s.TB;
    return TVSPEC_OK;
}

tvspec_status tvspec_plan_stats(tvspec_plan *plan, tvspec_stats *out) {
    if (!plan || !out) return fail(TVSPEC_EINVAL, "NULL argument");
    out->kernel_launches = plan->kernel_launches.load();
    out->graph_launches = plan->graph_launches.load();
    out->graphs_built = plan->graphs_built.load();
    out->decompositions = plan->decompositions.load();
    size_t ws = 0;
    {
        std::lock_guard<std::mutex> lock(plan->mu);
        for (auto &E : plan->cache)
            for (auto &s : E->slots) ws += s.bytes;
        for (auto &s : plan->scratch) ws += s.bytes;
    }
    out->workspace_bytes = ws;
    out->last_tile = plan->last_tile.load();
    out->last_temporal_block = plan->last_depth.load();
    return TVSPEC_OK;
}

const char *tvspec_status_str(tvspec_status status) {
    switch (status) {
        case TVSPEC_OK: return "TVSPEC_OK";
        case TVSPEC_EINVAL: return "TVSPEC_EINVAL";
        case TVSPEC_ENOMEM: return "TVSPEC_ENOMEM";
        case TVSPEC_ECUDA: return "TVSPEC_ECUDA";
        case TVSPEC_ETIMEOUT: return "TVSPEC_ETIMEOUT";
        case TVSPEC_ENOTREADY: return "TVSPEC_ENOTREADY";
        case TVSPEC_ECANCELLED: return "TVSPEC_ECANCELLED";
        case TVSPEC_ENOTSUP: return "TVSPEC_ENOTSUP";
        default: return "TVSPEC_UNKNOWN";
    }
}

const char *tvspec_last_error(void) { return g_last_error.c_str(); }

const char *tvspec_version(void) { return "tvspec 0.1 (sm_103a)"; }

}  // extern "C"
