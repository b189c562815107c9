// Host runtime shared by the plain, batched and served paths.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "tvspec.h"
#include "tvspec_internal.h"

namespace tvspec {

// A named NVTX range over a scope: the host runtime's phases (calls, autotuning, graph
// replays, serving ticks) show up by name in profilers; without one attached it costs nothing.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Records msg as the thread's last error and returns s.
tvspec_status fail(tvspec_status s, const std::string &msg);
tvspec_status fail_cuda(cudaError_t e, const char *what);

#define TV_CK(call)                                               \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::tvspec::fail_cuda(e_, #call); \
    } while (0)

// A validated request plus what the host derives from it in float64.
struct Job {
    tvspec_request r;
    std::vector<double> edges;
    std::vector<signed char> band_of_k;  // K entries (entry 0 unused)
    std::vector<double> filt_H, filt_res; // n_filters x (K-1), n_filters
};
tvspec_status make_job(const tvspec_request &req, Job *out);

// Device workspace of one image: one allocation carved into the arrays below.
struct Slot {
    int H = 0, W = 0, pitch = 0, K = 0, n_inner = 0, n_bands = 0, storage = 0;
    bool trace = false, naive = false, async_alloc = false;
    double dt = 0.0;
    char *base = nullptr;
    size_t bytes = 0;
    size_t zero_off = 0, zero_bytes = 0;  // region cleared at the start of every decomposition
    float *f = nullptr;
    void *p1[2] = {nullptr, nullptr}, *p2[2] = {nullptr, nullptr};  // two copies of p
    float *lo1[2] = {nullptr, nullptr}, *lo2[2] = {nullptr, nullptr};  // their low parts (fp32)
    float *gl = nullptr;
    double *ua = nullptr, *ub = nullptr, *u3 = nullptr, *acc = nullptr;
    float *bands = nullptr, *residual = nullptr;
    double *S = nullptr, *utrace = nullptr, *partials = nullptr;
    unsigned *counter = nullptr, *status = nullptr;
    unsigned *tile_flags = nullptr;  // epochs of the neighbour-synchronised persistent kernel
    signed char *band_of_k = nullptr;
    int n_filters = 0;
    double *filt_H = nullptr, *filt_res = nullptr, *facc = nullptr;
    float *filtered = nullptr;
    double *S_par = nullptr, *partials_par = nullptr;  // Parseval-type spectrum, if requested
    int acc_mode = 0;  // epilogue arithmetic (tvspec_config::acc_mode)
    int ep_blocks = 0;
    size_t p_bytes = 0;  // bytes of one pitched p array (one component, one copy)
    std::vector<std::pair<size_t, size_t>> guards;  // test_guard_bytes regions (offset, bytes)
};
constexpr unsigned char kGuardByte = 0xA5;
size_t slot_bytes_for(const Job &j, int storage, bool naive, int guard = 0);
tvspec_status slot_alloc(Slot *s, const Job &j, int storage, bool naive, cudaStream_t st,
                         bool async_alloc, int acc_mode = 0, int guard = 0);
// test_guard_bytes: every guard region of the slot still holds what it was given (zero inside
// the region cleared per decomposition, kGuardByte elsewhere); ECUDA naming the first byte
// written otherwise. Synchronises st.
tvspec_status slot_check_guards(const Slot &s, cudaStream_t st);
void slot_free(Slot *s, cudaStream_t st);
ImgDesc slot_desc(const Slot &s, int s0);

// Device tables of one set of images: descriptors, tiles of one tile shape, epilogue blocks.
// Images are kept in the given order; prefix arrays give the first tile / epilogue block of
// each image so that a prefix of the images maps to a prefix of each table.
struct LaunchSet {
    int n = 0, shape = -1, depth = 0;
    bool pdl = false;  // programmatic dependent launch for this set's kernels (autotuned)
    ImgDesc *d_descs = nullptr;
    TileRef *d_tiles = nullptr;
    int *d_ep_img = nullptr, *d_ep_base = nullptr;
    size_t cap_descs = 0, cap_tiles = 0, cap_ep = 0, cap_base = 0;
    std::vector<ImgDesc> h_descs;
    std::vector<int> tile_prefix, ep_prefix;
    void release();
};
// Builds and uploads (synchronously) the tables for descs with tile shape `shape` (-1: none).
tvspec_status launchset_build(LaunchSet *ls, const std::vector<ImgDesc> &descs, int shape,
                              int depth);

struct CacheEntry {
    std::string key;
    std::vector<Slot> slots;     // run order: tiled images by K (descending), then resident ones
    int n_tiled = 0;             // slots [0, n_tiled) run step by step, the rest resident
    int *d_res_idx = nullptr;    // slot indices of resident images, grouped by variant
    std::vector<std::pair<int, int>> res_groups;  // (variant, count) in d_res_idx order
    std::vector<int> order;      // order[i] = index of the caller's request in slot i
    LaunchSet ls;
    int maxK = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t graph_kernels = 0;
    int uses = 0;                  // decompositions run from this entry (captured on the 2nd)
    unsigned *h_status = nullptr;  // pinned, one word per image
};

struct Server;  // serving scheduler (serving.cu)

// The autotuner's choice for a set of image sizes.
struct TuneChoice {
    int shape = -1, depth = 1;
    bool pdl = false;
};

}  // namespace tvspec

struct tvspec_plan {
    // second copy of the dual field for tvspec_chambolle_iterate on caller buffers
    void *ping = nullptr;
    size_t ping_bytes = 0;
    int device = 0;
    tvspec_config cfg{};
    cudaStream_t stream = nullptr;
    // second stream and events of the split epilogue: the spectral part of step k runs on
    // `side` beside step k+1's dual iterations on the main stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::mutex mu;  // serialises the plain and batched paths
    std::list<std::unique_ptr<tvspec::CacheEntry>> cache;  // most recent first
    std::map<std::string, tvspec::TuneChoice> tune;          // key -> (shape, depth, pdl)
    std::string tune_cache;   // file keeping tune across processes ("" = none)
    double *h_word = nullptr; // page-locked scalar for small device-to-host reads (plan->mu held)
    std::string tune_prefix;  // this GPU model and shape table, first field of the file lines
    std::map<std::string, std::unique_ptr<tvspec::LaunchSet>> iter_sets;
    std::list<tvspec::Slot> scratch;                        // buffers of tvspec_rof_step etc.
    std::atomic<uint64_t> kernel_launches{0}, graph_launches{0}, graphs_built{0},
        decompositions{0};
    std::atomic<int> last_tile{-1}, last_depth{0};
    uint64_t alloc_count = 0;  // batch-workspace allocations so far (test_fail_alloc; plan->mu held)
    tvspec::Server *server = nullptr;  // created on first submit, freed by tvspec_server_stop
    std::mutex server_mu;
};

namespace tvspec {

// Chooses (shape, depth) for a set of slots (autotuned unless the config fixes them).
// table_form: time the tile-table kernel even for one image (the serving path always uses it).
// *pdl (if given) receives whether programmatic dependent launch paid for the chosen shape.
tvspec_status choose_tiles(tvspec_plan *plan, const std::vector<Slot *> &slots, cudaStream_t st,
                           int *shape, int *depth, bool table_form = false, bool *pdl = nullptr);

// Enqueues the device work of one ROF step at global step gstep for the first n_active images
// of the set (dual iterations + epilogue). Adds the kernels launched to *n_kernels.
tvspec_status enqueue_step(tvspec_plan *plan, LaunchSet &ls, std::vector<Slot *> &slots,
                           int n_active, int gstep, cudaStream_t st, uint64_t *n_kernels);

size_t plan_budget(const tvspec_plan *plan);

// The cached workspace, tables and graph of a set of jobs (built on first use; plan->mu held).
tvspec_status get_entry(tvspec_plan *plan, const std::vector<Job> &jobs, CacheEntry **out);
// Enqueues the whole decomposition of a cached entry on st (graph replay when captured).
tvspec_status launch_entry(tvspec_plan *plan, CacheEntry &E, cudaStream_t st);
// Device-to-device copies as one launch (stream-ordered table; zero-byte items skipped).
tvspec_status enqueue_copy_list(const std::vector<CopyItem> &items, cudaStream_t st);
// Makes `later` wait for the work enqueued on `earlier` so far.
tvspec_status order_after(cudaStream_t later, cudaStream_t earlier);

// n_inner dual iterations of the tiled kernel on one image's buffers d.p1/p2[0..1], d.gl
// (plan->mu held); *final_copy receives the copy of p that holds the result.
tvspec_status run_iterations(tvspec_plan *plan, ImgDesc d, cudaStream_t st, int *final_copy);

// Tile choice for an H x W image, tuned on plan-owned scratch buffers (takes the plan lock).
tvspec_status tune_for_size(tvspec_plan *plan, int H, int W, int *shape, int *depth,
                            bool *pdl = nullptr);

}  // namespace tvspec
