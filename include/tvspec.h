/*
 * tvspec.h -- C ABI of the GB300 (sm_103a) spectral total-variation decomposition library.
 *
 * The library computes the classical (model-driven) spectral TV decomposition of a greyscale
 * image (arXiv 2006.10004, Sec. 2):
 *
 *   u_0 = f;  u_{k+1} = argmin_v 1/2 |u_k - v|^2 + dt J_TV(v),  k = 0..K-1   (Eq. TVflow, Eq. ROF)
 *   each ROF step solved by n_inner Chambolle projection iterations (Sec. 4.3):
 *       w = div p - u_k/dt;  G = grad w;  p <- (p + tau G) / (1 + tau |G|);  u_{k+1} = u_k - dt div p
 *   (forward differences, Neumann boundary, isotropic |.|, p carried across steps by default)
 *   phi_k = t_k (u_{k+1} - 2 u_k + u_{k-1}) / dt^2,  t_k = k dt,  k = 1..K-1    (Eq. TVtrafo)
 *   S(t_k) = sum_ij |phi_k(i,j)|                                                  (Sec. 2.1)
 *   b^m = sum_{k: e_m <= t_k < e_{m+1}} phi_k dt                                  (Eq. spectral_bands)
 *   f_r = u_{K-1} - t_{K-1} (u_K - u_{K-1}) / dt                                  (Eq. finite_inverse_trafo)
 * so that sum_m b^m + f_r = f when the edges cover [0, t_{K-1}].
 *
 * Conventions shared by every call:
 *   - Images are row-major float32, H rows (index i) by W columns (index j), contiguous
 *     (row stride W) unless a pitch is given.
 *   - The caller owns every input and output buffer. The plan owns its device workspace,
 *     its streams and its CUDA graphs.
 *   - No call throws or aborts. Every call returns a tvspec_status; after TVSPEC_EINVAL the
 *     plan is unchanged and usable. tvspec_last_error() gives a one-line reason.
 *   - Arithmetic: the dual iterations run in float32 (p may be stored as fp16/bf16 between
 *     kernel launches, see tvspec_config.p_storage); u, phi, S, the band sums and the residual
 *     are computed in float64 (or float-float pairs, tvspec_config.acc_mode). Results do not
 *     depend on the tile shape, the iterations per kernel launch, the batch an image runs in,
 *     graph versus plain launches, TMA versus per-thread tile loads, or a checkpoint / resume
 *     in between (bit-identical).
 *   - The library never falls back to CPU arithmetic: without a usable CUDA device every
 *     compute call returns TVSPEC_ECUDA.
 */
#ifndef TVSPEC_H
#define TVSPEC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tvspec_plan tvspec_plan; /* opaque, owned by the library */

typedef enum {
    TVSPEC_OK = 0,
    TVSPEC_EINVAL = 1,      /* an argument is out of range; nothing was launched */
    TVSPEC_ENOMEM = 2,      /* device or host allocation failed, or the request exceeds the budget */
    TVSPEC_ECUDA = 3,       /* a CUDA call failed (no device, launch failure, ...) */
    TVSPEC_ETIMEOUT = 4,    /* a bounded wait ran out (tvspec_wait, or a device-side spin limit) */
    TVSPEC_ENOTREADY = 5,   /* tvspec_poll: the request is still queued or running */
    TVSPEC_ECANCELLED = 6,  /* the request was cancelled before it finished */
    TVSPEC_ENOTSUP = 7      /* the combination of options is not supported by this library */
} tvspec_status;

/* Storage type of the dual field p between kernel launches (config.p_storage). SNORM16 stores
 * q = round(32767 p) (|p| <= 1 always), a uniform step of 1/32767. The 16-bit forms move 12
 * instead of 20 bytes per pixel-iteration; their error is reported, not held to the bars. */
enum { TVSPEC_P_FP32 = 0, TVSPEC_P_FP16 = 1, TVSPEC_P_BF16 = 2, TVSPEC_P_SNORM16 = 3 };

/* Where the image and output pointers of a call live (mem_kind). */
enum { TVSPEC_MEM_HOST = 0, TVSPEC_MEM_DEVICE = 1 };

/* Kernel family for the dual iterations (config.kernel). */
enum {
    TVSPEC_KERNEL_AUTO = 0,      /* tiled kernel, tile and depth from the autotuner */
    TVSPEC_KERNEL_NAIVE = 1,     /* one iteration per launch, one thread per pixel */
    TVSPEC_KERNEL_TILED = 2      /* register-resident tiles, temporal blocking (tile/depth below) */
};

typedef struct {
    int p_storage;          /* TVSPEC_P_*; default TVSPEC_P_FP32 */
    int warm_start;         /* 1 (default): p carried from one ROF step to the next; 0: p = 0 each step */
    float tau;              /* Chambolle step, 0 < tau <= 0.25; default 0.125 (Chambolle 2004: tau <= 1/8) */
    int kernel;             /* TVSPEC_KERNEL_*; default TVSPEC_KERNEL_AUTO */
    int tile;               /* tile-shape index (see tvspec_tile_info), -1 = autotune; default -1 */
    int temporal_block;     /* dual iterations per tiled launch (1..16), 0 = autotune; default 0 */
    int use_graphs;         /* 1 (default): a problem signature used a second time is captured into
                               a CUDA graph then and replayed from then on (plan-level LRU of 4) */
    int fast_math;          /* 1 (default): hardware approximate sqrt/reciprocal; 0: IEEE-rounded */
    size_t mem_budget_bytes;/* device memory the serving scheduler may hold, and the bound on
                             * the batch workspaces a plan keeps cached for reuse (least
                             * recently used ones are freed first; a batch needing more than
                             * the budget still runs, alone); 0 = 60 GiB */
    int max_batch;          /* serving: most requests resident at once; 0 = 256 */
    int pdl;                /* 1 (default): programmatic dependent launch between the kernels of a
                               step (the next kernel is scheduled while the previous one drains;
                               each waits for its predecessor's results before reading them); 0 off */
    int persistent;         /* run a single image's step in one cooperative launch when all its
                               tiles fit on the GPU at once (tiles resident for the whole step):
                               1 with bounded-wait grid barriers between blocks of iterations,
                               2 with each tile waiting (bounded) only for its eight neighbours'
                               progress flags; 0 (default): one launch per block */
    int barrier_timeout_ms; /* longest wait at a grid barrier or for a neighbour before the kernel
                               gives up and the call returns TVSPEC_ETIMEOUT; default 2000 */
    int test_barrier_noshow;/* fault injection for tests: this CTA of the persistent kernel skips
                               its first barrier (persistent 1) or never publishes its progress
                               (persistent 2), so the others time out; default -1 (off) */
    int resident;           /* images up to 64x128 or 128x64 can run their whole decomposition
                               in one CTA (one launch for all of them): 1 (default) when a call
                               holds at least 32 such images (one CTA per image needs many images
                               to fill the GPU), 2 always, 0 never; with kernel = AUTO and fp32
                               storage of p */
    int resident_variant;   /* thread layout of the resident kernel: -1 (default) automatic,
                               else an index below tvspec_resident_variant_count(); an image the
                               variant cannot hold uses the automatic choice */
    int acc_mode;           /* per-step epilogue arithmetic (u, phi, bands, residual, filters):
                               0 (default) float64; 1 compensated float32 (float-float pairs,
                               about 48 significant bits, on the float32 pipes, which GB300 runs
                               many times faster than float64). S is reduced in float64 in both.
                               Results are bit-identical across all paths within one mode. */
    const char *tune_cache; /* optional path of a text file that keeps the autotuner's tile
                               choices across processes: read when the plan is created (lines of
                               another GPU model or library build are ignored), one line appended
                               per new choice; NULL (default) = in-memory only. The string is
                               copied by tvspec_plan_create. */
    int test_fail_alloc;    /* fault injection for tests, on the host: n > 0 makes the plan's
                               n-th batch-workspace allocation (counted from 1 over the plan's
                               life) fail once with TVSPEC_ENOMEM, as if the device were out of
                               memory; default 0 (off) */
    int test_guard_bytes;   /* write checks for tests (compute-sanitizer stands in): n > 0 puts a
                               guard region of n bytes (rounded up to 256) before and after
                               every array of each image's workspace, filled with a known
                               pattern, and checks every guard after each decomposition (plain,
                               batched, stepped, served); a guard byte found changed fails the
                               call with TVSPEC_ECUDA naming its offset. Default 0 (off). */
    int tma;                /* 1: single-image dual-iteration launches load their tiles with the
                               tensor memory accelerator (three 2-D TMA copies into shared
                               memory per CTA, completing on an mbarrier whose wait is bounded:
                               a wait that runs out fails the call with TVSPEC_ETIMEOUT) for
                               the tile shapes that allow it (float32 p, 16-byte aligned tile
                               columns, tile in static shared memory: shapes 8, 24, 25) and
                               images whose tile columns all start on 4 floats (with tiles
                               aligned to the image border, the last column of tiles starts at
                               W - 64: W a multiple of 4); other shapes, images and batches keep
                               per-thread loads. Same bits either way.
                               0 (default): per-thread loads. */
} tvspec_config;

/* One decomposition. Every pointer is in host memory when mem_kind == TVSPEC_MEM_HOST and in
 * device memory of the plan's device when mem_kind == TVSPEC_MEM_DEVICE, except band_edges,
 * which is always host memory. */
typedef struct {
    const float *f;         /* in:  H*W image */
    int H, W;               /* >= 1 each; H*W <= 2^28 */
    double dt;              /* time step = ROF weight lambda of every step; finite, > 0 */
    int K;                  /* number of ROF steps (u_0..u_K); 2 <= K <= 100000 */
    int n_inner;            /* Chambolle iterations per step; 0 <= n_inner <= 10^7 */
    const double *band_edges; /* n_edges edges in t: e_0 >= 0, strictly increasing, only the last may be +inf */
    int n_edges;            /* 2 <= n_edges <= 65 */
    float *bands;           /* out: (n_edges-1)*H*W, band m at offset m*H*W */
    float *residual;        /* out: H*W */
    double *S;              /* out: K-1 values, S[k-1] = S(t_k) */
    double *u_trace;        /* out, optional (NULL): (K+1)*H*W values of u_0..u_K in float64 */
    int mem_kind;           /* TVSPEC_MEM_HOST or TVSPEC_MEM_DEVICE */
    /* Spectral filtering (Eq. filteredTVtrafo substituted into Eq. finite_inverse_trafo),
     * fused into the per-step epilogue: filter q gives
     *     filtered_q = sum_{k=1}^{K-1} H_q(t_k) phi_k dt + h_q f_r
     * (H_q = 1, h_q = 1 reconstructs f; H_q = the indicator of a band, h_q = 0, gives that band). */
    int n_filters;              /* 0 <= n_filters <= 64 */
    const double *filter_H;     /* host: n_filters*(K-1) finite values, H_q(t_k) at q*(K-1) + k-1 */
    const double *filter_residual; /* host: n_filters finite weights h_q of the residual */
    float *filtered;            /* out: n_filters*H*W images (mem_kind memory) */
    /* Parseval-type spectrum (the alternative Sec. 2.1 names, after Burger et al. 2016), read
     * as the pairing <phi_k, f> = sum_ij phi_k(i,j) f(i,j), for which
     * sum_k <phi_k, f> dt + <f_r, f> = |f|^2. Reduced in float64 with the same fixed
     * partition as S. */
    double *S_parseval;         /* out, optional (NULL): K-1 values (mem_kind memory) */
} tvspec_request;

typedef struct {
    uint64_t kernel_launches;   /* kernels this plan launched (graph replays count their nodes) */
    uint64_t graph_launches;    /* CUDA graph replays */
    uint64_t graphs_built;      /* CUDA graphs captured and instantiated */
    uint64_t decompositions;    /* finished decompositions */
    size_t workspace_bytes;     /* device workspace currently held */
    int last_tile;              /* tile-shape index used by the last tiled launch */
    int last_temporal_block;    /* iterations per launch used by the last tiled launch */
} tvspec_stats;

/* Fill *cfg with the defaults listed above. */
void tvspec_config_init(tvspec_config *cfg);

/* Create a plan bound to CUDA device `device`. cfg may be NULL (defaults). On success *out
 * receives the plan. Errors: EINVAL (bad cfg or out == NULL), ECUDA (no such device). */
tvspec_status tvspec_plan_create(const tvspec_config *cfg, int device, tvspec_plan **out);

/* Stop the serving thread (cancelling queued requests), free the workspace and graphs, and
 * free the plan. NULL is a no-op. */
tvspec_status tvspec_plan_destroy(tvspec_plan *plan);

/* Host-only argument check of one request; launches nothing and needs no GPU.
 * Returns OK or EINVAL. With mem_kind == TVSPEC_MEM_HOST it also rejects a non-finite f. */
tvspec_status tvspec_validate(const tvspec_request *req);

/* One decomposition (the plain path). `stream` is a cudaStream_t (NULL = the plan's stream).
 * With TVSPEC_MEM_HOST the call copies f in, runs, copies the outputs back and returns when
 * they are in host memory. With TVSPEC_MEM_DEVICE the call enqueues the work on `stream` and
 * returns; the outputs are valid once the stream reaches that point, and the next call on this
 * plan must use the same stream (or synchronise first) because it reuses the workspace.
 * Errors: EINVAL, ENOMEM, ECUDA. */
tvspec_status tvspec_decompose(tvspec_plan *plan, const float *f, int H, int W, double dt, int K,
                               int n_inner, const double *band_edges, int n_edges, float *bands,
                               float *residual, double *S, int mem_kind, void *stream);

/* Same as tvspec_decompose for one request struct (adds the optional u_trace output). */
tvspec_status tvspec_decompose_ex(tvspec_plan *plan, const tvspec_request *req, void *stream);

/* n independent decompositions of mixed sizes and schedules, run together: every launch
 * covers the tiles of all images still inside their own K steps (Sec. 4.3 timing protocol is
 * per image; batching only shares the GPU). Each result is bit-identical to the same request
 * run alone. All requests must share one mem_kind. Synchronous for TVSPEC_MEM_HOST. */
tvspec_status tvspec_decompose_batch(tvspec_plan *plan, int n, const tvspec_request *reqs,
                                     void *stream);

/* Ground-truth generation for training (Sec. 4.1): greyscale crops of size x size pixels, some
 * taken from (scale*size)^2 windows and downsampled by averaging scale x scale blocks (the
 * paper's 128^2 crops downsampled by 2), standardised to zero mean and unit standard
 * deviation, then decomposed with one schedule (dt, K, n_inner, band edges) for all crops.
 *
 * A crop is (src, y, x, scale): the window of source image `src` with top-left pixel (y, x);
 * the block average sums a block in row-major order in float64 and rounds the mean to float32.
 * Random crop positions are drawn by the caller and passed in. */
typedef struct tvspec_crop {
    int src;    /* index into sources[] */
    int y, x;   /* top-left pixel of the window; the window must lie inside the source */
    int scale;  /* 1..16: window side = scale * size */
} tvspec_crop;

typedef struct tvspec_training_request {
    int n_sources;                  /* >= 1 */
    const float *const *sources;    /* host array of n_sources pointers to row-major images
                                       (mem_kind memory) */
    const int *source_H;            /* host, n_sources heights */
    const int *source_W;            /* host, n_sources widths */
    int n_crops;                    /* >= 1 */
    const tvspec_crop *crops;       /* host, n_crops */
    int size;                       /* crop side, 1..4096 */
    int standardize;                /* 0 none; 1 one mean / population standard deviation over
                                       all crops of this call (the data set); 2 each crop by its
                                       own; 3 by mean_std[0..1]. A zero deviation divides by 1.
                                       out = (float)((x - mean) / sd) in float64 */
    double mean_std[2];             /* in, for standardize == 3 */
    double dt;                      /* > 0 */
    int K;                          /* ROF steps, 2..100000 */
    int n_inner;                    /* dual iterations per step, >= 0 */
    const double *band_edges;       /* host, n_edges increasing t-edges (last may be +inf) */
    int n_edges;                    /* 2..65 */
    float *crops_out;               /* out, optional: n_crops*size*size standardised crops */
    float *bands;                   /* out: n_crops*(n_edges-1)*size*size, crop-major */
    float *residual;                /* out: n_crops*size*size */
    double *S;                      /* out: n_crops*(K-1) */
    double *stats;                  /* out, optional (host): 2 values (standardize 1, 3) or
                                       2*n_crops (standardize 2): mean, deviation pairs */
    int mem_kind;                   /* sources and the outputs above (stats: always host) */
} tvspec_training_request;

/* Runs the whole generation for one request: crop + downsample and standardisation kernels,
 * the decompositions of all crops as one batch (the resident one-CTA-per-image kernel for
 * small crops; results bit-identical to tvspec_decompose of each standardised crop), and one
 * gather of the outputs into the caller's crop-major arrays. Synchronous for TVSPEC_MEM_HOST
 * (and whenever stats is requested); otherwise enqueued on `stream` like tvspec_decompose.
 * Errors: EINVAL (bad request, window outside its source, non-finite mean_std), ENOMEM, ECUDA
 * (including a non-finite value in the flow, detected for TVSPEC_MEM_HOST). */
tvspec_status tvspec_training_set(tvspec_plan *plan, const tvspec_training_request *req,
                                  void *stream);

/* Serving (continuous batching). submit copies the request descriptor (not the buffers, which
 * must stay valid until poll returns OK) and returns a ticket at once. A scheduler thread
 * admits requests while their device memory fits mem_budget_bytes, runs one ROF step of every
 * resident request per scheduler tick, retires finished requests and admits waiting ones at
 * step boundaries. Results are bit-identical to tvspec_decompose_ex of the same request.
 * Only TVSPEC_MEM_HOST requests are accepted. Thread-safe. */
tvspec_status tvspec_submit(tvspec_plan *plan, const tvspec_request *req, uint64_t *ticket);

/* OK when the request finished (outputs written), ENOTREADY while queued or running,
 * ECANCELLED, or the request's own error status. EINVAL for an unknown ticket. A finished
 * ticket stays queryable until the plan is destroyed; it then holds its status only (its
 * workspace and band / filter tables are released when it finishes). Thread-safe. */
tvspec_status tvspec_poll(tvspec_plan *plan, uint64_t ticket);

/* Wait up to timeout_ms (< 0: no limit) for the request; returns like tvspec_poll, or
 * ETIMEOUT. Thread-safe. */
tvspec_status tvspec_wait(tvspec_plan *plan, uint64_t ticket, int timeout_ms);

/* Cancel a queued or running request; it is retired at the next step boundary with
 * ECANCELLED. OK, or EINVAL for an unknown or already finished ticket. */
tvspec_status tvspec_cancel(tvspec_plan *plan, uint64_t ticket);

/* Latency statistics of finished served requests since the plan was created (or the last
 * reset): count, p50 and p99 of submit-to-finish time in milliseconds. */
tvspec_status tvspec_serving_stats(tvspec_plan *plan, int reset, uint64_t *count, double *p50_ms,
                                   double *p99_ms);

/* Checkpoint / resume of one decomposition. The implicit-Euler flow (Eq. TVflow, one Eq. ROF
 * solve per step) is deterministic, so a request can stop after any ROF step, its state can
 * wait in host memory (or another process), and the run can continue from it to the same bits
 * as an uninterrupted tvspec_decompose_ex of the same request on a plan of the same
 * configuration.
 *
 * tvspec_checkpoint_bytes: size in bytes of the state of req under this plan's configuration
 * (a header, then the image's whole device workspace: about 62 + 4 n_bands bytes per pixel);
 * 0 for a NULL or invalid argument.
 *
 * tvspec_decompose_steps: runs ROF steps [k_begin, k_end) of req, 0 <= k_begin < k_end <= K.
 * k_begin == 0 starts from req->f; otherwise state_in (host memory, written by a call that
 * stopped at k_begin) is restored and req->f is not read. k_end < K: the state after step
 * k_end - 1 goes to state_out (host memory, tvspec_checkpoint_bytes(plan, req) bytes, owned
 * by the caller) and the request's outputs are not written; k_end == K: the outputs are
 * written as by tvspec_decompose_ex (req->mem_kind) and state_out is not used. Synchronous,
 * on the plan's stream. EINVAL for a bad range, a missing state buffer, or a state_in of
 * another request, configuration or step; ENOTSUP when the plan runs the request on the
 * one-CTA resident kernel (resident = 2), which has no step boundary; ECUDA for a non-finite
 * value in the flow. */
size_t tvspec_checkpoint_bytes(tvspec_plan *plan, const tvspec_request *req);
tvspec_status tvspec_decompose_steps(tvspec_plan *plan, const tvspec_request *req, int k_begin,
                                     int k_end, const void *state_in, void *state_out);

/* One ROF step (Eq. ROF) by n_iter Chambolle iterations on the plan's kernel: u = g - lambda div p.
 * g (H*W), p1/p2 (H*W, in: starting dual field, out: final) and u (H*W, out) are contiguous
 * float32 buffers in host or device memory per mem_kind. Synchronous for host memory.
 * Errors: EINVAL, ENOMEM, ECUDA, ENOTSUP (p_storage other than fp32). */
tvspec_status tvspec_rof_step(tvspec_plan *plan, const float *g, int H, int W, double lambda,
                              int n_iter, float *p1, float *p2, float *u, int mem_kind,
                              void *stream);

/* The dual iterations alone, on pitched device buffers, as the decomposition runs them:
 * n_iter iterations of p <- (p + tau G)/(1 + tau|G|), G = grad(div p - gl), with gl = g/lambda
 * precomputed by the caller. gl, p1, p2: device float32, row stride `pitch` elements
 * (pitch >= W, pitch % 4 == 0, 16-byte aligned base; columns W..pitch-1 must hold zeros).
 * Enqueued on `stream`, asynchronous. Used to time the hot kernel in isolation.
 * Errors: EINVAL, ECUDA, ENOTSUP (p_storage other than fp32). */
tvspec_status tvspec_chambolle_iterate(tvspec_plan *plan, const float *gl, float *p1, float *p2,
                                       int H, int W, int pitch, int n_iter, void *stream);

/* Inner solvers of one ROF step (Eq. ROF), for comparing accuracy per iteration and time:
 *   TVSPEC_SOLVER_CHAMBOLLE  Chambolle's projection (the decomposition's solver; the tiled,
 *                            temporally blocked kernel)
 *   TVSPEC_SOLVER_FGP        Beck and Teboulle's fast gradient projection on the same dual
 *                            (step 1/8, Nesterov momentum)
 *   TVSPEC_SOLVER_PDHG       Chambolle and Pock's primal-dual hybrid gradient method (the
 *                            family of the GPU toolbox timed in Sec. 4.3); accelerated when
 *                            pdhg_gamma > 0 (steps tau_n, sigma_n, theta_n updated per
 *                            iteration), basic with theta = 1 when pdhg_gamma == 0. */
enum {
    TVSPEC_SOLVER_CHAMBOLLE = 0,
    TVSPEC_SOLVER_FGP = 1,           /* temporally blocked register tiles, 8 iterations per launch */
    TVSPEC_SOLVER_PDHG = 2,
    TVSPEC_SOLVER_FGP_REFERENCE = 3  /* FGP one iteration per launch (same results as FGP) */
};

typedef struct tvspec_rof_request {
    const float *g;         /* in: H*W image (mem_kind memory) */
    int H, W;
    double lambda;          /* ROF weight (the flow's dt), > 0 */
    int solver;             /* TVSPEC_SOLVER_* */
    int max_iter;           /* 0..1e7 */
    double gap_tol;         /* > 0: stop at the first check with duality gap <= gap_tol (sum
                               over pixels); <= 0: run max_iter iterations */
    int check_every;        /* iterations between gap evaluations, >= 1 */
    float pdhg_tau, pdhg_sigma, pdhg_gamma;  /* PDHG steps, tau sigma <= 1/8, gamma >= 0 */
    const float *p1_in, *p2_in;  /* optional (NULL = 0): starting dual field, H*W each, in
                                    Chambolle's scaling |p| <= 1 */
    float *u;               /* out: H*W primal iterate (dual methods: g - lambda div p) */
    float *p1, *p2;         /* out, optional (NULL): final dual field, H*W each */
    int mem_kind;           /* g, p*_in, u, p1, p2 */
    int iterations;         /* out: iterations run */
    double gap;             /* out: duality gap P(u) - D(p) of the returned pair, float64 */
} tvspec_rof_request;

/* Runs one ROF step with the chosen solver. The duality gap of the pair (u, p) is
 * 1/2|u-g|^2 + lambda sum|grad u| - (1/2|g|^2 - 1/2|g - lambda div p|^2), reduced in float64
 * in a fixed order; it bounds 1/2|u - u*|^2. Checking it costs one host synchronisation per
 * check. Synchronous. Errors: EINVAL, ENOMEM, ECUDA, ENOTSUP (p_storage other than fp32). */
tvspec_status tvspec_rof_solve(tvspec_plan *plan, tvspec_rof_request *req, void *stream);

/* The decomposition without any device allocation. No counterpart in the paper: this entry
 * exists for callers that cannot call cudaMalloc/cudaFree where they run (a thread working
 * while another captures a CUDA graph in global mode, real-time loops that cannot take the
 * implicit synchronisation of an allocation, frameworks that own all device memory).
 *
 * f (H*W), bands ((n_edges-1)*H*W), residual (H*W) and S (K-1) are DEVICE pointers on the
 * current CUDA device, caller-owned; a pointer that is not device (or managed) memory of the
 * current device is rejected with TVSPEC_EINVAL before anything is enqueued. Every other
 * buffer comes from one file-scope device array of 48 MiB inside this library, which every GPU
 * that loads the library holds until the process exits. Arithmetic and defaults are those of a
 * default plan (float32 dual iterations, float64 epilogue, tau = 1/8, warm start) with the same
 * per-pixel operations, so the results are bit-identical to tvspec_decompose with such a plan.
 * The work enqueued reads no host memory (the tables travel in kernel parameters).
 *
 * Limits: 1 <= H, W <= 2048, 2 <= K <= 4096, and the workspace (about 44 bytes per pixel plus
 * small tables) must fit the 48 MiB array -- about 1.1 megapixels, so 1024x1024 fits and
 * 2048x2048 does not; larger requests return TVSPEC_EINVAL with the needed size in
 * tvspec_last_error().
 *
 * The call enqueues its work on `stream` (a cudaStream_t; NULL = the legacy default stream)
 * and returns; the outputs are valid once the stream reaches that point. It allocates nothing:
 * the first call on a device (and the first after that device's context was destroyed and
 * created again) looks up the array's device address (cudaGetSymbolAddress, which may load
 * the module) -- make that first call before any stream capture. Every call uses
 * the same array and finds the previous call's contents in it (the call clears what must
 * start at zero), so calls that overlap on the GPU race: issue them on one stream, or
 * synchronise between them. A non-finite value in f is not detected (it propagates).
 * Errors: EINVAL, ENOTSUP, ECUDA. */
tvspec_status tvspec_decompose_noalloc(const float *f, int H, int W, double dt, int K,
                                       int n_inner, const double *band_edges, int n_edges,
                                       float *bands, float *residual, double *S, void *stream);

/* Number of tile shapes this library provides for TVSPEC_KERNEL_TILED, and the geometry of
 * shape `index`: columns per lane, rows per thread, warps per block, maximum iterations per
 * launch. Returns EINVAL for an index out of range. */
int tvspec_tile_count(void);
tvspec_status tvspec_tile_info(int index, int *cols_per_lane, int *rows_per_thread, int *warps,
                               int *max_temporal_block);

/* Number of thread layouts of the resident small-image kernel, and the geometry of layout
 * `index`: the largest image it holds (max_H x max_W), threads per CTA and the CTAs per SM its
 * register budget is built for. Returns EINVAL for an index out of range. */
int tvspec_resident_variant_count(void);
tvspec_status tvspec_resident_variant_info(int index, int *max_H, int *max_W, int *threads,
                                           int *min_ctas_per_sm);

/* Counters of this plan (see tvspec_stats). */
tvspec_status tvspec_plan_stats(tvspec_plan *plan, tvspec_stats *out);

/* Human-readable name of a status code (static storage). */
const char *tvspec_status_str(tvspec_status status);

/* Reason for the last non-OK status returned on this plan (plan may be NULL for calls that
 * failed before a plan existed); thread-local, static storage until the next call. */
const char *tvspec_last_error(void);

/* Library version string (static storage). */
const char *tvspec_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TVSPEC_H */
