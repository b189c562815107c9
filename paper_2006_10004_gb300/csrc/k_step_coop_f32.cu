// Instantiations and launcher of the persistent per-step kernel (p stored as float32).
#include <algorithm>

#include "k_step_coop.cuh"

namespace tvspec {

#define TVSPEC_ENTRY_COOP(idx, V, R, RW, TB, MINB) \
    {&k_step_coop<V, R, RW, TB, MINB, true>, &k_step_coop<V, R, RW, TB, MINB, false>},

static StepCoopKernel coop_kernel(int shape, bool fast) {
    static const StepCoopKernel table[][2] = {TVSPEC_TILE_SHAPES(TVSPEC_ENTRY_COOP)};
    constexpr int n = sizeof(table) / sizeof(table[0]);
    if (shape < 0 || shape >= n) return nullptr;
    return table[shape][fast ? 0 : 1];
}

bool step_coop_fits(int shape, bool fast, int n_tiles) {
    StepCoopKernel k = coop_kernel(shape, fast);
    if (!k) return false;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * tiled_shape(shape).RW, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)per_sm * sms >= n_tiles;
}

cudaError_t launch_step_coop(int shape, bool fast, const ImgDesc &d, int gstep, int depth,
                             float tau, unsigned long long timeout_ns, int noshow_block,
                             cudaStream_t st) {
    StepCoopKernel k = coop_kernel(shape, fast);
    if (!k) return cudaErrorInvalidValue;
    int ow, oh;
    tiled_output_tile(tiled_shape(shape), &ow, &oh);
    const int ntx = (d.W + ow - 1) / ow, nty = (d.H + oh - 1) / oh;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntx * nty));
    cfg.blockDim = dim3((unsigned)(32 * tiled_shape(shape).RW));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, d, ntx, gstep, depth, tau, timeout_ns, noshow_block);
}

#define TVSPEC_ENTRY_NBR(idx, V, R, RW, TB, MINB) \
    {&k_step_nbr<V, R, RW, TB, MINB, true>, &k_step_nbr<V, R, RW, TB, MINB, false>},

static StepNbrKernel nbr_kernel(int shape, bool fast) {
    static const StepNbrKernel table[][2] = {TVSPEC_TILE_SHAPES(TVSPEC_ENTRY_NBR)};
    constexpr int n = sizeof(table) / sizeof(table[0]);
    if (shape < 0 || shape >= n) return nullptr;
    return table[shape][fast ? 0 : 1];
}

bool step_nbr_fits(int shape, bool fast, int n_tiles) {
    StepNbrKernel k = nbr_kernel(shape, fast);
    if (!k) return false;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 32 * tiled_shape(shape).RW, 0) !=
            cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (long long)per_sm * sms >= n_tiles;
}

cudaError_t launch_step_nbr(int shape, bool fast, const ImgDesc &d, int gstep, int depth,
                            float tau, unsigned long long timeout_ns, int noshow_block,
                            cudaStream_t st) {
    StepNbrKernel k = nbr_kernel(shape, fast);
    if (!k || !d.tile_flags) return cudaErrorInvalidValue;
    int ow, oh;
    tiled_output_tile(tiled_shape(shape), &ow, &oh);
    const int ntx = (d.W + ow - 1) / ow, nty = (d.H + oh - 1) / oh;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntx * nty));
    cfg.blockDim = dim3((unsigned)(32 * tiled_shape(shape).RW));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident: no wait on an unstarted one
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, d, ntx, nty, gstep, depth, tau, timeout_ns, noshow_block);
}

int max_tiles_for(int H, int W) {
    int most = 0;
    for (int i = 0; i < tiled_shape_count(); ++i) {
        int ow, oh;
        tiled_output_tile(tiled_shape(i), &ow, &oh);
        most = std::max(most, ((W + ow - 1) / ow) * ((H + oh - 1) / oh));
    }
    return most;
}

}  // namespace tvspec
