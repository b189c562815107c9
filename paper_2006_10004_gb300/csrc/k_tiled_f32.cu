// Instantiations of the tiled dual-iteration kernel for p stored as float.
#include "k_tiled.cuh"

namespace tvspec {

#define TVSPEC_ENTRY(idx, V, R, RW, TB, MINB) \
    {&k_tiled<V, R, RW, TB, MINB, float, true>, &k_tiled<V, R, RW, TB, MINB, float, false>},

TiledKernel tiled_kernel_f32(int shape, bool fast) {
    static const TiledKernel table[][2] = {TVSPEC_TILE_SHAPES(TVSPEC_ENTRY)};
    constexpr int n = sizeof(table) / sizeof(table[0]);
    if (shape < 0 || shape >= n) return nullptr;
    return table[shape][fast ? 0 : 1];
}

#define TVSPEC_ENTRY_ONE(idx, V, R, RW, TB, MINB) \
    {&k_tiled_one<V, R, RW, TB, MINB, float, true>, &k_tiled_one<V, R, RW, TB, MINB, float, false>},

TiledOneKernel tiled_one_kernel_f32(int shape, bool fast) {
    static const TiledOneKernel table[][2] = {TVSPEC_TILE_SHAPES(TVSPEC_ENTRY_ONE)};
    constexpr int n = sizeof(table) / sizeof(table[0]);
    if (shape < 0 || shape >= n) return nullptr;
    return table[shape][fast ? 0 : 1];
}

}  // namespace tvspec
