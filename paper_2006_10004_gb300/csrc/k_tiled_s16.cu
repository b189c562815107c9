// Instantiations of the tiled dual-iteration kernel for p stored as SNORM16 (short).
#include "k_tiled.cuh"

namespace tvspec {

#define TVSPEC_ENTRY(idx, V, R, RW, TB, MINB) \
    {&k_tiled<V, R, RW, TB, MINB, short, true>, &k_tiled<V, R, RW, TB, MINB, short, false>},

TiledKernel tiled_kernel_s16(int shape, bool fast) {
    static const TiledKernel table[][2] = {TVSPEC_TILE_SHAPES(TVSPEC_ENTRY)};
    constexpr int n = sizeof(table) / sizeof(table[0]);
    if (shape < 0 || shape >= n) return nullptr;
    return table[shape][fast ? 0 : 1];
}

}  // namespace tvspec
