// Instantiations of the temporally blocked flow kernel: float storage, zero boundary,
// 8 warps (a 128 x 32 region per CTA).
#include "wmc_tile.cuh"

namespace wmc {
cudaError_t launch_tile_f32_zero_w8(int steps, const CUtensorMap *map, const TileParams &p,
                                    int64_t batch_tiles, cudaStream_t st) {
    return launch_tile_steps_nw<float, BND_ZERO, 8>(steps, map, p, batch_tiles, st);
}
}  // namespace wmc
