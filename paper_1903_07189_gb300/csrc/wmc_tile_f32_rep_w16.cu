// Instantiations of the temporally blocked flow kernel: float storage, replicate boundary,
// 16 warps (a 128 x 64 region per CTA).
#include "wmc_tile.cuh"

namespace wmc {
cudaError_t launch_tile_f32_rep_w16(int steps, const CUtensorMap *map, const TileParams &p,
                                    int64_t batch_tiles, cudaStream_t st) {
    return launch_tile_steps_nw<float, BND_REPLICATE, 16>(steps, map, p, batch_tiles, st);
}
}  // namespace wmc
