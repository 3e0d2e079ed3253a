// Instantiations of the temporally blocked flow kernel: float storage, BND_REPLICATE.
#include "wmc_tile.cuh"

namespace wmc {
cudaError_t launch_tile_f32_rep(int steps, const CUtensorMap *map, const TileV2Params &p,
                                   int64_t batch_tiles, cudaStream_t st) {
    return launch_tile_v2_steps<float, BND_REPLICATE>(steps, map, p, batch_tiles, st);
}
}  // namespace wmc
