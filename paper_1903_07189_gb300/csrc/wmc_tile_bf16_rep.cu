// Instantiations of the temporally blocked flow kernel: __nv_bfloat16 storage, BND_REPLICATE.
#include "wmc_tile.cuh"

namespace wmc {
cudaError_t launch_tile_bf16_rep(int steps, const CUtensorMap *map, const TileV2Params &p,
                                   int64_t batch_tiles, cudaStream_t st) {
    return launch_tile_v2_steps<__nv_bfloat16, BND_REPLICATE>(steps, map, p, batch_tiles, st);
}
}  // namespace wmc
