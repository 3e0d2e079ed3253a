// Instantiations of the temporally blocked tile kernel for float storage.
#include "wmc_tile.cuh"

namespace wmc {
cudaError_t launch_tile_f32(int mode, int steps, const TileParams &p, cudaStream_t st) {
    return launch_tile_dtype<float>(mode, steps, p, st);
}
}  // namespace wmc
