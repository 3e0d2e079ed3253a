// Instantiations of the temporally blocked tile kernel for __half storage.
#include "wmc_tile.cuh"

namespace wmc {
cudaError_t launch_tile_f16(int mode, int steps, const TileParams &p, cudaStream_t st) {
    return launch_tile_dtype<__half>(mode, steps, p, st);
}
}  // namespace wmc
