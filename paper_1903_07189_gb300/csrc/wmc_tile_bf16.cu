// Instantiations of the temporally blocked tile kernel for __nv_bfloat16 storage.
#include "wmc_tile.cuh"

namespace wmc {
cudaError_t launch_tile_bf16(int mode, int steps, const TileParams &p, cudaStream_t st) {
    return launch_tile_dtype<__nv_bfloat16>(mode, steps, p, st);
}
}  // namespace wmc
