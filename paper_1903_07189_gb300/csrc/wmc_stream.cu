// Instantiations of the single-pass streaming kernels (evaluation and one flow step).
#include "wmc_stream.cuh"

namespace wmc {
cudaError_t launch_stream(int dtype, int mode, int bnd, const StreamParams &p, bool vec,
                          cudaStream_t st) {
    switch (dtype) {
        case 0: return launch_stream_dtype<float>(mode, bnd, p, vec, st);
        case 1: return launch_stream_dtype<__nv_bfloat16>(mode, bnd, p, vec, st);
        case 2: return launch_stream_dtype<__half>(mode, bnd, p, vec, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace wmc
