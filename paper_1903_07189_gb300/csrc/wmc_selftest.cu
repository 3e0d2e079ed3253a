// wmc_selftest.cu -- a wait that nothing completes, for testing the timeout report of the
// multi-step kernels' bounded mbarrier waits without faulting or hanging the GPU.
#include "wmc_window.cuh"

namespace wmc {

// Thread 0 arms the barrier for 16 bytes (arrival counted, transfer pending) and waits on phase 0
// with the same bounded wait the tile kernels use; no copy is issued, so the wait runs out after
// limit_ns and the status bit is set exactly as for a tile whose load timed out.
__global__ void selftest_wait_kernel(unsigned int *status, uint64_t limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_u32(&bar), 1);
    mbar_expect_tx(smem_u32(&bar), 16u);
    if (!mbar_wait_bounded(smem_u32(&bar), 0u, limit_ns)) atomicOr(status, 1u);
}

cudaError_t launch_selftest_wait(unsigned int *status, uint64_t limit_ns, cudaStream_t st) {
    selftest_wait_kernel<<<1, 32, 0, st>>>(status, limit_ns);
    return cudaGetLastError();
}

}  // namespace wmc
