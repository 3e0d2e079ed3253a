// wmc_internal.h -- host-side interfaces between the C ABI layer and the kernel launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace wmc {

// MODE_FD_*: the same passes with the conventional finite-difference WMC of Eq. rhs.
enum Mode { MODE_EVAL = 0, MODE_FLOW = 1, MODE_FD_EVAL = 2, MODE_FD_FLOW = 3 };

constexpr int kMaxSteps = 8;

struct StreamParams;   // wmc_stream.cuh
struct TileParams;     // wmc_tile.cuh

// Single-pass kernels (evaluation, one flow step).  dtype: 0 f32, 1 bf16, 2 f16.
// vec: every row start of u, f and out is aligned to two elements (2-element accesses).
cudaError_t launch_stream(int dtype, int mode, int bnd, const StreamParams &p, bool vec,
                          cudaStream_t st);

// Temporally blocked flow kernels, steps = 1..kMaxSteps, one function per storage type, boundary
// rule and tile shape (w16: 16 warps, a 128 x 64 region; w8: 8 warps, 128 x 32).
// map: single-image launches pass two tensor maps, U's window then f's (read when p.f_tma);
// batch launches (batch_tiles >= 0) pass nullptr and use the image descriptors' maps
#define WMC_DECLARE_TILE(name) \
    cudaError_t name(int steps, const CUtensorMap *map, const TileParams &p, int64_t batch_tiles, cudaStream_t st);
WMC_DECLARE_TILE(launch_tile_f32_rep_w16)
WMC_DECLARE_TILE(launch_tile_f32_zero_w16)
WMC_DECLARE_TILE(launch_tile_bf16_rep_w16)
WMC_DECLARE_TILE(launch_tile_bf16_zero_w16)
WMC_DECLARE_TILE(launch_tile_f16_rep_w16)
WMC_DECLARE_TILE(launch_tile_f16_zero_w16)
WMC_DECLARE_TILE(launch_tile_f32_rep_w8)
WMC_DECLARE_TILE(launch_tile_f32_zero_w8)
WMC_DECLARE_TILE(launch_tile_bf16_rep_w8)
WMC_DECLARE_TILE(launch_tile_bf16_zero_w8)
WMC_DECLARE_TILE(launch_tile_f16_rep_w8)
WMC_DECLARE_TILE(launch_tile_f16_zero_w8)
#undef WMC_DECLARE_TILE

// The whole flow of a small image (up to 256 x 256) in one launch of one thread-block cluster
// (wmc_cluster.cu).  cluster_ctas: the cluster size for h x w, 0 when the image is too large;
// cluster_fits: whether that cluster can be scheduled on the current device.
int cluster_ctas(int32_t h, int32_t w);
bool cluster_fits(int ctas);
cudaError_t launch_flow_cluster(int dtype, int bnd, const void *u0, const void *f, void *out,
                                unsigned int *status, int64_t ld, int64_t ldo, int32_t h, int32_t w,
                                int32_t iters, float c_keep, float c_f, float c_h, cudaStream_t st);

// Shape of the TMA box the flow kernel loads for tile shape `tile` (1 or 2), in elements of the
// storage type.
void tile_box(int dtype, int tile, int *box_w, int *box_h);

// FP64 energies; workspace: a 256-byte ticket block followed by 3 doubles per CTA.
int64_t energy_blocks(int32_t h, int32_t w);
// wmc_eval_tma.cu: FP32 evaluation fed by TMA (map: U's window map, as the tile kernel's); the
// status call reads and clears the word its bounded waits set
cudaError_t launch_eval_tma(const CUtensorMap *map, float *out, int64_t ldo, int32_t h, int32_t w,
                            int bnd, float scale, cudaStream_t st);
cudaError_t eval_tma_status(unsigned int *word, cudaStream_t st);
// device address of that word on the current device (for the timeout self-test)
cudaError_t eval_status_word(unsigned int **word);

// wmc_selftest.cu: one CTA waits (bounded) on a transfer that never comes and sets *status
cudaError_t launch_selftest_wait(unsigned int *status, uint64_t limit_ns, cudaStream_t st);

// FP32 energies fed by TMA: maps[0] is U's window map, maps[1] / maps[2] f's / clean's box maps
// (box size from energy_tma_box; read when has_f / has_clean)
void energy_tma_box(int *bw, int *bh);
cudaError_t launch_energy_tma(const CUtensorMap *maps, bool has_f, bool has_clean, int32_t h, int32_t w,
                              int bnd, double *out, void *ws, cudaStream_t st);

cudaError_t launch_energy(int dtype, const void *u, const void *f, const void *clean, int32_t h,
                          int32_t w, int64_t ld, int bnd, double *out, void *workspace,
                          cudaStream_t st);

// Adjoint (wmc_adjoint.cu).  Stacks: n images, image i at offset i * img_stride elements.
// adjoint_blocks: CTAs per image of one adjoint step (one dlambda partial each).
int64_t adjoint_blocks(int32_t h, int32_t w);
cudaError_t launch_stack_step(int bnd, const float *u, const float *f, float *out, const float *lam,
                              float step, int32_t n, int32_t h, int32_t w, int64_t ld,
                              int64_t img_stride, bool vec, cudaStream_t st);
cudaError_t launch_adjoint_step(int bnd, const float *U, const float *g_in, float *g_out,
                                float *grad_f, double *partials, const float *lam, float step,
                                int first, int last, int32_t n, int32_t h, int32_t w, int64_t ld,
                                int64_t img_stride, cudaStream_t st);
cudaError_t launch_energy_grad(int bnd, const float *U, float *grad, int32_t h, int32_t w, int64_t ld,
                               cudaStream_t st);
cudaError_t launch_lambda_grad(const double *partials, int32_t K, int32_t n, int64_t nb, float step,
                               float *grad_lambda, cudaStream_t st);

// One L1 primal-dual step (wmc_l1.cu): out = U^{t+1}, d updated in place.  FP32.
cudaError_t launch_l1_step(int bnd, const float *u, const float *f, float *d, float *out, int32_t h,
                           int32_t w, int64_t ld, float c_h, float c_d, float alpha, bool vec,
                           cudaStream_t st);

}  // namespace wmc
