// wmc_internal.h -- host-side interfaces between the C ABI layer and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace wmc {

enum Mode { MODE_EVAL = 0, MODE_FLOW = 1 };

// Geometry of the temporally blocked tile kernel: every step updates a CW x CH region of
// cells held in shared memory, surrounded by a one-cell ring that is read but not updated.
// After T steps the inner (CW + 2 - 2T) x (CH + 2 - 2T) cells are exact (each step's error
// front moves in by one cell), and those are written out.
constexpr int kTileCW = 64;
constexpr int kTileCH = 64;
constexpr int kTileThreads = 256;
constexpr int kMaxSteps = 8;

struct TileParams {
    const void *u;   // U^t (device)
    const void *f;   // f (device) or nullptr (mean-curvature flow / eval)
    void *out;       // U^{t+T} or H^w (device)
    int64_t ldu, ldf, ldo;
    int32_t h, w;
    int32_t bnd;     // Boundary
    float c_keep;    // 1 - step*mu
    float c_f;       // step*mu
    float c_h;       // step*lambda/12 (flow) or 1/12 (eval)
};

// dtype: 0 = f32, 1 = bf16, 2 = f16.  steps: 1..kMaxSteps (MODE_EVAL requires 1).
cudaError_t launch_tile(int dtype, int mode, int steps, const TileParams &p, cudaStream_t st);

// FP64 energies; partials: >= energy_partials_count() doubles * 3 + counter word.
int energy_grid_blocks();
cudaError_t launch_energy(int dtype, const void *u, const void *f, const void *clean, int32_t h,
                          int32_t w, int64_t ld, int bnd, double *out, void *workspace,
                          cudaStream_t st);

}  // namespace wmc
