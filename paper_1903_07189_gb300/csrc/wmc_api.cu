// wmc_api.cu -- the C ABI declared in include/wmc.h: argument checks, workspace layout and
// the host-side loop that drives the stencil kernels on the caller's stream.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include <cuda_runtime.h>

#include "../../include/wmc.h"
#include "wmc_internal.h"

namespace wmc {
cudaError_t launch_tile_f32(int mode, int steps, const TileParams &p, cudaStream_t st);
cudaError_t launch_tile_bf16(int mode, int steps, const TileParams &p, cudaStream_t st);
cudaError_t launch_tile_f16(int mode, int steps, const TileParams &p, cudaStream_t st);
}  // namespace wmc

namespace {

thread_local char g_last_error[512] = "";

wmc_status_t fail(wmc_status_t s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

wmc_status_t cuda_fail(cudaError_t e, const char *what) {
    return fail(WMC_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

size_t elem_size(wmc_dtype_t t) {
    switch (t) {
        case WMC_F32: return 4;
        case WMC_BF16:
        case WMC_F16: return 2;
        default: return 0;
    }
}

// Bytes spanned by an h x w image with pitch ld.
size_t span_bytes(int32_t h, int32_t w, int64_t ld, size_t es) {
    if (h <= 0 || w <= 0) return 0;
    return ((size_t)(h - 1) * (size_t)ld + (size_t)w) * es;
}

bool overlap(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b || na == 0 || nb == 0) return false;
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + nb && pb < pa + na;
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

wmc_status_t check_image(int32_t h, int32_t w, int64_t ld, const char *name) {
    if (h < 0 || w < 0) return fail(WMC_ERR_INVALID_ARG, "%s: negative size %d x %d", name, h, w);
    if (h > 0 && w > 0 && ld < w)
        return fail(WMC_ERR_INVALID_ARG, "%s: leading dimension %lld < width %d", name,
                    (long long)ld, w);
    // Grid rows are bounded by 65535 tiles of at least 50 rows.
    if (h > 3000000) return fail(WMC_ERR_INVALID_ARG, "%s: height %d too large", name, h);
    return WMC_OK;
}

wmc_status_t check_enums(wmc_dtype_t dtype, wmc_boundary_t bnd) {
    if (elem_size(dtype) == 0) return fail(WMC_ERR_INVALID_ARG, "unknown dtype %d", (int)dtype);
    if (bnd != WMC_BOUNDARY_REPLICATE && bnd != WMC_BOUNDARY_ZERO)
        return fail(WMC_ERR_INVALID_ARG, "unknown boundary %d", (int)bnd);
    return WMC_OK;
}

cudaError_t launch_tile(wmc_dtype_t dtype, int mode, int steps, const wmc::TileParams &p,
                        cudaStream_t st) {
    switch (dtype) {
        case WMC_F32: return wmc::launch_tile_f32(mode, steps, p, st);
        case WMC_BF16: return wmc::launch_tile_bf16(mode, steps, p, st);
        case WMC_F16: return wmc::launch_tile_f16(mode, steps, p, st);
        default: return cudaErrorInvalidValue;
    }
}

constexpr int kDefaultSteps = 4;

// The flow on device buffers; all checks done by the caller.
wmc_status_t run_flow(const void *f, const void *u0, void *u, int32_t h, int32_t w, int64_t ld,
                      wmc_dtype_t dtype, float lambda, float step, int32_t iters,
                      wmc_boundary_t bnd, int steps_per_launch, void *ws, cudaStream_t st) {
    const size_t es = elem_size(dtype);
    if (!u0) u0 = f;
    if (h == 0 || w == 0) return WMC_OK;
    if (iters == 0) {
        if (u0 != u) {
            cudaError_t e = cudaMemcpy2DAsync(u, ld * es, u0, ld * es, w * es, h,
                                              cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "copy U^0");
        }
        return WMC_OK;
    }
    const int T = steps_per_launch;
    const int nl = (iters + T - 1) / T;  // launches; the last takes the remainder
    const float mu = f ? 1.0f : 0.0f;
    wmc::TileParams p{};
    p.f = f;
    p.ldu = p.ldf = p.ldo = ld;
    p.h = h;
    p.w = w;
    p.bnd = (int)bnd;
    p.c_keep = 1.0f - step * mu;
    p.c_f = step * mu;
    p.c_h = step * lambda / 12.0f;
    // Ping-pong between u and the workspace so that the last launch writes u.  When U^0
    // already lives in u, the first launch must write the workspace; if the parity then
    // ends in the workspace, one copy finishes the job.
    void *bufs[2];
    bool copy_back = false;
    if (u0 == u) {
        bufs[0] = ws;
        bufs[1] = u;
        copy_back = (nl % 2) == 1;
    } else if (nl % 2 == 1) {
        bufs[0] = u;
        bufs[1] = ws;
    } else {
        bufs[0] = ws;
        bufs[1] = u;
    }
    const void *src = u0;
    int done = 0;
    for (int k = 0; k < nl; ++k) {
        const int s = (iters - done) < T ? (iters - done) : T;
        p.u = src;
        p.out = bufs[k & 1];
        cudaError_t e = launch_tile(dtype, wmc::MODE_FLOW, s, p, st);
        if (e != cudaSuccess) return cuda_fail(e, "flow kernel launch");
        src = p.out;
        done += s;
    }
    if (copy_back) {
        cudaError_t e =
            cudaMemcpy2DAsync(u, ld * es, src, ld * es, w * es, h, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy result");
    }
    return WMC_OK;
}

wmc_status_t check_flow_args(const void *f, const void *u0, void *u, int32_t h, int32_t w,
                             int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                             int32_t iters, wmc_boundary_t bnd, const wmc_config_t *cfg,
                             int *steps_out) {
    wmc_status_t s;
    if ((s = check_enums(dtype, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld, "image")) != WMC_OK) return s;
    if (!std::isfinite(lambda) || lambda < 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "lambda must be finite and >= 0 (got %g)", lambda);
    if (!std::isfinite(step) || step <= 0.0f)
        return fail(WMC_ERR_INVALID_ARG, "step must be finite and > 0 (got %g)", step);
    if (iters < 0) return fail(WMC_ERR_INVALID_ARG, "iters must be >= 0 (got %d)", iters);
    int T = kDefaultSteps;
    if (cfg) {
        if (cfg->steps_per_launch < 0 || cfg->steps_per_launch > wmc::kMaxSteps)
            return fail(WMC_ERR_INVALID_ARG, "steps_per_launch must be 0..%d (got %d)",
                        wmc::kMaxSteps, cfg->steps_per_launch);
        if (cfg->tile != 0) return fail(WMC_ERR_INVALID_ARG, "unknown tile %d", cfg->tile);
        if (cfg->steps_per_launch > 0) T = cfg->steps_per_launch;
    }
    *steps_out = T;
    if (h > 0 && w > 0) {
        if (!u) return fail(WMC_ERR_INVALID_ARG, "u is NULL");
        if (!f && !u0) return fail(WMC_ERR_INVALID_ARG, "f and u0 are both NULL");
        const size_t n = span_bytes(h, w, ld, elem_size(dtype));
        if (overlap(u, n, f, n)) return fail(WMC_ERR_ALIAS, "u overlaps f");
        if (u0 && u0 != u && overlap(u, n, u0, n)) return fail(WMC_ERR_ALIAS, "u overlaps u0");
    }
    return WMC_OK;
}

}  // namespace

extern "C" {

const char *wmc_status_string(wmc_status_t s) {
    switch (s) {
        case WMC_OK: return "WMC_OK";
        case WMC_ERR_INVALID_ARG: return "WMC_ERR_INVALID_ARG";
        case WMC_ERR_ALIAS: return "WMC_ERR_ALIAS";
        case WMC_ERR_UNSUPPORTED: return "WMC_ERR_UNSUPPORTED";
        case WMC_ERR_CUDA: return "WMC_ERR_CUDA";
        case WMC_ERR_TIMEOUT: return "WMC_ERR_TIMEOUT";
        case WMC_ERR_WORKSPACE: return "WMC_ERR_WORKSPACE";
        default: return "WMC_ERR_UNKNOWN";
    }
}

const char *wmc_last_error(void) { return g_last_error; }

int32_t wmc_version(void) { return 100; }

wmc_status_t wmc_eval(const void *u, void *hw, int32_t h, int32_t w, int64_t ld_u, int64_t ld_hw,
                      wmc_dtype_t dtype, wmc_boundary_t bnd, wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s;
    if ((s = check_enums(dtype, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld_u, "u")) != WMC_OK) return s;
    if ((s = check_image(h, w, ld_hw, "hw")) != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    if (!u || !hw) return fail(WMC_ERR_INVALID_ARG, "NULL image pointer");
    const size_t es = elem_size(dtype);
    if (overlap(u, span_bytes(h, w, ld_u, es), hw, span_bytes(h, w, ld_hw, es)))
        return fail(WMC_ERR_ALIAS, "hw overlaps u");
    wmc::TileParams p{};
    p.u = u;
    p.out = hw;
    p.ldu = ld_u;
    p.ldo = ld_hw;
    p.h = h;
    p.w = w;
    p.bnd = (int)bnd;
    p.c_h = 1.0f / 12.0f;
    cudaError_t e = launch_tile(dtype, wmc::MODE_EVAL, 1, p, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "eval kernel launch");
    return WMC_OK;
}

size_t wmc_denoise_workspace_size(int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype) {
    if (h <= 0 || w <= 0 || ld < w || elem_size(dtype) == 0) return 0;
    return round_up((size_t)h * (size_t)ld * elem_size(dtype), WMC_WORKSPACE_ALIGN);
}

wmc_status_t wmc_denoise_ex(const void *f, const void *u0, void *u, int32_t h, int32_t w,
                            int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                            int32_t iters, wmc_boundary_t bnd, const wmc_config_t *config,
                            void *workspace, size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    int T = 0;
    wmc_status_t s =
        check_flow_args(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, config, &T);
    if (s != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    if (iters > 0) {
        const size_t need = wmc_denoise_workspace_size(h, w, ld, dtype);
        if (!workspace || workspace_bytes < need)
            return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need,
                        workspace ? workspace_bytes : (size_t)0);
        if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
            return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
        const size_t n = span_bytes(h, w, ld, elem_size(dtype));
        if (overlap(workspace, need, f, n) || overlap(workspace, need, u, n) ||
            overlap(workspace, need, u0, n))
            return fail(WMC_ERR_ALIAS, "workspace overlaps an image");
    }
    return run_flow(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, T, workspace,
                    (cudaStream_t)stream);
}

wmc_status_t wmc_denoise(const void *f, const void *u0, void *u, int32_t h, int32_t w, int64_t ld,
                         wmc_dtype_t dtype, float lambda, float step, int32_t iters,
                         wmc_boundary_t bnd, void *workspace, size_t workspace_bytes,
                         wmc_stream_t stream) {
    return wmc_denoise_ex(f, u0, u, h, w, ld, dtype, lambda, step, iters, bnd, nullptr, workspace,
                          workspace_bytes, stream);
}

size_t wmc_denoise_host_workspace_size(int32_t h, int32_t w, int64_t ld, wmc_dtype_t dtype) {
    // f, U^0 (when given separately), U and the ping-pong buffer.
    const size_t one = wmc_denoise_workspace_size(h, w, ld, dtype);
    return 4 * one;
}

wmc_status_t wmc_denoise_host(const void *f_host, const void *u0_host, void *u_host, int32_t h,
                              int32_t w, int64_t ld, wmc_dtype_t dtype, float lambda, float step,
                              int32_t iters, wmc_boundary_t bnd, void *workspace,
                              size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    int T = 0;
    wmc_status_t s = check_flow_args(f_host, u0_host, u_host, h, w, ld, dtype, lambda, step, iters,
                                     bnd, nullptr, &T);
    if (s != WMC_OK) return s;
    if (h == 0 || w == 0) return WMC_OK;
    const size_t one = wmc_denoise_workspace_size(h, w, ld, dtype);
    const size_t need = 4 * one;
    if (!workspace || workspace_bytes < need)
        return fail(WMC_ERR_WORKSPACE, "device workspace of %zu bytes needed, %zu given", need,
                    workspace ? workspace_bytes : (size_t)0);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    char *base = static_cast<char *>(workspace);
    void *d_f = f_host ? base : nullptr;
    void *d_u0 = u0_host ? base + one : nullptr;
    void *d_u = base + 2 * one;
    void *d_ws = base + 3 * one;
    const size_t es = elem_size(dtype);
    const size_t pitch = (size_t)ld * es;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    if (d_f && (e = cudaMemcpy2DAsync(d_f, pitch, f_host, pitch, w * es, h, cudaMemcpyHostToDevice,
                                      st)) != cudaSuccess)
        return cuda_fail(e, "copy f to device");
    if (d_u0 && (e = cudaMemcpy2DAsync(d_u0, pitch, u0_host, pitch, w * es, h,
                                       cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "copy u0 to device");
    s = run_flow(d_f, d_u0, d_u, h, w, ld, dtype, lambda, step, iters, bnd, T, d_ws, st);
    if (s != WMC_OK) return s;
    if ((e = cudaMemcpy2DAsync(u_host, pitch, d_u, pitch, w * es, h, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return cuda_fail(e, "copy result to host");
    return WMC_OK;
}

size_t wmc_energy_workspace_size(int32_t h, int32_t w) {
    (void)h;
    (void)w;
    return round_up(3 * sizeof(double) * (size_t)wmc::energy_grid_blocks() + sizeof(unsigned int),
                    WMC_WORKSPACE_ALIGN);
}

wmc_status_t wmc_energy(const void *u, const void *f, const void *clean, int32_t h, int32_t w,
                        int64_t ld, wmc_dtype_t dtype, wmc_boundary_t bnd, double *out,
                        void *workspace, size_t workspace_bytes, wmc_stream_t stream) {
    g_last_error[0] = 0;
    wmc_status_t s;
    if ((s = check_enums(dtype, bnd)) != WMC_OK) return s;
    if ((s = check_image(h, w, ld, "u")) != WMC_OK) return s;
    if (!out) return fail(WMC_ERR_INVALID_ARG, "out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (h == 0 || w == 0) {
        cudaError_t e = cudaMemsetAsync(out, 0, 3 * sizeof(double), st);
        return e == cudaSuccess ? WMC_OK : cuda_fail(e, "clear out");
    }
    if (!u) return fail(WMC_ERR_INVALID_ARG, "u is NULL");
    const size_t need = wmc_energy_workspace_size(h, w);
    if (!workspace || workspace_bytes < need)
        return fail(WMC_ERR_WORKSPACE, "workspace of %zu bytes needed", need);
    if ((uintptr_t)workspace % WMC_WORKSPACE_ALIGN)
        return fail(WMC_ERR_WORKSPACE, "workspace not %d-byte aligned", WMC_WORKSPACE_ALIGN);
    cudaError_t e = wmc::launch_energy((int)dtype, u, f, clean, h, w, ld, (int)bnd, out, workspace, st);
    if (e != cudaSuccess) return cuda_fail(e, "energy kernel launch");
    return WMC_OK;
}

}  // extern "C"
