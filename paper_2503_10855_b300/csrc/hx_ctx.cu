// hx_ctx.cu -- context lifetime, error reporting and per-stream workspace
// slots of libhx.  A context plays the part of the Hercules runner: it owns
// the backing memory a call needs and allocates it once, up front
// (Hercules paper, Sec. 4.2 last paragraph and Sec. 4.6).
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "hx_internal.cuh"

namespace {
thread_local std::string g_last_error;
}

namespace hx {

hx_status fail(hx_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

hx_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(HX_ERR_CUDA, m);
}

hx_status slot_for(hx_ctx *ctx, hx_stream_t stream, WsSlot **slot) {
    std::lock_guard<std::mutex> lk(ctx->slot_mu);
    int free_i = -1;
    for (int i = 0; i < HX_MAX_STREAMS; ++i) {
        if (ctx->slot_used[i] && ctx->slot_stream[i] == stream) {
            *slot = ctx->ws + i;
            return HX_OK;
        }
        if (!ctx->slot_used[i] && free_i < 0) free_i = i;
    }
    if (free_i < 0) {
        return fail(HX_ERR_NOMEM, "more than HX_MAX_STREAMS distinct streams used with one context");
    }
    ctx->slot_used[free_i] = true;
    ctx->slot_stream[free_i] = stream;
    *slot = ctx->ws + free_i;
    return HX_OK;
}

void release_slot(hx_ctx *ctx, hx_stream_t stream) {
    std::lock_guard<std::mutex> lk(ctx->slot_mu);
    for (int i = 0; i < HX_MAX_STREAMS; ++i)
        if (ctx->slot_used[i] && ctx->slot_stream[i] == stream) ctx->slot_used[i] = false;
}

}  // namespace hx

extern "C" {

int hx_version(void) { return (0 << 16) | 3; }

const char *hx_last_error(void) { return g_last_error.c_str(); }

hx_status hx_create(hx_ctx **out, int device, size_t hbm_budget_bytes) {
    if (!out) return hx::fail(HX_ERR_INVALID, "hx_create: out is NULL");
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_create: cudaGetDeviceCount");
    if (device < 0 || device >= count) return hx::fail(HX_ERR_INVALID, "hx_create: no such device");
    hx::DeviceGuard g(device);
    hx_ctx *ctx = new (std::nothrow) hx_ctx();
    if (!ctx) return hx::fail(HX_ERR_NOMEM, "hx_create: host allocation failed");
    ctx->device = device;
    ctx->hbm_budget = hbm_budget_bytes;
    hx_tune_table_default(&ctx->tune);
    if (const char *tf = getenv("HX_TUNE_FILE")) {
        if (tf[0] && hx_tune_table_load(&ctx->tune, tf) != HX_OK) {
            const std::string msg = std::string("hx_create: HX_TUNE_FILE: ") + hx_last_error();
            delete ctx;
            return hx::fail(HX_ERR_INVALID, msg);
        }
    }
    e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete ctx;
        return hx::cuda_fail(e, "hx_create: SM count");
    }
    const size_t bytes = sizeof(hx::WsSlot) * HX_MAX_STREAMS;
    const size_t nest_bytes = sizeof(hx::NestWs) * HX_MAX_STREAMS;
    e = cudaMalloc(&ctx->ws, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->nest_ws, nest_bytes);
    if (e != cudaSuccess) {
        if (ctx->ws) cudaFree(ctx->ws);
        delete ctx;
        return hx::cuda_fail(e, "hx_create: workspace cudaMalloc");
    }
    e = cudaMemset(ctx->ws, 0, bytes);
    if (e == cudaSuccess) e = cudaMemset(ctx->nest_ws, 0, nest_bytes);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(ctx->ws);
        cudaFree(ctx->nest_ws);
        delete ctx;
        return hx::cuda_fail(e, "hx_create: workspace clear");
    }
    hx_status st = hx::histogram_setup(ctx);
    if (st == HX_OK) st = hx::batch_setup(ctx);
    if (st != HX_OK) {
        cudaFree(ctx->ws);
        cudaFree(ctx->nest_ws);
        delete ctx;
        return st;
    }
    *out = ctx;
    return HX_OK;
}

hx_status hx_debug_inject_launch_failures(hx_ctx *ctx, int32_t after, int32_t count) {
    if (!ctx) return hx::fail(HX_ERR_INVALID, "hx_debug_inject_launch_failures: ctx is NULL");
    if (after < 0 || count < 0) return hx::fail(HX_ERR_INVALID, "hx_debug_inject_launch_failures: negative count");
    std::lock_guard<std::mutex> lk(ctx->inject_mu);
    ctx->inject_after = after;
    ctx->inject_count = count;
    return HX_OK;
}

hx_status hx_debug_checks(int32_t *enabled, int32_t *code, int64_t *a, int64_t *b) {
    if (!enabled || !code || !a || !b) return hx::fail(HX_ERR_INVALID, "hx_debug_checks: NULL argument");
#ifdef HX_DEBUG_CHECKS
    *enabled = 1;
#else
    *enabled = 0;
#endif
    *code = 0;
    *a = 0;
    *b = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_debug_checks: synchronize");
    hx_status (*readers[])(int32_t *, int64_t *, int64_t *) = {hx::checks_map_reduce, hx::checks_stencil,
                                                                hx::checks_histogram, hx::checks_batch,
                                                                hx::checks_srad, hx::checks_noalloc,
                                                                hx::checks_nest};
    for (auto rd : readers) {
        int32_t c = 0;
        int64_t x = 0, y = 0;
        hx_status st = rd(&c, &x, &y);   // reads and clears every file's record
        if (st != HX_OK) return st;
        if (c != 0 && *code == 0) {
            *code = c;
            *a = x;
            *b = y;
        }
    }
    return HX_OK;
}

void hx_destroy(hx_ctx *ctx) {
    if (!ctx) return;
    hx::DeviceGuard g(ctx->device);
    if (!ctx->pending.empty()) {
        cudaDeviceSynchronize();
        for (auto &kv : ctx->pending) {
            cudaEventDestroy(kv.second.second);
            hx_batch_free(kv.second.first);
        }
        ctx->pending.clear();
    }
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->nest_ws) cudaFree(ctx->nest_ws);
    delete ctx;
}

}  // extern "C"
