// Context lifetime and error reporting of the GIPC C ABI.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "common.cuh"
#include "context.cuh"

namespace gipc {

static thread_local char g_last_error[512] = "";

gipc_status fail(gipc_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

gipc_status check_launch(const char* what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GIPC_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return GIPC_OK;
}

namespace {
std::mutex g_facts_mutex;
std::map<int, DeviceFacts> g_device_facts;
std::map<std::tuple<const void*, int, int, size_t>, int> g_occupancy;   // (kernel, device, threads, smem)
std::map<std::pair<const void*, int>, size_t> g_smem_limit;             // (kernel, device) -> raised limit
}  // namespace

DeviceFacts device_facts() {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return DeviceFacts{};
    std::lock_guard<std::mutex> lock(g_facts_mutex);
    auto it = g_device_facts.find(dev);
    if (it != g_device_facts.end()) return it->second;
    DeviceFacts f;
    int sms = 0, coop = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) {
        cudaGetLastError();
        return DeviceFacts{};
    }
    f.device = dev;
    f.sms = sms;
    f.coop = coop != 0;
    g_device_facts[dev] = f;
    return f;
}

int kernel_occupancy(const void* fn, int threads, size_t smem) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 0;
    std::lock_guard<std::mutex> lock(g_facts_mutex);
    const auto key = std::make_tuple(fn, dev, threads, smem);
    auto it = g_occupancy.find(key);
    if (it != g_occupancy.end()) return it->second;
    size_t& limit = g_smem_limit[std::make_pair(fn, dev)];
    if (smem > 48 * 1024 && smem > limit) {
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        limit = smem;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    g_occupancy[key] = occ;
    return occ;
}

unsigned grid_for(int64_t work, int64_t per_block, int per_sm) {
    const int sms = device_facts().sms;
    int64_t b = per_block > 0 ? (work + per_block - 1) / per_block : 1;
    const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace gipc

extern "C" const char* gipc_last_error(void) { return gipc::g_last_error; }

extern "C" gipc_status gipc_create(gipc_ctx** ctx_out_h) {
    if (!ctx_out_h) return gipc::fail(GIPC_ERR_INVALID_ARG, "gipc_create: null output pointer");
    gipc_ctx* c = new (std::nothrow) gipc_ctx();
    if (!c) return gipc::fail(GIPC_ERR_OOM, "gipc_create: host allocation failed");
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return gipc::fail(GIPC_ERR_CUDA, "gipc_create: no current CUDA device");
    }
    *ctx_out_h = c;
    return GIPC_OK;
}

extern "C" gipc_status gipc_destroy(gipc_ctx* ctx) {
    if (!ctx) return GIPC_OK;
    ctx->release_all();
    delete ctx;
    return GIPC_OK;
}

extern "C" gipc_status gipc_profile_begin(gipc_ctx* ctx) {
    if (!ctx) return gipc::fail(GIPC_ERR_INVALID_ARG, "gipc_profile_begin: null context");
    ctx->prof.on = true;
    ctx->prof.reset();
    return GIPC_OK;
}

extern "C" gipc_status gipc_profile_sampling(gipc_ctx* ctx, int kind, int every) {
    if (!ctx || kind < 0 || kind >= GIPC_PROF_KINDS || every < 0)
        return gipc::fail(GIPC_ERR_INVALID_ARG, "gipc_profile_sampling: bad arguments");
    ctx->prof.every[kind] = every;
    return GIPC_OK;
}

extern "C" gipc_status gipc_profile_stop(gipc_ctx* ctx) {
    if (!ctx) return gipc::fail(GIPC_ERR_INVALID_ARG, "gipc_profile_stop: null context");
    ctx->prof.on = false;
    return GIPC_OK;
}

extern "C" gipc_status gipc_profile_read(gipc_ctx* ctx, int kind, gipc_kernel_time* out) {
    if (!ctx || !out || kind < 0 || kind >= GIPC_PROF_KINDS)
        return gipc::fail(GIPC_ERR_INVALID_ARG, "gipc_profile_read: bad arguments");
    const auto& P = ctx->prof;
    out->launches = P.used[kind] / 2;
    out->total_ms = 0.0;
    for (int i = 0; i + 1 < P.used[kind]; i += 2) {
        if (cudaEventSynchronize(P.pool[kind][i + 1]) != cudaSuccess)
            return gipc::fail(GIPC_ERR_CUDA, "gipc_profile_read: event synchronisation failed");
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P.pool[kind][i], P.pool[kind][i + 1]) != cudaSuccess)
            return gipc::fail(GIPC_ERR_CUDA, "gipc_profile_read: elapsed time failed");
        out->total_ms += ms;
    }
    return GIPC_OK;
}
