// Context management for libmh.
#include "mh_internal.cuh"

mh_status mh_fail(mh_ctx* ctx, mh_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

extern "C" mh_status mh_create(int device, void* stream, mh_ctx** out) {
    if (!out) return MH_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return MH_ERR_CUDA;
    if (device < 0 || device >= n) return MH_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return MH_ERR_CUDA;
    mh_ctx* c = new mh_ctx();
    c->device = device;
    c->stream = (cudaStream_t)stream;
    *out = c;
    return MH_OK;
}

extern "C" mh_status mh_destroy(mh_ctx* ctx) {
    delete ctx;
    return MH_OK;
}

extern "C" const char* mh_last_error(const mh_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" int64_t mh_kernel_launches(const mh_ctx* ctx) { return ctx ? ctx->launches : 0; }

std::atomic<int64_t> g_mh_alloc_calls{0};

extern "C" mh_status mh_set_tensor_cores(mh_ctx* ctx, int on) {
    if (!ctx) return MH_ERR_INVALID_ARG;
    ctx->tensor_cores = on != 0;
    return MH_OK;
}

extern "C" int64_t mh_device_alloc_calls(void) { return g_mh_alloc_calls.load(std::memory_order_relaxed); }

mh_ctx::~mh_ctx() {
    for (auto& kv : prof)
        for (auto& e : kv.second.pending) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
}

prof_scope::prof_scope(mh_ctx* c, const char* n, double flops_, double bytes_)
    : ctx(c), name(n), flops(flops_), bytes(bytes_) {
    if (!ctx || !ctx->profiling) return;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
        a = b = nullptr;
        return;
    }
    cudaEventRecord(a, ctx->stream);
}

prof_scope::~prof_scope() {
    if (!a) return;
    cudaEventRecord(b, ctx->stream);
    prof_region& r = ctx->prof[name];
    r.pending.emplace_back(a, b);
    r.flops += flops;
    r.bytes += bytes;
}

extern "C" mh_status mh_profile_enable(mh_ctx* ctx, int on) {
    if (!ctx) return MH_ERR_INVALID_ARG;
    ctx->profiling = on != 0;
    return MH_OK;
}

extern "C" mh_status mh_profile_read(mh_ctx* ctx, const char* region, double* total_ms, int64_t* launches,
                                     double* flops, double* bytes, int reset) {
    if (!ctx || !region) return mh_fail(ctx, MH_ERR_INVALID_ARG, "null argument");
    MH_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (auto& kv : ctx->prof) {
        for (auto& e : kv.second.pending) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, e.first, e.second) == cudaSuccess) kv.second.total_ms += ms;
            kv.second.launches++;
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        kv.second.pending.clear();
    }
    auto it = ctx->prof.find(region);
    if (total_ms) *total_ms = it == ctx->prof.end() ? 0.0 : it->second.total_ms;
    if (launches) *launches = it == ctx->prof.end() ? 0 : it->second.launches;
    if (flops) *flops = it == ctx->prof.end() ? 0.0 : it->second.flops;
    if (bytes) *bytes = it == ctx->prof.end() ? 0.0 : it->second.bytes;
    if (reset) ctx->prof.clear();
    return MH_OK;
}
