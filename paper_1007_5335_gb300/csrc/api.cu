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
