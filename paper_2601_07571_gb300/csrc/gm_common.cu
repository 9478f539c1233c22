// gm_common.cu -- context lifecycle, error reporting, host/device staging.
#include <cstring>
#include <string>

#include "gm_internal.cuh"

static thread_local std::string g_last_error;

gm_status gm_set_error(gm_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

gm_status gm_cuda_error(cudaError_t e, const char* what) {
    gm_status st = (e == cudaErrorMemoryAllocation) ? GM_ERR_OOM : GM_ERR_CUDA;
    return gm_set_error(st, std::string(what) + ": " + cudaGetErrorName(e) + " (" +
                                cudaGetErrorString(e) + ")");
}

extern "C" const char* gm_last_error(void) { return g_last_error.c_str(); }

bool gm_is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

gm_status gm_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return gm_cuda_error(e, "cudaMallocAsync");
    }
    return GM_OK;
}

gm_status gm_stage_to_device(const void* src, size_t bytes, cudaStream_t s, void** dev, bool* owned) {
    *owned = false;
    *dev = nullptr;
    if (bytes == 0) return GM_OK;
    if (!src) return gm_set_error(GM_ERR_INVALID_ARG, "null input pointer");
    if (gm_is_device_ptr(src)) {
        *dev = const_cast<void*>(src);
        return GM_OK;
    }
    GM_TRY(gm_alloc(dev, bytes, s));
    *owned = true;
    GM_TRY_CUDA(cudaMemcpyAsync(*dev, src, bytes, cudaMemcpyHostToDevice, s));
    return GM_OK;
}

gm_status gm_copy_out(void* dst, const void* dev_src, size_t bytes, cudaStream_t s) {
    if (bytes == 0) return GM_OK;
    if (!dst) return gm_set_error(GM_ERR_INVALID_ARG, "null output pointer");
    bool dev = gm_is_device_ptr(dst);
    GM_TRY_CUDA(cudaMemcpyAsync(dst, dev_src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!dev) GM_TRY_CUDA(cudaStreamSynchronize(s));
    return GM_OK;
}

extern "C" gm_status gm_create(int device, gm_ctx** out) {
    if (!out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_create: out is null");
    *out = nullptr;
    int n = 0;
    GM_TRY_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_create: no such CUDA device");
    cudaDeviceProp prop;
    GM_TRY_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3)
        return gm_set_error(GM_ERR_UNSUPPORTED, std::string("gm_create: device is sm_") +
                                                    std::to_string(prop.major) + std::to_string(prop.minor) +
                                                    ", this library is built for sm_103a only");
    GM_TRY_CUDA(cudaSetDevice(device));
    // Keep freed stream-ordered allocations in the device's default pool instead of returning
    // them to the CUDA driver at every synchronisation: the scene, sample and map buffers of
    // successive calls then reuse the same memory without new mappings.
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    gm_ctx* c = new gm_ctx();
    c->device = device;
    c->n_sm = prop.multiProcessorCount;
    cudaError_t e = cudaMalloc(&c->dev_err, sizeof(int));
    if (e != cudaSuccess) {
        delete c;
        return gm_cuda_error(e, "cudaMalloc(dev_err)");
    }
    e = cudaMemset(c->dev_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(c->dev_err);
        delete c;
        return gm_cuda_error(e, "cudaMemset(dev_err)");
    }
    *out = c;
    return GM_OK;
}

extern "C" void gm_destroy(gm_ctx* c) {
    if (!c) return;
    cudaFree(c->dev_err);
    delete c;
}

extern "C" gm_status gm_sync(gm_ctx* c, gm_stream stream) {
    if (!c) return gm_set_error(GM_ERR_INVALID_ARG, "gm_sync: null context");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaStreamSynchronize(s));
    int err = 0;
    GM_TRY_CUDA(cudaMemcpy(&err, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (err == GM_DEV_STACK_OVERFLOW)
        return gm_set_error(GM_ERR_INTERNAL, "device: BVH traversal stack overflow");
    if (err == GM_DEV_WAIT_TIMEOUT) {
        cudaMemset(c->dev_err, 0, sizeof(int));
        return gm_set_error(GM_ERR_TIMEOUT, "device: an asynchronous copy or tensor-core product did not complete in time");
    }
    if (err == GM_DEV_TOO_MANY_SAMPLES) {
        cudaMemset(c->dev_err, 0, sizeof(int));
        return gm_set_error(GM_ERR_UNSUPPORTED, "device: the scene needs 2^31 - 16 or more samples (offsets set to 0)");
    }
    if (err != 0) return gm_set_error(GM_ERR_INTERNAL, "device: consistency check failed (" + std::to_string(err) + ")");
    return GM_OK;
}

extern "C" gm_status gm_ctx_launches(const gm_ctx* c, uint64_t* n) {
    if (!c || !n) return gm_set_error(GM_ERR_INVALID_ARG, "gm_ctx_launches: null argument");
    *n = c->launches;
    return GM_OK;
}
