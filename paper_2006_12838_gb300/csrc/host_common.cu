// host_common.cu -- status strings, thread-local error text, launch geometry.
#include <mutex>
#include <stdio.h>
#include <unordered_map>

#include "host_common.h"

namespace plic {

static thread_local char g_last_error[256] = "";

void set_last_error(const char* where, cudaError_t e) {
    snprintf(g_last_error, sizeof g_last_error, "%s: %s (%s)", where, cudaGetErrorName(e),
             cudaGetErrorString(e));
}

void set_limit_error(int64_t ncell) {
    snprintf(g_last_error, sizeof g_last_error,
             "vof_interface_compact_noalloc: field of %lld cells exceeds the limit of %lld cells "
             "of the built-in scratch; use vof_interface_compact with a workspace",
             (long long)ncell, (long long)PLIC_NOALLOC_MAX_CELLS);
}

plic_status check_launch(const char* where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(where, e);
        return PLIC_ERR_CUDA;
    }
    return PLIC_OK;
}

int sm_count() {
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
        n = 1;
    cache[dev] = n;
    return n;
}

int blocks_per_sm(const void* kernel, int threads, size_t smem) {
    static std::mutex mu;
    struct Key {
        const void* k; int t; size_t s; int dev;
        bool operator==(const Key& o) const { return k == o.k && t == o.t && s == o.s && dev == o.dev; }
    };
    struct H { size_t operator()(const Key& k) const {
        return std::hash<const void*>()(k.k) ^ ((size_t)k.t << 20) ^ (k.s << 4) ^ (size_t)k.dev; } };
    static std::unordered_map<Key, int, H> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    Key key{kernel, threads, smem, dev};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem) != cudaSuccess || b <= 0) {
        cudaGetLastError();
        b = 1;
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = b;
    return b;
}

cudaError_t launch_after(const void* kernel, dim3 grid, dim3 block, void** args, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, kernel, args);
}

int stream_grid(const void* kernel, int threads, int64_t work) {
    const int64_t need = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)stride_grid(kernel, threads, work) * STREAM_WAVES;
    const int64_t g = need < cap ? need : cap;
    return g < 1 ? 1 : (int)(g < 2147483647LL ? g : 2147483647LL);
}

int stride_grid(const void* kernel, int threads, int64_t work, size_t smem) {
    int64_t need = (work + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * blocks_per_sm(kernel, threads, smem);
    int64_t g = need < cap ? need : cap;
    return g < 1 ? 1 : (int)g;
}

}  // namespace plic

extern "C" {

const char* plic_status_string(plic_status s) {
    switch (s) {
        case PLIC_OK: return "PLIC_OK";
        case PLIC_ERR_ARG: return "PLIC_ERR_ARG: invalid argument";
        case PLIC_ERR_ALIGN: return "PLIC_ERR_ALIGN: misaligned pointer";
        case PLIC_ERR_CUDA: return "PLIC_ERR_CUDA: CUDA error (see plic_last_error)";
        case PLIC_ERR_UNSUPPORTED: return "PLIC_ERR_UNSUPPORTED: unsupported combination";
        case PLIC_ERR_TIMEOUT: return "PLIC_ERR_TIMEOUT: bounded device wait gave up";
    }
    return "unknown plic_status";
}

const char* plic_last_error(void) { return plic::g_last_error; }

int plic_abi_version(void) { return 1; }

plic_status plic_host_device_pointer(const void* host_ptr, void** dev_ptr) {
    if (!host_ptr || !dev_ptr) return PLIC_ERR_ARG;
    cudaPointerAttributes a;
    const cudaError_t e = cudaPointerGetAttributes(&a, host_ptr);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();           // an unknown address is an answer, not a failure
        return PLIC_ERR_ARG;
    }
    if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return PLIC_ERR_ARG;
    *dev_ptr = a.devicePointer;
    return PLIC_OK;
}

}  // extern "C"
