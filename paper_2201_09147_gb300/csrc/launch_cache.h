// Host-side cache of launch facts that depend only on (kernel, device,
// configuration): the function attributes a launcher sets and the number of
// resident CTAs it computes.  Filled on the first launch of each
// configuration, so that later launches make no attribute queries.
#pragma once

#include <cstdint>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

namespace sdfnn {

struct LaunchCacheEntry {
    const void* fn;
    int dev;
    uint64_t a, b;
    int value;
};

inline std::mutex& launch_cache_mutex() {
    static std::mutex m;
    return m;
}

inline std::vector<LaunchCacheEntry>& launch_cache_table() {
    static std::vector<LaunchCacheEntry> t;
    return t;
}

// Cached value of (fn, current device, a, b), or computes it with make(&v)
// (a cudaError_t-returning callable) and stores it on success.
template <class Make>
cudaError_t launch_cached(const void* fn, uint64_t a, uint64_t b, int* out, Make make) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lock(launch_cache_mutex());
        for (const auto& x : launch_cache_table())
            if (x.fn == fn && x.dev == dev && x.a == a && x.b == b) {
                *out = x.value;
                return cudaSuccess;
            }
    }
    int v = 0;
    e = make(&v);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(launch_cache_mutex());
    launch_cache_table().push_back({fn, dev, a, b, v});
    *out = v;
    return cudaSuccess;
}

// Sets the kernel's shared-memory attributes once per device: the dynamic
// limit to the device's opt-in maximum (the attribute belongs to the function,
// not to one launch, so launches with different sizes must not lower it) and
// the largest carveout.
template <class Kernel>
cudaError_t ensure_smem_attributes(Kernel k) {
    int done = 0;
    return launch_cached(reinterpret_cast<const void*>(k), ~uint64_t(0), 0, &done, [&](int* v) {
        int dev = 0, optin = 0;
        cudaError_t r = cudaGetDevice(&dev);
        if (r == cudaSuccess) r = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (r == cudaSuccess) r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
        *v = 1;
        return r;
    });
}

}  // namespace sdfnn
