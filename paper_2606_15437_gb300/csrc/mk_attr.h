// mk_attr.h -- host helper: raise a kernel's dynamic shared-memory limit
// once per (device, kernel).  cudaFuncSetAttribute acts on the current
// device, so a process that drives several GPUs needs it on each of them;
// the cache avoids repeating the call on every launch.  Thread-safe.
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>
#include <vector>

namespace mkd {

struct SmemAttr {
    int device;
    const void *kernel;
    size_t bytes;
};

inline void ensure_dynamic_smem(const void *kernel, size_t bytes) {
    static std::mutex mutex;
    static std::vector<SmemAttr> done;
    int device = 0;
    cudaGetDevice(&device);
    std::lock_guard<std::mutex> lock(mutex);
    for (auto &e : done)
        if (e.device == device && e.kernel == kernel) {
            if (bytes > e.bytes) {
                cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
                e.bytes = bytes;
            }
            return;
        }
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    done.push_back({device, kernel, bytes});
}

}  // namespace mkd
