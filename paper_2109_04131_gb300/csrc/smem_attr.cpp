// The dynamic shared-memory limit of a kernel is one attribute per function and device, shared
// by every host thread.  Plans run from several threads (usfft_increment_many) launch the same
// kernels with different shared-memory sizes, so the limit only ever grows here: a launch never
// finds it lowered below its own size by another thread.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "usfft_internal.h"

namespace usfft {

cudaError_t allow_dyn_smem(const void* func, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> granted;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    size_t& g = granted[std::make_pair(dev, func)];
    if (bytes <= g) return cudaSuccess;
    e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g = bytes;
    return e;
}

}  // namespace usfft
