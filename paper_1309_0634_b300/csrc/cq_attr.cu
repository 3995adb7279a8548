/*
 * cq_attr.cu -- the dynamic shared-memory limit of the library's kernels.
 *
 * cudaFuncAttributeMaxDynamicSharedMemorySize is a setting of a kernel on
 * the current device.  Every launch site asks for the bytes it needs through
 * raise_dyn_smem, which remembers, per (device, kernel), the largest value
 * already set, and only ever raises it: a launch planned with a larger
 * footprint stays valid after another thread plans a smaller one.  One mutex
 * covers the check, the driver call and the record, so threads that push
 * different queries at once (the serving loop's dispatcher beside a caller)
 * cannot leave the record above the kernel's real setting.
 */
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "cq_internal.h"

namespace cq {

namespace {
std::mutex g_attr_mu;
std::map<std::pair<int, const void *>, int> g_attr;   /* (device, kernel) -> bytes set */
}  // namespace

cudaError_t raise_dyn_smem(const void *fn, int bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mu);
    int &cur = g_attr[std::make_pair(dev, fn)];
    if (bytes <= cur) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) cur = bytes;
    return e;
}

}  // namespace cq
