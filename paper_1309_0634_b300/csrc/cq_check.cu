/*
 * cq_check.cu -- cq_check_avg: the AVG division of the finalisations
 * (cq_avg.cuh, integer long division) against the FP64 division, on the
 * device, over pseudo-random (sum, count) pairs.
 *
 * Pair i is drawn from two outputs of the splitmix64 generator (Steele,
 * Lea and Flood, "Fast splittable pseudorandom number generators", 2014) at
 * positions 2i and 2i + 1 of the stream seeded by `seed`: a sum whose
 * magnitude has a bit length uniform in 0 .. 63 (so sums at and above 2^53,
 * which take the FP64 path, are drawn too) and a random sign, and a count
 * whose bit length is uniform in 1 .. 31.  Every pair whose two doubles
 * differ in any bit is counted.
 */
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cq.h"
#include "cq_avg.cuh"

namespace cq {
namespace {

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__global__ void check_avg_kernel(int64_t n, unsigned long long seed, unsigned long long *mismatches) {
    unsigned long long bad = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long h1 = splitmix64(seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(2 * i));
        const unsigned long long h2 = splitmix64(seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(2 * i + 1));
        const int sbits = (int)(h1 & 63u);                    /* 0 .. 63 */
        const int cbits = 1 + (int)((h1 >> 8) % 31u);         /* 1 .. 31 */
        const unsigned long long mag = sbits ? (h2 >> (64 - sbits)) : 0ull;
        const long long s = ((h1 >> 16) & 1u) ? -(long long)mag : (long long)mag;
        uint32_t c = (uint32_t)(h2 & 0xFFFFFFFFu) >> (32 - cbits);
        if (c == 0u) c = 1u;
        const double want = __ddiv_rn(__ll2double_rn(s), (double)(int32_t)c);
        const double got = avg_rn(s, (int32_t)c);
        if (__double_as_longlong(want) != __double_as_longlong(got)) bad++;
    }
    if (bad) atomicAdd(mismatches, bad);
}

}  // namespace
}  // namespace cq

extern "C" CQ_API cq_status cq_check_avg(int64_t n, uint64_t seed, int64_t *mismatches) {
    if (n < 0 || !mismatches) return CQ_EINVAL;
    *mismatches = 0;
    if (n == 0) return CQ_OK;
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(unsigned long long));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CQ_ENOMEM : CQ_ECUDA;
    }
    unsigned long long h = 0;
    e = cudaMemset(d, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        int sms = 148;
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess)
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cq::check_avg_kernel<<<(unsigned)(sms * 8), 256>>>(n, (unsigned long long)seed, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CQ_ENOMEM : CQ_ECUDA;
    *mismatches = (int64_t)h;
    return CQ_OK;
}
