// Host-side launch facts that cost driver calls, computed once: a kernel's
// dynamic shared-memory limit is raised only when a launch needs more than
// the limit already set on the current device, and its co-resident CTAs
// per SM are computed once per (device, kernel, block size, shared memory).
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "internal.h"

namespace amc {

namespace {
std::mutex g_mu;
std::map<std::pair<int, const void *>, size_t> g_smem;
std::map<std::tuple<int, const void *, int, size_t>, int> g_occ;
}  // namespace

cudaError_t ensure_smem(const void *f, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_smem.find({dev, f});
    if (it != g_smem.end() && it->second >= smem) return cudaSuccess;
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) g_smem[{dev, f}] = smem;
    return e;
}

cudaError_t ctas_per_sm(const void *f, int threads, size_t smem, int *out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    const auto key = std::make_tuple(dev, f, threads, smem);
    auto it = g_occ.find(key);
    if (it != g_occ.end()) {
        *out = it->second;
        return cudaSuccess;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, f, threads, smem);
    if (e == cudaSuccess) g_occ[key] = *out;
    return e;
}

}  // namespace amc
