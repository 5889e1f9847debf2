// se_launch.cpp -- launch shapes of the persistent kernels, computed once per
// device: the SM count, resident CTAs per SM for a (kernel, block size,
// dynamic shared memory) triple, and the kernel's dynamic shared memory limit,
// so that a batch launch costs no attribute or occupancy queries.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>

#include "se_internal.h"

namespace se {
namespace {

std::mutex g_mu;
std::map<int, int> g_sms;                                        // device -> SMs
std::map<std::tuple<int, const void *>, size_t> g_smem;          // (device, kernel) -> limit set
std::map<std::tuple<int, const void *, int, size_t>, int> g_occ; // -> CTAs per SM
std::map<std::tuple<int, const void *>, bool> g_carve;           // (device, kernel) -> carveout set

}  // namespace

cudaError_t launch_grid(const void *kern, int threads, size_t smem, int want, int *grid, bool max_shared)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    auto s = g_sms.find(dev);
    if (s == g_sms.end()) {
        int sms = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        s = g_sms.emplace(dev, sms).first;
    }
    auto a = g_smem.find({dev, kern});
    if (a == g_smem.end() || a->second < smem) {
        if (smem > 48 * 1024 || a != g_smem.end()) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
            if (e != cudaSuccess) return e;
        }
        if (max_shared) {
            e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
            if (e != cudaSuccess) return e;
        }
        g_smem[{dev, kern}] = smem;
    }
    auto o = g_occ.find({dev, kern, threads, smem});
    if (o == g_occ.end()) {
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
        o = g_occ.emplace(std::make_tuple(dev, kern, threads, smem), per_sm > 0 ? per_sm : 1).first;
    }
    const int cap = s->second * o->second;
    *grid = want < 1 ? 1 : (want < cap ? want : cap);
    return cudaSuccess;
}

cudaError_t prefer_max_shared(const void *kern)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_carve.count({dev, kern})) return cudaSuccess;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    g_carve[{dev, kern}] = true;
    return cudaSuccess;
}

int sm_count()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    std::lock_guard<std::mutex> lk(g_mu);
    auto s = g_sms.find(dev);
    if (s == g_sms.end()) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return 1;
        s = g_sms.emplace(dev, sms).first;
    }
    return s->second;
}

}  // namespace se
