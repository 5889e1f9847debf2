// k_device.cuh -- device helpers shared by the fp32 iteration kernels:
// the 3-input absolute maximum and the bounded bulk (TMA) row copy.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace se {
namespace dev {

#ifndef SE_ITER_MAX3
#define SE_ITER_MAX3 1       // 1: three-input max instruction, 0: two fmaxf
#endif

// max(m, |a|, |b|); NaN inputs are ignored (maxNum semantics).
__device__ __forceinline__ float max3_abs(float m, float a, float b)
{
#if SE_ITER_MAX3
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(m), "f"(fabsf(a)), "f"(fabsf(b)));
    return r;
#else
    return fmaxf(m, fmaxf(fabsf(a), fabsf(b)));
#endif
}

// One bulk (TMA) copy of a whole row of T into shared memory, completing on
// an mbarrier; waits are bounded by %globaltimer (2 s unless given).
__device__ __forceinline__ void bulk_row(float *dst, const float *src, uint32_t bytes, uint64_t *bar)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const uint32_t m = static_cast<uint32_t>(__cvta_generic_to_shared(bar));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(m), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(d), "l"(src), "r"(bytes), "r"(m) : "memory");
}

__device__ __forceinline__ bool bar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns = 2000000000ull)
{
    const uint32_t m = static_cast<uint32_t>(__cvta_generic_to_shared(bar));
    uint32_t ok = 0;
    unsigned long long t0 = 0;
    for (uint32_t i = 0;; ++i) {
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(ok) : "r"(m), "r"(parity) : "memory");
        if (ok) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (i == 0) t0 = t;
        else if (t - t0 > limit_ns) return false;
    }
}

}  // namespace dev
}  // namespace se
