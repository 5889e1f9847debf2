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

// The hardware conversion, kept out of line so that the common path below
// carries no fp64-pipe instruction.
static __device__ __noinline__ float f64_to_f32_hw(double x) { return __double2float_rn(x); }

// fp64 -> fp32 with rounding to nearest, ties to even (IEEE 754), on the
// integer pipe: the 52-bit significand is cut to 23 bits and the 29 dropped
// bits decide the rounding; a carry out of the significand raises the
// exponent (and gives infinity above the largest float).  Doubles whose
// result is a normal float (biased exponents 897 .. 1150) take this path, and
// zeros and double subnormals (below half the smallest float subnormal) give
// a signed zero; the rest (subnormal float results, infinities, NaNs, values
// beyond the float range) take the hardware conversion.  The projection
// kernels convert every sample, and the fp64 pipe is narrow on this GPU.
__device__ __forceinline__ float f64_to_f32_rn(double x)
{
    const unsigned hi = static_cast<unsigned>(__double2hiint(x));
    const unsigned lo = static_cast<unsigned>(__double2loint(x));
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e - 897u < 254u) {
        const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);   // kept significand bits
        const unsigned r = lo & 0x1fffffffu;                       // dropped bits
        const unsigned up = (r > 0x10000000u) | ((r == 0x10000000u) & (m & 1u));
        return __uint_as_float(((((e - 896u) << 23) | m) + up) | (hi & 0x80000000u));
    }
    if (e == 0u) return __uint_as_float(hi & 0x80000000u);
    return f64_to_f32_hw(x);
}

// Split-TF32 tensor-core products (mma.sync m16n8k8): each fp32 operand x is
// x_b = tf32(x) plus x_s = tf32(x - x_b), and a product accumulates
// x_s y_b + x_b y_s + x_b y_b in fp32 (the dropped x_s y_s and the roundings
// leave about 2^-21 relative).  Fragments: g = lane / 4, q = lane mod 4;
// A (16 x 8) {(g, q), (g + 8, q), (g, q + 4), (g + 8, q + 4)}, B (8 x 8)
// {(q, g), (q + 4, g)}, C (16 x 8) {(g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1)}.
__device__ __forceinline__ uint32_t tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &b, uint32_t &sm)
{
    b = tf32_rna(x);
    sm = tf32_rna(x - __uint_as_float(b));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// d += A B in split TF32 (three products, small ones first)
__device__ __forceinline__ void mma3(float (&d)[4], const uint32_t (&ab)[4], const uint32_t (&as)[4], uint32_t bb0,
                                     uint32_t bb1, uint32_t bs0, uint32_t bs1)
{
    mma_tf32(d, as, bb0, bb1);
    mma_tf32(d, ab, bs0, bs1);
    mma_tf32(d, ab, bb0, bb1);
}

// fp32 -> fp64 (exact) on the integer pipe: a normal float's exponent is
// rebiased and its significand shifted into place, zeros keep their sign;
// subnormals, infinities and NaNs take the hardware conversion (out of line).
static __device__ __noinline__ double f32_to_f64_hw(float x) { return static_cast<double>(x); }

__device__ __forceinline__ double f32_to_f64(float x)
{
    const unsigned b = __float_as_uint(x);
    const unsigned e = (b >> 23) & 0xffu;
    const unsigned sign = b & 0x80000000u;
    if (e - 1u < 254u) {
        const unsigned m = b & 0x7fffffu;
        return __hiloint2double(static_cast<int>(sign | ((e + 896u) << 20) | (m >> 3)), static_cast<int>(m << 29));
    }
    if ((b & 0x7fffffffu) == 0u) return __hiloint2double(static_cast<int>(sign), 0);
    return f32_to_f64_hw(x);
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
