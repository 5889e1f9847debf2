// k_sym.cu -- the fp32 iterations (Alg. 3) when the weighting function is
// symmetric about the area's centre in both directions and every atom is
// even or odd in each direction (DCT and sequency-ordered WHT rows).  Then
// C(k,u) = sum w phi_k phi_u vanishes unless atoms k and u have the same
// parity class (p mod 2, q mod 2): the product of an odd and an even function
// summed against a symmetric weight is zero.  The update of eq. (20) changes
// only the R_k of the selected atom's class, so each iteration reads a row of
// K/4 entries and updates a quarter of the projections; the three other
// classes keep their maxima.
//
// Atoms are permuted so that the classes are contiguous (perm[new] = original
// index, original order kept inside a class); lane l of the warp that owns a
// block holds, for each class c, the atoms c K/4 + ch 128 + 4 l + e.
// Everything else follows iterate_f32_kernel: D-scaled projections in
// registers, packed FMAs, three-input maxima, one redux for the maximum, a
// scan of the winning lane's class for the smallest index, bounded TMA row
// copies into shared memory.
#include <cuda_runtime.h>

#include <climits>

#include "k_device.cuh"
#include "se_internal.h"

namespace se {
namespace {

using dev::bar_wait;
using dev::bulk_row;
using dev::max3_abs;

constexpr int kBPC = 4;   // blocks (warps) per CTA

template <int VPT>
__global__ void __launch_bounds__(32 * kBPC, 4) iterate_sym_kernel(const IterArgs a)
{
    constexpr int NCH = VPT / 4;           // float4 chunks per lane
    constexpr int NCC = NCH / 4;           // chunks per lane and class
    constexpr int Q = 32 * 4 * NCC;        // atoms per class (K / 4)
    static_assert(NCC >= 1 && NCH % 4 == 0, "whole chunks per class");
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sBar = reinterpret_cast<uint64_t *>(smem);                 // [kBPC][2]
    float *sT = reinterpret_cast<float *>(smem + 16 * kBPC);              // [kBPC][Q]
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *myT = sT + g * Q;
    uint64_t *myBar = sBar + 2 * g;
    if (lane == 0) {
        const uint32_t m = static_cast<uint32_t>(__cvta_generic_to_shared(myBar));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    uint32_t phase = 0;
    bool failed = false;
    const float gamma = static_cast<float>(a.gamma);

    for (int b = blockIdx.x * kBPC + g; b < a.n; b += gridDim.x * kBPC) {
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const float *R0 = static_cast<const float *>(a.R0) + static_cast<size_t>(b) * a.Kp;
        // R2[c][2 ch + h]: atoms c Q + ch 128 + 4 lane + 2 h + {0, 1}, R'_k = R_k D_k
        float2 R2[4][2 * NCC];
        float m[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            m[c] = 0.0f;
#pragma unroll
            for (int ch = 0; ch < NCC; ++ch) {
                const int j = c * Q + ch * 128 + 4 * lane;
                float v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    v[e] = R0[__ldg(a.perm + j + e)] * __ldg(a.Dkp + j + e);
                    m[c] = fmaxf(m[c], fabsf(v[e]));
                }
                R2[c][2 * ch] = make_float2(v[0], v[1]);
                R2[c][2 * ch + 1] = make_float2(v[2], v[3]);
            }
        }

        for (int nu = 0; nu < I; ++nu) {
            // eq. (18): the maximum over the class maxima, then the smallest index
            const float mx = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
            const float M = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
            int kc = INT_MAX;
            float rc = 0.0f;
            if (mx == M) {
                // the first class holding the maximum, then its first atom holding it
                // (k grows with c, ch and e, so this is the lane's smallest index)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (m[c] != M) continue;
#pragma unroll
                    for (int ch = 0; ch < NCC; ++ch) {
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 q = R2[c][2 * ch + (e >> 1)];
                            const float r = (e & 1) ? q.y : q.x;
                            if (fabsf(r) == M) {
                                kc = c * Q + ch * 128 + 4 * lane + e;
                                rc = r;
                                goto found;
                            }
                        }
                    }
                }
            found:;
            }
            int u = static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<unsigned>(kc)));
            const int owner = u == INT_MAX ? 0 : (u % Q) / 4 % 32;
            float ru = __shfl_sync(0xffffffffu, rc, owner);
            if (u < 0 || u >= a.K) {
                if (lane == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
                ru = 0.0f;
            }
            const int cu = u / Q;
            const bool more = nu + 1 < I;
            if (more && lane == 0)
                bulk_row(myT, a.Cc + static_cast<size_t>(u) * Q, static_cast<uint32_t>(Q * sizeof(float)), myBar);
            // eq. (19): c = gamma R'_u D_u
            const float c = gamma * ru * __ldg(a.Dkp + u);
            if (lane == 0) {   // the selection log in original atom indices (model kernel, user logs)
                a.log_u[static_cast<size_t>(b) * a.I_max + nu] = __ldg(a.perm + u);
                a.log_c[static_cast<size_t>(b) * a.I_max + nu] = c;
            }
            if (!more) break;
            if (!bar_wait(myBar, phase)) {
                if (lane == 0) atomicOr(a.err, 1 << DEV_ERR_WAIT_TIMEOUT);
                failed = true;
                bar_wait(myBar, phase);   // let the copy in flight land before leaving
            }
            phase ^= 1u;
            if (failed) break;
            // eq. (20) on the selected class only; its maximum is formed again
            const float2 nc = make_float2(-c, -c);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {   // static register indices: one case runs
                if (cc != cu) continue;
                float mc[2] = {0.0f, 0.0f};
#pragma unroll
                for (int ch = 0; ch < NCC; ++ch) {
                    const float4 t = *reinterpret_cast<const float4 *>(myT + ch * 128 + 4 * lane);
                    float2 &x0 = R2[cc][2 * ch], &x1 = R2[cc][2 * ch + 1];
                    x0 = __ffma2_rn(nc, make_float2(t.x, t.y), x0);
                    x1 = __ffma2_rn(nc, make_float2(t.z, t.w), x1);
                    mc[0] = max3_abs(mc[0], x0.x, x0.y);
                    mc[1] = max3_abs(mc[1], x1.x, x1.y);
                }
                m[cc] = fmaxf(mc[0], mc[1]);
            }
        }
        __syncwarp();
        if (failed) break;
    }
}

__global__ void sym_gather_kernel(const float *__restrict__ C, const float *__restrict__ Dk,
                                  const int *__restrict__ perm, int K, int Kp, float *__restrict__ Cc,
                                  float *__restrict__ Dkp)
{
    const int Q = K / 4;
    const int u = blockIdx.x;
    const int cu = u / Q;
    const float *row = C + static_cast<size_t>(perm[u]) * Kp;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) Cc[static_cast<size_t>(u) * Q + j] = row[perm[cu * Q + j]];
    if (threadIdx.x == 0) Dkp[u] = Dk[perm[u]];
}

}  // namespace

cudaError_t launch_sym_gather(const float *C, const float *Dk, const int *perm, int K, int Kp, float *Cc, float *Dkp,
                              cudaStream_t st)
{
    if (K <= 0 || K % 4) return cudaErrorInvalidValue;
    sym_gather_kernel<<<K, 128, 0, st>>>(C, Dk, perm, K, Kp, Cc, Dkp);
    return cudaGetLastError();
}

template <int VPT>
static cudaError_t launch_sym_vpt(const IterArgs &a, cudaStream_t st, int *launches)
{
    constexpr int Q = 32 * VPT / 4;
    if (a.K != 4 * Q || a.Kp != a.K || !a.log_u || !a.log_c || !a.perm || !a.Cc || !a.Dkp)
        return cudaErrorInvalidValue;
    const size_t smem = 16 * kBPC + sizeof(float) * kBPC * Q + 16;
    auto kern = iterate_sym_kernel<VPT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kBPC, smem)) != cudaSuccess) return e;
    const int need = (a.n + kBPC - 1) / kBPC;
    const int cap = sms * (per_sm > 0 ? per_sm : 1);
    kern<<<need < cap ? need : cap, 32 * kBPC, smem, st>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_iterate_sym(const IterArgs &a, cudaStream_t st, int *launches)
{
    if (a.n <= 0) return cudaSuccess;
    switch (a.Kp) {
    case 512: return launch_sym_vpt<16>(a, st, launches);
    case 1024: return launch_sym_vpt<32>(a, st, launches);
    case 2048: return launch_sym_vpt<64>(a, st, launches);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace se
