// k_iterate.cu -- the iteration loop of Fast Selective Extrapolation (Alg. 3)
// for blocks that share one weighting pattern and its full table C.
//
// Per block, starting from R^(0) (eq. 12):
//   u   = argmax_k |R_k| D_k                (eq. 18; ties -> smallest k)
//   c   = gamma R_u / C_uu                  (eq. 19, 1/C_uu tabulated)
//   R_k = R_k - c C(k, u)   for all k       (eq. 20; one row of the
//                                            symmetric C, coalesced)
// repeated I times, then the model of eq. (9) is evaluated on the loss
// pixels, g = sum_nu c_nu phi_{u_nu}, and written over B (last step of
// Alg. 3); the support pixels are copied from the samples.
//
// Layout: a group of W warps owns one block; the block's K projections live
// in registers (VPT per thread, Kp = 32 W VPT).  Element k sits in thread
// (k / VE) % (32 W), vector chunk k / (32 W VE), so one 16-byte vector load
// per thread and chunk reads a whole row of C coalesced.  The update and the
// next selection are fused into one pass over the registers.  The argmax is
// a warp butterfly on (score, index, R) followed, for W > 1, by one
// shared-memory exchange and a single barrier per iteration.  D and 1/C_kk
// sit in shared memory (shared by the CTA's blocks); the selection log
// (u, c) stays in shared memory until the model is evaluated.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "se_internal.h"

namespace se {
namespace {

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void vget(const typename Vec<T>::type &v, T *o);
template <>
__device__ __forceinline__ void vget<float>(const float4 &v, float *o)
{
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <>
__device__ __forceinline__ void vget<double>(const double2 &v, double *o)
{
    o[0] = v.x; o[1] = v.y;
}

template <typename T> struct Cand { T s; int k; T r; };

// (a) beats (b): larger score, then smaller index.
template <typename T>
__device__ __forceinline__ bool better(T sa, int ka, T sb, int kb)
{
    return sa > sb || (sa == sb && ka < kb);
}

template <typename T>
__device__ __forceinline__ void warp_argmax(T &s, int &k, T &r)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T so = __shfl_xor_sync(0xffffffffu, s, o);
        const int ko = __shfl_xor_sync(0xffffffffu, k, o);
        const T ro = __shfl_xor_sync(0xffffffffu, r, o);
        if (better(so, ko, s, k)) { s = so; k = ko; r = ro; }
    }
}

template <typename T, int W, int VPT, int BPC>
__global__ void __launch_bounds__(32 * W * BPC)
iterate_full_kernel(const IterArgs a)
{
    static_assert(W == 1 || BPC == 1, "multi-warp blocks use one block per CTA");
    constexpr int NT = 32 * W;                 // threads per block group
    constexpr int VE = Vec<T>::n;
    constexpr int NCH = VPT / VE;
    using VT = typename Vec<T>::type;
    const int Kp = a.Kp;                       // == NT * VPT (checked on the host)

    extern __shared__ __align__(16) unsigned char smem[];
    T *sD = reinterpret_cast<T *>(smem);
    T *sInvC = sD + Kp;
    Cand<T> *sRed = reinterpret_cast<Cand<T> *>(sInvC + Kp);            // [2][W]
    T *sC = reinterpret_cast<T *>(sRed + 2 * W);                         // [BPC][I_max]
    int *sU = reinterpret_cast<int *>(sC + BPC * a.I_max);               // [BPC][I_max]

    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        sD[k] = static_cast<const T *>(a.Dk)[k];
        sInvC[k] = static_cast<const T *>(a.invC)[k];
    }
    __syncthreads();

    const int g = threadIdx.x / NT;
    const int tid = threadIdx.x % NT;
    const int lane = threadIdx.x & 31;
    const int warp = tid >> 5;
    T *logC = sC + g * a.I_max;
    int *logU = sU + g * a.I_max;
    const T *Ctab = static_cast<const T *>(a.C);
    const T gamma = static_cast<T>(a.gamma);

    for (int b = blockIdx.x * BPC + g; b < a.n; b += gridDim.x * BPC) {
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const T *R0 = static_cast<const T *>(a.R0) + static_cast<size_t>(b) * Kp;

        T R[VPT];
        T s = T(-1);
        int kbest = INT_MAX;
        T rbest = T(0);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            const int k0 = ch * NT * VE + tid * VE;
            VT v = *reinterpret_cast<const VT *>(R0 + k0);
            vget<T>(v, R + ch * VE);
            T dv[VE];
            vget<T>(*reinterpret_cast<const VT *>(sD + k0), dv);
#pragma unroll
            for (int j = 0; j < VE; ++j) {
                const T sc = fabs(R[ch * VE + j]) * dv[j];
                if (sc > s) { s = sc; kbest = k0 + j; rbest = R[ch * VE + j]; }
            }
        }

        for (int nu = 0; nu < I; ++nu) {
            // ---- block-wide argmax of the scores of R^(nu) (eq. 18)
            warp_argmax<T>(s, kbest, rbest);
            if constexpr (W > 1) {
                Cand<T> *slot = sRed + (nu & 1) * W;
                if (lane == 0) slot[warp] = Cand<T>{s, kbest, rbest};
                __syncthreads();
                s = slot[0].s; kbest = slot[0].k; rbest = slot[0].r;
#pragma unroll
                for (int w = 1; w < W; ++w) {
                    const Cand<T> c = slot[w];
                    if (better(c.s, c.k, s, kbest)) { s = c.s; kbest = c.k; rbest = c.r; }
                }
            }
            int u = kbest;
            if (u < 0 || u >= a.K) {          // no admissible atom: cannot happen after host checks
                if (tid == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
                rbest = T(0);
            }
            // ---- coefficient (eq. 19)
            const T c = gamma * rbest * sInvC[u];
            if (tid == 0) { logU[nu] = u; logC[nu] = c; }
            if (nu + 1 == I) break;

            // ---- update (eq. 20) fused with the next selection
            const T *crow = Ctab + static_cast<size_t>(u) * Kp;
            s = T(-1);
            kbest = INT_MAX;
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
                const int k0 = ch * NT * VE + tid * VE;
                VT v = __ldg(reinterpret_cast<const VT *>(crow + k0));
                T cv[VE], dv[VE];
                vget<T>(v, cv);
                vget<T>(*reinterpret_cast<const VT *>(sD + k0), dv);
#pragma unroll
                for (int j = 0; j < VE; ++j) {
                    T &r = R[ch * VE + j];
                    r = fma(-c, cv[j], r);
                    const T sc = fabs(r) * dv[j];
                    if (sc > s) { s = sc; kbest = k0 + j; rbest = r; }
                }
            }
        }
        if constexpr (W > 1) __syncthreads(); else __syncwarp();

        // ---- model on the loss pixels (eq. 9) and replacement of B
        const double *smp = bd.samples;
        double *out = bd.out;
        const T *PhiB = static_cast<const T *>(a.PhiB);
        for (int j = tid; j < a.nB; j += NT) {
            T acc = T(0);
            for (int nu = 0; nu < I; ++nu)
                acc = fma(logC[nu], PhiB[static_cast<size_t>(logU[nu]) * a.nB + j], acc);
            out[a.b_idx[j]] = static_cast<double>(acc);
        }
        for (int p = tid; p < a.MN; p += NT)
            if (a.pat_support[p]) out[p] = smp[p];
        if (bd.sel_idx)
            for (int nu = tid; nu < I; nu += NT) bd.sel_idx[nu] = logU[nu];
        if (bd.sel_coef)
            for (int nu = tid; nu < I; nu += NT) bd.sel_coef[nu] = static_cast<double>(logC[nu]);
        if constexpr (W > 1) __syncthreads(); else __syncwarp();
    }
}

template <typename T, int W, int VPT, int BPC>
cudaError_t launch_cfg(const IterArgs &a, cudaStream_t st, int *launches)
{
    constexpr int threads = 32 * W * BPC;
    if (a.Kp != 32 * W * VPT) return cudaErrorInvalidValue;
    const size_t smem = sizeof(T) * 2 * a.Kp + sizeof(Cand<T>) * 2 * W +
                        (sizeof(T) + sizeof(int)) * BPC * a.I_max + 16;
    auto kern = iterate_full_kernel<T, W, VPT, BPC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int need = (a.n + BPC - 1) / BPC;
    const int grid = need < sms * per_sm ? need : sms * per_sm;
    kern<<<grid, threads, smem, st>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

}  // namespace

// Kp per precision: fp32 keeps up to 64 projections per thread, fp64 up to
// 32; the block group grows to more warps for larger dictionaries.
int iterate_kp(int K, bool fp64)
{
    const int caps32[] = {512, 1024, 2048, 4096, 8192, 16384};
    const int caps64[] = {512, 1024, 2048, 4096, 8192, 16384};
    const int *caps = fp64 ? caps64 : caps32;
    for (int i = 0; i < 6; ++i)
        if (K <= caps[i]) return caps[i];
    return -1;
}

template <>
cudaError_t launch_iterate_full<float>(const IterArgs &a, cudaStream_t st, int *launches)
{
    switch (a.Kp) {
    case 512: return launch_cfg<float, 1, 16, 4>(a, st, launches);
    case 1024: return launch_cfg<float, 1, 32, 4>(a, st, launches);
    case 2048: return launch_cfg<float, 1, 64, 4>(a, st, launches);
    case 4096: return launch_cfg<float, 2, 64, 1>(a, st, launches);
    case 8192: return launch_cfg<float, 4, 64, 1>(a, st, launches);
    case 16384: return launch_cfg<float, 8, 64, 1>(a, st, launches);
    default: return cudaErrorInvalidValue;
    }
}

template <>
cudaError_t launch_iterate_full<double>(const IterArgs &a, cudaStream_t st, int *launches)
{
    switch (a.Kp) {
    case 512: return launch_cfg<double, 1, 16, 4>(a, st, launches);
    case 1024: return launch_cfg<double, 1, 32, 4>(a, st, launches);
    case 2048: return launch_cfg<double, 2, 32, 1>(a, st, launches);
    case 4096: return launch_cfg<double, 4, 32, 1>(a, st, launches);
    case 8192: return launch_cfg<double, 8, 32, 1>(a, st, launches);
    case 16384: return launch_cfg<double, 16, 32, 1>(a, st, launches);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace se
