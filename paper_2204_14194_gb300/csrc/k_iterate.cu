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

#include "k_device.cuh"
#include "se_internal.h"

#ifndef SE_ITER_ASYNC
#define SE_ITER_ASYNC 2      // 0: row of T in registers, 1: cp.async to shared, 2: TMA bulk copy
#endif

namespace se {
namespace {

using dev::bar_wait;
using dev::bulk_row;
using dev::max3_abs;

template <typename T> struct Vec;
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void vget(const typename Vec<T>::type &v, T *o);
template <>
__device__ __forceinline__ void vget<double>(const double2 &v, double *o)
{
    o[0] = v.x; o[1] = v.y;
}


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

// ---------------------------------------------------------------------------
// fp32 form, on D-scaled quantities.  With R'_k = R_k D_k and the table row
// T[u][k] = C(k, u) D_k (both scaled in the GEMM epilogues), eq. (18) is
// u = argmax |R'_k|, eq. (19) is c = gamma R'_u D_u (since 1/C_uu = D_u^2)
// and eq. (20) is R'_k -= c T[u][k]: one FFMA and one FMNMX per atom and
// iteration, no per-atom loads besides the row of T.  Inadmissible atoms have
// D = NaN, so their R' is NaN and fmaxf never selects them.
//
// Scores |R'| are >= 0, so their IEEE bit patterns order like unsigned
// integers and the warp maximum is one redux.sync.  The fused update keeps
// four independent running maxima (one per position of the float4) instead
// of a compare-and-select chain; only the lane(s) holding the maximum then
// look for its smallest index, scanning the chain(s) whose maximum matched.
// Ties therefore still go to the smallest k, as in the generic path.
#ifndef SE_ITER_SCAN_BREAK
#define SE_ITER_SCAN_BREAK 1  // 1: the winning lane stops its scan at the first match
#endif
template <int W, int VPT, bool CERT = false>
__device__ __forceinline__ void select_f32(const float2 (&R2)[VPT / 2], const float (&m)[4], int tid,
                                           int lane, int warp, Cand<float> *slot, int &u, float &ru,
                                           float *second = nullptr)
{
    constexpr int NT = 32 * W;
    constexpr int NCH = VPT / 4;
    const float mx = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
    const float M = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
    // key: the index above the sign bit of R' (the winner's |R'| is M, so the
    // warp minimum of the keys gives both the smallest index and R'_u)
    unsigned key = 0xffffffffu;
    if (mx == M) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (m[j] == M) {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int k = ch * NT * 4 + tid * 4 + j;
                    const float2 q = R2[ch * 2 + (j >> 1)];
                    const float r = (j & 1) ? q.y : q.x;
                    if (static_cast<unsigned>(k) < (key >> 1) && fabsf(r) == M) {
                        key = (static_cast<unsigned>(k) << 1) | (__float_as_uint(r) >> 31);
#if SE_ITER_SCAN_BREAK
                        break;   // k grows with ch: the first match is this chain's smallest index
#endif
                    }
                }
            }
        }
    }
    const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
    const int kw = static_cast<int>(kmin >> 1);   // INT_MAX when no lane holds M
    const float rw = (kmin & 1u) ? -M : M;
    if constexpr (CERT) {
        const int owner = kw == INT_MAX ? 0 : (kw >> 2) % NT % 32;
        static_assert(W == 1, "the runner-up is formed within one warp");
        // runner-up: the largest |R'| over every atom but the winner (the other
        // chains of each lane by their maxima, the winner's own chain in full)
        float sl = 0.0f;
        if (lane == owner && kw != INT_MAX) {
            const int jw = kw & 3;
#pragma unroll
            for (int j = 0; j < 4; ++j) {   // static register indices: j is unrolled
                if (j != jw) {
                    sl = fmaxf(sl, m[j]);
                    continue;
                }
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    const int k = ch * NT * 4 + tid * 4 + j;
                    const float2 q = R2[ch * 2 + (j >> 1)];
                    if (k != kw) sl = fmaxf(sl, fabsf((j & 1) ? q.y : q.x));
                }
            }
        } else {
            sl = mx;
        }
        *second = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(sl)));
    }
    if constexpr (W == 1) {
        u = kw;
        ru = rw;
    } else {
        if (lane == 0) slot[warp] = Cand<float>{M, kw, rw};
        __syncthreads();
        float sb = slot[0].s;
        int kb = slot[0].k;
        float rb = slot[0].r;
#pragma unroll
        for (int w = 1; w < W; ++w) {
            const Cand<float> c = slot[w];
            if (better(c.s, c.k, sb, kb)) { sb = c.s; kb = c.k; rb = c.r; }
        }
        u = kb;
        ru = rb;
    }
}


// The row of T is copied global -> shared with cp.async (16 bytes per
// thread and chunk, L1-allocating), so the in-flight row holds no registers;
// each thread later reads back exactly the chunks it copied itself, so only
// its own cp.async group has to complete.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}


// Register budget: VPT projections (the row of T is staged in shared memory
// when SE_ITER_ASYNC, in registers otherwise); the launch bound keeps at
// least SE_ITER_MIN_WARPS warps per SM resident.
#ifndef SE_ITER_MIN_WARPS
#define SE_ITER_MIN_WARPS 16
#endif
template <int W, int VPT, int BPC, bool CERT = false>
__global__ void __launch_bounds__(32 * W * BPC, (SE_ITER_MIN_WARPS + W * BPC - 1) / (W * BPC))
iterate_f32_kernel(const IterArgs a)
{
    static_assert(W == 1 || BPC == 1, "multi-warp blocks use one block per CTA");
    static_assert(VPT % 4 == 0, "whole float4 chunks");
    constexpr int NT = 32 * W;
    constexpr int NCH = VPT / 4;
    const int Kp = a.Kp;

    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sBar = reinterpret_cast<uint64_t *>(smem);                     // [BPC] (bulk copies)
    float *sT = reinterpret_cast<float *>(smem + 16 * BPC);                  // [BPC][Kp] if async
    Cand<float> *sRed = reinterpret_cast<Cand<float> *>(sT + (SE_ITER_ASYNC ? BPC * Kp : 0));

    const int g = threadIdx.x / NT;
    const int tid = threadIdx.x % NT;
    const int lane = threadIdx.x & 31;
    const int warp = tid >> 5;
    float *myT = sT + g * Kp;
    uint64_t *myBar = sBar + 2 * g;
    if (SE_ITER_ASYNC == 2 && tid == 0) {
        const uint32_t m = static_cast<uint32_t>(__cvta_generic_to_shared(myBar));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(m) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if constexpr (W > 1) __syncthreads(); else __syncwarp();
    uint32_t phase = 0;
    bool failed = false;
    const float *Ttab = static_cast<const float *>(a.C);
    const float *Dk = static_cast<const float *>(a.Dk);
    const float gamma = static_cast<float>(a.gamma);

    for (int b = blockIdx.x * BPC + g; b < a.n; b += gridDim.x * BPC) {
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const float *R0 = static_cast<const float *>(a.R0) + static_cast<size_t>(b) * Kp;

        // R2[2 ch + h] holds projections k = ch*NT*4 + tid*4 + 2h + {0, 1}
        float2 R2[VPT / 2];
        float m[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            float4 v = *reinterpret_cast<const float4 *>(R0 + ch * NT * 4 + tid * 4);
            if (a.r0_scale) {   // R^(0) stored unscaled: R'_k = R_k D_k here
                const float4 d = *reinterpret_cast<const float4 *>(a.r0_scale + ch * NT * 4 + tid * 4);
                v.x *= d.x; v.y *= d.y; v.z *= d.z; v.w *= d.w;
            }
            R2[ch * 2 + 0] = make_float2(v.x, v.y);
            R2[ch * 2 + 1] = make_float2(v.z, v.w);
            m[0] = fmaxf(m[0], fabsf(v.x));
            m[1] = fmaxf(m[1], fabsf(v.y));
            m[2] = fmaxf(m[2], fabsf(v.z));
            m[3] = fmaxf(m[3], fabsf(v.w));
        }

        int first_close = -1;
        int lu = 0;
        float lc = 0.0f;
        for (int nu = 0; nu < I; ++nu) {
            int u;
            float ru;
            if constexpr (CERT) {
                float s2;
                select_f32<W, VPT, true>(R2, m, tid, lane, warp, sRed + (nu & 1) * W, u, ru, &s2);
                const float s1 = fabsf(ru);
                if (first_close < 0 && !(s1 - s2 > a.cert_delta * s1)) first_close = nu;
            } else {
                select_f32<W, VPT>(R2, m, tid, lane, warp, sRed + (nu & 1) * W, u, ru);
            }
            if (u < 0 || u >= a.K) {
                if (tid == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
                ru = 0.0f;
            }
            const float *trow = Ttab + static_cast<size_t>(u) * Kp;
            const bool more = nu + 1 < I;
            if (SE_ITER_ASYNC == 1 && more) {
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch)
                    cp_async16(myT + ch * NT * 4 + tid * 4, trow + ch * NT * 4 + tid * 4);
            }
            if (SE_ITER_ASYNC == 2 && more && tid == 0)
                bulk_row(myT, trow, static_cast<uint32_t>(Kp * sizeof(float)), myBar);
            const float c = gamma * ru * __ldg(Dk + u);
            // the selection log, read by the model kernel (eq. 9): lane nu mod 32 of
            // warp 0 holds entry nu, written 32 entries at a time
            if (tid == (nu & 31)) {
                lu = u;
                lc = c;
            }
            if (((nu & 31) == 31 || !more) && tid <= (nu & 31)) {
                const size_t o = static_cast<size_t>(b) * a.I_max + (nu & ~31) + tid;
                a.log_u[o] = lu;
                a.log_c[o] = lc;
            }
            if (!more) break;

            m[0] = m[1] = m[2] = m[3] = 0.0f;
            if (SE_ITER_ASYNC == 1) cp_async_wait_all();
            if (SE_ITER_ASYNC == 2) {
                if (!bar_wait(myBar, phase)) {
                    if (tid == 0) atomicOr(a.err, 1 << DEV_ERR_WAIT_TIMEOUT);
                    failed = true;
                    bar_wait(myBar, phase);   // let the copy in flight land before leaving
                }
                phase ^= 1u;
                if (failed) break;
            }
            const float2 nc = make_float2(-c, -c);
            static_assert(NCH % 2 == 0, "chunks are processed in pairs");
#pragma unroll
            for (int ch = 0; ch < NCH; ch += 2) {
                const int off0 = ch * NT * 4 + tid * 4, off1 = off0 + NT * 4;
                const float4 v0 = SE_ITER_ASYNC ? *reinterpret_cast<const float4 *>(myT + off0)
                                                : __ldg(reinterpret_cast<const float4 *>(trow + off0));
                const float4 v1 = SE_ITER_ASYNC ? *reinterpret_cast<const float4 *>(myT + off1)
                                                : __ldg(reinterpret_cast<const float4 *>(trow + off1));
                float2 &a0 = R2[ch * 2 + 0], &a1 = R2[ch * 2 + 1];
                float2 &b0 = R2[ch * 2 + 2], &b1 = R2[ch * 2 + 3];
                a0 = __ffma2_rn(nc, make_float2(v0.x, v0.y), a0);
                a1 = __ffma2_rn(nc, make_float2(v0.z, v0.w), a1);
                b0 = __ffma2_rn(nc, make_float2(v1.x, v1.y), b0);
                b1 = __ffma2_rn(nc, make_float2(v1.z, v1.w), b1);
                m[0] = max3_abs(m[0], a0.x, b0.x);
                m[1] = max3_abs(m[1], a0.y, b0.y);
                m[2] = max3_abs(m[2], a1.x, b1.x);
                m[3] = max3_abs(m[3], a1.y, b1.y);
            }
        }
        if constexpr (W > 1) __syncthreads(); else __syncwarp();
        if (CERT && tid == 0) a.cert_flag[b] = first_close;
        if (failed) break;
        if constexpr (W > 1) __syncthreads(); else __syncwarp();
    }
}


// Model on the loss pixels (eq. 9) and replacement for the fp32 form, from
// the selection log: one warp per block, each lane owning 8 loss pixels per
// pass, the log walked once with the 8 row gathers of four logged atoms in
// flight; support pixels are copied from the samples; user logs filled.
__global__ void __launch_bounds__(256) model_f32_kernel(const IterArgs a)
{
    const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= a.n) return;
    const BlockDesc bd = a.blocks[b];
    const int I = bd.iterations;
    const int *lu = a.log_u + static_cast<size_t>(b) * a.I_max;
    const float *lc = a.log_c + static_cast<size_t>(b) * a.I_max;
    const float *PhiB = static_cast<const float *>(a.PhiB);

    // support pixels keep their samples; the loads of a round of 8 pixels per
    // lane are all issued before the first store
    for (int p0 = 0; p0 < a.MN; p0 += 256) {
        bool on[8];
        double v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int p = p0 + q * 32 + lane;
            on[q] = p < a.MN && a.pat_support[p];
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) v[q] = on[q] ? bd.samples[p0 + q * 32 + lane] : 0.0;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (on[q]) bd.out[p0 + q * 32 + lane] = v[q];
    }

    // g on B (eq. 9): lane j0 + 32 q of a chunk of 256 loss pixels sums c_nu
    // phi_u_nu over the log; 32 log entries per coalesced load, broadcast by
    // shuffles, 8 atoms' rows in flight
    for (int c0 = 0; c0 < a.nB; c0 += 256) {   // every lane runs every chunk (shuffles)
        const int j0 = c0 + lane;
        float acc[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        for (int nu0 = 0; nu0 < I; nu0 += 32) {
            const bool live = nu0 + lane < I;
            const int my_u = live ? lu[nu0 + lane] : 0;
            const float my_c = live ? lc[nu0 + lane] : 0.0f;   // padded entries add 0 * phi_0
            const int cnt = min(32, I - nu0);
            for (int t0 = 0; t0 < cnt; t0 += 8) {
                float cn[8], ph[8][8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int u = __shfl_sync(0xffffffffu, my_u, t0 + t);
                    cn[t] = __shfl_sync(0xffffffffu, my_c, t0 + t);
                    const float *r = PhiB + static_cast<size_t>(u) * a.nB + j0;
#pragma unroll
                    for (int q = 0; q < 8; ++q) ph[t][q] = j0 + q * 32 < a.nB ? __ldg(r + q * 32) : 0.0f;
                }
#pragma unroll
                for (int t = 0; t < 8; ++t)
#pragma unroll
                    for (int q = 0; q < 8; ++q) acc[q] = fmaf(cn[t], ph[t][q], acc[q]);
            }
        }
#pragma unroll
        for (int q = 0; q < 8; ++q)
            if (j0 + q * 32 < a.nB) bd.out[a.b_idx[j0 + q * 32]] = static_cast<double>(acc[q]);
    }
    if (bd.sel_idx)
        for (int nu = lane; nu < I; nu += 32) bd.sel_idx[nu] = lu[nu];
    if (bd.sel_coef)
        for (int nu = lane; nu < I; nu += 32) bd.sel_coef[nu] = static_cast<double>(lc[nu]);
}

template <int W, int VPT, int BPC, bool CERT = false>
cudaError_t launch_f32(const IterArgs &a, cudaStream_t st, int *launches)
{
    constexpr int threads = 32 * W * BPC;
    if (a.Kp != 32 * W * VPT) return cudaErrorInvalidValue;
    if (!a.log_u || !a.log_c) return cudaErrorInvalidValue;   // the model kernel reads the log
    const size_t smem = 16 * BPC + (SE_ITER_ASYNC ? sizeof(float) * BPC * a.Kp : 0) + sizeof(Cand<float>) * 2 * W + 16;
    auto kern = iterate_f32_kernel<W, VPT, BPC, CERT>;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(kern), threads, smem, (a.n + BPC - 1) / BPC, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, st>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <typename T, int W, int VPT, int BPC>
cudaError_t launch_cfg(const IterArgs &a, cudaStream_t st, int *launches)
{
    constexpr int threads = 32 * W * BPC;
    if (a.Kp != 32 * W * VPT) return cudaErrorInvalidValue;
    const size_t smem = sizeof(T) * 2 * a.Kp + sizeof(Cand<T>) * 2 * W +
                        (sizeof(T) + sizeof(int)) * BPC * a.I_max + 16;
    auto kern = iterate_full_kernel<T, W, VPT, BPC>;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(kern), threads, smem, (a.n + BPC - 1) / BPC, &grid);
    if (e != cudaSuccess) return e;
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

cudaError_t launch_model_f32(const IterArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    model_f32_kernel<<<(a.n + 7) / 8, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <>
cudaError_t launch_iterate_full<float>(const IterArgs &a, cudaStream_t st, int *launches, int variant)
{
    if (a.cert_flag) {   // certified form: one warp per block, K <= 2048
        switch (a.Kp) {
        case 512: return launch_f32<1, 16, 4, true>(a, st, launches);
        case 1024: return launch_f32<1, 32, 4, true>(a, st, launches);
        case 2048: return launch_f32<1, 64, 4, true>(a, st, launches);
        default: return cudaErrorInvalidValue;
        }
    }
    // variant 1: twice the warps per block with half the projections per
    // lane (same selections and updates, another occupancy / latency balance)
    switch (a.Kp) {
    case 512: return launch_f32<1, 16, 4>(a, st, launches);
    case 1024: return launch_f32<1, 32, 4>(a, st, launches);
    case 2048: return variant == 1 ? launch_f32<2, 32, 1>(a, st, launches) : launch_f32<1, 64, 4>(a, st, launches);
    case 4096: return variant == 1 ? launch_f32<4, 32, 1>(a, st, launches) : launch_f32<2, 64, 1>(a, st, launches);
    case 8192: return variant == 1 ? launch_f32<8, 32, 1>(a, st, launches) : launch_f32<4, 64, 1>(a, st, launches);
    case 16384: return launch_f32<8, 64, 1>(a, st, launches);
    default: return cudaErrorInvalidValue;
    }
}

int iterate_variants(int Kp, bool fp64)
{
    return !fp64 && (Kp == 2048 || Kp == 4096 || Kp == 8192) ? 2 : 1;
}

int iterate_cert_max_kp()
{
    return 2048;
}

template <>
cudaError_t launch_iterate_full<double>(const IterArgs &a, cudaStream_t st, int *launches, int)
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
