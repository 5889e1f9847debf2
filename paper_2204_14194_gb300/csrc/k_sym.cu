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
// index, original order kept inside a class); R^(0) and the compact table come
// in this order from the folded transforms below.  Lane l of the warp that
// owns a block holds, for each class c, the atoms c K/4 + ch 128 + 4 l + e.
//
// The file holds four forms of the iterations with identical results (the
// tuner picks one per batch size): the projections in registers
// (iterate_sym_kernel: the row by a bounded TMA copy into shared memory), in
// shared memory (iterate_sym_smem_kernel: 27 blocks per SM, the row loaded
// straight into registers), in tensor memory (iterate_sym_tmem_kernel), and the
// last-updated class in registers with the other three in shared memory
// (iterate_sym_hot_kernel);
// the folded transforms of the table (sym_rows_kernel: diagonal, D_k and the
// compact rows) and of eq. (12) (sym_r0_kernel, sym_r0_32_kernel on the CUDA
// cores, sym_r0_32tc_kernel on the tensor cores).  All forms share the
// arithmetic of iterate_f32_kernel: D-scaled projections, packed FMAs,
// three-input maxima, one redux for the maximum and one for the smallest index.
#include <cuda_runtime.h>

#include <climits>

#include "k_device.cuh"
#include "k_model.cuh"
#include "se_internal.h"

namespace se {
namespace {

using dev::bar_wait;
using dev::mma3;
using dev::split_tf32;
using dev::bulk_row;
using dev::max3_abs;

constexpr int kBPC = 4;   // blocks (warps) per CTA

// Selection key of eq. (18): the atom index above the sign bit of its R'
// (the winner's |R'| is the warp maximum M, so index and sign give R'_u), and
// the warp minimum of the keys is the smallest index attaining M.
__device__ __forceinline__ unsigned sel_key(int k, float r)
{
    return (static_cast<unsigned>(k) << 1) | (__float_as_uint(r) >> 31);
}

// The selection log, lane nu mod 32 holding entry nu: written 32 entries at a
// time (and at the last iteration) in original atom indices.
__device__ __forceinline__ void log_entry(const IterArgs &a, int b, int nu, bool more, int lane, int u, float c,
                                          int &lu, float &lc)
{
    if (lane == (nu & 31)) {
        lu = u;
        lc = c;
    }
    if ((nu & 31) == 31 || !more) {
        const size_t o = static_cast<size_t>(b) * a.I_max + (nu & ~31) + lane;
        if (lane <= (nu & 31)) {
            a.log_u[o] = __ldg(a.perm + lu);
            a.log_c[o] = lc;
        }
    }
}

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
                    v[e] = R0[j + e] * __ldg(a.Dkp + j + e);
                    m[c] = fmaxf(m[c], fabsf(v[e]));
                }
                R2[c][2 * ch] = make_float2(v[0], v[1]);
                R2[c][2 * ch + 1] = make_float2(v[2], v[3]);
            }
        }

        int lu = 0;
        float lc = 0.0f;
        for (int nu = 0; nu < I; ++nu) {
            // eq. (18): the maximum over the class maxima, then the smallest index
            const float mx = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
            const float M = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
            unsigned key = 0xffffffffu;
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
                                key = sel_key(c * Q + ch * 128 + 4 * lane + e, r);
                                goto found;
                            }
                        }
                    }
                }
            found:;
            }
            const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
            int u = static_cast<int>(kmin >> 1);
            float ru = (kmin & 1u) ? -M : M;   // the winner's R' is +-M: its sign rides in the key
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
            log_entry(a, b, nu, more, lane, u, c, lu, lc);
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

// The same iterations with the block's projections in shared memory instead of
// registers: a warp still owns one block, lane l keeps its float4 chunks at
// [c][ch][l] (a warp's accesses are 512 contiguous bytes), and the selected
// class's compact row is read straight into registers (four 16-byte loads per
// lane, no copy engine and no barrier).  With 8 KiB per block at K = 2048 and
// few registers, 27 blocks fit on an SM instead of 16, which is what an
// iteration chain bound by the row's L2 latency needs.  Every arithmetic step
// (R0 scaling, packed FMAs, three-input maxima, selection order) is the one of
// iterate_sym_kernel, so both give the same bits.
template <int VPT, int BPC, int MINB>
__global__ void __launch_bounds__(32 * BPC, MINB) iterate_sym_smem_kernel(const IterArgs a)
{
    constexpr int NCH = VPT / 4;
    constexpr int NCC = NCH / 4;
    constexpr int Q = 32 * 4 * NCC;
    static_assert(NCC >= 1 && NCH % 4 == 0, "whole chunks per class");
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *myR = reinterpret_cast<float4 *>(smem) + static_cast<size_t>(g) * (4 * NCC * 32) + lane;
    const float gamma = static_cast<float>(a.gamma);
    // the model kernel (a programmatic dependent) may be scheduled now; it waits for
    // this grid to complete before it reads the log
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    for (int b = blockIdx.x * BPC + g; b < a.n; b += gridDim.x * BPC) {
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const float *R0 = static_cast<const float *>(a.R0) + static_cast<size_t>(b) * a.Kp;
        float m[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float mm = 0.0f;
#pragma unroll 1
            for (int ch = 0; ch < NCC; ++ch) {
                const int j = c * Q + ch * 128 + 4 * lane;
                const float4 rj = *reinterpret_cast<const float4 *>(R0 + j);
                const float4 dj = __ldg(reinterpret_cast<const float4 *>(a.Dkp + j));
                const float v[4] = {rj.x * dj.x, rj.y * dj.y, rj.z * dj.z, rj.w * dj.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) mm = fmaxf(mm, fabsf(v[e]));
                myR[(c * NCC + ch) * 32] = make_float4(v[0], v[1], v[2], v[3]);
            }
            m[c] = mm;
        }

        int lu = 0;
        float lc = 0.0f;
        for (int nu = 0; nu < I; ++nu) {
            const float mx = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
            const float M = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
            unsigned key = 0xffffffffu;
            if (mx == M) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (m[c] != M) continue;
#pragma unroll
                    for (int ch = 0; ch < NCC; ++ch) {
                        const float4 q = myR[(c * NCC + ch) * 32];
                        const float r4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            if (fabsf(r4[e]) == M) {
                                key = sel_key(c * Q + ch * 128 + 4 * lane + e, r4[e]);
                                goto found;
                            }
                        }
                    }
                }
            found:;
            }
            const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
            int u = static_cast<int>(kmin >> 1);
            float ru = (kmin & 1u) ? -M : M;
            if (u < 0 || u >= a.K) {
                if (lane == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
                ru = 0.0f;
            }
            const int cu = u / Q;
            const bool more = nu + 1 < I;
            float4 t[NCC];
            if (more) {
                const float4 *row = reinterpret_cast<const float4 *>(a.Cc + static_cast<size_t>(u) * Q) + lane;
#pragma unroll
                for (int ch = 0; ch < NCC; ++ch) t[ch] = __ldg(row + ch * 32);
            }
            const float c = gamma * ru * __ldg(a.Dkp + u);
            log_entry(a, b, nu, more, lane, u, c, lu, lc);
            if (!more) break;
            const float2 nc = make_float2(-c, -c);
            float mc[2] = {0.0f, 0.0f};
            float4 *Rc = myR + cu * NCC * 32;
#pragma unroll
            for (int ch = 0; ch < NCC; ++ch) {
                const float4 x = Rc[ch * 32];
                const float2 x0 = __ffma2_rn(nc, make_float2(t[ch].x, t[ch].y), make_float2(x.x, x.y));
                const float2 x1 = __ffma2_rn(nc, make_float2(t[ch].z, t[ch].w), make_float2(x.z, x.w));
                Rc[ch * 32] = make_float4(x0.x, x0.y, x1.x, x1.y);
                mc[0] = max3_abs(mc[0], x0.x, x0.y);
                mc[1] = max3_abs(mc[1], x1.x, x1.y);
            }
            const float mn = fmaxf(mc[0], mc[1]);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) m[cc] = cc == cu ? mn : m[cc];
        }
    }
}

// The same iterations with the class that was updated last ("hot") kept in
// registers and the other three classes in three shared-memory slots per block
// (6 KiB at K = 2048).  When the next selection falls in the hot class (about
// 30 % of the iterations) the update touches no shared memory; otherwise
// the selected class is read from its slot, the hot class is written into that
// slot chunk by chunk, and the selected class becomes the hot one.  A packed
// map (2 bits per class, the hot class in bits 8-9) tells which slot holds
// which class; it is always a permutation of the three cold classes.  One
// block per warp, the grid covering the batch.  Arithmetic and selection
// order are those of the other forms (same bits).
//
// With MT > 0 the kernel also evaluates the model of eq. (9) on the loss box
// once a block's iterations are done (dev::model_tc_block, the body of the
// tensor-core model kernel, so the same bits): the block's class slots are
// free by then and hold the warp's log table and output tile.
template <int VPT, int BPC, int MINB, int MT = 0, int NT = 0>
__global__ void __launch_bounds__(32 * BPC, MINB) iterate_sym_hot_kernel(const IterArgs a, const FusedModel fm)
{
    constexpr int NCH = VPT / 4;
    constexpr int NCC = NCH / 4;
    constexpr int Q = 32 * 4 * NCC;
    static_assert(NCC >= 1 && NCH % 4 == 0, "whole chunks per class");
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *myR = reinterpret_cast<float4 *>(smem) + static_cast<size_t>(g) * (3 * NCC * 32) + lane;
    const float gamma = static_cast<float>(a.gamma);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    {
        const int b = blockIdx.x * BPC + g;
        if (b >= a.n) return;
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const float *R0 = static_cast<const float *>(a.R0) + static_cast<size_t>(b) * a.Kp;
        float4 H[NCC];
        float m[4];
        {
            float mm = 0.0f;
#pragma unroll
            for (int ch = 0; ch < NCC; ++ch) {
                const int j = ch * 128 + 4 * lane;
                const float4 rj = *reinterpret_cast<const float4 *>(R0 + j);
                const float4 dj = __ldg(reinterpret_cast<const float4 *>(a.Dkp + j));
                const float v[4] = {rj.x * dj.x, rj.y * dj.y, rj.z * dj.z, rj.w * dj.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) mm = fmaxf(mm, fabsf(v[e]));
                H[ch] = make_float4(v[0], v[1], v[2], v[3]);
            }
            m[0] = mm;
        }
#pragma unroll
        for (int c = 1; c < 4; ++c) {
            float mm = 0.0f;
#pragma unroll 1
            for (int ch = 0; ch < NCC; ++ch) {
                const int j = c * Q + ch * 128 + 4 * lane;
                const float4 rj = *reinterpret_cast<const float4 *>(R0 + j);
                const float4 dj = __ldg(reinterpret_cast<const float4 *>(a.Dkp + j));
                const float v[4] = {rj.x * dj.x, rj.y * dj.y, rj.z * dj.z, rj.w * dj.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) mm = fmaxf(mm, fabsf(v[e]));
                myR[((c - 1) * NCC + ch) * 32] = make_float4(v[0], v[1], v[2], v[3]);
            }
            m[c] = mm;
        }
        // slot of class c at bits 2c; the class held in H at bits 8-9
        unsigned smap = (0u << 2) | (1u << 4) | (2u << 6);

        int lu = 0;
        float lc = 0.0f;
        for (int nu = 0; nu < I; ++nu) {
            const float mx = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
            const float M = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
            unsigned key = 0xffffffffu;
            if (mx == M) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    if (m[c] != M) continue;
                    if (c == static_cast<int>(smap >> 8)) {
#pragma unroll
                        for (int ch = 0; ch < NCC; ++ch) {
                            const float r4[4] = {H[ch].x, H[ch].y, H[ch].z, H[ch].w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (fabsf(r4[e]) == M) {
                                    key = sel_key(c * Q + ch * 128 + 4 * lane + e, r4[e]);
                                    goto found;
                                }
                        }
                    } else {
                        const float4 *Rs = myR + ((smap >> (2 * c)) & 3u) * (NCC * 32);
#pragma unroll
                        for (int ch = 0; ch < NCC; ++ch) {
                            const float4 q = Rs[ch * 32];
                            const float r4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (fabsf(r4[e]) == M) {
                                    key = sel_key(c * Q + ch * 128 + 4 * lane + e, r4[e]);
                                    goto found;
                                }
                        }
                    }
                }
            found:;
            }
            const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
            int u = static_cast<int>(kmin >> 1);
            float ru = (kmin & 1u) ? -M : M;
            if (u < 0 || u >= a.K) {
                if (lane == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
                ru = 0.0f;
            }
            const int cu = u / Q;
            const bool more = nu + 1 < I;
            float4 t[NCC];
            if (more) {
                const float4 *row = reinterpret_cast<const float4 *>(a.Cc + static_cast<size_t>(u) * Q) + lane;
#pragma unroll
                for (int ch = 0; ch < NCC; ++ch) t[ch] = __ldg(row + ch * 32);
            }
            const float c = gamma * ru * __ldg(a.Dkp + u);
            log_entry(a, b, nu, more, lane, u, c, lu, lc);
            if (!more) break;
            const float2 nc = make_float2(-c, -c);
            float mc[2] = {0.0f, 0.0f};
            const unsigned hc = smap >> 8;
            if (static_cast<unsigned>(cu) == hc) {
#pragma unroll
                for (int ch = 0; ch < NCC; ++ch) {
                    const float2 x0 = __ffma2_rn(nc, make_float2(t[ch].x, t[ch].y), make_float2(H[ch].x, H[ch].y));
                    const float2 x1 = __ffma2_rn(nc, make_float2(t[ch].z, t[ch].w), make_float2(H[ch].z, H[ch].w));
                    H[ch] = make_float4(x0.x, x0.y, x1.x, x1.y);
                    mc[0] = max3_abs(mc[0], x0.x, x0.y);
                    mc[1] = max3_abs(mc[1], x1.x, x1.y);
                }
            } else {
                const unsigned s = (smap >> (2 * cu)) & 3u;
                float4 *Rs = myR + s * (NCC * 32);
#pragma unroll
                for (int ch = 0; ch < NCC; ++ch) {
                    const float4 x = Rs[ch * 32];
                    Rs[ch * 32] = H[ch];
                    const float2 x0 = __ffma2_rn(nc, make_float2(t[ch].x, t[ch].y), make_float2(x.x, x.y));
                    const float2 x1 = __ffma2_rn(nc, make_float2(t[ch].z, t[ch].w), make_float2(x.z, x.w));
                    H[ch] = make_float4(x0.x, x0.y, x1.x, x1.y);
                    mc[0] = max3_abs(mc[0], x0.x, x0.y);
                    mc[1] = max3_abs(mc[1], x1.x, x1.y);
                }
                smap = ((smap & 0xffu & ~(3u << (2 * hc))) | (s << (2 * hc))) | (static_cast<unsigned>(cu) << 8);
            }
            const float mn = fmaxf(mc[0], mc[1]);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) m[cc] = cc == cu ? mn : m[cc];
        }
        if constexpr (MT > 0) {
            static_assert(4 * 32 + dev::model_tile_floats(MT, NT) <= 3 * NCC * 32 * 4, "table and tile fit the slots");
            __syncwarp();   // the log is stored and the slots are no longer read
            float *base = reinterpret_cast<float *>(myR - lane);
            if (fm.compact) {
                // square area, box rows and columns from m0 = n0: the rows t_p[m0 .. m0 + RA)
                // of every transform serve both factors; staged in the warp's slots
                constexpr int RA = 16 * MT;
                const int M = fm.s.M, cs = M * M + fm.s.N * fm.s.N, rows = fm.s.ntr * M;
                for (int tp = lane / RA; tp < rows; tp += 32 / RA) {
                    const int t = tp >= M ? 1 : 0, p = tp - t * M;
                    base[tp * RA + lane % RA] = __ldg(fm.tab + t * cs + p * M + fm.m0 + lane % RA);
                }
                __syncwarp();
                const dev::ModelLayout L{-fm.m0, M * RA, RA, -fm.n0, M * RA, RA};
                int4 *Etab = reinterpret_cast<int4 *>(base + rows * RA);
                dev::model_tc_block<MT, NT>(a, fm.s, base, L, Etab, reinterpret_cast<float *>(Etab + 32), b, fm.m0,
                                            fm.Mb, fm.n0, fm.Nb, lane);
            } else {
                int4 *Etab = reinterpret_cast<int4 *>(base);
                dev::model_tc_block<MT, NT>(a, fm.s, fm.tab, dev::model_full_layout(fm.s.M, fm.s.N), Etab,
                                            reinterpret_cast<float *>(Etab + 32), b, fm.m0, fm.Mb, fm.n0, fm.Nb, lane);
            }
        }
    }
}


// The same iterations with the block's projections in tensor memory: a CTA of
// four warps allocates 64 TMEM columns, warp w keeps its block's R' in TMEM
// lanes 32 w .. 32 w + 31 (lane l, column c 16 + ch 4 + e: the atom
// c K/4 + ch 128 + 4 l + e, the layout of the other two forms).  An iteration
// finds the class of the winner (the smallest class holding the maximum),
// loads that class's 16 columns with tcgen05.ld, scans it, updates it with the
// row and stores it back with tcgen05.st: the class traffic leaves the
// shared-memory/L1 pipe, which then carries only the row.  The arithmetic and
// the selection order are those of the other forms (same bits).  At most
// eight CTAs (512 columns) fit on an SM: the launch bounds and a shared-memory
// reservation guarantee it, so tcgen05.alloc never waits.
constexpr int kTmemCols = 64;
constexpr int kTmemGuard = 26 * 1024;   // dynamic shared memory that keeps an SM at <= 8 CTAs

__device__ __forceinline__ void tm_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tm_st16(uint32_t taddr, const float (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                 ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                   "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                   "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                   "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                   "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                   "r"(__float_as_uint(v[15]))
                 : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(128, 8) iterate_sym_tmem_kernel(const IterArgs a)
{
    constexpr int NCC = 4;       // float4 chunks per lane and class (K = 2048)
    constexpr int Q = 512;       // atoms per class
    __shared__ uint32_t tmem_base;
    const int g = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (g == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(&tmem_base))), "r"(kTmemCols) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tw = tmem_base + (static_cast<uint32_t>(g * 32) << 16);   // this warp's lane quarter
    const float gamma = static_cast<float>(a.gamma);
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    for (int b = blockIdx.x * 4 + g; b < a.n; b += gridDim.x * 4) {
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const float *R0 = static_cast<const float *>(a.R0) + static_cast<size_t>(b) * a.Kp;
        float m[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float v[16];
            float mm = 0.0f;
#pragma unroll
            for (int ch = 0; ch < NCC; ++ch) {
                const int j = c * Q + ch * 128 + 4 * lane;
                const float4 rj = *reinterpret_cast<const float4 *>(R0 + j);
                const float4 dj = __ldg(reinterpret_cast<const float4 *>(a.Dkp + j));
                v[4 * ch] = rj.x * dj.x;
                v[4 * ch + 1] = rj.y * dj.y;
                v[4 * ch + 2] = rj.z * dj.z;
                v[4 * ch + 3] = rj.w * dj.w;
#pragma unroll
                for (int e = 0; e < 4; ++e) mm = fmaxf(mm, fabsf(v[4 * ch + e]));
            }
            m[c] = mm;
            tm_st16(tw + c * 16, v);
        }

        int lu = 0;
        float lc = 0.0f;
        for (int nu = 0; nu < I; ++nu) {
            const float mx = fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3]));
            const float M = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(mx)));
            // the class of the winner: the smallest class holding M (indices grow with the class)
            int cl = 4;
            if (mx == M) cl = m[0] == M ? 0 : m[1] == M ? 1 : m[2] == M ? 2 : 3;
            const int cw = static_cast<int>(__reduce_min_sync(0xffffffffu, static_cast<unsigned>(cl)));
            float v[16];
            tm_ld16(tw + (cw & 3) * 16, v);
            unsigned key = 0xffffffffu;
            if (cl == cw) {
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (fabsf(v[j]) == M) {
                        key = sel_key(cw * Q + (j >> 2) * 128 + 4 * lane + (j & 3), v[j]);
                        break;
                    }
            }
            const unsigned kmin = __reduce_min_sync(0xffffffffu, key);
            int u = static_cast<int>(kmin >> 1);
            float ru = (kmin & 1u) ? -M : M;
            if (u < 0 || u >= a.K) {
                if (lane == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
                ru = 0.0f;
            }
            const int cu = u / Q;   // == cw for a valid selection
            const bool more = nu + 1 < I;
            float4 t[NCC];
            if (more) {
                const float4 *row = reinterpret_cast<const float4 *>(a.Cc + static_cast<size_t>(u) * Q) + lane;
#pragma unroll
                for (int ch = 0; ch < NCC; ++ch) t[ch] = __ldg(row + ch * 32);
            }
            const float c = gamma * ru * __ldg(a.Dkp + u);
            log_entry(a, b, nu, more, lane, u, c, lu, lc);
            if (!more) break;
            if (cu != cw) tm_ld16(tw + cu * 16, v);   // only after a recorded bad index
            const float2 nc = make_float2(-c, -c);
            float mc[2] = {0.0f, 0.0f};
#pragma unroll
            for (int ch = 0; ch < NCC; ++ch) {
                const float2 x0 = __ffma2_rn(nc, make_float2(t[ch].x, t[ch].y), make_float2(v[4 * ch], v[4 * ch + 1]));
                const float2 x1 =
                    __ffma2_rn(nc, make_float2(t[ch].z, t[ch].w), make_float2(v[4 * ch + 2], v[4 * ch + 3]));
                v[4 * ch] = x0.x;
                v[4 * ch + 1] = x0.y;
                v[4 * ch + 2] = x1.x;
                v[4 * ch + 3] = x1.y;
                mc[0] = max3_abs(mc[0], x0.x, x0.y);
                mc[1] = max3_abs(mc[1], x1.x, x1.y);
            }
            tm_st16(tw + cu * 16, v);
            const float mn = fmaxf(mc[0], mc[1]);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) m[cc] = cc == cu ? mn : m[cc];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (g == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------- folded transforms
// With w symmetric and t_p[M-1-m] = (-1)^p t_p[m] (DCT-II and sequency-ordered
// Walsh rows), the separable transform of Sec. VI splits into four
// quarter-size ones: for p = 2i + a and q = 2j + b,
//   Y[p][q] = sum_{m < M/2, n < N/2} t_p[m] X_ab[m][n] t'_q[n],
//   X_ab[m][n] = x[m][n] + (-1)^a x[M-1-m][n] + (-1)^b x[m][N-1-n]
//                + (-1)^(a+b) x[M-1-m][N-1-n].
// For R^(0) (x = w s) all four classes are formed, half the multiply-adds of
// the full transform.  For a table row (x = w phi_u) only the class (a, b) of
// atom u is non-zero and X_ab = 4 x on the quadrant, so a compact row costs an
// eighth of a full one.  Outputs are written in the class order of the
// iteration kernel: class c = 2a + b, then transform t, then (i, j).
//
// One warp per item; per transform t the constants A_t[m][a][i] = t_{2i+a}[m]
// (m, i < M/2) and B_t[n][b][j] = t'_{2j+b}[n] (n, j < N/2) sit in shared
// memory, then the unmasked weights rho[MN].  Lane l handles column
// l mod QN and rows h RI .. h RI + RI - 1 (h = l / QN) of each quarter product.
template <int QM, int QN>
struct Fold {
    static constexpr int QMN = QM * QN;
    static constexpr int G = 32 / QN;     // row groups
    static constexpr int RI = QM / G;     // rows per lane
    static constexpr int RO = QMN / 32;   // quadrant points per lane
    static_assert(QN <= 32 && 32 % QN == 0 && QM % G == 0 && QMN % 32 == 0 && RI % 2 == 0, "fold shape");
    static constexpr int cst = 2 * QM * QM + 2 * QN * QN;   // floats per transform
};

template <int Nv>
__device__ __forceinline__ void lds_v(const float *p, float (&v)[Nv])
{
    if constexpr (Nv % 4 == 0) {
#pragma unroll
        for (int j = 0; j < Nv; j += 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p + j);
            v[j] = t.x; v[j + 1] = t.y; v[j + 2] = t.z; v[j + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < Nv; j += 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p + j);
            v[j] = t.x; v[j + 1] = t.y;
        }
    }
}

template <int Nv>
__device__ __forceinline__ void sts_v(float *p, const float (&v)[Nv])
{
    if constexpr (Nv % 4 == 0) {
#pragma unroll
        for (int j = 0; j < Nv; j += 4) *reinterpret_cast<float4 *>(p + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < Nv; j += 2) *reinterpret_cast<float2 *>(p + j) = make_float2(v[j], v[j + 1]);
    }
}

// The quarter product Y = A_a X B_b^T of one class and transform for this
// lane: acc[r] = Y[h RI + r][lane mod QN].  UT is the warp's [QN][QM] buffer.
template <int QM, int QN>
__device__ __forceinline__ void fold_product(const float *Ct, int a, int b, const float *X, float *UT, int lane,
                                             float (&acc)[Fold<QM, QN>::RI])
{
    using F = Fold<QM, QN>;
    constexpr int RI = F::RI;
    const int col = lane % QN, h = lane / QN;
    const float *A = Ct + a * QM + h * RI;                  // A[m][a][h RI ..] at m 2QM
    const float *B = Ct + 2 * QM * QM + b * QN + col;       // B[n][b][col] at n 2QN
    float u[RI];
#pragma unroll
    for (int r = 0; r < RI; ++r) u[r] = 0.0f;
#pragma unroll 4
    for (int m = 0; m < QM; ++m) {
        float av[RI];
        lds_v<RI>(A + m * 2 * QM, av);
        const float xv = X[m * QN + col];
#pragma unroll
        for (int r = 0; r < RI; r += 2) {
            const float2 o = __ffma2_rn(make_float2(av[r], av[r + 1]), make_float2(xv, xv), make_float2(u[r], u[r + 1]));
            u[r] = o.x;
            u[r + 1] = o.y;
        }
    }
    __syncwarp();   // the previous product's reads of UT are done
    sts_v<RI>(UT + col * QM + h * RI, u);
    __syncwarp();
#pragma unroll
    for (int r = 0; r < RI; ++r) acc[r] = 0.0f;
#pragma unroll 4
    for (int n = 0; n < QN; ++n) {
        float uv[RI];
        lds_v<RI>(UT + n * QM + h * RI, uv);
        const float bv = B[n * 2 * QN];
#pragma unroll
        for (int r = 0; r < RI; r += 2) {
            const float2 o = __ffma2_rn(make_float2(uv[r], uv[r + 1]), make_float2(bv, bv), make_float2(acc[r], acc[r + 1]));
            acc[r] = o.x;
            acc[r + 1] = o.y;
        }
    }
}

__device__ __forceinline__ void stage_consts(const float *src, float *dst, int nfloats)
{
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    for (int e = threadIdx.x; e < nfloats / 4; e += blockDim.x) d4[e] = __ldg(s4 + e);
}

// The table of Alg. 2 for a parity-class plan in one launch.  Every CTA first
// forms the diagonal of eq. (16) for all atoms as a folded separable sum of
// non-negative terms, C_kk = 4 sum_{m < M/2, n < N/2} w t_p[m]^2 t'_q[n]^2
// (no cancellation, so fp32 keeps its relative accuracy down to the
// admissibility threshold), the largest C_kk of the non-duplicate atoms, and
// D_k of eq. (17) (NaN for inadmissible atoms); CTA 0 also stores D_k and
// 1/C_kk.  Then the compact rows: item u (class order) is atom perm[u];
// Cc[u][j] = C(perm[c Q + j], perm[u]) D_{perm[c Q + j]}, Dkp[u] = D_{perm[u]}.
template <int QM, int QN>
__global__ void __launch_bounds__(512) sym_rows_kernel(const SymSepArgs a)
{
    using F = Fold<QM, QN>;
    constexpr int QMN = F::QMN, RI = F::RI, RO = F::RO;
    constexpr int M = 2 * QM, N = 2 * QN, MN = M * N;
    extern __shared__ __align__(16) float fsm[];
    __shared__ float red[32];
    const int ncst = a.ntr * F::cst;
    float *cst = fsm;                          // constants, then rho
    const float *rho = cst + ncst;
    float *wq = cst + ncst + MN;               // [QM][QN] w on the first quadrant
    float *Dsh = wq + QMN;                     // [K] C_kk, then D_k
    float *V = Dsh + a.K;                      // [ntr][M][QN] stage 1 of the diagonal
    float *X = V + a.ntr * M * QN + (threadIdx.x >> 5) * 2 * QMN;
    float *UT = X + QMN;
    stage_consts(a.img, cst, ncst + MN);
    __syncthreads();
    for (int o = threadIdx.x; o < QMN; o += blockDim.x) {
        const int m = o / QN, n = o % QN;
        wq[o] = a.pattern[m * N + n] ? rho[m * N + n] : 0.0f;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
    const int Q = a.K / 4;

    for (int e = threadIdx.x; e < a.ntr * M * QN; e += blockDim.x) {
        const int t = e / (M * QN), p = (e / QN) % M, n = e % QN;
        const float *At = cst + t * F::cst + (p & 1) * QM + (p >> 1);
        float v = 0.0f;
#pragma unroll 4
        for (int m = 0; m < QM; ++m) {
            const float tp = At[m * 2 * QM];
            v = fmaf(tp * tp, wq[m * QN + n], v);
        }
        V[e] = v;
    }
    __syncthreads();
    float lmax = 0.0f;
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const int t = k / MN, p = (k % MN) / N, q = k % N;
        const float *Bt = cst + t * F::cst + 2 * QM * QM + (q & 1) * QN + (q >> 1);
        const float *Vp = V + (t * M + p) * QN;
        float d = 0.0f;
#pragma unroll 4
        for (int n = 0; n < QN; ++n) {
            const float tq = Bt[n * 2 * QN];
            d = fmaf(Vp[n], tq * tq, d);
        }
        d *= 4.0f;
        Dsh[k] = d;
        if (!a.dup[k]) lmax = fmaxf(lmax, d);
    }
    for (int o = 16; o > 0; o >>= 1) lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    if (lane == 0) red[threadIdx.x >> 5] = lmax;
    __syncthreads();
    float dmax = 0.0f;
    for (int w = 0; w < wpc; ++w) dmax = fmaxf(dmax, red[w]);
    for (int k = threadIdx.x; k < a.K; k += blockDim.x) {
        const float d = Dsh[k];
        const bool adm = !a.dup[k] && dmax > 0.0f && d > 1e-14f * dmax;
        const float D = adm ? 1.0f / sqrtf(d) : NAN;
        Dsh[k] = D;
        if (blockIdx.x == 0) {
            a.Dk[k] = D;
            a.invC[k] = adm ? 1.0f / d : 0.0f;
        }
    }
    __syncthreads();

    for (int u = blockIdx.x * wpc + (threadIdx.x >> 5); u < a.K; u += gridDim.x * wpc) {
        const int k = __ldg(a.perm + u);
        const int t = k >= MN ? 1 : 0;
        const int kk = k - t * MN, pu = kk / N, qu = kk % N;
        const int ca = pu & 1, cb = qu & 1;
        const float *Ct = cst + t * F::cst;
        __syncwarp();   // the previous item's reads of X are done
#pragma unroll
        for (int r = 0; r < RO; ++r) {
            const int o = lane + 32 * r, m = o / QN, n = o % QN;
            const float ex = Ct[m * 2 * QM + ca * QM + (pu >> 1)] * Ct[2 * QM * QM + n * 2 * QN + cb * QN + (qu >> 1)];
            X[o] = wq[o] * ex;
        }
        __syncwarp();
        float *row = a.Cc + static_cast<size_t>(u) * Q;
        for (int to = 0; to < a.ntr; ++to) {
            float acc[RI];
            fold_product<QM, QN>(cst + to * F::cst, ca, cb, X, UT, lane, acc);
            // entry (i, jj) is atom (to, 2 i + ca, 2 jj + cb) of the class order
            const int i0 = (lane / QN) * RI, jj = lane % QN;
            const int base = to * QMN + i0 * QN + jj;
            const float *Dr = Dsh + to * MN + (2 * i0 + ca) * N + 2 * jj + cb;
#pragma unroll
            for (int r = 0; r < RI; ++r) row[base + r * QN] = 4.0f * acc[r] * Dr[2 * r * N];
        }
        if (lane == 0) a.Dkp[u] = Dsh[k];
    }
}

// R^(0) of eq. (12) for pattern blocks, all four classes, unscaled, in class
// order (R0[b][c Q + t QM QN + i QN + j]); also copies the support samples to
// the block's output.
template <int QM, int QN>
__global__ void __launch_bounds__(256) sym_r0_kernel(const SymSepArgs a)
{
    using F = Fold<QM, QN>;
    constexpr int QMN = F::QMN, RI = F::RI, RO = F::RO;
    constexpr int M = 2 * QM, N = 2 * QN, MN = M * N;
    extern __shared__ __align__(16) float fsm[];
    const int ncst = a.ntr * F::cst;
    float *cst = fsm;
    const float *rho = cst + ncst;
    float *X = cst + ncst + MN + (threadIdx.x >> 5) * 5 * QMN;   // X_00, X_01, X_10, X_11
    float *UT = X + 4 * QMN;
    stage_consts(a.img, cst, ncst + MN);
    __syncthreads();
    const int lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
    const int Q = a.K / 4;
    for (int b = blockIdx.x * wpc + (threadIdx.x >> 5); b < a.n; b += gridDim.x * wpc) {
        const BlockDesc bd = a.blocks[b];
        const uint8_t *mask = bd.support ? bd.support : a.pattern;
        const double *smp = bd.samples;
        // in place (out is samples): the support samples are already there
        double *dst = a.copy_support && bd.out != bd.samples ? bd.out : nullptr;
        __syncwarp();   // the previous block's reads of X are done
#pragma unroll 2
        for (int r = 0; r < RO; ++r) {
            const int o = lane + 32 * r, m = o / QN, n = o % QN;
            const int p[4] = {m * N + n, (M - 1 - m) * N + n, m * N + N - 1 - n, (M - 1 - m) * N + N - 1 - n};
            float x[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const bool on = mask[p[e]] != 0;
                const double sv = on ? smp[p[e]] : 0.0;
                x[e] = on ? rho[p[e]] * dev::f64_to_f32_rn(sv) : 0.0f;
                if (dst && on) dst[p[e]] = sv;
            }
            const float s0 = x[0] + x[1], d0 = x[0] - x[1];   // fold in m
            const float s1 = x[2] + x[3], d1 = x[2] - x[3];
            X[o] = s0 + s1;                                     // (a, b) = (0, 0)
            X[QMN + o] = s0 - s1;                               // (0, 1)
            X[2 * QMN + o] = d0 + d1;                           // (1, 0)
            X[3 * QMN + o] = d0 - d1;                           // (1, 1)
        }
        __syncwarp();
        float *R = a.R0 + static_cast<size_t>(b) * a.K;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            for (int t = 0; t < a.ntr; ++t) {
                float acc[RI];
                fold_product<QM, QN>(cst + t * F::cst, c >> 1, c & 1, X + c * QMN, UT, lane, acc);
                const int base = c * Q + t * QMN + (lane / QN) * RI * QN + lane % QN;
#pragma unroll
                for (int r = 0; r < RI; ++r) R[base + r * QN] = acc[r];
            }
        }
    }
}

// The same R^(0) pass for 32 x 32 areas with the lane as the column: lane n
// reads rows r and 31 - r of column n for all r < 16 at once (no load waits
// on another), folds in m in its registers and in n with the lane 31 - n
// (shuffle); lanes < 16 write X_00 and X_10, lanes >= 16 X_01 and X_11.  The
// quarter products run two at a time, one per half-warp (column parity b =
// half), in 4 x 4 register tiles: two 16-byte shared loads per 16
// multiply-adds.  Every output is the same chain of fused multiply-adds
// (same operands, same order) as in sym_r0_kernel<16, 16>, so both give the
// same bits.
constexpr int kR0Plane = 272;   // X_ab plane pitch: 256 + 16 (lanes >= 16 store to the other 16 banks)
constexpr int kR0UT = 20;       // pitch of a row n of the transposed stage-1 result
__global__ void __launch_bounds__(288, 3) sym_r0_32_kernel(const SymSepArgs a)
{
    constexpr int M = 32, N = 32, MN = 1024, QMN = 256, CST = 1024;   // floats of one transform's constants
    extern __shared__ __align__(16) float fsm[];
    const int ncst = a.ntr * CST;
    float *cst = fsm;
    const float *rho = cst + ncst;
    float *X = cst + ncst + MN + (threadIdx.x >> 5) * (4 * kR0Plane + 2 * 16 * kR0UT);
    float *UT = X + 4 * kR0Plane;   // per half-warp [n][kR0UT]: the transposed stage-1 result
    stage_consts(a.img, cst, ncst + MN);
    __syncthreads();
    const int lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
    const int hw = lane >> 4, iq = (lane >> 2) & 3, jq = lane & 3;
    const int Q = a.K / 4;
    for (int b = blockIdx.x * wpc + (threadIdx.x >> 5); b < a.n; b += gridDim.x * wpc) {
        const BlockDesc bd = a.blocks[b];
        const uint8_t *mask = (bd.support ? bd.support : a.pattern) + lane;
        const double *smp = bd.samples + lane;
        double *dst = a.copy_support && bd.out != bd.samples ? bd.out + lane : nullptr;   // none in place
        __syncwarp();   // the previous block's reads of X and UT are done
#pragma unroll 1
        for (int r0 = 0; r0 < M / 2; r0 += 8) {
            double s0[8], s1[8];
            bool o0[8], o1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {   // the loss samples are not read
                const int r = r0 + k;
                o0[k] = mask[r * N] != 0;
                o1[k] = mask[(M - 1 - r) * N] != 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = r0 + k;
                s0[k] = o0[k] ? smp[r * N] : 0.0;
                s1[k] = o1[k] ? smp[(M - 1 - r) * N] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = r0 + k;
                const float x0 = o0[k] ? rho[r * N + lane] * dev::f64_to_f32_rn(s0[k]) : 0.0f;
                const float x1 = o1[k] ? rho[(M - 1 - r) * N + lane] * dev::f64_to_f32_rn(s1[k]) : 0.0f;
                if (dst) {
                    if (o0[k]) dst[r * N] = s0[k];
                    if (o1[k]) dst[(M - 1 - r) * N] = s1[k];
                }
                const float sm = x0 + x1, dm = x0 - x1;
                const float smo = __shfl_xor_sync(0xffffffffu, sm, 31), dmo = __shfl_xor_sync(0xffffffffu, dm, 31);
                if (lane < 16) {
                    X[r * 16 + lane] = sm + smo;                          // (0, 0)
                    X[2 * kR0Plane + r * 16 + lane] = dm + dmo;           // (1, 0)
                } else {
                    X[kR0Plane + r * 16 + 31 - lane] = smo - sm;          // (0, 1)
                    X[3 * kR0Plane + r * 16 + 31 - lane] = dmo - dm;      // (1, 1)
                }
            }
        }
        __syncwarp();
        float *R = a.R0 + static_cast<size_t>(b) * a.K;
        // pass (ca, t): half-warp hw takes column parity cb = hw; lane hl = 4 iq + jq
        // holds the 4 x 4 tile rows 4 iq .., columns 4 jq ..
        float *UTh = UT + hw * 16 * kR0UT;
#pragma unroll 1
        for (int ca = 0; ca < 2; ++ca) {
#pragma unroll 1
            for (int t = 0; t < a.ntr; ++t) {
                const float *A = cst + t * CST + ca * 16 + 4 * iq;                 // A[m][ca][4 iq ..] at m 32
                const float *Bt = cst + t * CST + 2 * 16 * 16 + hw * 16 + 4 * jq;  // B[n][cb][4 jq ..] at n 32
                const float *Xp = X + (2 * ca + hw) * kR0Plane + 4 * jq;
                float u[4][4];
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int k = 0; k < 4; ++k) u[ii][k] = 0.0f;
#pragma unroll 4
                for (int m = 0; m < 16; ++m) {
                    const float4 av = *reinterpret_cast<const float4 *>(A + m * 32);
                    const float4 xv = *reinterpret_cast<const float4 *>(Xp + m * 16);
                    const float ai[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        float2 o = __ffma2_rn(make_float2(ai[ii], ai[ii]), make_float2(xv.x, xv.y),
                                              make_float2(u[ii][0], u[ii][1]));
                        u[ii][0] = o.x;
                        u[ii][1] = o.y;
                        o = __ffma2_rn(make_float2(ai[ii], ai[ii]), make_float2(xv.z, xv.w),
                                       make_float2(u[ii][2], u[ii][3]));
                        u[ii][2] = o.x;
                        u[ii][3] = o.y;
                    }
                }
                __syncwarp();   // the previous pass is done reading UT
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    *reinterpret_cast<float4 *>(UTh + (4 * jq + k) * kR0UT + 4 * iq) =
                        make_float4(u[0][k], u[1][k], u[2][k], u[3][k]);
                __syncwarp();
                float y[4][4];
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int k = 0; k < 4; ++k) y[ii][k] = 0.0f;
#pragma unroll 4
                for (int n = 0; n < 16; ++n) {
                    const float4 uv = *reinterpret_cast<const float4 *>(UTh + n * kR0UT + 4 * iq);
                    const float4 bv = *reinterpret_cast<const float4 *>(Bt + n * 32);
                    const float ui[4] = {uv.x, uv.y, uv.z, uv.w};
#pragma unroll
                    for (int ii = 0; ii < 4; ++ii) {
                        float2 o = __ffma2_rn(make_float2(ui[ii], ui[ii]), make_float2(bv.x, bv.y),
                                              make_float2(y[ii][0], y[ii][1]));
                        y[ii][0] = o.x;
                        y[ii][1] = o.y;
                        o = __ffma2_rn(make_float2(ui[ii], ui[ii]), make_float2(bv.z, bv.w),
                                       make_float2(y[ii][2], y[ii][3]));
                        y[ii][2] = o.x;
                        y[ii][3] = o.y;
                    }
                }
                float *Rc = R + (2 * ca + hw) * Q + t * QMN + 4 * jq;
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
                    *reinterpret_cast<float4 *>(Rc + (4 * iq + ii) * 16) = make_float4(y[ii][0], y[ii][1], y[ii][2], y[ii][3]);
            }
        }
    }
}

// R^(0) of 32 x 32 parity-class blocks on the tensor cores: the sixteen
// quarter products of a block (Y = A^T X_ab B per class and transform) as
// mma.sync m16n8k8 products in split TF32: each fp32 operand x is
// x_b = tf32(x) plus x_s = tf32(x - x_b), and a product accumulates
// x_s y_b + x_b y_s + x_b y_b in fp32 (the dropped x_s y_s and the two
// roundings leave about 2^-21 relative), accurate like the fp32 transforms.
// The fold is the one of sym_r0_kernel (lane = column, shuffle across the
// centre); the constant operands come as per-lane fragments from the plan's
// table (conflict-free 16- and 8-byte loads).  Fragments of m16n8k8: g = lane / 4,
// q = lane mod 4; A(16 x 8) {(g, q), (g + 8, q), (g, q + 4), (g + 8, q + 4)},
// B(8 x 8) {(q, g), (q + 4, g)}, C(16 x 8) {(g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1)}.
constexpr int kTcPlane = 272;   // X_ab plane pitch (rows of 16; lanes >= 16 store to the other banks)
constexpr int kTcU = 20;        // pitch of the stage-1 result rows

__global__ void __launch_bounds__(288, 3) sym_r0_32tc_kernel(const SymSepArgs a)
{
    constexpr int M = 32, N = 32, MN = 1024, QMN = 256;
    extern __shared__ __align__(16) float fsm[];
    const int ntr = a.ntr;
    // constants, split into TF32 parts by the plan: AF[t][ca][ks][lane] (uint4 large,
    // uint4 small), BF[t][cb][ks][nt][lane] (b0, b1 large, b0, b1 small), rho[MN]
    const int nconst = ntr * 2048 + MN;
    float *cst = fsm;
    const uint4 *AF = reinterpret_cast<const uint4 *>(cst);
    const uint4 *BF = reinterpret_cast<const uint4 *>(cst + ntr * 1024);
    const float *rho = cst + ntr * 2048;
    float *X = cst + nconst + (threadIdx.x >> 5) * (4 * kTcPlane + 16 * kTcU);
    float *U = X + 4 * kTcPlane;
    for (int e = threadIdx.x; e < nconst / 4; e += blockDim.x)
        reinterpret_cast<float4 *>(cst)[e] = __ldg(reinterpret_cast<const float4 *>(a.img) + e);
    __syncthreads();
    const int lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
    const int g = lane >> 2, q = lane & 3;
    const int Q = a.K / 4;
    for (int b = blockIdx.x * wpc + (threadIdx.x >> 5); b < a.n; b += gridDim.x * wpc) {
        const BlockDesc bd = a.blocks[b];
        const uint8_t *mask = (bd.support ? bd.support : a.pattern) + lane;
        const double *smp = bd.samples + lane;
        double *dst = a.copy_support && bd.out != bd.samples ? bd.out + lane : nullptr;   // none in place
        __syncwarp();   // the previous block's reads of X and U are done
#pragma unroll 1
        for (int r0 = 0; r0 < M / 2; r0 += 8) {
            double s0[8], s1[8];
            bool o0[8], o1[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {   // the loss samples are not read
                const int r = r0 + k;
                o0[k] = mask[r * N] != 0;
                o1[k] = mask[(M - 1 - r) * N] != 0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = r0 + k;
                s0[k] = o0[k] ? smp[r * N] : 0.0;
                s1[k] = o1[k] ? smp[(M - 1 - r) * N] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int r = r0 + k;
                const float x0 = o0[k] ? rho[r * N + lane] * dev::f64_to_f32_rn(s0[k]) : 0.0f;
                const float x1 = o1[k] ? rho[(M - 1 - r) * N + lane] * dev::f64_to_f32_rn(s1[k]) : 0.0f;
                if (dst) {
                    if (o0[k]) dst[r * N] = s0[k];
                    if (o1[k]) dst[(M - 1 - r) * N] = s1[k];
                }
                const float sm = x0 + x1, dm = x0 - x1;
                const float smo = __shfl_xor_sync(0xffffffffu, sm, 31), dmo = __shfl_xor_sync(0xffffffffu, dm, 31);
                if (lane < 16) {
                    X[r * 16 + lane] = sm + smo;                          // (0, 0)
                    X[2 * kTcPlane + r * 16 + lane] = dm + dmo;           // (1, 0)
                } else {
                    X[kTcPlane + r * 16 + 31 - lane] = smo - sm;          // (0, 1)
                    X[3 * kTcPlane + r * 16 + 31 - lane] = dmo - dm;      // (1, 1)
                }
            }
        }
        __syncwarp();
        float *R = a.R0 + static_cast<size_t>(b) * a.K;
#pragma unroll 1
        for (int t = 0; t < ntr; ++t) {
#pragma unroll 1
            for (int ca = 0; ca < 2; ++ca) {
                // A^T fragments of this (t, ca) for both k-steps, split
                uint32_t Ab[2][4], As[2][4];
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    const uint4 fb = AF[(((t * 2 + ca) * 2 + ks) * 2 + 0) * 32 + lane];
                    const uint4 fs = AF[(((t * 2 + ca) * 2 + ks) * 2 + 1) * 32 + lane];
                    Ab[ks][0] = fb.x; Ab[ks][1] = fb.y; Ab[ks][2] = fb.z; Ab[ks][3] = fb.w;
                    As[ks][0] = fs.x; As[ks][1] = fs.y; As[ks][2] = fs.z; As[ks][3] = fs.w;
                }
#pragma unroll 1
                for (int cb = 0; cb < 2; ++cb) {
                    const float *Xp = X + (2 * ca + cb) * kTcPlane;
                    // stage 1: U = A^T X_ab (16 x 16), two column tiles of 8
                    float d[2][4];
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        d[nt][0] = d[nt][1] = d[nt][2] = d[nt][3] = 0.0f;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
                            uint32_t bb0, bs0, bb1, bs1;
                            split_tf32(Xp[(8 * ks + q) * 16 + 8 * nt + g], bb0, bs0);
                            split_tf32(Xp[(8 * ks + q + 4) * 16 + 8 * nt + g], bb1, bs1);
                            mma3(d[nt], Ab[ks], As[ks], bb0, bb1, bs0, bs1);
                        }
                    }
                    __syncwarp();   // the previous product is done reading U
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        *reinterpret_cast<float2 *>(U + g * kTcU + 8 * nt + 2 * q) = make_float2(d[nt][0], d[nt][1]);
                        *reinterpret_cast<float2 *>(U + (g + 8) * kTcU + 8 * nt + 2 * q) = make_float2(d[nt][2], d[nt][3]);
                    }
                    __syncwarp();
                    // stage 2: Y = U B (16 x 16)
                    uint32_t Ub[2][4], Us[2][4];
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
                        split_tf32(U[g * kTcU + 8 * ks + q], Ub[ks][0], Us[ks][0]);
                        split_tf32(U[(g + 8) * kTcU + 8 * ks + q], Ub[ks][1], Us[ks][1]);
                        split_tf32(U[g * kTcU + 8 * ks + q + 4], Ub[ks][2], Us[ks][2]);
                        split_tf32(U[(g + 8) * kTcU + 8 * ks + q + 4], Ub[ks][3], Us[ks][3]);
                    }
                    float *Rc = R + (2 * ca + cb) * Q + t * QMN;
#pragma unroll
                    for (int nt = 0; nt < 2; ++nt) {
                        float y[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks) {
                            const uint4 f = BF[(((t * 2 + cb) * 2 + ks) * 2 + nt) * 32 + lane];
                            mma3(y, Ub[ks], Us[ks], f.x, f.y, f.z, f.w);
                        }
                        *reinterpret_cast<float2 *>(Rc + g * 16 + 8 * nt + 2 * q) = make_float2(y[0], y[1]);
                        *reinterpret_cast<float2 *>(Rc + (g + 8) * 16 + 8 * nt + 2 * q) = make_float2(y[2], y[3]);
                    }
                }
            }
        }
    }
}

}  // namespace

template <int QM, int QN>
static cudaError_t launch_fold(const SymSepArgs &a, bool rows, cudaStream_t st)
{
    using F = Fold<QM, QN>;
    const int wpc = rows ? 16 : 8;
    const size_t smem = sizeof(float) * (static_cast<size_t>(a.ntr) * F::cst + 4 * QM * QN +
                                         (rows ? F::QMN + static_cast<size_t>(a.K) + a.ntr * 2 * QM * QN : 0) +
                                         static_cast<size_t>(wpc) * (rows ? 2 : 5) * F::QMN);
    const int items = rows ? a.K : a.n;
    if (items <= 0) return cudaSuccess;
    auto kern = rows ? sym_rows_kernel<QM, QN> : sym_r0_kernel<QM, QN>;
    const int need = (items + wpc - 1) / wpc;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(kern), 32 * wpc, smem, need, &grid);
    if (e != cudaSuccess) return e;
    if (rows) {   // the table kernel repeats the diagonal in every CTA: at most one CTA per SM
        const int sms = sm_count();
        grid = need < sms ? need : sms;
    }
    kern<<<grid, 32 * wpc, smem, st>>>(a);
    return cudaGetLastError();
}

bool sym_fold_supported(int M, int N)
{
    return (M == 16 || M == 32) && (N == 16 || N == 32);
}

static cudaError_t launch_fold_any(const SymSepArgs &a, bool rows, cudaStream_t st)
{
    if (a.K != a.ntr * a.M * a.N || a.K % 4 || !a.img || !a.perm) return cudaErrorInvalidValue;
    if (a.M == 32 && a.N == 32) return launch_fold<16, 16>(a, rows, st);
    if (a.M == 16 && a.N == 16) return launch_fold<8, 8>(a, rows, st);
    if (a.M == 32 && a.N == 16) return launch_fold<16, 8>(a, rows, st);
    if (a.M == 16 && a.N == 32) return launch_fold<8, 16>(a, rows, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_sym_rows(const SymSepArgs &a, cudaStream_t st)
{
    if (!a.Dk || !a.invC || !a.dup || !a.Cc || !a.Dkp) return cudaErrorInvalidValue;
    return launch_fold_any(a, true, st);
}

int sym_r0_variants(int M, int N) { return M == 32 && N == 32 ? 2 : 1; }

cudaError_t launch_sym_r0_tc(const SymSepArgs &a, cudaStream_t st)
{
    if (!a.blocks || !a.R0 || !a.tc_img || a.M != 32 || a.N != 32 || a.K != a.ntr * 1024) return cudaErrorInvalidValue;
    if (a.n <= 0) return cudaSuccess;
    constexpr int wpc = 9;   // 3 CTAs of 9 warps per SM: 4104 blocks in one wave
    const size_t smem = sizeof(float) * (static_cast<size_t>(a.ntr) * 2048 + 1024 +
                                         wpc * static_cast<size_t>(4 * kTcPlane + 16 * kTcU));
    SymSepArgs b = a;
    b.img = a.tc_img;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(sym_r0_32tc_kernel), 32 * wpc, smem,
                                (a.n + wpc - 1) / wpc, &grid);
    if (e != cudaSuccess) return e;
    sym_r0_32tc_kernel<<<grid, 32 * wpc, smem, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_sym_r0(const SymSepArgs &a, cudaStream_t st, int variant)
{
    if (!a.blocks || !a.R0) return cudaErrorInvalidValue;
    if (variant == 1 && a.M == 32 && a.N == 32) {
        if (a.K != a.ntr * 1024 || !a.img) return cudaErrorInvalidValue;
        if (a.n <= 0) return cudaSuccess;
        constexpr int wpc = 9;   // 3 CTAs of 9 warps per SM: 4104 blocks in one wave
        const size_t smem = sizeof(float) * (static_cast<size_t>(a.ntr) * 1024 + 1024 +
                                             wpc * static_cast<size_t>(4 * kR0Plane + 2 * 16 * kR0UT));
        int grid = 0;
        cudaError_t e = launch_grid(reinterpret_cast<const void *>(sym_r0_32_kernel), 32 * wpc, smem,
                                    (a.n + wpc - 1) / wpc, &grid);
        if (e != cudaSuccess) return e;
        sym_r0_32_kernel<<<grid, 32 * wpc, smem, st>>>(a);
        return cudaGetLastError();
    }
    return launch_fold_any(a, false, st);
}

template <int VPT>
static cudaError_t launch_sym_vpt(const IterArgs &a, cudaStream_t st, int *launches)
{
    constexpr int Q = 32 * VPT / 4;
    if (a.K != 4 * Q || a.Kp != a.K || !a.log_u || !a.log_c || !a.perm || !a.Cc || !a.Dkp)
        return cudaErrorInvalidValue;
    const size_t smem = 16 * kBPC + sizeof(float) * kBPC * Q + 16;
    auto kern = iterate_sym_kernel<VPT>;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(kern), 32 * kBPC, smem, (a.n + kBPC - 1) / kBPC, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, 32 * kBPC, smem, st>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

template <int VPT, int BPC, int MINB>
static cudaError_t launch_sym_smem(const IterArgs &a, cudaStream_t st, int *launches)
{
    constexpr int Q = 32 * VPT / 4;
    if (a.K != 4 * Q || a.Kp != a.K || !a.log_u || !a.log_c || !a.perm || !a.Cc || !a.Dkp)
        return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * static_cast<size_t>(BPC) * a.Kp;
    auto kern = iterate_sym_smem_kernel<VPT, BPC, MINB>;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(kern), 32 * BPC, smem, (a.n + BPC - 1) / BPC, &grid,
                                true);
    if (e != cudaSuccess) return e;
    kern<<<grid, 32 * BPC, smem, st>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

int iterate_sym_variants(int Kp) { return Kp == 2048 ? 4 : 2; }

template <int MT, int NT>
static cudaError_t launch_sym_hot(const IterArgs &a, const FusedModel &fm, cudaStream_t st, int *launches)
{
    constexpr int BPC = 3, Q = 512;
    if (a.K != 4 * Q || a.Kp != a.K || !a.log_u || !a.log_c || !a.perm || !a.Cc || !a.Dkp)
        return cudaErrorInvalidValue;
    if (MT > 0 && (!fm.tab || fm.Mb <= 0 || fm.Nb <= 0 || fm.Mb > 16 * MT || fm.Nb > 8 * NT || fm.m0 < 0 ||
                   fm.n0 < 0 || fm.m0 + fm.Mb > fm.s.M || fm.n0 + fm.Nb > fm.s.N || !a.pat_support))
        return cudaErrorInvalidValue;
    const size_t smem = sizeof(float) * static_cast<size_t>(BPC) * 3 * Q;   // three class slots per block
    const int grid = (a.n + BPC - 1) / BPC;                                   // one block per warp
    auto kern = iterate_sym_hot_kernel<64, BPC, 9, MT, NT>;
    // the carveout of the other parity-class forms: batches that run side by side on
    // several streams (the chunks of a host-buffer call) can then share the SMs
    cudaError_t e = prefer_max_shared(reinterpret_cast<const void *>(kern));
    if (e != cudaSuccess) return e;
    kern<<<grid, 32 * BPC, smem, st>>>(a, fm);
    if (launches) ++*launches;
    return cudaGetLastError();
}

bool sym_model_box(int Mb, int Nb) { return Mb > 0 && Nb > 0 && ((Mb <= 16 && Nb <= 16) || (Mb <= 32 && Nb <= 8)); }

cudaError_t launch_iterate_sym_model(const IterArgs &a, const FusedModel &fm, cudaStream_t st, int *launches)
{
    if (a.n <= 0) return cudaSuccess;
    if (!sym_model_box(fm.Mb, fm.Nb)) return cudaErrorInvalidValue;
    // the tile shapes of the tensor-core model kernel for the same box (at most two
    // tiles: the model's accumulators then fit the iteration kernel's registers)
    if (fm.Mb > 16) return launch_sym_hot<2, 1>(a, fm, st, launches);
    return fm.Nb <= 8 ? launch_sym_hot<1, 1>(a, fm, st, launches) : launch_sym_hot<1, 2>(a, fm, st, launches);
}

static cudaError_t launch_sym_tmem(const IterArgs &a, cudaStream_t st, int *launches)
{
    if (a.K != 2048 || a.Kp != 2048 || !a.log_u || !a.log_c || !a.perm || !a.Cc || !a.Dkp)
        return cudaErrorInvalidValue;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(iterate_sym_tmem_kernel), 128, kTmemGuard,
                                (a.n + 3) / 4, &grid, true);
    if (e != cudaSuccess) return e;
    // the registers (64 x 128 per CTA) and the shared-memory guard bound the
    // residency at 8 CTAs per SM, which is also the TMEM limit (8 x 64 columns)
    const int want = (a.n + 3) / 4, cap = 8 * sm_count();
    grid = want < cap ? want : cap;
    iterate_sym_tmem_kernel<<<grid, 128, kTmemGuard, st>>>(a);
    if (launches) ++*launches;
    return cudaGetLastError();
}

cudaError_t launch_iterate_sym(const IterArgs &a, cudaStream_t st, int *launches, int variant)
{
    if (a.n <= 0) return cudaSuccess;
    if (variant == 2 && a.Kp == 2048) return launch_sym_tmem(a, st, launches);   // projections in tensor memory
    if (variant == 3 && a.Kp == 2048) return launch_sym_hot<0, 0>(a, FusedModel{}, st, launches);   // hot class in registers
    if (variant == 1) {   // projections in shared memory
        switch (a.Kp) {
        case 512: return launch_sym_smem<16, 4, 12>(a, st, launches);
        case 1024: return launch_sym_smem<32, 4, 10>(a, st, launches);
        case 2048: return launch_sym_smem<64, 3, 9>(a, st, launches);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (a.Kp) {
    case 512: return launch_sym_vpt<16>(a, st, launches);
    case 1024: return launch_sym_vpt<32>(a, st, launches);
    case 2048: return launch_sym_vpt<64>(a, st, launches);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace se
