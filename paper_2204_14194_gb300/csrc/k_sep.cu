// k_sep.cu -- transform-domain scalar products for DCT / WHT dictionaries
// (Sec. VI, eqs. 21-23): for atoms that are products of 1-D basis rows,
// phi_(p,q)[m,n] = t_p[m] t'_q[n], every weighted scalar product with a
// weighted M x N signal x is an entry of the separable transform
//     Y = T_M x T_N^T,   Y[p][q] = sum_m sum_n t_p[m] x[m][n] t'_q[n],
// so all K products of one signal cost 2 M N (M + N) flops instead of
// 2 K M N.  Used by the per-block-mask path for
//   mode 0  R^(0)_b       x = rho m_b s_b                 (eq. 12)
//   mode 1  C_b(k, k)     x = rho m_b with squared rows    (eq. 16 diagonal:
//                          sum w phi_k^2 = sum w t_p^2 t'_q^2)
//   mode 2  C_b(:, u)     x = rho m_b phi_u               (eq. 16 column; phi_u
//                          rebuilt from its two 1-D rows)
//   mode 3  C(:, i)       x = rho m phi_i on the shared pattern (table rows of
//                          Alg. 2 one atom per item)
// A dictionary may hold two transforms (the DCT u WHT union); transform t
// writes atoms koff[t] + p N + q.
#include <algorithm>
#include <cstdlib>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "k_device.cuh"
#include "k_model.cuh"
#include "se_internal.h"

namespace se {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) sep_kernel(const SepArgs a)
{
    const int i = blockIdx.x;
    if (a.n_dev && i >= *a.n_dev) return;
    if (i >= a.n) return;
    const int M = a.M, N = a.N, MN = M * N;
    extern __shared__ __align__(16) unsigned char smem[];
    T *X = reinterpret_cast<T *>(smem);          // [M][N]
    T *Z = X + MN;                                // [M][N]
    T *Tm = Z + MN;                               // [M][M]
    T *Tn = Tm + M * M;                           // [N][N]

    const int b = a.item_blk ? a.item_blk[i] : i;
    const uint8_t *mask;
    const double *smp = nullptr;
    double *dst = nullptr;
    const T *rowM = nullptr, *rowN = nullptr;
    if (a.mode == 3) {
        mask = a.pattern;
    } else {
        const BlockDesc bd = a.blocks[b];
        mask = bd.support ? bd.support : a.pattern;
        smp = bd.samples;
        if (a.mode == 0 && a.copy_support && bd.out != bd.samples) dst = bd.out;   // none in place
    }
    if (a.mode >= 2) {
        const int u = a.mode == 3 ? i : a.cur_u[b];
        const int t = (a.ntr > 1 && u >= a.koff[1]) ? 1 : 0;
        const int ku = u - a.koff[t];
        rowM = static_cast<const T *>(a.TM[t]) + static_cast<size_t>(ku / N) * M;
        rowN = static_cast<const T *>(a.TN[t]) + static_cast<size_t>(ku % N) * N;
    }
    for (int p = threadIdx.x; p < MN; p += blockDim.x) {
        const int m = p / N, n = p - m * N;
        T v = mask[p] ? static_cast<T>(a.rho[p]) : T(0);
        if (a.mode == 0) {
            const double sp = mask[p] ? smp[p] : 0.0;
            v = mask[p] ? v * static_cast<T>(sp) : T(0);
            if (dst && mask[p]) dst[p] = sp;
        } else if (a.mode >= 2) {
            v *= rowM[m] * rowN[n];
        }
        X[p] = v;
    }
    T *out = static_cast<T *>(a.out) + (a.out_rows ? a.out_rows[i] : static_cast<long long>(b) * a.ldo);

    for (int t = 0; t < a.ntr; ++t) {
        const T *gm = static_cast<const T *>(a.TM[t]);
        const T *gn = static_cast<const T *>(a.TN[t]);
        __syncthreads();   // X ready / previous transform done with Tm, Tn, Z
        for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
            const T v = gm[e];
            Tm[e] = a.mode == 1 ? v * v : v;
        }
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const T v = gn[e];
            const int q = e / N, n = e - q * N;
            Tn[n * N + q] = a.mode == 1 ? v * v : v;      // stored transposed: Tn[n][q]
        }
        __syncthreads();
        // Z[m][q] = sum_n X[m][n] t'_q[n]; consecutive threads take consecutive q,
        // so X[m][n] is a broadcast and Tn[n][q] a conflict-free row read
        for (int e = threadIdx.x; e < MN; e += blockDim.x) {
            const int m = e / N, q = e - m * N;
            const T *xr = X + m * N;
            T acc = T(0);
            for (int n = 0; n < N; ++n) acc = fma(xr[n], Tn[n * N + q], acc);
            Z[e] = acc;
        }
        __syncthreads();
        // Y[p][q] = sum_m Tm[p][m] Z[m][q]
        for (int e = threadIdx.x; e < MN; e += blockDim.x) {
            const int p = e / N, q = e - p * N;
            const T *tr = Tm + p * M;
            T acc = T(0);
            for (int m = 0; m < M; ++m) acc = fma(tr[m], Z[m * N + q], acc);
            out[a.koff[t] + e] = acc * (sizeof(T) == 4 && a.scale ? static_cast<T>(a.scale[a.koff[t] + e]) : T(1));
        }
    }
    for (int k = a.koff[a.ntr - 1] + MN + threadIdx.x; k < a.kfill; k += blockDim.x)
        out[k] = a.scale ? static_cast<T>(NAN) : T(0);
}

// fp32 form: transform rows resident in shared memory for the CTA's
// lifetime, one item per group of 64 threads (named barriers per group),
// TS x TS register tiles with paired FMAs.  Per item and transform t:
//   U[p][n] = sum_m t_p[m] x[m][n]      (k = m: TmT[m][p..], X[m][n..]),
//             kept transposed, UT[n][p];
//   Y[p][q] = sum_n U[p][n] t'_q[n]     (k = n: UT[n][p..], TnT[n][q..]),
// written to global memory straight from the registers.  x is staged row-major
// (conflict-free, coalesced); the constant rows are staged transposed once.
constexpr int kSepGroup = 64;

template <int TS> struct VecT;
template <> struct VecT<4> {
    using type = float4;
    __device__ static void get(const float *p, float (&v)[4])
    {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    __device__ static void put(float *p, const float (&v)[4])
    {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct VecT<2> {
    using type = float2;
    __device__ static void get(const float *p, float (&v)[2])
    {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        v[0] = t.x; v[1] = t.y;
    }
    __device__ static void put(float *p, const float (&v)[2])
    {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    }
};

// barrier of one group (ids 1-4; 0 is __syncthreads), immediate ids so that
// the kernel holds five hardware barriers rather than all sixteen
__device__ __forceinline__ void group_sync(int id)
{
    switch (id) {
    case 1: asm volatile("bar.sync 1, %0;" ::"n"(kSepGroup) : "memory"); break;
    case 2: asm volatile("bar.sync 2, %0;" ::"n"(kSepGroup) : "memory"); break;
    case 3: asm volatile("bar.sync 3, %0;" ::"n"(kSepGroup) : "memory"); break;
    default: asm volatile("bar.sync 4, %0;" ::"n"(kSepGroup) : "memory"); break;
    }
}

// acc[r][c] += a[r] * b[c] for a TS x TS tile, two columns per paired FMA
template <int TS>
__device__ __forceinline__ void outer_fma(float (&acc)[TS][TS], const float (&av)[TS], const float (&bv)[TS])
{
#pragma unroll
    for (int r = 0; r < TS; ++r)
#pragma unroll
        for (int c = 0; c < TS; c += 2) {
            const float2 o = __ffma2_rn(make_float2(av[r], av[r]), make_float2(bv[c], bv[c + 1]),
                                        make_float2(acc[r][c], acc[r][c + 1]));
            acc[r][c] = o.x;
            acc[r][c + 1] = o.y;
        }
}

// Copy the constants' shared-memory image (TmT, TnT per transform, then
// rho) with coalesced 16-byte loads, eight in flight per thread; mode 1 uses
// the squared transform rows.
__device__ __forceinline__ void stage_image(const SepArgs &a, float *dst, int cst_floats, int total_floats)
{
    const float4 *src = reinterpret_cast<const float4 *>(a.img);
    float4 *d4 = reinterpret_cast<float4 *>(dst);
    const int n4 = (total_floats + 3) / 4;
    for (int e0 = threadIdx.x; e0 < n4; e0 += 8 * blockDim.x) {
        float4 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = e0 + j * blockDim.x;
            if (e < n4) v[j] = __ldg(src + e);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int e = e0 + j * blockDim.x;
            if (e >= n4) continue;
            float4 w = v[j];
            if (a.mode == 1 && 4 * e < cst_floats) {
                w.x *= w.x; w.y *= w.y; w.z *= w.z; w.w *= w.w;
            }
            d4[e] = w;
        }
    }
}

template <int TS, int MC, int NC>
__global__ void __launch_bounds__(256) sep_group_kernel(const SepArgs a, int groups)
{
    // MC, NC: compile-time area size (0 = taken from the arguments)
    const int M = MC ? MC : a.M, N = NC ? NC : a.N, MN = M * N;
    extern __shared__ __align__(16) unsigned char smem[];
    float *cst = reinterpret_cast<float *>(smem);       // per transform: TmT [M][M], TnT [N][N]
    const int cstride = M * M + N * N;
    float *Wr = cst + a.ntr * cstride;                  // [MN] rho (unmasked weights)
    const int g = threadIdx.x / kSepGroup, tg = threadIdx.x % kSepGroup;
    float *X = Wr + MN + static_cast<size_t>(g) * 2 * MN;   // [M][N]
    float *UT = X + MN;                                     // [N][M]

    stage_image(a, cst, a.ntr * cstride, a.ntr * cstride + MN);
    __syncthreads();

    const int n_items = a.n_dev ? min(a.n, *a.n_dev) : a.n;
    constexpr int tilesMC = MC / TS, tilesNC = NC / TS;
    const int tilesM = MC ? tilesMC : M / TS, tilesN = NC ? tilesNC : N / TS;
    for (int i = blockIdx.x * groups + g; i < n_items; i += gridDim.x * groups) {
        const int b = a.item_blk ? a.item_blk[i] : i;
        const uint8_t *mask;
        const double *smp = nullptr;
        double *dst = nullptr;
        const float *rowM = nullptr, *rowN = nullptr;   // the 1-D rows of atom u (global)
        if (a.mode == 3) {
            mask = a.pattern;
        } else {
            const BlockDesc bd = a.blocks[b];
            mask = bd.support ? bd.support : a.pattern;
            smp = bd.samples;
            if (a.mode == 0 && a.copy_support && bd.out != bd.samples) dst = bd.out;   // none in place
        }
        if (a.mode >= 2) {
            const int u = a.mode == 3 ? i : a.cur_u[b];
            const int t = (a.ntr > 1 && u >= a.koff[1]) ? 1 : 0;
            const int ku = u - a.koff[t];
            rowM = static_cast<const float *>(a.TM[t]) + static_cast<size_t>(ku / N) * M;
            rowN = static_cast<const float *>(a.TN[t]) + static_cast<size_t>(ku % N) * N;
        }
        // x on the item's support; 8 pixels per thread per round, every load
        // of a round issued before the first use (samples on B are not read)
        for (int p0 = 0; p0 < MN; p0 += 8 * kSepGroup) {
            bool on[8];
            float ex[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int p = p0 + j * kSepGroup + tg;
                on[j] = p < MN && mask[p] != 0;
                ex[j] = (a.mode >= 2 && p < MN) ? rowM[p / N] * rowN[p % N] : 1.0f;
            }
            double sv[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) sv[j] = (a.mode == 0 && on[j]) ? smp[p0 + j * kSepGroup + tg] : 0.0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int p = p0 + j * kSepGroup + tg;
                if (p >= MN) continue;
                float v = on[j] ? Wr[p] : 0.0f;
                if (a.mode == 0) v = on[j] ? v * dev::f64_to_f32_rn(sv[j]) : 0.0f;
                else if (a.mode >= 2) v *= ex[j];
                X[p] = v;
                if (dst && on[j]) dst[p] = sv[j];
            }
        }
        float *out = static_cast<float *>(a.out) + (a.out_rows ? a.out_rows[i] : static_cast<long long>(b) * a.ldo);
        group_sync(1 + g);

        for (int t = 0; t < a.ntr; ++t) {
            const float *TmT = cst + t * cstride, *TnT = TmT + M * M;
            if (t) group_sync(1 + g);   // the previous transform is done reading UT
            for (int tile = tg; tile < tilesM * tilesN; tile += kSepGroup) {
                const int p0 = TS * (tile / tilesN), n0 = TS * (tile % tilesN);
                float acc[TS][TS] = {};
#pragma unroll 8
                for (int m = 0; m < M; ++m) {
                    float av[TS], bv[TS];
                    VecT<TS>::get(TmT + m * M + p0, av);
                    VecT<TS>::get(X + m * N + n0, bv);
                    outer_fma<TS>(acc, av, bv);
                }
#pragma unroll
                for (int c = 0; c < TS; ++c) {
                    float col[TS];
#pragma unroll
                    for (int r = 0; r < TS; ++r) col[r] = acc[r][c];
                    VecT<TS>::put(UT + (n0 + c) * M + p0, col);
                }
            }
            group_sync(1 + g);
            for (int tile = tg; tile < tilesM * tilesN; tile += kSepGroup) {
                const int p0 = TS * (tile / tilesN), q0 = TS * (tile % tilesN);
                float acc[TS][TS] = {};
#pragma unroll 8
                for (int n = 0; n < N; ++n) {
                    float av[TS], bv[TS];
                    VecT<TS>::get(UT + n * M + p0, av);
                    VecT<TS>::get(TnT + n * N + q0, bv);
                    outer_fma<TS>(acc, av, bv);
                }
#pragma unroll
                for (int r = 0; r < TS; ++r) {
                    const int k0 = a.koff[t] + (p0 + r) * N + q0;
                    if (a.scale) {
                        float sv[TS];
                        VecT<TS>::get(a.scale + k0, sv);
#pragma unroll
                        for (int c = 0; c < TS; ++c) acc[r][c] *= sv[c];
                    }
                    VecT<TS>::put(out + k0, acc[r]);
                }
            }
        }
        for (int k = a.koff[a.ntr - 1] + MN + tg; k < a.kfill; k += kSepGroup)
            out[k] = a.scale ? NAN : 0.0f;
        // the next item's X is written only after every thread of the group has
        // passed the barrier that follows it, i.e. finished this item
    }
}

// The lazy columns of eq. (16) for 32 x 32 and 64 x 64 areas (mode 2: the
// column of atom u for block b, C_b(k, u) = sum_mn rho m_b phi_u phi_k) on the
// tensor cores.  Per item and transform the two M x M x M products U = T_M x
// and Y = U T_N^T run as mma.sync m16n8k16 products of two-part fp16 splits:
// each fp32 operand, scaled by a power of two that puts its largest entry in
// [2^14, 2^15), is v = v_h + v_l with fp16 parts, and v_l w_h + v_h w_l +
// v_h w_h is accumulated in fp32 (about 2^-22 of the largest entry per
// product); the scales are undone exactly on the result.  The 1-D rows take
// one scale per CTA, x one per item, U one per warp.
// One item per group of M / 16 warps; warp w computes rows 16 w .. 16 w + 15
// of U and then the same rows of Y, which need only its own rows of U, so the
// two products of a warp are separated by warp synchronisation alone.  Shared
// memory per CTA: the 1-D rows of every transform, split and packed in pairs
// along the sample index (square areas: the same rows serve both directions),
// rho, and per item the split x and U; rows are padded so that the fragment
// loads of a warp hit 32 different banks.  Global reads are issued in
// batches: the constants as float4 together with the first item's
// descriptor, mask and atom rows, and each next item's before the current
// item's products.
template <int M> struct ColCfg {
    static constexpr int MN = M * M;
    static constexpr int Groups = M == 64 ? 4 : 8;     // items per CTA (512 threads)
    static constexpr int Threads = 2 * M;              // threads per item (M / 16 warps)
    static constexpr int NT = Threads * Groups;
    static constexpr int W = M + 8;                    // words per row of a pair-packed operand with M columns
    static constexpr int V = M / 2 + 4;                // words per row of the pair-packed U (M / 2 pairs)
    static constexpr int Op = (M / 2) * W;             // words of one pair-packed M x M part
    static constexpr int Up = M * V;                   // words of one part of U
    static constexpr int ItemWords = 2 * Op + 2 * Up;
    static constexpr int Red = 64;                     // words of reduction scratch
    static constexpr int Q = M / 4;                    // column quads per row
    static constexpr int Units = M / 16;               // x units (row pair, column quad) per thread
    static constexpr int KS = M / 16;                  // k-steps of 16
    static constexpr int NTile = M / 8;                // n tiles of 8
    static constexpr int CK = (MN / 4 + NT - 1) / NT;  // float4 of the constants per thread and part
    static constexpr int MinBlocks = M == 64 ? 1 : 2;
};

// barrier of one item's warps (ids 1-8; 0 is __syncthreads)
template <int NTH>
__device__ __forceinline__ void col_sync(int id)
{
    switch (id) {
    case 1: asm volatile("bar.sync 1, %0;" ::"n"(NTH) : "memory"); break;
    case 2: asm volatile("bar.sync 2, %0;" ::"n"(NTH) : "memory"); break;
    case 3: asm volatile("bar.sync 3, %0;" ::"n"(NTH) : "memory"); break;
    case 4: asm volatile("bar.sync 4, %0;" ::"n"(NTH) : "memory"); break;
    case 5: asm volatile("bar.sync 5, %0;" ::"n"(NTH) : "memory"); break;
    case 6: asm volatile("bar.sync 6, %0;" ::"n"(NTH) : "memory"); break;
    case 7: asm volatile("bar.sync 7, %0;" ::"n"(NTH) : "memory"); break;
    default: asm volatile("bar.sync 8, %0;" ::"n"(NTH) : "memory"); break;
    }
}

template <int M> struct ColItem {
    uint32_t w[2 * ColCfg<M>::Units];   // mask bytes of rows 2 jp, 2 jp + 1 at columns n0 .. n0 + 3
    float2 rm[ColCfg<M>::Units];        // t_p[2 jp], t_p[2 jp + 1] of the atom's first factor
    float4 rn;                          // t'_q[n0 .. n0 + 3] of its second factor
};

// thread tg of an item takes the units jp = tg / Q + 8 i (row pairs) at the
// column quad tg % Q
template <int M>
__device__ __forceinline__ void col_load_item(const SepArgs &a, int i, int tg, ColItem<M> &it)
{
    using C = ColCfg<M>;
    const int b = a.item_blk ? a.item_blk[i] : i;
    const uint8_t *sup = a.blocks[b].support;
    const uint8_t *mask = sup ? sup : a.pattern;
    const int u = a.cur_u[b];
    const int tu = (a.ntr > 1 && u >= a.koff[1]) ? 1 : 0;
    const int ku = min(max(u - a.koff[tu], 0), C::MN - 1);   // valid atoms only reach here
    const float *rowM = static_cast<const float *>(a.TM[tu]) + (ku / M) * M;
    const float *rowN = static_cast<const float *>(a.TN[tu]) + (ku % M) * M;
    const int cq = tg % C::Q;
    it.rn = __ldg(reinterpret_cast<const float4 *>(rowN) + cq);
#pragma unroll
    for (int i4 = 0; i4 < C::Units; ++i4)
        it.rm[i4] = __ldg(reinterpret_cast<const float2 *>(rowM) + tg / C::Q + 8 * i4);
    if ((reinterpret_cast<uintptr_t>(mask) & 3) == 0) {
        const uint32_t *m4 = reinterpret_cast<const uint32_t *>(mask);
#pragma unroll
        for (int i4 = 0; i4 < C::Units; ++i4) {
            const int jp = tg / C::Q + 8 * i4;
            it.w[2 * i4] = __ldg(m4 + (2 * jp) * C::Q + cq);
            it.w[2 * i4 + 1] = __ldg(m4 + (2 * jp + 1) * C::Q + cq);
        }
    } else {
#pragma unroll
        for (int i4 = 0; i4 < C::Units; ++i4)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const uint8_t *q = mask + (2 * (tg / C::Q + 8 * i4) + h) * M + 4 * cq;
                it.w[2 * i4 + h] = static_cast<uint32_t>(q[0]) | static_cast<uint32_t>(q[1]) << 8 |
                                   static_cast<uint32_t>(q[2]) << 16 | static_cast<uint32_t>(q[3]) << 24;
            }
    }
}

// Exponent e with 2^e mx in [2^14, 2^15) (mx > 0 normal), clamped so that 2^e
// is a normal float; 0 when mx is zero.
__device__ __forceinline__ int col_scale_exp(float mx)
{
    if (!(mx > 0.0f)) return 0;
    const int ex = static_cast<int>((__float_as_uint(mx) >> 23) & 0xffu) - 127;
    return min(max(14 - ex, -126), 127);
}
__device__ __forceinline__ float col_pow2(int e) { return __uint_as_float(static_cast<uint32_t>(e + 127) << 23); }

// fp16 parts of two scaled values, packed as the pair (lo16 = first, hi16 = second)
__device__ __forceinline__ void col_split2(float v0, float v1, uint32_t &hw, uint32_t &lw)
{
    const __half h0 = __float2half_rn(v0), h1 = __float2half_rn(v1);
    const __half l0 = __float2half_rn(v0 - __half2float(h0)), l1 = __float2half_rn(v1 - __half2float(h1));
    hw = static_cast<uint32_t>(__half_as_ushort(h0)) | static_cast<uint32_t>(__half_as_ushort(h1)) << 16;
    lw = static_cast<uint32_t>(__half_as_ushort(l0)) | static_cast<uint32_t>(__half_as_ushort(l1)) << 16;
}

__device__ __forceinline__ void mma_f16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
                 "{%8, %9}, {%0, %1, %2, %3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// acc[nt] += A B over k = M from pair-packed parts, A rows r0 + (gq, gq + 8),
// B columns 8 nt + gq.  A word (r, j) (the pair A(r, 2j), A(r, 2j + 1)) at
// r APITCH + j when A_BY_ROW, else at j APITCH + r; B word (j, c) at j W + c.
template <int M, int APITCH, bool A_BY_ROW>
__device__ __forceinline__ void col_mma_pass(float (&acc)[ColCfg<M>::NTile][4], const uint32_t *Ah,
                                             const uint32_t *Al, const uint32_t *Bh, const uint32_t *Bl, int r0,
                                             int gq, int q)
{
    constexpr int W = ColCfg<M>::W;
#pragma unroll 2
    for (int ks = 0; ks < ColCfg<M>::KS; ++ks) {
        const int j0 = 8 * ks + q, r = r0 + gq;
        const int o0 = A_BY_ROW ? r * APITCH + j0 : j0 * APITCH + r;
        const int o1 = A_BY_ROW ? (r + 8) * APITCH + j0 : j0 * APITCH + r + 8;
        const int o2 = A_BY_ROW ? r * APITCH + j0 + 4 : (j0 + 4) * APITCH + r;
        const int o3 = A_BY_ROW ? (r + 8) * APITCH + j0 + 4 : (j0 + 4) * APITCH + r + 8;
        const uint32_t ah[4] = {Ah[o0], Ah[o1], Ah[o2], Ah[o3]};
        const uint32_t al[4] = {Al[o0], Al[o1], Al[o2], Al[o3]};
#pragma unroll
        for (int nt = 0; nt < ColCfg<M>::NTile; ++nt) {
            const int c = 8 * nt + gq;
            const uint32_t bh0 = Bh[j0 * W + c], bh1 = Bh[(j0 + 4) * W + c];
            const uint32_t bl0 = Bl[j0 * W + c], bl1 = Bl[(j0 + 4) * W + c];
            mma_f16(acc[nt], al, bh0, bh1);
            mma_f16(acc[nt], ah, bl0, bl1);
            mma_f16(acc[nt], ah, bh0, bh1);
        }
    }
}

template <int M>
__global__ void __launch_bounds__(ColCfg<M>::NT, ColCfg<M>::MinBlocks) sep_col_tc_kernel(const SepArgs a)
{
    using C = ColCfg<M>;
    constexpr int N = M, MN = C::MN, NT = C::NT;
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *Tp = reinterpret_cast<uint32_t *>(smem);                  // per transform: hi part, lo part
    float *Wr = reinterpret_cast<float *>(Tp + a.ntr * 2 * C::Op);       // [MN] rho
    float *red = Wr + MN;                                                 // [16] CTA, then [groups][4]
    const int g = threadIdx.x / C::Threads, tg = threadIdx.x % C::Threads;
    uint32_t *XH = reinterpret_cast<uint32_t *>(red + C::Red) + g * C::ItemWords;
    uint32_t *XL = XH + C::Op, *UH = XL + C::Op, *UL = UH + C::Up;
    float *gred = red + 16 + 4 * g;
    const int n_items = a.n_dev ? min(a.n, *a.n_dev) : a.n;
    int i = blockIdx.x * C::Groups + g;
    ColItem<M> it;
    int eT;
    {
        // TmT [M][M] of the image holds t_p[m] at m M + p; unit (t, j, quad of p):
        // rows 2 j and 2 j + 1, packed in pairs along m
        const float4 *img4 = static_cast<const float4 *>(static_cast<const void *>(a.img));
        const int cstride4 = 2 * MN / 4, units = a.ntr * (M / 2) * C::Q;
        float4 v0[C::CK], v1[C::CK], wv[C::CK];
#pragma unroll
        for (int k = 0; k < C::CK; ++k) {
            const int e = threadIdx.x + k * NT;
            if (e < units) {
                const int t = e / (MN / 8), j = (e / C::Q) % (M / 2), c4 = e % C::Q;
                v0[k] = __ldg(img4 + t * cstride4 + (2 * j) * C::Q + c4);
                v1[k] = __ldg(img4 + t * cstride4 + (2 * j + 1) * C::Q + c4);
            }
            if (e < MN / 4) wv[k] = __ldg(img4 + a.ntr * cstride4 + e);
        }
        if (i < n_items) col_load_item<M>(a, i, tg, it);
        float mx = 0.0f;
#pragma unroll
        for (int k = 0; k < C::CK; ++k)
            if (threadIdx.x + k * NT < units)
                mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(fabsf(v0[k].x), fabsf(v0[k].y)), fmaxf(fabsf(v0[k].z), fabsf(v0[k].w))),
                                     fmaxf(fmaxf(fabsf(v1[k].x), fabsf(v1[k].y)), fmaxf(fabsf(v1[k].z), fabsf(v1[k].w)))));
        mx = warp_max(mx);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
#pragma unroll
        for (int k = 0; k < C::CK; ++k)
            if (threadIdx.x + k * NT < MN / 4) reinterpret_cast<float4 *>(Wr)[threadIdx.x + k * NT] = wv[k];
        __syncthreads();
        mx = red[0];
        for (int w = 1; w < NT / 32; ++w) mx = fmaxf(mx, red[w]);
        eT = col_scale_exp(mx);
        const float sT = col_pow2(eT);
#pragma unroll
        for (int k = 0; k < C::CK; ++k) {
            const int e = threadIdx.x + k * NT;
            if (e < units) {
                const int t = e / (MN / 8), j = (e / C::Q) % (M / 2), c4 = e % C::Q;
                uint4 h, l;
                col_split2(v0[k].x * sT, v1[k].x * sT, h.x, l.x);
                col_split2(v0[k].y * sT, v1[k].y * sT, h.y, l.y);
                col_split2(v0[k].z * sT, v1[k].z * sT, h.z, l.z);
                col_split2(v0[k].w * sT, v1[k].w * sT, h.w, l.w);
                uint32_t *dst = Tp + t * 2 * C::Op + j * C::W + 4 * c4;
                *reinterpret_cast<uint4 *>(dst) = h;
                *reinterpret_cast<uint4 *>(dst + C::Op) = l;
            }
        }
    }
    __syncthreads();
    const int wg = tg >> 5, lane = tg & 31, gq = lane >> 2, q = lane & 3;
    const int cq = tg % C::Q, r0 = 16 * wg;
    for (; i < n_items; i += gridDim.x * C::Groups) {
        // x = rho m_b phi_u on the item's support, rows 2 jp, 2 jp + 1 and columns n0 .. n0 + 3
        float xv[C::Units][2][4];
        float mx = 0.0f;
#pragma unroll
        for (int i4 = 0; i4 < C::Units; ++i4) {
            const int jp = tg / C::Q + 8 * i4;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float4 w = reinterpret_cast<const float4 *>(Wr)[(2 * jp + h) * C::Q + cq];
                const float rm = h ? it.rm[i4].y : it.rm[i4].x;
                const uint32_t mw = it.w[2 * i4 + h];
                xv[i4][h][0] = (mw & 0xffu) ? w.x * (rm * it.rn.x) : 0.0f;
                xv[i4][h][1] = (mw & 0xff00u) ? w.y * (rm * it.rn.y) : 0.0f;
                xv[i4][h][2] = (mw & 0xff0000u) ? w.z * (rm * it.rn.z) : 0.0f;
                xv[i4][h][3] = (mw & 0xff000000u) ? w.w * (rm * it.rn.w) : 0.0f;
#pragma unroll
                for (int c = 0; c < 4; ++c) mx = fmaxf(mx, fabsf(xv[i4][h][c]));
            }
        }
        mx = warp_max(mx);
        if (lane == 0) gred[wg] = mx;
        const int b = a.item_blk ? a.item_blk[i] : i;
        float *out = static_cast<float *>(a.out) + (a.out_rows ? a.out_rows[i] : static_cast<long long>(b) * a.ldo);
        col_sync<C::Threads>(1 + g);   // also: every warp is done with the previous item's x
        float gm = gred[0];
#pragma unroll
        for (int w = 1; w < M / 16; ++w) gm = fmaxf(gm, gred[w]);
        const int ex = col_scale_exp(gm);
        {
            const float sx = col_pow2(ex);
#pragma unroll
            for (int i4 = 0; i4 < C::Units; ++i4) {
                const int jp = tg / C::Q + 8 * i4;
                uint4 h, l;
                col_split2(xv[i4][0][0] * sx, xv[i4][1][0] * sx, h.x, l.x);
                col_split2(xv[i4][0][1] * sx, xv[i4][1][1] * sx, h.y, l.y);
                col_split2(xv[i4][0][2] * sx, xv[i4][1][2] * sx, h.z, l.z);
                col_split2(xv[i4][0][3] * sx, xv[i4][1][3] * sx, h.w, l.w);
                *reinterpret_cast<uint4 *>(XH + jp * C::W + 4 * cq) = h;
                *reinterpret_cast<uint4 *>(XL + jp * C::W + 4 * cq) = l;
            }
        }
        if (i + static_cast<int>(gridDim.x) * C::Groups < n_items)
            col_load_item<M>(a, i + gridDim.x * C::Groups, tg, it);   // in flight during the products
        col_sync<C::Threads>(1 + g);   // x complete; gred read by every warp

        for (int t = 0; t < a.ntr; ++t) {
            const uint32_t *TH = Tp + t * 2 * C::Op, *TL = TH + C::Op;
            float acc[C::NTile][4];
#pragma unroll
            for (int nt = 0; nt < C::NTile; ++nt)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[nt][k] = 0.0f;
            // U[p][n] = sum_m t_p[m] x[m][n] for p = r0 + (gq, gq + 8): A(p, m) = t_p[m]
            col_mma_pass<M, C::W, false>(acc, TH, TL, XH, XL, r0, gq, q);
            float mu = 0.0f;
#pragma unroll
            for (int nt = 0; nt < C::NTile; ++nt)
#pragma unroll
                for (int k = 0; k < 4; ++k) mu = fmaxf(mu, fabsf(acc[nt][k]));
            const int eu = col_scale_exp(warp_max(mu));
            {
                const float su = col_pow2(eu);
                const int r = r0 + gq;
                __syncwarp();   // the previous transform's reads of these rows of U are done
#pragma unroll
                for (int nt = 0; nt < C::NTile; ++nt) {
                    uint32_t h, l;
                    col_split2(acc[nt][0] * su, acc[nt][1] * su, h, l);
                    UH[r * C::V + 4 * nt + q] = h;
                    UL[r * C::V + 4 * nt + q] = l;
                    col_split2(acc[nt][2] * su, acc[nt][3] * su, h, l);
                    UH[(r + 8) * C::V + 4 * nt + q] = h;
                    UL[(r + 8) * C::V + 4 * nt + q] = l;
                }
                __syncwarp();
            }
            // Y[p][q'] = sum_n U[p][n] t'_q'[n] (square area: the rows of T_N are those of T_M)
#pragma unroll
            for (int nt = 0; nt < C::NTile; ++nt)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[nt][k] = 0.0f;
            col_mma_pass<M, C::V, true>(acc, UH, UL, TH, TL, r0, gq, q);
            // Y = acc 2^-(2 eT + ex + eu)
            const int etot = 2 * eT + ex + eu;
            const bool onef = etot >= -126 && etot <= 127;
            const float f = onef ? col_pow2(-etot) : 1.0f;
#pragma unroll
            for (int nt = 0; nt < C::NTile; ++nt)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = a.koff[t] + (r0 + gq + 8 * h) * N + 8 * nt + 2 * q;
                    float2 y = onef ? make_float2(acc[nt][2 * h] * f, acc[nt][2 * h + 1] * f)
                                    : make_float2(ldexpf(acc[nt][2 * h], -etot), ldexpf(acc[nt][2 * h + 1], -etot));
                    if (a.scale) {
                        const float2 sv = __ldg(reinterpret_cast<const float2 *>(a.scale + k));
                        y.x *= sv.x;
                        y.y *= sv.y;
                    }
                    *reinterpret_cast<float2 *>(out + k) = y;
                }
        }
        for (int k = a.koff[a.ntr - 1] + MN + tg; k < a.kfill; k += C::Threads)
            out[k] = a.scale ? NAN : 0.0f;
    }
}

// fp32 form, one warp per item: lane tiles of TP x TQ outputs (the 32 lanes
// cover (M / TP) x (N / TQ) tiles exactly), so the phases need only warp
// synchronisation and the 16 warps of an SM work on independent items.
// Same arithmetic order as sep_group_kernel: U = T_M x over m, then
// Y = U T_N^T over n.
template <int Nv>
__device__ __forceinline__ void lds_vec(const float *p, float (&v)[Nv])
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
__device__ __forceinline__ void sts_vec(float *p, const float (&v)[Nv])
{
    if constexpr (Nv % 4 == 0) {
#pragma unroll
        for (int j = 0; j < Nv; j += 4)
            *reinterpret_cast<float4 *>(p + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
    } else {
#pragma unroll
        for (int j = 0; j < Nv; j += 2) *reinterpret_cast<float2 *>(p + j) = make_float2(v[j], v[j + 1]);
    }
}

template <int TP, int TQ>
__device__ __forceinline__ void outer_fma_pq(float (&acc)[TP][TQ], const float (&av)[TP], const float (&bv)[TQ])
{
#pragma unroll
    for (int r = 0; r < TP; ++r)
#pragma unroll
        for (int c = 0; c < TQ; c += 2) {
            const float2 o = __ffma2_rn(make_float2(av[r], av[r]), make_float2(bv[c], bv[c + 1]),
                                        make_float2(acc[r][c], acc[r][c + 1]));
            acc[r][c] = o.x;
            acc[r][c + 1] = o.y;
        }
}

// UT[n][p] position: with SW the 4-float slots of a row are XOR-permuted by
// (n / 4) mod 8, so that the 8 lanes storing one row each (different n, same
// p) hit different banks; reads of a row stay aligned 16-byte slots.
template <int M, bool SW>
__device__ __forceinline__ int ut_index(int n, int p)
{
    if constexpr (SW) return n * M + ((((p >> 2) ^ (n >> 2)) & 7) << 2) + (p & ~31) + (p & 3);
    else return n * M + p;
}

template <int M, int N, int TP, int TQ, int WPC>
__global__ void __launch_bounds__(32 * WPC) sep_warp_kernel(const SepArgs a)
{
    constexpr int MN = M * N, tilesN = N / TQ;
    static_assert((M / TP) * (N / TQ) == 32, "one tile per lane");
    constexpr bool SW = M == 32 && TP % 4 == 0;
    extern __shared__ __align__(16) unsigned char smem[];
    float *cst = reinterpret_cast<float *>(smem);        // per transform: TmT [M][M], TnT [N][N]
    constexpr int cstride = M * M + N * N;
    float *Wr = cst + a.ntr * cstride;                   // [MN] rho (unmasked weights)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wpc = blockDim.x >> 5;
    float *X = Wr + MN + w * 2 * MN;                     // [M][N]
    float *UT = X + MN;                                  // [N][M]

    stage_image(a, cst, a.ntr * cstride, a.ntr * cstride + MN);
    __syncthreads();

    const int n_items = a.n_dev ? min(a.n, *a.n_dev) : a.n;
    const int p0 = TP * (lane / tilesN), c0 = TQ * (lane % tilesN);
    for (int i = blockIdx.x * wpc + w; i < n_items; i += gridDim.x * wpc) {
        const int b = a.item_blk ? a.item_blk[i] : i;
        const uint8_t *mask;
        const double *smp = nullptr;
        double *dst = nullptr;
        const float *rowM = nullptr, *rowN = nullptr;
        if (a.mode == 3) {
            mask = a.pattern;
        } else {
            const BlockDesc bd = a.blocks[b];
            mask = bd.support ? bd.support : a.pattern;
            smp = bd.samples;
            if (a.mode == 0 && a.copy_support && bd.out != bd.samples) dst = bd.out;   // none in place
        }
        if (a.mode >= 2) {
            const int u = a.mode == 3 ? i : a.cur_u[b];
            const int t = (a.ntr > 1 && u >= a.koff[1]) ? 1 : 0;
            const int ku = u - a.koff[t];
            rowM = static_cast<const float *>(a.TM[t]) + static_cast<size_t>(ku / N) * M;
            rowN = static_cast<const float *>(a.TN[t]) + static_cast<size_t>(ku % N) * N;
        }
        __syncwarp();   // the previous item's last reads of X and UT are done
        constexpr int R = MN / 32 < 16 ? MN / 32 : 16;
#pragma unroll 1
        for (int q0 = 0; q0 < MN; q0 += 32 * R) {
            bool on[R];
            float ex[R];
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int p = q0 + j * 32 + lane;
                on[j] = mask[p] != 0;
                ex[j] = a.mode >= 2 ? rowM[p / N] * rowN[p % N] : 1.0f;
            }
            double sv[R];
#pragma unroll
            for (int j = 0; j < R; ++j) sv[j] = (a.mode == 0 && on[j]) ? smp[q0 + j * 32 + lane] : 0.0;
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const int p = q0 + j * 32 + lane;
                float v = on[j] ? Wr[p] : 0.0f;
                if (a.mode == 0) v = on[j] ? v * dev::f64_to_f32_rn(sv[j]) : 0.0f;
                else if (a.mode >= 2) v *= ex[j];
                X[p] = v;
                if (dst && on[j]) dst[p] = sv[j];
            }
        }
        float *out = static_cast<float *>(a.out) + (a.out_rows ? a.out_rows[i] : static_cast<long long>(b) * a.ldo);
        __syncwarp();

        for (int t = 0; t < a.ntr; ++t) {
            const float *TmT = cst + t * cstride, *TnT = TmT + M * M;
            if (t) __syncwarp();   // the previous transform is done reading UT
            {
                float acc[TP][TQ] = {};
#pragma unroll 8
                for (int m = 0; m < M; ++m) {
                    float av[TP], bv[TQ];
                    lds_vec<TP>(TmT + m * M + p0, av);
                    lds_vec<TQ>(X + m * N + c0, bv);
                    outer_fma_pq<TP, TQ>(acc, av, bv);
                }
#pragma unroll
                for (int c = 0; c < TQ; ++c) {
#pragma unroll
                    for (int r0 = 0; r0 < TP; r0 += 4) {
                        float col[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) col[r] = acc[r0 + r][c];
                        sts_vec<4>(UT + ut_index<M, SW>(c0 + c, p0 + r0), col);
                    }
                }
            }
            __syncwarp();
            {
                float acc[TP][TQ] = {};
#pragma unroll 8
                for (int n = 0; n < N; ++n) {
                    float av[TP], bv[TQ];
#pragma unroll
                    for (int r0 = 0; r0 < TP; r0 += 4) {
                        float v4[4];
                        lds_vec<4>(UT + ut_index<M, SW>(n, p0 + r0), v4);
#pragma unroll
                        for (int r = 0; r < 4; ++r) av[r0 + r] = v4[r];
                    }
                    lds_vec<TQ>(TnT + n * N + c0, bv);
                    outer_fma_pq<TP, TQ>(acc, av, bv);
                }
#pragma unroll
                for (int r = 0; r < TP; ++r) {
                    const int k0 = a.koff[t] + (p0 + r) * N + c0;
                    if (a.scale) {
                        float sv[TQ];
                        lds_vec<TQ>(a.scale + k0, sv);
#pragma unroll
                        for (int c = 0; c < TQ; ++c) acc[r][c] *= sv[c];
                    }
                    sts_vec<TQ>(out + k0, acc[r]);
                }
            }
        }
        for (int k = a.koff[a.ntr - 1] + MN + lane; k < a.kfill; k += 32)
            out[k] = a.scale ? NAN : 0.0f;
    }
}

// Model (eq. 9) for separable dictionaries, one warp per block (the launcher
// requires a non-empty box, so the first pass over it always runs and also
// writes the caller's copies of the log).  Shared
// memory holds the 1-D rows of every transform, T_t[p][m] then T'_t[q][n];
// a log entry u = koff[t] + p N + q contributes c t_p[m] t'_q[n].  The
// entries of the log pass through a per-warp table (row offsets and c, one
// 16-byte broadcast read per entry).  Outputs of the loss bounding box
// (Mb x Nb) are taken RP per lane: with COL (Nb divides 32, whole chunks of
// 32 RP outputs, row runs aligned to RP floats) every lane keeps one column n
// and RP consecutive rows, reading t_p[m..m+RP) as vectors; otherwise each
// output reads both factors.
template <bool COL, int RP>
__global__ void __launch_bounds__(256) sep_model_kernel(const IterArgs a, const SepArgs s, int m0, int Mb,
                                                        int n0, int Nb)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *Ts = reinterpret_cast<float *>(smem);
    const int M = s.M, N = s.N, MN = M * N, cstride = M * M + N * N;
    int4 *Etab = reinterpret_cast<int4 *>(Ts + ((s.ntr * cstride + 3) & ~3)) + (threadIdx.x >> 5) * 32;
    for (int t = 0; t < s.ntr; ++t) {
        const float *gm = static_cast<const float *>(s.TM[t]);
        const float *gn = static_cast<const float *>(s.TN[t]);
        for (int e = threadIdx.x; e < M * M; e += blockDim.x) Ts[t * cstride + e] = gm[e];
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) Ts[t * cstride + M * M + e] = gn[e];
    }
    __syncthreads();
    // launched as a programmatic dependent of the iteration kernel: the rows above
    // are staged while it drains; its log is read only after it has completed
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
    const int nbox = Mb * Nb;
    constexpr int CH = 32 * RP;   // outputs per chunk
    for (int b = blockIdx.x * wpc + (threadIdx.x >> 5); b < a.n; b += gridDim.x * wpc) {
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const int *lu = a.log_u + static_cast<size_t>(b) * a.I_max;
        const float *lc = a.log_c + static_cast<size_t>(b) * a.I_max;

        for (int o0 = 0; o0 < nbox; o0 += CH) {
            // COL: column n0 + lane % Nb, rows mb .. mb + RP - 1
            const int mb = m0 + o0 / Nb + RP * (lane / Nb);
            int mo[RP], no[RP];
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                const int o = o0 + lane + 32 * r;
                const int oc = o < nbox ? o : 0;
                mo[r] = COL ? mb + r : m0 + oc / Nb;
                no[r] = COL ? n0 + lane % Nb : n0 + oc % Nb;
            }
            static_assert(RP % 2 == 0, "outputs in pairs");
            float2 acc2[RP / 2];
#pragma unroll
            for (int r = 0; r < RP / 2; ++r) acc2[r] = make_float2(0.0f, 0.0f);
            // the log in rounds of 32 entries, the next round's loads in flight
            // while this one is evaluated; the first pass over the box also
            // writes the caller's copies of the log
            int un = lane < I ? lu[lane] : -1;
            float cn = lane < I ? lc[lane] : 0.0f;
            for (int nu0 = 0; nu0 < I; nu0 += 32) {
                int u = un;
                const float cl = cn;
                if (nu0 + 32 + lane < I) {
                    un = lu[nu0 + 32 + lane];
                    cn = lc[nu0 + 32 + lane];
                }
                if (o0 == 0 && nu0 + lane < I) {
                    if (bd.sel_idx) bd.sel_idx[nu0 + lane] = u;
                    if (bd.sel_coef) bd.sel_coef[nu0 + lane] = static_cast<double>(cl);
                }
                float cf = 0.0f;                                   // padded entries add 0
                if (nu0 + lane < I && u >= 0 && u < s.koff[s.ntr - 1] + MN) cf = cl;
                else u = 0;
                const int t = (s.ntr > 1 && u >= s.koff[1]) ? 1 : 0;
                const int ku = u - s.koff[t];
                __syncwarp();   // the previous round's reads of the table are done
                Etab[lane] = make_int4(t * cstride + (ku / N) * M, t * cstride + M * M + (ku % N) * N,
                                       __float_as_int(cf), 0);
                __syncwarp();
                // padded entries (coefficient 0) add exact zeros: whole groups of 4
                const int cnt = (min(32, I - nu0) + 3) & ~3;
#pragma unroll 4
                for (int k = 0; k < cnt; ++k) {
                    const int4 e = Etab[k];
                    const float c = __int_as_float(e.z);
                    if (COL) {
                        const float cb = c * Ts[e.y + no[0]];
                        float tv[RP];
                        lds_vec<RP>(Ts + e.x + mb, tv);
#pragma unroll
                        for (int r = 0; r < RP; r += 2)   // paired: the same fma per output
                            acc2[r / 2] = __ffma2_rn(make_float2(cb, cb), make_float2(tv[r], tv[r + 1]), acc2[r / 2]);
                    } else {
#pragma unroll
                        for (int r = 0; r < RP; ++r) {
                            float &x = (r & 1) ? acc2[r / 2].y : acc2[r / 2].x;
                            x = fmaf(c * Ts[e.y + no[r]], Ts[e.x + mo[r]], x);
                        }
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < RP; ++r) {
                const int o = o0 + lane + 32 * r;
                if (o >= nbox) continue;
                const int p = mo[r] * N + no[r];
                if (!a.pat_support[p]) bd.out[p] = static_cast<double>((r & 1) ? acc2[r / 2].y : acc2[r / 2].x);
            }
        }
    }
}

// The same model on the tensor cores (the per-block body is dev::model_tc_block):
// one warp per block, the 1-D rows of the transforms staged in shared memory
// while the iteration kernel drains, a per-warp log table and output tile.
template <int MT, int NT>
__global__ void __launch_bounds__(256) sep_model_tc_kernel(const IterArgs a, const SepArgs s, int m0, int Mb,
                                                           int n0, int Nb)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float *Ts = reinterpret_cast<float *>(smem);
    const int M = s.M, N = s.N, cstride = M * M + N * N;
    int4 *Etab = reinterpret_cast<int4 *>(Ts + ((s.ntr * cstride + 3) & ~3)) + (threadIdx.x >> 5) * 32;
    float *Gt = reinterpret_cast<float *>(reinterpret_cast<int4 *>(Ts + ((s.ntr * cstride + 3) & ~3)) +
                                          (blockDim.x >> 5) * 32) +
                (threadIdx.x >> 5) * dev::model_tile_floats(MT, NT);
    for (int t = 0; t < s.ntr; ++t) {
        const float *gm = static_cast<const float *>(s.TM[t]);
        const float *gn = static_cast<const float *>(s.TN[t]);
        for (int e = threadIdx.x; e < M * M; e += blockDim.x) Ts[t * cstride + e] = gm[e];
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) Ts[t * cstride + M * M + e] = gn[e];
    }
    __syncthreads();
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const int lane = threadIdx.x & 31, wpc = blockDim.x >> 5;
    const dev::ModelLayout L = dev::model_full_layout(M, N);
    for (int b = blockIdx.x * wpc + (threadIdx.x >> 5); b < a.n; b += gridDim.x * wpc)
        dev::model_tc_block<MT, NT>(a, s, Ts, L, Etab, Gt, b, m0, Mb, n0, Nb, lane);
}

}  // namespace

template <int TS, int MC, int NC>
cudaError_t launch_sep_group(const SepArgs &a, cudaStream_t st, bool *done)
{
    *done = false;
    const size_t MN = static_cast<size_t>(a.M) * a.N;
    const size_t cst = 4 * a.ntr * (static_cast<size_t>(a.M) * a.M + static_cast<size_t>(a.N) * a.N) + 4 * MN;
    int groups = 4;
    while (groups > 0 && cst + 8 * MN * groups > 227 * 1024) groups /= 2;
    if (groups == 0) return cudaSuccess;
    const size_t smem = cst + 8 * MN * groups;
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(sep_group_kernel<TS, MC, NC>), kSepGroup * groups, smem,
                                (a.n + groups - 1) / groups, &grid);
    if (e != cudaSuccess) return e;
    sep_group_kernel<TS, MC, NC><<<grid, kSepGroup * groups, smem, st>>>(a, groups);
    *done = true;
    return cudaGetLastError();
}

template <int M, int N, int TP, int TQ>
cudaError_t launch_sep_warp(const SepArgs &a, cudaStream_t st)
{
    constexpr int wpc = 10;   // 2 CTAs of 10 warps per SM at 32 x 32 (shared memory bound)
    const size_t smem = 4 * (a.ntr * static_cast<size_t>(M * M + N * N) + M * N + 2 * M * N * wpc);
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(sep_warp_kernel<M, N, TP, TQ, wpc>), 32 * wpc, smem,
                                (a.n + wpc - 1) / wpc, &grid);
    if (e != cudaSuccess) return e;
    sep_warp_kernel<M, N, TP, TQ, wpc><<<grid, 32 * wpc, smem, st>>>(a);
    return cudaGetLastError();
}

int sep_variants(const SepArgs &a, bool fp64)
{
    return !fp64 && ((a.M == 32 && a.N == 32) || (a.M == 16 && a.N == 16)) ? 2 : 1;
}

// The tensor-core lazy columns of 32 x 32 and 64 x 64 areas (SE_COL_FFMA=1:
// the fp32 transform kernels); *done stays false if the launch does not apply.
template <int M>
static cudaError_t launch_col_tc_m(const SepArgs &a, cudaStream_t st)
{
    using C = ColCfg<M>;
    const size_t smem = sizeof(uint32_t) * (static_cast<size_t>(a.ntr) * 2 * C::Op + C::MN + C::Red +
                                            static_cast<size_t>(C::Groups) * C::ItemWords);
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(sep_col_tc_kernel<M>), C::NT, smem,
                                (a.n + C::Groups - 1) / C::Groups, &grid);
    if (e != cudaSuccess) return e;
    sep_col_tc_kernel<M><<<grid, C::NT, smem, st>>>(a);
    return cudaGetLastError();
}

static cudaError_t launch_col_tc(const SepArgs &a, cudaStream_t st, bool *done)
{
    *done = false;
    const char *env = std::getenv("SE_COL_FFMA");   // read at every launch: tests switch it per plan
    const bool ffma = env && env[0] == '1';
    auto al16 = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    if (ffma || a.mode != 2 || a.M != a.N || (a.M != 64 && a.M != 32) || !a.img || a.ntr < 1 || a.ntr > 2 ||
        !a.cur_u || (a.out_rows == nullptr && a.ldo < a.kfill) || !al16(a.img))
        return cudaSuccess;
    for (int t = 0; t < a.ntr; ++t)
        if (a.koff[t] % 2 || !al16(a.TM[t]) || !al16(a.TN[t])) return cudaSuccess;   // float2 / float4 accesses
    *done = true;
    return a.M == 64 ? launch_col_tc_m<64>(a, st) : launch_col_tc_m<32>(a, st);
}

template <typename T>
cudaError_t launch_sep(const SepArgs &a, cudaStream_t st, int variant)
{
    if (a.n <= 0) return cudaSuccess;
    if (sizeof(T) == 4) {
        bool done = false;
        cudaError_t e = launch_col_tc(a, st, &done);
        if (e != cudaSuccess || done) return e;
        if (a.M == 32 && a.N == 32 && variant == 0)
            return launch_sep_warp<32, 32, 8, 4>(a, st);
        if (a.M == 16 && a.N == 16 && variant == 0)
            return launch_sep_warp<16, 16, 4, 2>(a, st);
        if (a.M == 32 && a.N == 32)
            e = launch_sep_group<4, 32, 32>(a, st, &done);
        else if (a.M == 64 && a.N == 64)
            e = launch_sep_group<4, 64, 64>(a, st, &done);
        else if (a.M == 16 && a.N == 16)
            e = launch_sep_group<2, 16, 16>(a, st, &done);
        else if (a.M % 4 == 0 && a.N % 4 == 0 && a.M * a.N >= 1024)
            e = launch_sep_group<4, 0, 0>(a, st, &done);
        else if (a.M % 2 == 0 && a.N % 2 == 0)
            e = launch_sep_group<2, 0, 0>(a, st, &done);
        if (e != cudaSuccess || done) return e;
    }
    const size_t smem = sizeof(T) * (2 * static_cast<size_t>(a.M) * a.N + a.M * a.M + a.N * a.N);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    int unused = 0;   // one CTA per item; the call only raises the shared memory limit (per device)
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(sep_kernel<T>), 256, smem, 1, &unused);
    if (e != cudaSuccess) return e;
    sep_kernel<T><<<a.n, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template <bool COL, int RP>
cudaError_t launch_sep_model_t(const IterArgs &a, const SepArgs &s, int m0, int Mb, int n0, int Nb, size_t smem,
                               cudaStream_t st)
{
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(sep_model_kernel<COL, RP>), 256, smem, (a.n + 7) / 8,
                                &grid);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // may start while the
    attr[0].val.programmaticStreamSerializationAllowed = 1;             // previous kernel drains
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sep_model_kernel<COL, RP>, a, s, m0, Mb, n0, Nb);
}

template <int MT, int NT>
cudaError_t launch_sep_model_tc(const IterArgs &a, const SepArgs &s, int m0, int Mb, int n0, int Nb, size_t smem0,
                                cudaStream_t st)
{
    const size_t smem = smem0 + sizeof(float) * 8 * (16 * MT) * (8 * NT + 1);   // eight warps' output tiles
    int grid = 0;
    cudaError_t e = launch_grid(reinterpret_cast<const void *>(sep_model_tc_kernel<MT, NT>), 256, smem,
                                (a.n + 7) / 8, &grid);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // may start while the
    attr[0].val.programmaticStreamSerializationAllowed = 1;             // previous kernel drains
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, sep_model_tc_kernel<MT, NT>, a, s, m0, Mb, n0, Nb);
}

// Boxes up to 32 x 32 take the tensor-core form (SE_MODEL_FFMA=1: the fp32 FMA kernel).
bool sep_model_tc_box(int Mb, int Nb)
{
    static const bool ffma = [] {
        const char *env = std::getenv("SE_MODEL_FFMA");
        return env && env[0] == '1';
    }();
    return !ffma && Mb > 0 && Nb > 0 && Mb <= 32 && Nb <= 32;
}

cudaError_t launch_sep_model(const IterArgs &a, const SepArgs &s, int m0, int m1, int n0, int n1,
                             cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    const int Mb = m1 - m0, Nb = n1 - n0;
    if (Mb <= 0 || Nb <= 0 || m0 < 0 || n0 < 0 || m1 > s.M || n1 > s.N) return cudaErrorInvalidValue;
    const size_t smem = 4 * ((s.ntr * (static_cast<size_t>(s.M) * s.M + static_cast<size_t>(s.N) * s.N) + 3) & ~size_t(3)) +
                        8 * 32 * sizeof(int4);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if (sep_model_tc_box(Mb, Nb)) {
        const int nt = Nb <= 8 ? 1 : Nb <= 16 ? 2 : 4;
        if (Mb <= 16)
            return nt == 1 ? launch_sep_model_tc<1, 1>(a, s, m0, Mb, n0, Nb, smem, st)
                 : nt == 2 ? launch_sep_model_tc<1, 2>(a, s, m0, Mb, n0, Nb, smem, st)
                           : launch_sep_model_tc<1, 4>(a, s, m0, Mb, n0, Nb, smem, st);
        return nt == 1 ? launch_sep_model_tc<2, 1>(a, s, m0, Mb, n0, Nb, smem, st)
             : nt == 2 ? launch_sep_model_tc<2, 2>(a, s, m0, Mb, n0, Nb, smem, st)
                       : launch_sep_model_tc<2, 4>(a, s, m0, Mb, n0, Nb, smem, st);
    }
    // small boxes take 2 outputs per lane, else 8; one column and RP
    // consecutive rows per lane when Nb divides 32, the box holds whole
    // chunks and the row runs are aligned for vector reads
    const int nbox = Mb * Nb;
    const int rp = nbox <= 64 ? 2 : 8;
    const bool col = 32 % Nb == 0 && nbox % (32 * rp) == 0 && m0 % (rp == 8 ? 4 : 2) == 0 &&
                     s.M % (rp == 8 ? 4 : 2) == 0 && s.N % 2 == 0;
    if (rp == 2)
        return col ? launch_sep_model_t<true, 2>(a, s, m0, Mb, n0, Nb, smem, st)
                   : launch_sep_model_t<false, 2>(a, s, m0, Mb, n0, Nb, smem, st);
    return col ? launch_sep_model_t<true, 8>(a, s, m0, Mb, n0, Nb, smem, st)
               : launch_sep_model_t<false, 8>(a, s, m0, Mb, n0, Nb, smem, st);
}

template cudaError_t launch_sep<float>(const SepArgs &, cudaStream_t, int);
template cudaError_t launch_sep<double>(const SepArgs &, cudaStream_t, int);

}  // namespace se
