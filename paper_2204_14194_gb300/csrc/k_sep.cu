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

template <typename T>
cudaError_t launch_sep(const SepArgs &a, cudaStream_t st, int variant)
{
    if (a.n <= 0) return cudaSuccess;
    if (sizeof(T) == 4) {
        bool done = false;
        cudaError_t e = cudaSuccess;
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
