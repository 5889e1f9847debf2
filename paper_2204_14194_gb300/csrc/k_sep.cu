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
// writes atoms koff[t] + p N + q.  One CTA per item, the item's x and the
// intermediate Z = x T_N^T staged in shared memory with the 1-D bases.
#include <cuda_runtime.h>

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
    const T *rowM = nullptr, *rowN = nullptr;
    if (a.mode == 3) {
        mask = a.pattern;
    } else {
        const BlockDesc bd = a.blocks[b];
        mask = bd.support ? bd.support : a.pattern;
        smp = bd.samples;
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
        if (a.mode == 0) v = mask[p] ? v * static_cast<T>(smp[p]) : T(0);
        else if (a.mode >= 2) v *= rowM[m] * rowN[n];
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
}

// fp32 form with 4 x 4 register tiles (M, N multiples of 4).  Operands are
// staged transposed so that every shared-memory read is a float4 shared by
// the threads of a tile row or column:
//   XT[n][m] = x[m][n],  TnT[n][q] = t'_q[n],  TmT[m][p] = t_p[m],
//   Z[m][q] = sum_n XT[n][m] TnT[n][q],   Y[p][q] = sum_m TmT[m][p] Z[m][q].
__global__ void __launch_bounds__(256) sep_tiled_kernel(const SepArgs a)
{
    const int i = blockIdx.x;
    if (a.n_dev && i >= *a.n_dev) return;
    if (i >= a.n) return;
    const int M = a.M, N = a.N, MN = M * N;
    extern __shared__ __align__(16) unsigned char smem[];
    float *XT = reinterpret_cast<float *>(smem);    // [N][M]
    float *Z = XT + MN;                             // [M][N]
    float *TmT = Z + MN;                            // [M][M]
    float *TnT = TmT + M * M;                       // [N][N]

    const int b = a.item_blk ? a.item_blk[i] : i;
    const uint8_t *mask;
    const double *smp = nullptr;
    const float *rowM = nullptr, *rowN = nullptr;
    if (a.mode == 3) {
        mask = a.pattern;
    } else {
        const BlockDesc bd = a.blocks[b];
        mask = bd.support ? bd.support : a.pattern;
        smp = bd.samples;
    }
    if (a.mode >= 2) {
        const int u = a.mode == 3 ? i : a.cur_u[b];
        const int t = (a.ntr > 1 && u >= a.koff[1]) ? 1 : 0;
        const int ku = u - a.koff[t];
        rowM = static_cast<const float *>(a.TM[t]) + static_cast<size_t>(ku / N) * M;
        rowN = static_cast<const float *>(a.TN[t]) + static_cast<size_t>(ku % N) * N;
    }
    for (int p = threadIdx.x; p < MN; p += blockDim.x) {
        const int m = p / N, n = p - m * N;
        float v = mask[p] ? static_cast<float>(a.rho[p]) : 0.0f;
        if (a.mode == 0) v = mask[p] ? v * static_cast<float>(smp[p]) : 0.0f;
        else if (a.mode >= 2) v *= rowM[m] * rowN[n];
        XT[n * M + m] = v;
    }
    float *out = static_cast<float *>(a.out) + (a.out_rows ? a.out_rows[i] : static_cast<long long>(b) * a.ldo);
    const float *scale = a.scale;
    const int tilesM = M / 4, tilesN = N / 4;

    for (int t = 0; t < a.ntr; ++t) {
        const float *gm = static_cast<const float *>(a.TM[t]);
        const float *gn = static_cast<const float *>(a.TN[t]);
        __syncthreads();
        for (int e = threadIdx.x; e < M * M; e += blockDim.x) {
            const float v = gm[e];
            const int p = e / M, m = e - p * M;
            TmT[m * M + p] = a.mode == 1 ? v * v : v;
        }
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
            const float v = gn[e];
            const int q = e / N, n = e - q * N;
            TnT[n * N + q] = a.mode == 1 ? v * v : v;
        }
        __syncthreads();
        for (int tile = threadIdx.x; tile < tilesM * tilesN; tile += blockDim.x) {
            const int m0 = 4 * (tile / tilesN), q0 = 4 * (tile % tilesN);
            float acc[4][4] = {};
            for (int n = 0; n < N; ++n) {
                const float4 xv = *reinterpret_cast<const float4 *>(XT + n * M + m0);
                const float4 tv = *reinterpret_cast<const float4 *>(TnT + n * N + q0);
                const float xs[4] = {xv.x, xv.y, xv.z, xv.w}, ts[4] = {tv.x, tv.y, tv.z, tv.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(xs[r], ts[c], acc[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                *reinterpret_cast<float4 *>(Z + (m0 + r) * N + q0) =
                    make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        }
        __syncthreads();
        for (int tile = threadIdx.x; tile < tilesM * tilesN; tile += blockDim.x) {
            const int p0 = 4 * (tile / tilesN), q0 = 4 * (tile % tilesN);
            float acc[4][4] = {};
            for (int m = 0; m < M; ++m) {
                const float4 tv = *reinterpret_cast<const float4 *>(TmT + m * M + p0);
                const float4 zv = *reinterpret_cast<const float4 *>(Z + m * N + q0);
                const float ts[4] = {tv.x, tv.y, tv.z, tv.w}, zs[4] = {zv.x, zv.y, zv.z, zv.w};
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(ts[r], zs[c], acc[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int k0 = a.koff[t] + (p0 + r) * N + q0;
                if (scale) {
                    const float4 sv = *reinterpret_cast<const float4 *>(scale + k0);
                    acc[r][0] *= sv.x; acc[r][1] *= sv.y; acc[r][2] *= sv.z; acc[r][3] *= sv.w;
                }
                *reinterpret_cast<float4 *>(out + k0) = make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
            }
        }
    }
}

}  // namespace

template <typename T>
cudaError_t launch_sep(const SepArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    const size_t smem = sizeof(T) * (2 * static_cast<size_t>(a.M) * a.N + a.M * a.M + a.N * a.N);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    const bool tiled = sizeof(T) == 4 && a.M % 4 == 0 && a.N % 4 == 0;
    static bool attr[2] = {false, false};
    if (!attr[tiled]) {
        cudaError_t e = tiled ? cudaFuncSetAttribute(sep_tiled_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     227 * 1024)
                              : cudaFuncSetAttribute(sep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     227 * 1024);
        if (e != cudaSuccess) return e;
        attr[tiled] = true;
    }
    if (tiled) sep_tiled_kernel<<<a.n, 256, smem, st>>>(a);
    else sep_kernel<T><<<a.n, 256, smem, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_sep<float>(const SepArgs &, cudaStream_t);
template cudaError_t launch_sep<double>(const SepArgs &, cudaStream_t);

}  // namespace se
