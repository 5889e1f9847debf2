// k_simt.cu -- CUDA-core kernels: operand packing, the diagonal of the table
// (eq. 17), and the plain fp64 GEMM used by the fp64 form.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "se_internal.h"

namespace se {
namespace {

__device__ __forceinline__ uint16_t bf16_bits(double v)
{
    __nv_bfloat16 h = __float2bfloat16_rn(static_cast<float>(v));
    return *reinterpret_cast<uint16_t *>(&h);
}

__device__ __forceinline__ double bf16_value(uint16_t bits)
{
    __nv_bfloat16 h = *reinterpret_cast<__nv_bfloat16 *>(&bits);
    return static_cast<double>(__bfloat162float(h));
}

// Weighted samples of the shared pattern, x_b[j] = sqrt(w[j]) s_b[a_idx[j]]
// on the support pixels (so that sum_j G[k][j] x_b[j] = sum s phi_k w, eq. 12),
// zero in the padding.  Split parts: v = h + m + l with each part the bf16
// rounding of what the previous parts left; part p of block b lives at
// x_bf16[b][p * ka_pad + j].
__global__ void pack_x_kernel(const BlockDesc *__restrict__ blocks, const int *__restrict__ a_idx,
                              const double *__restrict__ sqrtw, int nA, int ka_pad, int nparts,
                              uint16_t *__restrict__ xb, double *__restrict__ xd)
{
    const int b = blockIdx.x;
    const double *s = blocks[b].samples;
    const size_t rowb = static_cast<size_t>(b) * nparts * ka_pad;
    for (int j = threadIdx.x; j < ka_pad; j += blockDim.x) {
        const double v = j < nA ? sqrtw[j] * s[a_idx[j]] : 0.0;
        if (xd) xd[static_cast<size_t>(b) * ka_pad + j] = v;
        if (xb) {
            double rest = v;
            for (int p = 0; p < nparts; ++p) {
                const uint16_t h = bf16_bits(rest);
                xb[rowb + static_cast<size_t>(p) * ka_pad + j] = h;
                rest -= bf16_value(h);
            }
        }
    }
}

// Split fp64 rows into bf16 parts (same rule as pack_x_kernel).
__global__ void split_bf16_kernel(const double *__restrict__ in, int cols, int ld_in, int ka_pad,
                                  int nparts, uint16_t *__restrict__ out)
{
    const int r = blockIdx.x;
    const size_t rowo = static_cast<size_t>(r) * nparts * ka_pad;
    for (int j = threadIdx.x; j < ka_pad; j += blockDim.x) {
        double rest = j < cols ? in[static_cast<size_t>(r) * ld_in + j] : 0.0;
        for (int p = 0; p < nparts; ++p) {
            const uint16_t h = bf16_bits(rest);
            out[rowo + static_cast<size_t>(p) * ka_pad + j] = h;
            rest -= bf16_value(h);
        }
    }
}

// diag[k] = sum_j G[k][j]^2 = sum phi_k^2 w = C_kk (eq. 16 on the diagonal),
// one warp per atom, fp64.
__global__ void diag_kernel(const double *__restrict__ G, int ldg, int Kp, int nA,
                            double *__restrict__ diag)
{
    const int k = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (k >= Kp) return;
    double acc = 0.0;
    for (int j = lane; j < nA; j += 32) {
        const double g = G[static_cast<size_t>(k) * ldg + j];
        acc = fma(g, g, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) diag[k] = acc;
}

// Admissibility and the per-atom constants of eqs. (17)-(19): atom k may be
// selected if k < K, it is not a collinear duplicate of a lower index, and
// C_kk > 1e-14 max_j C_jj.  invC = 1/C_kk (0 if inadmissible), D = 1/sqrt(C_kk)
// (NaN if inadmissible, so |R_k| D_k never wins a comparison).
template <typename T>
__global__ void finalize_kernel(const double *__restrict__ diag, const uint8_t *__restrict__ dup,
                                int K, int Kp, T *__restrict__ invC, T *__restrict__ Dk,
                                int *__restrict__ n_adm)
{
    __shared__ double smax[32];
    __shared__ int scnt[32];
    double mx = 0.0;
    for (int k = threadIdx.x; k < K; k += blockDim.x)
        if (!dup[k]) mx = fmax(mx, diag[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) smax[threadIdx.x / 32] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < blockDim.x / 32 ? smax[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (threadIdx.x == 0) smax[0] = v;
    }
    __syncthreads();
    mx = smax[0];
    int cnt = 0;
    for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
        const double d = k < K ? diag[k] : 0.0;
        const bool adm = k < K && !dup[k] && mx > 0.0 && d > 1e-14 * mx;
        invC[k] = adm ? static_cast<T>(1.0 / d) : static_cast<T>(0);
        Dk[k] = adm ? static_cast<T>(1.0 / sqrt(d)) : static_cast<T>(NAN);
        cnt += adm;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) scnt[threadIdx.x / 32] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) t += scnt[w];
        *n_adm = t;
    }
}

// Plain tiled GEMM on CUDA cores: D[m][n] = sum_k A[m][k] B[n][k], 64 x 64
// tiles, 256 threads with 4 x 4 outputs each.  symmetric: upper tiles of a
// square D, stored mirrored (each entry written once); otherwise D is
// stored transposed, out[n * ldo + m].
template <typename T>
__global__ void __launch_bounds__(256)
simt_gemm_kernel(const T *__restrict__ A, int lda, const T *__restrict__ B, int ldb, int M, int N,
                 int Kd, T *__restrict__ out, long long ldo, int symmetric, int mt)
{
    __shared__ T As[16][65];
    __shared__ T Bs[16][65];
    int tm, tn;
    if (symmetric) {
        int t = blockIdx.x;
        tm = 0;
        while (t >= mt - tm) { t -= mt - tm; ++tm; }
        tn = tm + t;
    } else {
        tm = blockIdx.x % mt;
        tn = blockIdx.x / mt;
    }
    const int tx = threadIdx.x & 15;
    const int ty = threadIdx.x >> 4;
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int k0 = 0; k0 < Kd; k0 += 16) {
        for (int i = threadIdx.x; i < 1024; i += 256) {
            const int r = i >> 4, c = i & 15;
            const int m = tm * 64 + r, n = tn * 64 + r, k = k0 + c;
            As[c][r] = (m < M && k < Kd) ? A[static_cast<size_t>(m) * lda + k] : T(0);
            Bs[c][r] = (n < N && k < Kd) ? B[static_cast<size_t>(n) * ldb + k] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            T av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }
    const bool diag_tile = symmetric && tm == tn;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = tm * 64 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = tn * 64 + tx + 16 * j;
            if (n >= N) continue;
            if (!symmetric) {
                out[static_cast<long long>(n) * ldo + m] = acc[i][j];
            } else if (!diag_tile || n >= m) {
                out[static_cast<long long>(m) * ldo + n] = acc[i][j];
                out[static_cast<long long>(n) * ldo + m] = acc[i][j];
            }
        }
    }
}

}  // namespace

cudaError_t launch_pack_x(const BlockDesc *blocks, int n, const int *a_idx, const double *sqrtw,
                          int nA, int ka_pad, int nparts, uint16_t *x_bf16, double *x_f64,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    pack_x_kernel<<<n, 256, 0, st>>>(blocks, a_idx, sqrtw, nA, ka_pad, nparts, x_bf16, x_f64);
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(const double *in, int rows, int cols, int ld_in, int ka_pad,
                              int nparts, uint16_t *out, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    split_bf16_kernel<<<rows, 256, 0, st>>>(in, cols, ld_in, ka_pad, nparts, out);
    return cudaGetLastError();
}

cudaError_t launch_tables_diag(const double *G64, int ldg, int Kp, int nA, double *diag,
                               cudaStream_t st)
{
    diag_kernel<<<(Kp + 7) / 8, 256, 0, st>>>(G64, ldg, Kp, nA, diag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tables_finalize(const double *diag, const uint8_t *dup, int K, int Kp, T *invC,
                                   T *Dk, int *n_admissible, cudaStream_t st)
{
    finalize_kernel<T><<<1, 1024, 0, st>>>(diag, dup, K, Kp, invC, Dk, n_admissible);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_simt_gemm(const T *A, int lda, const T *B, int ldb, int M, int N, int Kd, T *out,
                             long long ldo, int symmetric, cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int mt = (M + 63) / 64, nt = (N + 63) / 64;
    const int grid = symmetric ? mt * (mt + 1) / 2 : mt * nt;
    simt_gemm_kernel<T><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, Kd, out, ldo, symmetric, mt);
    return cudaGetLastError();
}

template cudaError_t launch_tables_finalize<float>(const double *, const uint8_t *, int, int, float *,
                                                   float *, int *, cudaStream_t);
template cudaError_t launch_tables_finalize<double>(const double *, const uint8_t *, int, int,
                                                    double *, double *, int *, cudaStream_t);
template cudaError_t launch_simt_gemm<double>(const double *, int, const double *, int, int, int, int,
                                              double *, long long, int, cudaStream_t);
template cudaError_t launch_simt_gemm<float>(const float *, int, const float *, int, int, int, int,
                                             float *, long long, int, cudaStream_t);

}  // namespace se
