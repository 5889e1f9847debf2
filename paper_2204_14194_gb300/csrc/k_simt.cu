// k_simt.cu -- CUDA-core kernels: operand packing, the diagonal of the table
// (eq. 17), and the plain fp64 GEMM used by the fp64 form.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>

#include "k_device.cuh"
#include "se_internal.h"

namespace se {
namespace {

// Exact split of a double into bf16 parts without fp64 arithmetic (GB300's
// fp64 pipe is narrow).  From the IEEE-754 binary64 fields, hi is x truncated
// to 24 significant bits (a float, exact) and lo the remaining 29 mantissa
// bits scaled by 2^(e - 1075) (one int->float rounding, < 2^-47 |x|).  Then
// h = bf16(hi), m = bf16(hi - h), l = bf16((hi - h - m) + lo): the first two
// differences are exact in fp32, so x - (h + m + l) is below ~2^-26 |x|.
// Zeros, subnormals, infinities, NaN and values outside the fp32 range go
// through the ordinary conversion (lo = 0).
__device__ __forceinline__ void f64_split_pair(double x, float &hi, float &lo)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
    const int e = static_cast<int>((b >> 52) & 0x7FF);
    const int ef = e - 1023 + 127;
    if (e == 0 || e == 0x7FF || ef <= 0 || ef >= 255) {
        hi = __double2float_rn(x);
        lo = 0.0f;
        return;
    }
    const unsigned long long mant = b & ((1ull << 52) - 1);
    hi = __uint_as_float(sign | (static_cast<uint32_t>(ef) << 23) | static_cast<uint32_t>(mant >> 29));
    const uint32_t rest = static_cast<uint32_t>(mant & ((1u << 29) - 1));
    const int es = e - 1075 + 127;                         // exponent of 2^(e - 1075)
    const float scale = es >= 1 ? __uint_as_float(static_cast<uint32_t>(es) << 23) : 0.0f;
    lo = __uint_as_float(sign | __float_as_uint(static_cast<float>(rest) * scale));
}

__device__ __forceinline__ uint16_t bf16_of(float v)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t *>(&h);
}

__device__ __forceinline__ float bf16_to_f(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

// Parts of x: part 0 = h, 1 = m, 2 = l (nparts <= 3; fewer parts simply
// drop the smaller ones).
__device__ __forceinline__ void split_parts(double x, uint16_t (&p)[3])
{
    float hi, lo;
    f64_split_pair(x, hi, lo);
    p[0] = bf16_of(hi);
    const float r = hi - bf16_to_f(p[0]);
    p[1] = bf16_of(r);
    p[2] = bf16_of((r - bf16_to_f(p[1])) + lo);
}

__device__ __forceinline__ void split_store2(double v0, double v1, int nparts, uint16_t *dst,
                                             int ka_pad)
{
    uint16_t a[3], b[3];
    split_parts(v0, a);
    split_parts(v1, b);
    for (int p = 0; p < nparts; ++p)
        *reinterpret_cast<uint32_t *>(dst + static_cast<size_t>(p) * ka_pad) =
            static_cast<uint32_t>(a[p]) | (static_cast<uint32_t>(b[p]) << 16);
}

// One warp per block: the block's samples are staged in shared memory with
// coalesced loads, then gathered at the support pixels two at a time, so the
// bf16 parts are written as 4-byte pairs (128 bytes per warp store).  The
// split path packs the raw samples s (the weights sit in the dictionary
// operand Phi_A w); the fp64 path (x_f64) packs sqrt(w) s in double.
__global__ void __launch_bounds__(256)
pack_x_staged_kernel(const BlockDesc *__restrict__ blocks, int n, const int *__restrict__ a_idx,
                     const double *__restrict__ sqrtw, int nA, int ka_pad, int nparts, int MN,
                     uint16_t *__restrict__ xb, double *__restrict__ xd)
{
    extern __shared__ double stage[];
    const int warps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = blockIdx.x * warps + warp;
    if (b >= n) return;
    double *sm = stage + static_cast<size_t>(warp) * MN;
    const double *s = blocks[b].samples;
    for (int i = lane; i < MN; i += 32) sm[i] = s[i];
    __syncwarp();
    const size_t rowb = static_cast<size_t>(b) * nparts * ka_pad;
    for (int j = 2 * lane; j < ka_pad; j += 64) {
        const double s0 = j < nA ? sm[a_idx[j]] : 0.0;
        const double s1 = j + 1 < nA ? sm[a_idx[j + 1]] : 0.0;
        if (xd)
            *reinterpret_cast<double2 *>(xd + static_cast<size_t>(b) * ka_pad + j) =
                make_double2(j < nA ? sqrtw[j] * s0 : 0.0, j + 1 < nA ? sqrtw[j + 1] * s1 : 0.0);
        if (xb) split_store2(s0, s1, nparts, xb + rowb + j, ka_pad);
    }
}

// Direct-gather form for areas too large to stage.
__global__ void pack_x_kernel(const BlockDesc *__restrict__ blocks, const int *__restrict__ a_idx,
                              const double *__restrict__ sqrtw, int nA, int ka_pad, int nparts,
                              uint16_t *__restrict__ xb, double *__restrict__ xd)
{
    const int b = blockIdx.x;
    const double *s = blocks[b].samples;
    const size_t rowb = static_cast<size_t>(b) * nparts * ka_pad;
    for (int j = 2 * threadIdx.x; j < ka_pad; j += 2 * blockDim.x) {
        const double s0 = j < nA ? s[a_idx[j]] : 0.0;
        const double s1 = j + 1 < nA ? s[a_idx[j + 1]] : 0.0;
        if (xd)
            *reinterpret_cast<double2 *>(xd + static_cast<size_t>(b) * ka_pad + j) =
                make_double2(j < nA ? sqrtw[j] * s0 : 0.0, j + 1 < nA ? sqrtw[j + 1] * s1 : 0.0);
        if (xb) split_store2(s0, s1, nparts, xb + rowb + j, ka_pad);
    }
}

// Split fp64 rows into bf16 parts (same rule as the sample packing).
__global__ void split_bf16_kernel(const double *__restrict__ in, int cols, int ld_in, int ka_pad,
                                  int nparts, uint16_t *__restrict__ out)
{
    const int r = blockIdx.x;
    const size_t rowo = static_cast<size_t>(r) * nparts * ka_pad;
    for (int j = threadIdx.x; j < ka_pad; j += blockDim.x) {
        uint16_t q[3];
        split_parts(j < cols ? in[static_cast<size_t>(r) * ld_in + j] : 0.0, q);
        for (int p = 0; p < nparts; ++p) out[rowo + static_cast<size_t>(p) * ka_pad + j] = q[p];
    }
}

// diag[k] = sum_j G[k][j]^2 = sum phi_k^2 w = C_kk (eq. 16 on the diagonal),
// one warp per atom, fp64.  The largest diagonal entry of the non-duplicate
// atoms is accumulated in *dmax as an unsigned 64-bit maximum (non-negative
// doubles order like their bit patterns); *dmax must start at 0.
__global__ void diag_kernel(const double *__restrict__ G, int ldg, int K, int Kp, int nA,
                            const uint8_t *__restrict__ dup, double *__restrict__ diag,
                            unsigned long long *__restrict__ dmax)
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
    if (lane == 0) {
        diag[k] = acc;
        if (k < K && !dup[k]) atomicMax(dmax, static_cast<unsigned long long>(__double_as_longlong(acc)));
    }
}

// Admissibility and the per-atom constants of eqs. (17)-(19): atom k may be
// selected if k < K, it is not a collinear duplicate of a lower index, and
// C_kk > 1e-14 max_j C_jj.  invC = 1/C_kk (0 if inadmissible), D = 1/sqrt(C_kk)
// (NaN if inadmissible, so |R_k| D_k never wins a comparison).
template <typename T>
__global__ void finalize_kernel(const double *__restrict__ diag, const uint8_t *__restrict__ dup,
                                const unsigned long long *__restrict__ dmax, int K, int Kp,
                                T *__restrict__ invC, T *__restrict__ Dk, int *__restrict__ n_adm)
{
    const double mx = __longlong_as_double(static_cast<long long>(*dmax));
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    bool adm = false;
    if (k < Kp) {
        const double d = k < K ? diag[k] : 0.0;
        adm = k < K && !dup[k] && mx > 0.0 && d > 1e-14 * mx;
        invC[k] = adm ? static_cast<T>(1.0 / d) : static_cast<T>(0);
        Dk[k] = adm ? static_cast<T>(1.0 / sqrt(d)) : static_cast<T>(NAN);
    }
    const unsigned cnt = __popc(__ballot_sync(0xffffffffu, adm));
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(n_adm, static_cast<int>(cnt));
}

// Plain tiled GEMM on CUDA cores: D[m][n] = sum_k A[m][k] B[n][k], 64 x 64
// tiles, 256 threads with 4 x 4 outputs each.  symmetric: upper tiles of a
// square D, stored mirrored (each entry written once); otherwise D is
// stored transposed, out[n * ldo + m].
template <typename T>
__global__ void __launch_bounds__(256)
simt_gemm_kernel(const T *__restrict__ A, int lda, const T *__restrict__ B, int ldb, int M, int N,
                 int Kd, T *__restrict__ out, long long ldo, int symmetric, int mt,
                 const long long *__restrict__ out_rows, const int *__restrict__ n_dev)
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
    if (n_dev) {
        const int nd = *n_dev;
        N = nd < N ? nd : N;
        if (tn * 64 >= N) return;
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
                out[(out_rows ? out_rows[n] : static_cast<long long>(n) * ldo) + m] = acc[i][j];
            } else if (!diag_tile || n >= m) {
                out[static_cast<long long>(m) * ldo + n] = acc[i][j];
                out[static_cast<long long>(n) * ldo + m] = acc[i][j];
            }
        }
    }
}

// Seeded synthetic samples in [0, 255) for probe batches (a 32-bit integer
// hash of the element index and the seed; no dependence on the method).
__global__ void probe_samples_kernel(double *s, long long total, uint32_t seed)
{
    const long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x;
    if (i >= total) return;
    uint32_t h = static_cast<uint32_t>(i) * 0x9E3779B1u ^ (static_cast<uint32_t>(i >> 32) + seed) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    s[i] = 255.0 * static_cast<double>(h >> 8) / 16777216.0;
}

}  // namespace

cudaError_t launch_pack_x(const BlockDesc *blocks, int n, const int *a_idx, const double *sqrtw,
                          int nA, int ka_pad, int nparts, int MN, uint16_t *x_bf16, double *x_f64,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const size_t per_warp = sizeof(double) * static_cast<size_t>(MN);
    if (per_warp <= 48 * 1024) {
        int warps = static_cast<int>(96 * 1024 / per_warp);
        warps = warps < 1 ? 1 : (warps > 8 ? 8 : warps);
        const size_t smem = per_warp * warps;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(pack_x_staged_kernel,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem));
            if (e != cudaSuccess) return e;
        }
        pack_x_staged_kernel<<<(n + warps - 1) / warps, 32 * warps, smem, st>>>(
            blocks, n, a_idx, sqrtw, nA, ka_pad, nparts, MN, x_bf16, x_f64);
    } else {
        pack_x_kernel<<<n, 256, 0, st>>>(blocks, a_idx, sqrtw, nA, ka_pad, nparts, x_bf16, x_f64);
    }
    return cudaGetLastError();
}

cudaError_t launch_split_bf16(const double *in, int rows, int cols, int ld_in, int ka_pad,
                              int nparts, uint16_t *out, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    split_bf16_kernel<<<rows, 256, 0, st>>>(in, cols, ld_in, ka_pad, nparts, out);
    return cudaGetLastError();
}

cudaError_t launch_tables_diag(const double *G64, int ldg, int K, int Kp, int nA, const uint8_t *dup,
                               double *diag, unsigned long long *dmax, int *n_adm, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(dmax, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_adm, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    diag_kernel<<<(Kp + 7) / 8, 256, 0, st>>>(G64, ldg, K, Kp, nA, dup, diag, dmax);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_tables_finalize(const double *diag, const uint8_t *dup,
                                   const unsigned long long *dmax, int K, int Kp, T *invC, T *Dk,
                                   int *n_admissible, cudaStream_t st)
{
    finalize_kernel<T><<<(Kp + 255) / 256, 256, 0, st>>>(diag, dup, dmax, K, Kp, invC, Dk, n_admissible);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_simt_gemm_ex(const T *A, int lda, const T *B, int ldb, int M, int N, int Kd,
                                T *out, long long ldo, const long long *out_rows, const int *n_dev,
                                cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int mt = (M + 63) / 64, nt = (N + 63) / 64;
    simt_gemm_kernel<T><<<mt * nt, 256, 0, st>>>(A, lda, B, ldb, M, N, Kd, out, ldo, 0, mt, out_rows,
                                                  n_dev);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_simt_gemm(const T *A, int lda, const T *B, int ldb, int M, int N, int Kd, T *out,
                             long long ldo, int symmetric, cudaStream_t st)
{
    if (M <= 0 || N <= 0) return cudaSuccess;
    const int mt = (M + 63) / 64, nt = (N + 63) / 64;
    const int grid = symmetric ? mt * (mt + 1) / 2 : mt * nt;
    simt_gemm_kernel<T><<<grid, 256, 0, st>>>(A, lda, B, ldb, M, N, Kd, out, ldo, symmetric, mt,
                                              nullptr, nullptr);
    return cudaGetLastError();
}

template cudaError_t launch_tables_finalize<float>(const double *, const uint8_t *,
                                                   const unsigned long long *, int, int, float *,
                                                   float *, int *, cudaStream_t);
template cudaError_t launch_tables_finalize<double>(const double *, const uint8_t *,
                                                    const unsigned long long *, int, int, double *,
                                                    double *, int *, cudaStream_t);
template cudaError_t launch_simt_gemm<double>(const double *, int, const double *, int, int, int, int,
                                              double *, long long, int, cudaStream_t);
template cudaError_t launch_simt_gemm<float>(const float *, int, const float *, int, int, int, int,
                                             float *, long long, int, cudaStream_t);
template cudaError_t launch_simt_gemm_ex<double>(const double *, int, const double *, int, int, int,
                                                 int, double *, long long, const long long *,
                                                 const int *, cudaStream_t);

cudaError_t launch_probe_samples(double *s, long long total, uint32_t seed, cudaStream_t st)
{
    if (total <= 0) return cudaSuccess;
    probe_samples_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, st>>>(s, total, seed);
    return cudaGetLastError();
}

namespace {

__global__ void fill_desc_kernel(BlockDesc *d, int n, StridedSpec s, int MN)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    BlockDesc x;
    x.samples = s.samples + static_cast<size_t>(MN) * b;
    x.support = nullptr;
    x.out = s.out + static_cast<size_t>(MN) * b;
    x.sel_idx = s.sel_idx ? s.sel_idx + static_cast<size_t>(s.I) * b : nullptr;
    x.sel_coef = s.sel_coef ? s.sel_coef + static_cast<size_t>(s.I) * s.coef * b : nullptr;
    x.iterations = s.I;
    x.pad_ = 0;
    d[b] = x;
}

}  // namespace

cudaError_t launch_fill_desc(BlockDesc *d, int n, const StridedSpec &s, int MN, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    fill_desc_kernel<<<(n + 255) / 256, 256, 0, st>>>(d, n, s, MN);
    return cudaGetLastError();
}

namespace {

// The device failure path, exercised on purpose: one thread waits on an
// mbarrier that nothing arrives at; the bounded wait gives up after limit_ns,
// the kernel records the timeout in the status word and returns.
__global__ void wait_probe_kernel(int *err, unsigned long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    const uint32_t m = static_cast<uint32_t>(__cvta_generic_to_shared(&bar));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(m) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!dev::bar_wait(&bar, 0, limit_ns)) atomicOr(err, 1 << DEV_ERR_WAIT_TIMEOUT);
}

// The projection kernels' fp64 -> fp32 sample conversion applied to n values,
// and (back != NULL) the model kernels' fp32 -> fp64 output conversion of the
// results.
__global__ void convert_probe_kernel(const double *in, float *out, double *back, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float f = dev::f64_to_f32_rn(in[i]);
        out[i] = f;
        if (back) back[i] = dev::f32_to_f64(f);
    }
}

}  // namespace

cudaError_t launch_convert_probe(const double *in, float *out, double *back, int n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int grid = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    convert_probe_kernel<<<grid, 256, 0, st>>>(in, out, back, n);
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(int *err, unsigned long long limit_ns, cudaStream_t st)
{
    wait_probe_kernel<<<1, 32, 0, st>>>(err, limit_ns);
    return cudaGetLastError();
}

}  // namespace se
