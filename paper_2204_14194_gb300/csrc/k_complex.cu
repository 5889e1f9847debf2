// k_complex.cu -- FaSE iterations for complex-valued atoms (the paper's
// general case, Sec. III): R_k and C(k,u) are complex, the selection of
// eq. (18) takes |R_k|^2 / C_kk, the coefficient of eq. (19) is complex and
// the update of eq. (20) subtracts c C(k,u).  Samples are real; the model
// g = sum c phi_u (eq. 9) is complex and its real part replaces the loss
// area (the output of a real image).
//
// Layouts (T = float in the fp32 form, double in the fp64 form):
//   R0  [n][2][Kp]   real plane then imaginary plane of R^(0) per block
//   C   [Kp][2][Kp]  row u = (Re, Im) of C(k, u) for all k (eq. 16,
//                    C(k, u) = sum conj(phi_k) w phi_u, Hermitian)
//   invC [Kp]        1 / C_kk, 0 for inadmissible atoms (never selected)
//   PhiB [Kp][2][nB] the atoms on the pattern's loss pixels
// One warp per block; the block's R planes and its selection log live in
// shared memory; rows of C stream from L2 with coalesced loads.
#include <cuda_runtime.h>

#include <climits>

#include "se_internal.h"

namespace se {
namespace {

template <typename T>
__global__ void __launch_bounds__(256) iterate_cplx_kernel(const IterArgs a, int wpc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Kp = a.Kp, K = a.K;
    T *Rr = reinterpret_cast<T *>(smem) + static_cast<size_t>(warp) * (2 * Kp + 2 * a.I_max);
    T *Ri = Rr + Kp;
    T *lc = Ri + Kp;                                  // [I_max][2] coefficients
    int *lu = reinterpret_cast<int *>(reinterpret_cast<T *>(smem) + static_cast<size_t>(wpc) * (2 * Kp + 2 * a.I_max)) +
              static_cast<size_t>(warp) * a.I_max;
    const T *C = static_cast<const T *>(a.C);
    const T *invC = static_cast<const T *>(a.invC);
    const T gamma = static_cast<T>(a.gamma);

    for (int b = blockIdx.x * wpc + warp; b < a.n; b += gridDim.x * wpc) {
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const T *R0 = static_cast<const T *>(a.R0) + static_cast<size_t>(b) * 2 * Kp;
        for (int k = lane; k < Kp; k += 32) {
            Rr[k] = R0[k];
            Ri[k] = R0[Kp + k];
        }
        __syncwarp();
        for (int nu = 0; nu < I; ++nu) {
            // eq. (18): argmax |R_k|^2 / C_kk over admissible k, ties to the smallest k
            T best = T(-1);
            int kb = INT_MAX;
            for (int k = lane; k < K; k += 32) {
                const T ic = invC[k];
                const T s = ic > T(0) ? (Rr[k] * Rr[k] + Ri[k] * Ri[k]) * ic : T(-1);
                if (s > best) { best = s; kb = k; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int ok = __shfl_xor_sync(0xffffffffu, kb, off);
                if (ob > best || (ob == best && ok < kb)) { best = ob; kb = ok; }
            }
            int u = kb;
            if (u < 0 || u >= K) {
                if (lane == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
            }
            // eq. (19): c = gamma R_u / C_uu (complex)
            const T ic = invC[u];
            const T cr = gamma * Rr[u] * ic, ci = gamma * Ri[u] * ic;
            if (lane == 0) {
                lu[nu] = u;
                lc[2 * nu] = cr;
                lc[2 * nu + 1] = ci;
            }
            __syncwarp();   // every lane has read R_u before the update below
            // eq. (20): R_k -= c C(k, u)
            const T *row = C + static_cast<size_t>(u) * 2 * Kp;
            for (int k = lane; k < Kp; k += 32) {
                const T xr = row[k], xi = row[Kp + k];
                Rr[k] -= cr * xr - ci * xi;
                Ri[k] -= cr * xi + ci * xr;
            }
            __syncwarp();
        }
        // eq. (9) on the loss pixels, real part; support pixels keep their samples
        const T *PhiB = static_cast<const T *>(a.PhiB);
        for (int j = lane; j < a.nB; j += 32) {
            T g = T(0);
            for (int nu = 0; nu < I; ++nu) {
                const T *pr = PhiB + static_cast<size_t>(lu[nu]) * 2 * a.nB;
                g += lc[2 * nu] * pr[j] - lc[2 * nu + 1] * pr[a.nB + j];
            }
            bd.out[a.b_idx[j]] = static_cast<double>(g);
        }
        for (int p = lane; p < a.MN; p += 32)
            if (a.pat_support[p]) bd.out[p] = bd.samples[p];
        if (bd.sel_idx)
            for (int nu = lane; nu < I; nu += 32) bd.sel_idx[nu] = lu[nu];
        if (bd.sel_coef)
            for (int nu = lane; nu < I; nu += 32) {
                bd.sel_coef[2 * nu] = static_cast<double>(lc[2 * nu]);
                bd.sel_coef[2 * nu + 1] = static_cast<double>(lc[2 * nu + 1]);
            }
        __syncwarp();   // the log is read before the next block overwrites it
    }
}

}  // namespace

template <typename T>
cudaError_t launch_iterate_cplx(const IterArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    const size_t per_warp = sizeof(T) * (2 * static_cast<size_t>(a.Kp) + 2 * static_cast<size_t>(a.I_max)) +
                            sizeof(int) * static_cast<size_t>(a.I_max);
    int wpc = 8;
    while (wpc > 1 && per_warp * wpc > 200 * 1024) wpc /= 2;
    const size_t smem = per_warp * wpc + 16;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(iterate_cplx_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, iterate_cplx_kernel<T>, 32 * wpc, smem)) !=
        cudaSuccess)
        return e;
    const int need = (a.n + wpc - 1) / wpc;
    const int grid = need < sms * (per_sm > 0 ? per_sm : 1) ? need : sms * (per_sm > 0 ? per_sm : 1);
    iterate_cplx_kernel<T><<<grid, 32 * wpc, smem, st>>>(a, wpc);
    return cudaGetLastError();
}

template cudaError_t launch_iterate_cplx<float>(const IterArgs &, cudaStream_t);
template cudaError_t launch_iterate_cplx<double>(const IterArgs &, cudaStream_t);

}  // namespace se
