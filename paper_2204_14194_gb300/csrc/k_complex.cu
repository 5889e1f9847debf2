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
// shared memory; rows of C stream from L2 with coalesced loads.  For DFT
// atoms the table is not needed: C(k,u) = sum w exp(j 2 pi ((mu_u - mu_k) m / M
// + (eta_u - eta_k) n / N)) / MN is one value of the 2-D DFT of w (Sec. VI),
// held in shared memory (What).
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "se_internal.h"

namespace se {
namespace {

template <typename T> struct CandC { T s; int k; T rr, ri; };

// W warps per block (W = 1: each warp its own block).  Candidates of the
// argmax carry R_u, so one barrier per iteration suffices: the reduction
// slots alternate between iterations, and every thread updates only its own
// atoms k = tid + 32 W j.
template <typename T, int W>
__global__ void __launch_bounds__(256) iterate_cplx_kernel(const IterArgs a, int bpc)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int NT = 32 * W;
    const int g = threadIdx.x / NT, tid = threadIdx.x % NT, lane = threadIdx.x & 31, warp = tid >> 5;
    const int Kp = a.Kp, K = a.K;
    // DFT plans: the DFT of w (Sec. VI), [2][MN], first in shared memory, for the whole CTA
    const int MNd = a.What ? a.Mdft * a.Ndft : 0;
    T *Wr = reinterpret_cast<T *>(smem), *Wi = Wr + MNd;
    for (int i = threadIdx.x; i < 2 * MNd; i += blockDim.x) Wr[i] = static_cast<const T *>(a.What)[i];
    const size_t per = 2 * static_cast<size_t>(Kp) + 2 * static_cast<size_t>(a.I_max);
    T *Rr = Wr + 2 * MNd + static_cast<size_t>(g) * per;
    T *Ri = Rr + Kp;
    T *lc = Ri + Kp;                                                        // [I_max][2]
    int *lu = reinterpret_cast<int *>(Wr + 2 * MNd + static_cast<size_t>(bpc) * per) + static_cast<size_t>(g) * a.I_max;
    const uintptr_t after_logs = reinterpret_cast<uintptr_t>(
        reinterpret_cast<int *>(Wr + 2 * MNd + static_cast<size_t>(bpc) * per) + static_cast<size_t>(bpc) * a.I_max);
    CandC<T> *red = reinterpret_cast<CandC<T> *>((after_logs + 15) & ~static_cast<uintptr_t>(15)) +
                    static_cast<size_t>(g) * 2 * W;                          // [2][W], 16-byte aligned
    __syncthreads();
    const T *C = static_cast<const T *>(a.C);
    const T *invC = static_cast<const T *>(a.invC);
    const T gamma = static_cast<T>(a.gamma);
    auto sync_block = [&]() {
        if constexpr (W == 1) __syncwarp(); else __syncthreads();
    };

    for (int b0 = blockIdx.x * bpc; b0 < a.n; b0 += gridDim.x * bpc) {
        const int b = b0 + g;
        const bool live = b < a.n;     // W > 1 runs one block per CTA (bpc = 1), so live holds
        if (!live) continue;
        const BlockDesc bd = a.blocks[b];
        const int I = bd.iterations;
        const T *R0 = static_cast<const T *>(a.R0) + static_cast<size_t>(b) * 2 * Kp;
        for (int k = tid; k < Kp; k += NT) {
            Rr[k] = R0[k];
            Ri[k] = R0[Kp + k];
        }
        for (int nu = 0; nu < I; ++nu) {
            // eq. (18): argmax |R_k|^2 / C_kk over admissible k, ties to the smallest k
            T best = T(-1), br = T(0), bi = T(0);
            int kb = INT_MAX;
            for (int k = tid; k < K; k += NT) {
                const T ic = invC[k];
                const T s = ic > T(0) ? (Rr[k] * Rr[k] + Ri[k] * Ri[k]) * ic : T(-1);
                if (s > best) { best = s; kb = k; br = Rr[k]; bi = Ri[k]; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const T ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int ok = __shfl_xor_sync(0xffffffffu, kb, off);
                const T orr = __shfl_xor_sync(0xffffffffu, br, off);
                const T oii = __shfl_xor_sync(0xffffffffu, bi, off);
                if (ob > best || (ob == best && ok < kb)) { best = ob; kb = ok; br = orr; bi = oii; }
            }
            if constexpr (W > 1) {
                CandC<T> *slot = red + (nu & 1) * W;
                if (lane == 0) slot[warp] = CandC<T>{best, kb, br, bi};
                __syncthreads();
                best = slot[0].s; kb = slot[0].k; br = slot[0].rr; bi = slot[0].ri;
#pragma unroll
                for (int w2 = 1; w2 < W; ++w2) {
                    const CandC<T> c = slot[w2];
                    if (c.s > best || (c.s == best && c.k < kb)) { best = c.s; kb = c.k; br = c.rr; bi = c.ri; }
                }
            }
            int u = kb;
            if (u < 0 || u >= K) {
                if (tid == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
                u = 0;
                br = bi = T(0);
            }
            // eq. (19): c = gamma R_u / C_uu (complex); R_u came with the candidate
            const T ic = invC[u];
            const T cr = gamma * br * ic, ci = gamma * bi * ic;
            if (tid == 0) {
                lu[nu] = u;
                lc[2 * nu] = cr;
                lc[2 * nu + 1] = ci;
            }
            // eq. (20): R_k -= c C(k, u), each thread on its own atoms
            if (MNd) {
                // C(k, u) of DFT atoms depends on the frequency difference only
                const int N = a.Ndft, M = a.Mdft;
                const int mu_u = u / N, eta_u = u - (u / N) * N;
                int mu = tid / N, eta = tid - (tid / N) * N;   // of k = tid, advanced by NT below
                for (int k = tid; k < K; k += NT) {
                    int dm = mu - mu_u, dn = eta - eta_u;
                    dm += dm < 0 ? M : 0;
                    dn += dn < 0 ? N : 0;
                    const T xr = Wr[dm * N + dn], xi = Wi[dm * N + dn];
                    Rr[k] -= cr * xr - ci * xi;
                    Ri[k] -= cr * xi + ci * xr;
                    eta += NT;
                    while (eta >= N) { eta -= N; ++mu; }
                }
            } else {
                const T *row = C + static_cast<size_t>(u) * 2 * Kp;
                for (int k = tid; k < Kp; k += NT) {
                    const T xr = row[k], xi = row[Kp + k];
                    Rr[k] -= cr * xr - ci * xi;
                    Ri[k] -= cr * xi + ci * xr;
                }
            }
            if constexpr (W == 1) __syncwarp();
        }
        sync_block();   // the log is complete
        // eq. (9) on the loss pixels, real part; support pixels keep their samples
        const T *PhiB = static_cast<const T *>(a.PhiB);
        for (int j = tid; j < a.nB; j += NT) {
            T gv = T(0);
            for (int nu = 0; nu < I; ++nu) {
                const T *pr = PhiB + static_cast<size_t>(lu[nu]) * 2 * a.nB;
                gv += lc[2 * nu] * pr[j] - lc[2 * nu + 1] * pr[a.nB + j];
            }
            bd.out[a.b_idx[j]] = static_cast<double>(gv);
        }
        for (int p = tid; p < a.MN; p += NT)
            if (a.pat_support[p]) bd.out[p] = bd.samples[p];
        if (bd.sel_idx)
            for (int nu = tid; nu < I; nu += NT) bd.sel_idx[nu] = lu[nu];
        if (bd.sel_coef)
            for (int nu = tid; nu < I; nu += NT) {
                bd.sel_coef[2 * nu] = static_cast<double>(lc[2 * nu]);
                bd.sel_coef[2 * nu + 1] = static_cast<double>(lc[2 * nu + 1]);
            }
        sync_block();   // the log and R are read before the next block overwrites them
    }
}

}  // namespace

template <typename T, int W>
cudaError_t launch_cplx_w(const IterArgs &a, cudaStream_t st)
{
    const size_t per_block = sizeof(T) * (2 * static_cast<size_t>(a.Kp) + 2 * static_cast<size_t>(a.I_max)) +
                             sizeof(int) * static_cast<size_t>(a.I_max) + sizeof(CandC<T>) * 2 * W;
    const size_t shared = a.What ? sizeof(T) * 2 * static_cast<size_t>(a.Mdft) * a.Ndft : 0;
    int bpc = W == 1 ? 8 : 1;   // blocks per CTA (one warp each when W = 1)
    while (bpc > 1 && shared + per_block * bpc > 200 * 1024) bpc /= 2;
    const size_t smem = shared + per_block * bpc + 64;
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    auto kern = iterate_cplx_kernel<T, W>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * W * bpc, smem)) != cudaSuccess) return e;
    const int need = (a.n + bpc - 1) / bpc;
    const int cap = sms * (per_sm > 0 ? per_sm : 1);
    kern<<<need < cap ? need : cap, 32 * W * bpc, smem, st>>>(a, bpc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_iterate_cplx(const IterArgs &a, cudaStream_t st)
{
    if (a.n <= 0) return cudaSuccess;
    // large dictionaries: 4 warps share a block's R (more resident warps per SM)
    return a.Kp >= 2048 ? launch_cplx_w<T, 4>(a, st) : launch_cplx_w<T, 1>(a, st);
}

template cudaError_t launch_iterate_cplx<float>(const IterArgs &, cudaStream_t);
template cudaError_t launch_iterate_cplx<double>(const IterArgs &, cudaStream_t);

}  // namespace se
