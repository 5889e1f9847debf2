// k_model.cuh -- the model of eq. (9) on the loss box of one block, for
// separable dictionaries, on the tensor cores: the body shared by the model
// kernel (one warp per block after the iterations) and the parity-class
// iteration kernel that evaluates the model itself once a block's iterations
// are done.  Both run the same operations in the same order, so their outputs
// are the same bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "k_device.cuh"
#include "se_internal.h"

namespace se {
namespace dev {

// On the loss box (Mb x Nb, at most 32 x 32) the model is a matrix product
// G = A B^T over the log entries nu: A[i][nu] = c_nu t_p[m0 + i] (p the atom's
// row index) and B[j][nu] = t'_q[n0 + j], taken in steps of 8 entries as
// mma.sync m16n8k8 products in split TF32 (x_s y_b + x_b y_s + x_b y_b, about
// 2^-21 relative, like fp32 sums; the small products accumulate apart from the
// large one), MT x NT output tiles of 16 x 8.  Ts (shared or
// global memory) holds the 1-D rows of the transforms as ModelLayout says.  The
// block's log (written by its iteration kernel) is read 32 entries at a time,
// the next 32 in flight, through the warp's table Etab (32 entries); the
// caller's copies of the log are written on the way.  The output tile passes
// through Gt (16 MT x (8 NT + 1) floats) so that the stores to the output are
// whole row segments: the output may be host memory reached over the host
// link, where short scattered writes are slow.  Only the loss pixels of the
// pattern are written.
// Where Ts holds the 1-D rows: t_p[m] of transform t at aoff + t a_t + p a_p + m
// and t'_q[n] at boff + t b_t + q b_q + n (only the rows and columns of the loss
// box are read).
struct ModelLayout {
    int aoff, a_t, a_p;
    int boff, b_t, b_q;
};

// The layout of the whole rows: T_t[p][m] at t (M M + N N) + p M + m, then
// T'_t[q][n] at t (M M + N N) + M M + q N + n.
__host__ __device__ inline ModelLayout model_full_layout(int M, int N)
{
    return ModelLayout{0, M * M + N * N, M, M * M, M * M + N * N, N};
}

template <int MT, int NT>
__device__ __forceinline__ void model_tc_block(const IterArgs &a, const SepArgs &s, const float *Ts,
                                               const ModelLayout &L, int4 *Etab, float *Gt, int b, int m0, int Mb,
                                               int n0, int Nb, int lane)
{
    const int M = s.M, N = s.N, MN = M * N;
    const int lgN = (N & (N - 1)) == 0 ? __ffs(N) - 1 : -1;   // atom index split by a shift when N = 2^j
    constexpr int GP = 8 * NT + 1;   // pitch of the output tile (padded)
    const int g = lane >> 2, q = lane & 3;
    // rows of the A fragments and columns of the B fragments (clamped into the
    // area; the clamped lanes compute values that are not stored)
    int ra[MT][2], cb[NT];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) ra[mt][h] = min(m0 + 16 * mt + g + 8 * h, M - 1);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) cb[nt] = min(n0 + 8 * nt + g, N - 1);

    const BlockDesc bd = a.blocks[b];
    const int I = bd.iterations;
    const int *lu = a.log_u + static_cast<size_t>(b) * a.I_max;
    const float *lc = a.log_c + static_cast<size_t>(b) * a.I_max;
    // the large-part products x_b y_b and the two small-part products in separate
    // accumulators (two independent chains of tensor-core products per tile),
    // added once at the end
    float acc[MT][NT][4], acs[MT][NT][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[mt][nt][k] = acs[mt][nt][k] = 0.0f;
    int un = lane < I ? lu[lane] : -1;
    float cn = lane < I ? lc[lane] : 0.0f;
    for (int nu0 = 0; nu0 < I; nu0 += 32) {
        int u = un;
        const float cl = cn;
        if (nu0 + 32 + lane < I) {
            un = lu[nu0 + 32 + lane];
            cn = lc[nu0 + 32 + lane];
        }
        if (nu0 + lane < I) {
            if (bd.sel_idx) bd.sel_idx[nu0 + lane] = u;
            if (bd.sel_coef) bd.sel_coef[nu0 + lane] = f32_to_f64(cl);
        }
        float cf = 0.0f;   // padded entries add 0
        if (nu0 + lane < I && u >= 0 && u < s.koff[s.ntr - 1] + MN) cf = cl;
        else u = 0;
        const int t = (s.ntr > 1 && u >= s.koff[1]) ? 1 : 0;
        const int ku = u - s.koff[t];
        const int pu = lgN >= 0 ? ku >> lgN : ku / N, qu = lgN >= 0 ? ku & (N - 1) : ku - pu * N;
        __syncwarp();   // the previous round's reads of the table are done
        Etab[lane] = make_int4(L.aoff + t * L.a_t + pu * L.a_p, L.boff + t * L.b_t + qu * L.b_q, __float_as_int(cf), 0);
        __syncwarp();
        const int steps = (min(32, I - nu0) + 7) >> 3;
        constexpr int UF = MT * NT <= 2 ? 2 : 1;   // two steps in flight where the registers allow
#pragma unroll UF
        for (int ks = 0; ks < steps; ++ks) {
            const int4 e0 = Etab[8 * ks + q], e1 = Etab[8 * ks + q + 4];
            const float c0 = __int_as_float(e0.z), c1 = __int_as_float(e1.z);
            uint32_t bb[NT][2], bs[NT][2];
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                split_tf32(Ts[e0.y + cb[nt]], bb[nt][0], bs[nt][0]);
                split_tf32(Ts[e1.y + cb[nt]], bb[nt][1], bs[nt][1]);
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt) {
                uint32_t ab[4], as[4];
                split_tf32(c0 * Ts[e0.x + ra[mt][0]], ab[0], as[0]);
                split_tf32(c0 * Ts[e0.x + ra[mt][1]], ab[1], as[1]);
                split_tf32(c1 * Ts[e1.x + ra[mt][0]], ab[2], as[2]);
                split_tf32(c1 * Ts[e1.x + ra[mt][1]], ab[3], as[3]);
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) {
                    mma_tf32(acs[mt][nt], as, bb[nt][0], bb[nt][1]);
                    mma_tf32(acs[mt][nt], ab, bs[nt][0], bs[nt][1]);
                    mma_tf32(acc[mt][nt], ab, bb[nt][0], bb[nt][1]);
                }
            }
        }
    }
    // C fragments (g, 2q), (g, 2q + 1), (g + 8, 2q), (g + 8, 2q + 1) of each tile
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                Gt[(16 * mt + g + 8 * (k >> 1)) * GP + 8 * nt + 2 * q + (k & 1)] = acc[mt][nt][k] + acs[mt][nt][k];
    __syncwarp();
    // 32 / (8 NT) rows of the box per pass, a lane per column
    constexpr int CW = 8 * NT, RPP = 32 / CW;
    const int jr = lane / CW, j = lane % CW;
    if (j < Nb) {
        for (int i = jr; i < Mb; i += RPP) {
            const int p = (m0 + i) * N + n0 + j;
            if (!a.pat_support[p]) bd.out[p] = f32_to_f64(Gt[i * GP + j]);
        }
    }
    __syncwarp();   // the tile is read before the next block overwrites it
}

// Floats of a warp's output tile for MT x NT tiles.
__host__ __device__ constexpr int model_tile_floats(int MT, int NT) { return 16 * MT * (8 * NT + 1); }

}  // namespace dev
}  // namespace se
