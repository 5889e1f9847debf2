// k_lazy.cu -- Fast Selective Extrapolation with per-block weighting patterns.
//
// When every block has its own support mask, the table C of eq. (16) is
// different for every block and building it whole (Alg. 2) would cost
// 2 K^2 |A| per block.  This path builds only what the iterations use:
//   * R^(0)_b = Phi (rho m_b s_b)          (eq. 12, one GEMM over the batch)
//   * C_b(k, k) = (Phi^2 rho) m_b          (eq. 16 diagonal, one GEMM)
//   * C_b(:, u) = (Phi rho)(m_b phi_u)     (eq. 16 column, on the first
//                                           selection of atom u by block b,
//                                           batched over the blocks that
//                                           need one in the same round)
// Columns are cached per block, so an atom selected again costs nothing.
// The iterations advance in lock-step rounds over the batch: a round kernel
// applies the previous update (eq. 20), selects (eq. 18) and records the
// coefficient (eq. 19), and queues a column request when the selected atom
// has no cached column; a packing kernel and a GEMM whose tiles past the
// device-side request count exit at once serve the requests before the next
// round.  Projections are kept D-scaled (R'_k = R_k D_b,k) as in the full
// path.  The model on the block's loss pixels is evaluated at the end.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "k_device.cuh"
#include "se_internal.h"

namespace se {
namespace {

template <typename T> __device__ __forceinline__ T nan_of();
template <> __device__ __forceinline__ float nan_of<float>() { return __int_as_float(0x7fc00000); }
template <> __device__ __forceinline__ double nan_of<double>() { return __longlong_as_double(0x7ff8000000000000ll); }

__device__ __forceinline__ uint16_t bf16b(float v)
{
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<const uint16_t *>(&h);
}
__device__ __forceinline__ float bf16f(uint16_t b) { return __uint_as_float(static_cast<uint32_t>(b) << 16); }

// Exact-enough split of a double into three bf16 parts (same rule as the
// shared-pattern packing; see k_simt.cu).
__device__ __forceinline__ void split3(double x, uint16_t (&p)[3])
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t sign = static_cast<uint32_t>(b >> 32) & 0x80000000u;
    const int e = static_cast<int>((b >> 52) & 0x7FF);
    const int ef = e - 1023 + 127;
    float hi, lo;
    if (e == 0 || e == 0x7FF || ef <= 0 || ef >= 255) {
        hi = __double2float_rn(x);
        lo = 0.0f;
    } else {
        const unsigned long long mant = b & ((1ull << 52) - 1);
        hi = __uint_as_float(sign | (static_cast<uint32_t>(ef) << 23) | static_cast<uint32_t>(mant >> 29));
        const uint32_t rest = static_cast<uint32_t>(mant & ((1u << 29) - 1));
        const int es = e - 1075 + 127;
        const float scale = es >= 1 ? __uint_as_float(static_cast<uint32_t>(es) << 23) : 0.0f;
        lo = __uint_as_float(sign | __float_as_uint(static_cast<float>(rest) * scale));
    }
    p[0] = bf16b(hi);
    const float r = hi - bf16f(p[0]);
    p[1] = bf16b(r);
    p[2] = bf16b((r - bf16f(p[1])) + lo);
}

// x 2^s (s a power of two chosen by the plan so that |x 2^s| <= 2^14) as two
// fp16 parts h + l: y = fp32(x 2^s), h = fp16(y), l = fp16(y - h).  The two
// parts keep 22 significant bits; the products h h', h l', l h' then carry a
// relative error of about 2^-21 (the dropped l l' and the roundings).
__device__ __forceinline__ void split2h(double x, float scale, uint16_t (&p)[2])
{
    const float y = dev::f64_to_f32_rn(x) * scale;
    const __half h = __float2half_rn(y);
    const __half l = __float2half_rn(y - __half2float(h));
    p[0] = __half_as_ushort(h);
    p[1] = __half_as_ushort(l);
}

// Masked samples x_b[p] = m_b[p] s_b[p] (as 3 bf16 parts or fp64) and the
// mask itself as one exact bf16 part (1 or 0).  Rows are [part][MN_pad].
__global__ void lazy_pack_kernel(const BlockDesc *__restrict__ blocks, int MN, int MN_pad,
                                 uint16_t *__restrict__ xb, double *__restrict__ xd,
                                 uint16_t *__restrict__ mb, double *__restrict__ md)
{
    const int b = blockIdx.x;
    const double *s = blocks[b].samples;
    const uint8_t *m = blocks[b].support;
    for (int p = threadIdx.x; p < MN_pad; p += blockDim.x) {
        const bool in = p < MN && m[p];
        const double v = in ? s[p] : 0.0;
        if (xb) {
            uint16_t q[3];
            split3(v, q);
            for (int t = 0; t < 3; ++t) xb[(static_cast<size_t>(b) * 3 + t) * MN_pad + p] = q[t];
        }
        if (xd) xd[static_cast<size_t>(b) * MN_pad + p] = v;
        if (mb) mb[static_cast<size_t>(b) * MN_pad + p] = in ? 0x3F80 : 0;   // bf16 1.0 / 0.0
        if (md) md[static_cast<size_t>(b) * MN_pad + p] = in ? 1.0 : 0.0;
    }
}

// Column requests: v_j[p] = m_b[p] phi_u[p] for request j (block b, atom u),
// as three bf16 parts (vb), two scaled fp16 parts (vh) or fp64 (vd).
__global__ void lazy_pack_cols_kernel(const BlockDesc *__restrict__ blocks, const int *__restrict__ miss_n,
                                      const int *__restrict__ miss_blk, const int *__restrict__ cur_u,
                                      const double *__restrict__ Phi64, int MN, int MN_pad,
                                      uint16_t *__restrict__ vb, double *__restrict__ vd,
                                      uint16_t *__restrict__ vh, float hscale)
{
    const int j = blockIdx.x;
    if (j >= *miss_n) return;
    const int b = miss_blk[j];
    const int u = cur_u[b];
    const uint8_t *m = blocks[b].support;
    const double *phi = Phi64 + static_cast<size_t>(u) * MN;
    for (int p = threadIdx.x; p < MN_pad; p += blockDim.x) {
        const double v = (p < MN && m[p]) ? phi[p] : 0.0;
        if (vb) {
            uint16_t q[3];
            split3(v, q);
            for (int t = 0; t < 3; ++t) vb[(static_cast<size_t>(j) * 3 + t) * MN_pad + p] = q[t];
        }
        if (vh) {
            uint16_t q[2];
            split2h(v, hscale, q);
            vh[(static_cast<size_t>(j) * 2 + 0) * MN_pad + p] = q[0];
            vh[(static_cast<size_t>(j) * 2 + 1) * MN_pad + p] = q[1];
        }
        if (vd) vd[static_cast<size_t>(j) * MN_pad + p] = v;
    }
}

// Rows of a plan operand as two scaled fp16 parts: out[r][t][ka_pad].
__global__ void split_f16_kernel(const double *__restrict__ in, int cols, int ld_in, int ka_pad, float scale,
                                 uint16_t *__restrict__ out)
{
    const int r = blockIdx.x;
    for (int j = threadIdx.x; j < ka_pad; j += blockDim.x) {
        uint16_t q[2];
        split2h(j < cols ? in[static_cast<size_t>(r) * ld_in + j] : 0.0, scale, q);
        out[(static_cast<size_t>(r) * 2 + 0) * ka_pad + j] = q[0];
        out[(static_cast<size_t>(r) * 2 + 1) * ka_pad + j] = q[1];
    }
}

template <typename T>
__device__ __forceinline__ void block_argmax(T &s, int &k, T &r, Cand<T> *red)
{
    for (int o = 16; o > 0; o >>= 1) {
        const T so = __shfl_xor_sync(0xffffffffu, s, o);
        const int ko = __shfl_xor_sync(0xffffffffu, k, o);
        const T ro = __shfl_xor_sync(0xffffffffu, r, o);
        if (so > s || (so == s && ko < k)) { s = so; k = ko; r = ro; }
    }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0) red[warp] = Cand<T>{s, k, r};
    __syncthreads();
    s = red[0].s; k = red[0].k; r = red[0].r;
    for (int w = 1; w < nw; ++w) {
        const Cand<T> c = red[w];
        if (c.s > s || (c.s == s && c.k < k)) { s = c.s; k = c.k; r = c.r; }
    }
    __syncthreads();
}

// The lo part of a compensated pair hi + lo kept as fp16 in units of
// 2^(e - 24), e the exponent of hi: round to nearest gives |lo| <= 2^(e - 24),
// so the unit value lies in [-1, 1] and keeps 11 significant bits (hi + lo
// then carries about 35).  Zero where |hi| < 2^-100.
__device__ __forceinline__ uint16_t lo_encode(float hi, float lo)
{
    const int e = static_cast<int>((__float_as_uint(hi) >> 23) & 0xffu) - 127;
    if (e < -100) return 0;
    return __half_as_ushort(__float2half_rn(lo * __uint_as_float(static_cast<uint32_t>(127 + 24 - e) << 23)));
}
__device__ __forceinline__ float lo_decode(float hi, uint16_t q)
{
    const int e = static_cast<int>((__float_as_uint(hi) >> 23) & 0xffu) - 127;
    if (e < -100) return 0.0f;
    return __half2float(__ushort_as_half(q)) * __uint_as_float(static_cast<uint32_t>(127 - 24 + e) << 23);
}

// Per block: admissibility (not a duplicate, C_kk > 1e-14 max C_jj), D = 1 /
// sqrt(C_kk) (NaN if inadmissible) and R' = R0 D, in place.
template <typename T>
__global__ void lazy_init_kernel(LazyArgs a)
{
    __shared__ T red[32];
    const int b = blockIdx.x;
    const T *diag = static_cast<const T *>(a.diag) + static_cast<size_t>(b) * a.Kp;
    T *R = static_cast<T *>(a.R) + static_cast<size_t>(b) * a.Kp;
    T *D = static_cast<T *>(a.Dk) + static_cast<size_t>(b) * a.Kp;
    T mx = T(0);
    for (int k = threadIdx.x; k < a.K; k += blockDim.x)
        if (!a.dup[k]) mx = fmax(mx, diag[k]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = red[0];
    for (int w = 1; w < static_cast<int>(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    int cnt = 0;
    for (int k = threadIdx.x; k < a.Kp; k += blockDim.x) {
        const T d = diag[k];
        const bool adm = k < a.K && !a.dup[k] && mx > T(0) && d > T(1e-14) * mx;
        const T Dv = adm ? T(1) / sqrt(d) : nan_of<T>();
        D[k] = Dv;
        if (a.Rlo && sizeof(T) == 4) {
            // R' = R0 D as hi + lo (lo the product's exact rounding error)
            const float r0 = static_cast<float>(R[k]), dv = static_cast<float>(Dv);
            const float hi = r0 * dv;
            R[k] = static_cast<T>(hi);
            a.Rlo[static_cast<size_t>(b) * a.Kp + k] = lo_encode(hi, fmaf(r0, dv, -hi));
        } else {
            R[k] = R[k] * Dv;
        }
        a.slot_of[static_cast<size_t>(b) * a.Kp + k] = -1;
        cnt += adm;
    }
    cnt = __syncthreads_count(cnt > 0);
    if (threadIdx.x == 0) {
        a.n_slots[b] = cnt > 0 ? 0 : -1;       // -1: no admissible atom, block is skipped
        if (cnt == 0) atomicOr(a.err, 1 << DEV_ERR_EMPTY_SUPPORT);
    }
}

// One round nu for every block: R' -= c_prev D col(u_prev); select u; record
// c; request the column of u if it is not cached and another round follows.
// The recurrence R'_k -= c_prev D_k col_k of eq. (20).  In T, or, for long
// fp32 runs (a.Rlo set), compensated: R'_k = hi + lo and c = ch + cl as pairs
// of floats, updated with exact products (fma) and exact sums (two-sum) on the
// fp32 pipe, lo stored in 16 bits between rounds (about 35 significant bits in
// all); the product D_k col_k of two floats enters with its exact rounding
// error.  The selection compares the hi parts.
__device__ __forceinline__ float2 df_update(float2 r, float2 c, float col, float d)
{
    const float v = col * d, ev = fmaf(col, d, -v);          // v + ev = col d exactly
    const float p = c.x * v, pe = fmaf(c.x, v, -p);          // p + pe = ch v exactly
    const float corr = pe + fmaf(c.x, ev, c.y * v);          // the small terms of c (col d)
    const float s = r.x - p, bb = s - r.x;                    // two-sum of hi - p
    const float err = (r.x - (s - bb)) + (-p - bb);
    const float lo = (r.y - corr) + err;
    const float hi = s + lo;
    return make_float2(hi, lo - (hi - s));
}

template <typename T>
__global__ void lazy_round_kernel(LazyArgs a, int nu)
{
    __shared__ Cand<T> red[32];
    const bool df = a.Rlo != nullptr && sizeof(T) == 4;
    const int b = blockIdx.x;
    if (b == 0 && threadIdx.x == 0) a.miss_n[(nu + 1) & 1] = 0;   // unused since round nu - 1
    const int Ib = a.blocks[b].iterations;
    if (nu >= Ib || a.n_slots[b] < 0) return;
    T *R = static_cast<T *>(a.R) + static_cast<size_t>(b) * a.Kp;
    uint16_t *Rl = df ? a.Rlo + static_cast<size_t>(b) * a.Kp : nullptr;
    const T *D = static_cast<const T *>(a.Dk) + static_cast<size_t>(b) * a.Kp;
    int *slot_of = a.slot_of + static_cast<size_t>(b) * a.Kp;
    const T *col = nullptr;
    T cprev = T(0);
    float2 c2 = make_float2(0.0f, 0.0f);
    if (nu > 0) {
        const int up = a.cur_u[b];
        if (df) c2 = reinterpret_cast<const float2 *>(a.cur_c64)[b];
        else cprev = static_cast<const T *>(a.cur_c)[b];
        col = static_cast<const T *>(a.cache) +
              (static_cast<size_t>(b) * a.slots + slot_of[up]) * a.Kp;
    }
    T s = T(-1), rb = T(0);
    int kb = INT_MAX;
    for (int k = threadIdx.x; k < a.Kp; k += blockDim.x) {
        T r;
        if (df) {
            const float h = static_cast<float>(R[k]);
            float2 r2 = make_float2(h, lo_decode(h, Rl[k]));
            if (col) {
                r2 = df_update(r2, c2, static_cast<float>(col[k]), static_cast<float>(D[k]));
                R[k] = static_cast<T>(r2.x);
                Rl[k] = lo_encode(r2.x, r2.y);
            }
            r = static_cast<T>(r2.x);
        } else {
            r = R[k];
            if (col) {
                r = fma(-cprev, col[k] * D[k], r);
                R[k] = r;
            }
        }
        const T sc = fabs(r);
        if (sc > s) { s = sc; kb = k; rb = r; }
    }
    block_argmax<T>(s, kb, rb, red);
    int u = kb;
    if (u < 0 || u >= a.K) {
        if (threadIdx.x == 0) atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
        u = 0;
        rb = T(0);
    }
    if (threadIdx.x == 0) {
        T c;
        if (df) {
            // c = gamma R'_u D_u from the pair (the winner's lo part is in global
            // memory, written by this CTA before the barriers of the argmax)
            const float hu = static_cast<float>(R[u]);
            const float2 ru = (u == kb) ? make_float2(hu, lo_decode(hu, Rl[u])) : make_float2(0.0f, 0.0f);
            const double cd = a.gamma * (static_cast<double>(ru.x) + static_cast<double>(ru.y)) *
                              static_cast<double>(D[u]);
            const float ch = static_cast<float>(cd);
            reinterpret_cast<float2 *>(a.cur_c64)[b] = make_float2(ch, static_cast<float>(cd - ch));
            a.c_log64[static_cast<size_t>(b) * a.I_max + nu] = cd;
            c = static_cast<T>(ch);
        } else {
            c = static_cast<T>(a.gamma) * rb * D[u];
            static_cast<T *>(a.cur_c)[b] = c;
        }
        a.cur_u[b] = u;
        a.u_log[static_cast<size_t>(b) * a.I_max + nu] = u;
        static_cast<T *>(a.c_log)[static_cast<size_t>(b) * a.I_max + nu] = c;
        if (nu + 1 < Ib && slot_of[u] < 0) {
            const int sl = a.n_slots[b]++;
            if (sl >= a.slots) {
                atomicOr(a.err, 1 << DEV_ERR_LAZY_CACHE);
                a.n_slots[b] = -1;
            } else {
                slot_of[u] = sl;
                const int j = atomicAdd(a.miss_n + (nu & 1), 1);
                a.miss_blk[j] = b;
                a.miss_rows[j] = (static_cast<long long>(b) * a.slots + sl) * a.Kp;
            }
        }
    }
}

// The same round in fp32 with vector accesses: a worker of NW threads takes
// atoms 4 t + 4 NW j .. + 3 (float4 rows of D, the column and R' (its hi parts
// in the compensated form), four 16-bit lo parts as one uint2), two steps j per pass with every load of the pass
// issued before its first use, and the loads that do not need the cached
// column ahead of those that do.  Rows must be 16-byte aligned (the host
// checks).  Same arithmetic per atom as lazy_round_kernel, so the same results.
struct RoundRow {
    const float4 *D4;
    float4 *R4;
    uint2 *L4;   // lo parts of R', four per uint2 (compensated form)
    const float4 *C4;
    float cprev;
    float2 c2;
};

template <bool DF, int NW>
__device__ __forceinline__ void round_scan(const RoundRow &w, int q4, int t, float &s, int &kb, float &rb)
{
    for (int j0 = t; j0 < q4; j0 += 2 * NW) {
        float4 dv[2], cv[2], rv[2];
        uint2 lv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + NW * h;
            if (j < q4) {
                rv[h] = w.R4[j];
                if (DF) lv[h] = w.L4[j];
                if (w.C4) dv[h] = __ldg(w.D4 + j);
            }
        }
        if (w.C4) {
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (j0 + NW * h < q4) cv[h] = __ldg(w.C4 + j0 + NW * h);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + NW * h;
            if (j >= q4) continue;
            float r[4];
            if (DF) {
                const uint16_t lq[4] = {static_cast<uint16_t>(lv[h].x & 0xffffu), static_cast<uint16_t>(lv[h].x >> 16),
                                        static_cast<uint16_t>(lv[h].y & 0xffffu), static_cast<uint16_t>(lv[h].y >> 16)};
                const float hq[4] = {rv[h].x, rv[h].y, rv[h].z, rv[h].w};
                float2 p[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) p[e] = make_float2(hq[e], lo_decode(hq[e], lq[e]));
                if (w.C4) {
                    const float cc[4] = {cv[h].x, cv[h].y, cv[h].z, cv[h].w};
                    const float dd[4] = {dv[h].x, dv[h].y, dv[h].z, dv[h].w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) p[e] = df_update(p[e], w.c2, cc[e], dd[e]);
                    w.R4[j] = make_float4(p[0].x, p[1].x, p[2].x, p[3].x);
                    w.L4[j] = make_uint2(static_cast<uint32_t>(lo_encode(p[0].x, p[0].y)) |
                                             static_cast<uint32_t>(lo_encode(p[1].x, p[1].y)) << 16,
                                         static_cast<uint32_t>(lo_encode(p[2].x, p[2].y)) |
                                             static_cast<uint32_t>(lo_encode(p[3].x, p[3].y)) << 16);
                }
#pragma unroll
                for (int e = 0; e < 4; ++e) r[e] = p[e].x;
            } else {
                r[0] = rv[h].x; r[1] = rv[h].y; r[2] = rv[h].z; r[3] = rv[h].w;
                if (w.C4) {
                    r[0] = fmaf(-w.cprev, cv[h].x * dv[h].x, r[0]);
                    r[1] = fmaf(-w.cprev, cv[h].y * dv[h].y, r[1]);
                    r[2] = fmaf(-w.cprev, cv[h].z * dv[h].z, r[2]);
                    r[3] = fmaf(-w.cprev, cv[h].w * dv[h].w, r[3]);
                    w.R4[j] = make_float4(r[0], r[1], r[2], r[3]);
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float sc = fabsf(r[e]);
                if (sc > s) { s = sc; kb = 4 * j + e; rb = r[e]; }
            }
        }
    }
}

// Row pointers of block b for round nu (false: the block takes no round).
template <bool DF>
__device__ __forceinline__ bool round_row(const LazyArgs &a, int b, int nu, int &Ib, int &ns, RoundRow &w)
{
    Ib = a.blocks[b].iterations;
    ns = a.n_slots[b];
    if (nu >= Ib || ns < 0) return false;
    const size_t row = static_cast<size_t>(b) * a.Kp;
    w.D4 = reinterpret_cast<const float4 *>(static_cast<const float *>(a.Dk) + row);
    w.R4 = reinterpret_cast<float4 *>(static_cast<float *>(a.R) + row);
    w.L4 = DF ? reinterpret_cast<uint2 *>(a.Rlo + row) : nullptr;
    w.C4 = nullptr;
    w.cprev = 0.0f;
    w.c2 = make_float2(0.0f, 0.0f);
    if (nu > 0) {
        const int up = a.cur_u[b];
        if (DF) w.c2 = reinterpret_cast<const float2 *>(a.cur_c64)[b];
        else w.cprev = static_cast<const float *>(a.cur_c)[b];
        w.C4 = reinterpret_cast<const float4 *>(static_cast<const float *>(a.cache) +
                                                (static_cast<size_t>(b) * a.slots + a.slot_of[row + up]) * a.Kp);
    }
    return true;
}

// Selection bookkeeping of one block (one thread): the coefficient of eq. (19),
// the logs and the column request of the next round.
template <bool DF>
__device__ __forceinline__ void round_tail(const LazyArgs &a, int b, int nu, int Ib, int ns, int kb, float rb)
{
    const size_t row = static_cast<size_t>(b) * a.Kp;
    int u = kb;
    if (u < 0 || u >= a.K) {
        atomicOr(a.err, 1 << DEV_ERR_BAD_INDEX);
        u = 0;
        rb = 0.0f;
    }
    const float du = static_cast<const float *>(a.Dk)[row + u];
    int *slot_of = a.slot_of + row;
    const int su = slot_of[u];
    float c;
    if (DF) {
        // c = gamma R'_u D_u from the pair (the winner's parts are in global
        // memory, written by this block's threads before the argmax's exchange)
        const float hu = static_cast<const float *>(a.R)[row + u];
        const float2 ru = (u == kb) ? make_float2(hu, lo_decode(hu, a.Rlo[row + u])) : make_float2(0.0f, 0.0f);
        const double cd = a.gamma * (static_cast<double>(ru.x) + static_cast<double>(ru.y)) *
                          static_cast<double>(du);
        const float ch = static_cast<float>(cd);
        reinterpret_cast<float2 *>(a.cur_c64)[b] = make_float2(ch, static_cast<float>(cd - ch));
        a.c_log64[static_cast<size_t>(b) * a.I_max + nu] = cd;
        c = ch;
    } else {
        c = static_cast<float>(a.gamma) * rb * du;
        static_cast<float *>(a.cur_c)[b] = c;
    }
    a.cur_u[b] = u;
    a.u_log[static_cast<size_t>(b) * a.I_max + nu] = u;
    static_cast<float *>(a.c_log)[static_cast<size_t>(b) * a.I_max + nu] = c;
    if (nu + 1 < Ib && su < 0) {
        // n_slots[b] is written only by this block's worker, one round at a time
        if (ns >= a.slots) {
            atomicOr(a.err, 1 << DEV_ERR_LAZY_CACHE);
            a.n_slots[b] = -1;
        } else {
            a.n_slots[b] = ns + 1;
            slot_of[u] = ns;
            const int jm = atomicAdd(a.miss_n + (nu & 1), 1);
            a.miss_blk[jm] = b;
            a.miss_rows[jm] = (static_cast<long long>(b) * a.slots + ns) * a.Kp;
        }
    }
}

// One CTA of 256 threads per block (long rows).
template <bool DF>
__global__ void __launch_bounds__(256) lazy_round_f32v_kernel(LazyArgs a, int nu)
{
    __shared__ Cand<float> red[8];
    const int b = blockIdx.x;
    if (b == 0 && threadIdx.x == 0) a.miss_n[(nu + 1) & 1] = 0;   // unused since round nu - 1
    int Ib, ns;
    RoundRow w;
    if (!round_row<DF>(a, b, nu, Ib, ns, w)) return;
    float s = -1.0f, rb = 0.0f;
    int kb = INT_MAX;
    round_scan<DF, 256>(w, a.Kp / 4, threadIdx.x, s, kb, rb);
    block_argmax<float>(s, kb, rb, red);
    if (threadIdx.x == 0) round_tail<DF>(a, b, nu, Ib, ns, kb, rb);
}

// One warp per block (short rows: many blocks' rounds in flight per SM, the
// argmax within the warp).
template <bool DF>
__global__ void __launch_bounds__(256) lazy_round_f32w_kernel(LazyArgs a, int nu)
{
    const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && threadIdx.x == 0) a.miss_n[(nu + 1) & 1] = 0;   // unused since round nu - 1
    if (b >= a.n) return;
    int Ib, ns;
    RoundRow w;
    if (!round_row<DF>(a, b, nu, Ib, ns, w)) return;
    float s = -1.0f, rb = 0.0f;
    int kb = INT_MAX;
    round_scan<DF, 32>(w, a.Kp / 4, lane, s, kb, rb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float so = __shfl_xor_sync(0xffffffffu, s, o);
        const int ko = __shfl_xor_sync(0xffffffffu, kb, o);
        const float ro = __shfl_xor_sync(0xffffffffu, rb, o);
        if (so > s || (so == s && ko < kb)) { s = so; kb = ko; rb = ro; }
    }
    __syncwarp();   // the lanes' stores of R' are visible to lane 0
    if (lane == 0) round_tail<DF>(a, b, nu, Ib, ns, kb, rb);
}

// Model on the block's loss pixels (eq. 9) and replacement; logs out.
template <typename T>
__global__ void lazy_model_kernel(LazyArgs a)
{
    const int b = blockIdx.x;
    const BlockDesc bd = a.blocks[b];
    const int I = a.n_slots[b] < 0 ? 0 : bd.iterations;
    const int *ul = a.u_log + static_cast<size_t>(b) * a.I_max;
    const T *cl = static_cast<const T *>(a.c_log) + static_cast<size_t>(b) * a.I_max;
    const T *Phi = static_cast<const T *>(a.Phi);
    for (int p = threadIdx.x; p < a.MN; p += blockDim.x) {
        if (bd.support[p]) {
            if (bd.out != bd.samples) bd.out[p] = bd.samples[p];
        } else {
            T acc = T(0);
            for (int nu = 0; nu < I; ++nu) acc = fma(cl[nu], Phi[static_cast<size_t>(ul[nu]) * a.MN + p], acc);
            bd.out[p] = static_cast<double>(acc);
        }
    }
    if (bd.sel_idx)
        for (int nu = threadIdx.x; nu < I; nu += blockDim.x) bd.sel_idx[nu] = ul[nu];
    if (bd.sel_coef) {
        const double *c64 = a.c_log64 ? a.c_log64 + static_cast<size_t>(b) * a.I_max : nullptr;
        for (int nu = threadIdx.x; nu < I; nu += blockDim.x)
            bd.sel_coef[nu] = c64 ? c64[nu] : static_cast<double>(cl[nu]);
    }
}

}  // namespace

cudaError_t launch_lazy_pack(const BlockDesc *blocks, int n, int MN, int MN_pad, uint16_t *xb,
                             double *xd, uint16_t *mb, double *md, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    lazy_pack_kernel<<<n, 256, 0, st>>>(blocks, MN, MN_pad, xb, xd, mb, md);
    return cudaGetLastError();
}

cudaError_t launch_lazy_pack_cols(const BlockDesc *blocks, int n, const int *miss_n, const int *miss_blk,
                                  const int *cur_u, const double *Phi64, int MN, int MN_pad,
                                  uint16_t *vb, double *vd, cudaStream_t st, uint16_t *vh, float hscale)
{
    if (n <= 0) return cudaSuccess;
    lazy_pack_cols_kernel<<<n, 256, 0, st>>>(blocks, miss_n, miss_blk, cur_u, Phi64, MN, MN_pad, vb, vd, vh,
                                             hscale);
    return cudaGetLastError();
}

cudaError_t launch_split_f16(const double *in, int rows, int cols, int ld_in, int ka_pad, float scale,
                             uint16_t *out, cudaStream_t st)
{
    if (rows <= 0) return cudaSuccess;
    split_f16_kernel<<<rows, 256, 0, st>>>(in, cols, ld_in, ka_pad, scale, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lazy_init(const LazyArgs &a, cudaStream_t st)
{
    lazy_init_kernel<T><<<a.n, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lazy_round(const LazyArgs &a, int nu, cudaStream_t st)
{
    auto al16 = [](const void *p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
    if (sizeof(T) == 4 && a.Kp % 4 == 0 && al16(a.R) && al16(a.Dk) && al16(a.cache) && (!a.Rlo || al16(a.Rlo))) {
        if (a.Kp <= 2048) {
            const int grid = (a.n + 7) / 8;
            if (a.Rlo) lazy_round_f32w_kernel<true><<<grid, 256, 0, st>>>(a, nu);
            else lazy_round_f32w_kernel<false><<<grid, 256, 0, st>>>(a, nu);
        } else {
            if (a.Rlo) lazy_round_f32v_kernel<true><<<a.n, 256, 0, st>>>(a, nu);
            else lazy_round_f32v_kernel<false><<<a.n, 256, 0, st>>>(a, nu);
        }
        return cudaGetLastError();
    }
    lazy_round_kernel<T><<<a.n, 256, 0, st>>>(a, nu);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lazy_model(const LazyArgs &a, cudaStream_t st)
{
    lazy_model_kernel<T><<<a.n, 256, 0, st>>>(a);
    return cudaGetLastError();
}

template cudaError_t launch_lazy_init<float>(const LazyArgs &, cudaStream_t);
template cudaError_t launch_lazy_init<double>(const LazyArgs &, cudaStream_t);
template cudaError_t launch_lazy_round<float>(const LazyArgs &, int, cudaStream_t);
template cudaError_t launch_lazy_round<double>(const LazyArgs &, int, cudaStream_t);
template cudaError_t launch_lazy_model<float>(const LazyArgs &, cudaStream_t);
template cudaError_t launch_lazy_model<double>(const LazyArgs &, cudaStream_t);

}  // namespace se
