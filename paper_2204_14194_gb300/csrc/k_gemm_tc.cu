// k_gemm_tc.cu -- tcgen05 tensor-core GEMM for the scalar-product stages.
//
// Computes D[m][n] = sum_pairs sum_k A[m][pa*ka + k] * B[n][pb*ka + k] with
// bf16 or fp16 operands (both K-major) and fp32 accumulation in tensor memory.
// The "pairs" implement split-precision products: an fp64 operand v is stored
// as bf16 parts v = h + m + l, and the partial products h*h, h*m, m*h, ... are
// accumulated into the same TMEM tile, so a 3-part split with 6 products
// gives ~fp32 accuracy from the bf16 tensor pipe.  With fp16 parts (11
// significant bits each) two parts v = h + l and the 3 products h*h, h*l,
// l*h give about 2^-21 relative, half the tensor work; the operands are then
// scaled by powers of two into the fp16 range and the epilogue undoes it.
//
// Used for
//   * the table of eq. (16), C = G G^T with G = Phi_A diag(sqrt(w)) (Alg. 2;
//     symmetric mode computes the upper tiles only and mirrors them), and
//   * the initial projections of eq. (12), R0[b][k] = sum_j G[k][j] X[b][j]
//     with X = sqrt(w) * s on the support (stored transposed, block-major).
// An optional per-atom factor (D_k = 1/sqrt(C_kk) of eq. 17) is applied in
// the epilogue, so the fp32 iteration works on D-scaled projections.
//
// Structure (one CTA per 128 x BN output tile, 128 threads):
//   warp 0 lane 0  TMA producer: cp.async.bulk.tensor 2-D loads of the A and
//                  B k-slices (64 bf16 = 128 B rows, 128-byte swizzle) into
//                  a STAGES-deep shared-memory ring, mbarrier complete_tx;
//   warp 1 lane 0  MMA issuer: tcgen05.mma.cta_group::1.kind::f16, M=128,
//                  N=BN, K=16 per instruction, accumulator in TMEM;
//                  tcgen05.commit frees a ring slot when its MMAs retire;
//   warps 0-3      epilogue: tcgen05.ld 32x32b of their TMEM lane quarter,
//                  fp32 stores (transposed for R0, mirrored for C).
// Every mbarrier wait is bounded by %globaltimer; on timeout the CTA records
// DEV_ERR_WAIT_TIMEOUT, drains what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "se_internal.h"

namespace se {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;                       // bf16 per row of a k-slice (128 bytes)
constexpr int THREADS = 128;
constexpr unsigned long long WAIT_NS = 2000000000ull;   // 2 s
constexpr unsigned long long DRAIN_NS = 200000000ull;   // 0.2 s

__device__ __forceinline__ uint32_t saddr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier; false on timeout or abort.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                          unsigned long long limit_ns)
{
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 63u) == 0) {
            if (abort_flag && *abort_flag) return false;
            if (gtimer() - t0 > limit_ns) return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// Bulk tensor store of a shared-memory box to global memory (bulk async-group
// completion); the box is the tensor map's, the coordinates its origin.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, uint32_t src)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<unsigned long long>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}

__device__ __forceinline__ void tma_store_commit_and_wait_read()
{
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile whose rows are 128 bytes
// with the 128-byte swizzle (the layout TMA writes with SWIZZLE_128B):
// start address >> 4 in bits 0-13, leading byte offset (unused for this
// layout, 16 B) in bits 16-29, stride byte offset between 8-row groups
// (1024 B) in bits 32-45, descriptor version 1 in bits 46-47, swizzle mode
// 2 (128-byte) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr)
{
    uint64_t d = 0;
    d |= static_cast<uint64_t>((addr >> 4) & 0x3FFFu);
    d |= static_cast<uint64_t>(16u >> 4) << 16;
    d |= static_cast<uint64_t>(1024u >> 4) << 32;
    d |= static_cast<uint64_t>(1u) << 46;
    d |= static_cast<uint64_t>(2u) << 61;
    return d;
}

// Instruction descriptor for kind::f16: fp32 accumulator (bits 4-5 = 1),
// A and B bf16 (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 =
// 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
           (static_cast<uint32_t>(M >> 4) << 24);
}

#define TMEM_LD_32x32b_X32(taddr, r)                                                              \
    asm volatile(                                                                                  \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14," \
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"              \
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),      \
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), \
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),          \
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),          \
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])           \
        : "r"(taddr))

// Two stage layouts.  GROUPED: a pipeline stage holds one 64-wide k-slice
// of every split part of A (NP x 16 KiB) and of B (NP x BN*128 B) and the MMA
// issuer runs all partial products on it, so each part is fetched once per
// k-slice.  Otherwise a stage holds the A and B slices of one partial product
// (pair-major), which needs less shared memory per stage and so allows a
// deeper ring and wider BN.
// CPS CTAs share an SM: the ring is sized to 200 KiB / CPS.  With two CTAs of
// one stage each, one CTA's loads, prologue and epilogue overlap the other's
// products (the grouped table layout needs 96 KiB per stage).
template <int BN, int NP, bool GROUPED, int CPS = 1>
struct TcCfg {
    static constexpr int A_PART = BM * BK * 2;
    static constexpr int B_PART = BN * BK * 2;
    static constexpr int STAGE = (GROUPED ? NP : 1) * (A_PART + B_PART);
    static constexpr int BUDGET = (200 * 1024) / CPS;
    static constexpr int STAGES = BUDGET / STAGE < 2 ? 1 : (BUDGET / STAGE > 6 ? 6 : BUDGET / STAGE);
    static constexpr size_t SMEM = static_cast<size_t>(STAGES) * STAGE + 1024 + 256;
};

template <int BN, int NP, bool GROUPED, int CPS = 1>
__global__ void __launch_bounds__(THREADS, CPS)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmO, const __grid_constant__ TcGemmArgs p, int mt, int nt,
               int tma_out)
{
    using Cfg = TcCfg<BN, NP, GROUPED, CPS>;
    constexpr int STAGES = Cfg::STAGES;
    static_assert(STAGES >= (CPS > 1 ? 1 : 2), "double buffering, in the CTA or across the CTAs of an SM");
    static_assert(STAGES * Cfg::STAGE >= 4 * 32 * 33 * 4, "the epilogue's transpose fits in the ring");
    // Two fp32 accumulators of BN columns: acc0 takes the leading product
    // (the pair of the two largest parts, main_pair), acc1 every smaller
    // cross product, so the small terms are summed among themselves and added
    // to the large ones only once, in the epilogue.
    constexpr uint32_t TMEM_COLS = 2 * BN;
    // A and B formats (bits 7-9, 10-12): 1 = bf16, 0 = fp16
    const uint32_t IDESC = p.f16 ? make_idesc(BM, BN) & ~((7u << 7) | (7u << 10)) : make_idesc(BM, BN);

    extern __shared__ uint8_t smem_raw[];
    const uint32_t raw = saddr(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    uint64_t *bars = reinterpret_cast<uint64_t *>(gbase + STAGES * Cfg::STAGE);
    const uint32_t full0 = saddr(bars);
    const uint32_t empty0 = full0 + 8 * STAGES;
    const uint32_t accum = full0 + 16 * STAGES;
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 2 * STAGES + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    int tm, tn;
    if (p.symmetric) {
        int t = blockIdx.x;
        tm = 0;
        while (t >= mt - tm) { t -= mt - tm; ++tm; }
        tn = tm + t;
    } else {
        tm = blockIdx.x % mt;
        tn = blockIdx.x / mt;
    }
    (void)nt;
    int n_eff = p.N;
    if (p.n_dev) {
        const int nd = *p.n_dev;
        n_eff = nd < p.N ? nd : p.N;
        if (tn * BN >= n_eff) return;   // whole tile beyond the live rows: nothing to do
    }

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(accum, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         saddr(tmem_holder)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_holder;

    const int kblocks = p.ka_pad / BK;
    const int units = GROUPED ? kblocks : p.npairs * kblocks;   // pipeline units
    int main_pair = 0, first_small = -1;
    for (int q = 0; q < p.npairs; ++q)
        if (p.pa[q] + p.pb[q] < p.pa[main_pair] + p.pb[main_pair]) main_pair = q;
    for (int q = 0; q < p.npairs; ++q)
        if (q != main_pair) { first_small = q; break; }
    const bool has_small = first_small >= 0;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------- producer
            int issued = 0;
            for (int i = 0; i < units; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (i / STAGES) & 1;
                if (!mbar_wait(empty0 + 8 * s, ph ^ 1u, abort_flag, WAIT_NS)) {
                    *abort_flag = 1;
                    atomicOr(p.err, 1 << DEV_ERR_WAIT_TIMEOUT);
                    break;
                }
                mbar_expect_tx(full0 + 8 * s, Cfg::STAGE);
                const uint32_t st0 = base + s * Cfg::STAGE;
                if (GROUPED) {
#pragma unroll
                    for (int q = 0; q < NP; ++q) {
                        tma_load_2d(st0 + q * Cfg::A_PART, &tmA, q * p.ka_pad + i * BK, tm * BM, full0 + 8 * s);
                        tma_load_2d(st0 + NP * Cfg::A_PART + q * Cfg::B_PART, &tmB, q * p.ka_pad + i * BK,
                                    tn * BN, full0 + 8 * s);
                    }
                } else {
                    const int pair = i / kblocks, kb = i - pair * kblocks;
                    tma_load_2d(st0, &tmA, p.pa[pair] * p.ka_pad + kb * BK, tm * BM, full0 + 8 * s);
                    tma_load_2d(st0 + Cfg::A_PART, &tmB, p.pb[pair] * p.ka_pad + kb * BK, tn * BN,
                                full0 + 8 * s);
                }
                issued = i + 1;
            }
            if (*abort_flag) {
                for (int i = issued - STAGES < 0 ? 0 : issued - STAGES; i < issued; ++i)
                    mbar_wait(full0 + 8 * (i % STAGES), (i / STAGES) & 1, nullptr, DRAIN_NS);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------- MMA issuer
            for (int i = 0; i < units; ++i) {
                const int s = i % STAGES;
                const uint32_t ph = (i / STAGES) & 1;
                if (!mbar_wait(full0 + 8 * s, ph, abort_flag, WAIT_NS)) {
                    *abort_flag = 1;
                    atomicOr(p.err, 1 << DEV_ERR_WAIT_TIMEOUT);
                    break;
                }
                tc_fence_after();
                const uint32_t st0 = base + s * Cfg::STAGE;
                if (GROUPED) {
                    for (int q = 0; q < p.npairs; ++q) {
                        const uint32_t a0 = st0 + p.pa[q] * Cfg::A_PART;
                        const uint32_t b0 = st0 + NP * Cfg::A_PART + p.pb[q] * Cfg::B_PART;
                        const bool big = q == main_pair;
                        const uint32_t d = big ? tmem : tmem + BN;
#pragma unroll
                        for (int kk = 0; kk < BK / 16; ++kk) {
                            const bool first = i == 0 && kk == 0 && (big || q == first_small);
                            tc_mma(d, smem_desc(a0 + kk * 32), smem_desc(b0 + kk * 32), IDESC,
                                   first ? 0u : 1u);
                        }
                    }
                } else {
                    const int pair = i / kblocks, kb = i - pair * kblocks;
                    const bool big = pair == main_pair;
                    const uint32_t d = big ? tmem : tmem + BN;
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const bool first = kb == 0 && kk == 0 && (big || pair == first_small);
                        tc_mma(d, smem_desc(st0 + kk * 32), smem_desc(st0 + Cfg::A_PART + kk * 32), IDESC,
                               first ? 0u : 1u);
                    }
                }
                tc_commit(empty0 + 8 * s);
            }
            tc_commit(accum);   // arrives once every MMA issued above has retired
        }
        __syncwarp();
    }

    // -------------------------------------------------------------- epilogue
    bool ok = mbar_wait(accum, 0, nullptr, WAIT_NS);
    if (!ok) atomicOr(p.err, 1 << DEV_ERR_WAIT_TIMEOUT);
    ok = __syncthreads_and(ok && !*abort_flag) != 0;   // one outcome for the whole CTA
    tc_fence_after();
    __syncwarp();

    const int m = tm * BM + warp * 32 + lane;
    const bool diag_tile = p.symmetric && tm == tn;
    if (BN == BM && p.symmetric && tma_out) {
        // Gram mode through shared memory and bulk tensor stores: the pipeline ring
        // (idle once the accumulator is complete) holds the tile as four boxes of
        // 128 rows x 32 floats in the 128-byte swizzled layout of the output map
        // (16-byte chunk c of row r at r * 128 + ((c ^ (r mod 8)) * 16)).  Pass 0
        // writes the direct half out[m][n] = D[m][n] scale[n]; pass 1 the mirrored
        // half out[n][m] = D[m][n] scale[m] (a diagonal tile takes both triangles
        // in one pass: n >= m direct, n > m mirrored).  Two buffers when the ring
        // holds them, else one reused after the first stores have read it.
        constexpr int BOX = BM * 32 * 4;                                   // 16 KiB
        constexpr bool TWO = STAGES * Cfg::STAGE >= 8 * BOX;
        static_assert(BN != BM || STAGES * Cfg::STAGE >= 4 * BOX, "one tile buffer fits the ring");
        const int r = warp * 32 + lane;                                    // tile row of this thread
        const float sm = p.scale && m < p.M ? p.scale[m] : 1.0f;
#pragma unroll 1
        for (int pass = 0; pass < (diag_tile ? 1 : 2); ++pass) {
            const uint32_t buf = base + (TWO ? pass * 4 * BOX : 0);
            if (pass == 1 && !TWO) {
                // the first pass's stores have read the buffer (thread 0 waited)
                __syncthreads();
            }
#pragma unroll 1
            for (int c = 0; c < BN / 32; ++c) {
                uint32_t v[32];
                const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + c * 32;
                TMEM_LD_32x32b_X32(taddr, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (has_small) {
                    uint32_t q[32];
                    TMEM_LD_32x32b_X32(taddr + BN, q);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__uint_as_float(q[j]) + __uint_as_float(v[j]));
                }
                if (p.post != 0.0f) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) * p.post);
                }
                const int n0 = tn * BN + c * 32;
                if (pass == 0) {
                    // row r of box c: 8 chunks of 4 floats, scaled by the column's factor
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float f[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int n = n0 + 4 * q + e;
                            const float sn = p.scale && n < p.N ? __ldg(p.scale + n) : 1.0f;
                            f[e] = __uint_as_float(v[4 * q + e]) * sn;
                        }
                        const bool keep = !diag_tile || c * 32 + 4 * q + 3 >= r;   // some n >= m in the chunk
                        if (keep) {
                            const uint32_t a = buf + c * BOX + r * 128 + ((q ^ (r & 7)) << 4);
                            if (!diag_tile || c * 32 + 4 * q >= r) {
                                asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(f[0]),
                                             "f"(f[1]), "f"(f[2]), "f"(f[3])
                                             : "memory");
                            } else {
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (c * 32 + 4 * q + e >= r)
                                        asm volatile("st.shared.f32 [%0], %1;" ::"r"(a + 4 * e), "f"(f[e]) : "memory");
                            }
                        }
                    }
                }
                if (pass == 1 || diag_tile) {
                    // mirrored: element (row n - tn BN, column r) of box r / 32, scaled by
                    // this row's factor; a diagonal tile keeps the rows below its diagonal
                    const uint32_t bx = buf + (r >> 5) * BOX;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int rn = c * 32 + j;   // tile row of the mirrored element
                        if (diag_tile && rn <= r) continue;
                        const uint32_t a = bx + rn * 128 + ((((r & 31) >> 2) ^ (rn & 7)) << 4) + ((r & 3) << 2);
                        asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(__uint_as_float(v[j]) * sm) : "memory");
                    }
                }
            }
            if (!ok) continue;   // the same for every thread of the CTA
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0) {
#pragma unroll 1
                for (int b = 0; b < BN / 32; ++b) {
                    if (pass == 0) tma_store_2d(&tmO, tn * BN + 32 * b, tm * BM, buf + b * BOX);   // direct
                    else tma_store_2d(&tmO, tm * BM + 32 * b, tn * BN, buf + b * BOX);            // mirrored
                }
                tma_store_commit_and_wait_read();
            }
        }
        if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // stores complete
        __syncthreads();
    } else {
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t r[32];
        const uint32_t taddr = tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0;
        TMEM_LD_32x32b_X32(taddr, r);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (has_small) {
            uint32_t q[32];
            TMEM_LD_32x32b_X32(taddr + BN, q);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(q[j]) + __uint_as_float(r[j]));
        }
        if (!ok) continue;   // the same for every thread of the CTA
        if (p.post != 0.0f) {
#pragma unroll
            for (int j = 0; j < 32; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) * p.post);
        }
        const int n0 = tn * BN + c0;
        const bool live = m < p.M;
        const float sm = p.scale && live ? p.scale[m] : 1.0f;
        if (!p.symmetric) {
            if (!live) continue;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int n = n0 + j;
                if (n < n_eff) {
                    const long long row = p.out_rows ? p.out_rows[n] : static_cast<long long>(n) * p.ldo;
                    p.out[row + m] = __uint_as_float(r[j]) * sm;
                }
            }
        } else {
            // the mirrored half out[n][m]: lanes hold consecutive m, so each store
            // is one coalesced row segment
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int n = n0 + j;
                if (live && n < p.N && !(diag_tile && n < m))
                    p.out[static_cast<long long>(n) * p.ldo + m] = __uint_as_float(r[j]) * sm;
            }
            // the direct half out[m][n]: through a 32 x 32 transpose in shared memory
            // (the pipeline stages are free once the accumulator is complete), so
            // that lanes hold consecutive n and each store is coalesced as well
            float *tr = reinterpret_cast<float *>(gbase) + warp * (32 * 33);
#pragma unroll
            for (int j = 0; j < 32; ++j) tr[lane * 33 + j] = __uint_as_float(r[j]);
            __syncwarp();
            const int n = n0 + lane;
            const float sn = p.scale && n < p.N ? p.scale[n] : 1.0f;
#pragma unroll 4
            for (int i = 0; i < 32; ++i) {
                const int mi = tm * BM + warp * 32 + i;
                if (mi < p.M && n < p.N && !(diag_tile && n < mi))
                    p.out[static_cast<long long>(mi) * p.ldo + n] = tr[i * 33 + lane] * sn;
            }
            __syncwarp();
        }
    }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TMEM_COLS)
                     : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn(std::string *why)
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    if (!fn && why) *why = "cuTensorMapEncodeTiled is not available from the driver";
    return fn;
}

// Encoded tensor maps of recent operands: the lazy rounds launch the same
// products (same operands, same shapes) hundreds of times per batch, and an
// encoding costs host time on every launch that is not replayed from a graph.
struct MapKey {
    const void *base;
    int rows, cols, pitch, box_rows;
    bool f16;
    bool operator==(const MapKey &o) const
    {
        return base == o.base && rows == o.rows && cols == o.cols && pitch == o.pitch && box_rows == o.box_rows &&
               f16 == o.f16;
    }
};
constexpr int kMapCache = 64;
std::mutex g_map_mu;
MapKey g_map_key[kMapCache];
CUtensorMap g_map_val[kMapCache];
int g_map_n = 0, g_map_next = 0;

bool encode_map(CUtensorMap *map, const void *base, int rows, int cols, int pitch_elems, int box_rows,
                std::string *why, bool f16);

bool make_map(CUtensorMap *map, const void *base, int rows, int cols, int pitch_elems, int box_rows,
              std::string *why, bool f16)
{
    const MapKey k{base, rows, cols, pitch_elems, box_rows, f16};
    {
        std::lock_guard<std::mutex> lk(g_map_mu);
        for (int i = 0; i < g_map_n; ++i)
            if (g_map_key[i] == k) {
                *map = g_map_val[i];
                return true;
            }
    }
    if (!encode_map(map, base, rows, cols, pitch_elems, box_rows, why, f16)) return false;
    std::lock_guard<std::mutex> lk(g_map_mu);
    const int slot = g_map_n < kMapCache ? g_map_n++ : (g_map_next++ % kMapCache);
    g_map_key[slot] = k;
    g_map_val[slot] = *map;
    return true;
}

bool encode_map(CUtensorMap *map, const void *base, int rows, int cols, int pitch_elems, int box_rows,
                std::string *why, bool f16)
{
    auto fn = encode_fn(why);
    if (!fn) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (pitch_elems * 2) % 16 || cols % BK) {
        if (why) *why = "tensor map: misaligned base, pitch or width";
        return false;
    }
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(pitch_elems) * 2};
    cuuint32_t box[2] = {static_cast<cuuint32_t>(BK), static_cast<cuuint32_t>(box_rows)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void *>(base), dims,
                    strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        if (why) *why = "cuTensorMapEncodeTiled failed with code " + std::to_string(static_cast<int>(r));
        return false;
    }
    return true;
}

// The fp32 output of a Gram product for bulk tensor stores: boxes of 128 rows x
// 32 floats (128 bytes, the 128-byte swizzle); false if the layout does not
// allow it (the epilogue then stores element by element).
bool encode_out_map(CUtensorMap *map, const float *out, int rows, int cols, long long ldo)
{
    auto fn = encode_fn(nullptr);
    if (!fn || (reinterpret_cast<uintptr_t>(out) & 15u) || (ldo * 4) % 16 || ldo < cols || rows <= 0 || cols <= 0)
        return false;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ldo) * 4};
    cuuint32_t box[2] = {32, static_cast<cuuint32_t>(BM)};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(out), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int NP, bool GROUPED, int CPS = 1>
cudaError_t launch_bn(const TcGemmArgs &a, cudaStream_t st, std::string *why)
{
    using Cfg = TcCfg<BN, NP, GROUPED, CPS>;
    CUtensorMap mA, mB, mO;
    if (!make_map(&mA, a.A, a.M, a.lda, a.lda, BM, why, a.f16 != 0)) return cudaErrorInvalidValue;
    if (!make_map(&mB, a.B, a.N, a.ldb, a.ldb, BN, why, a.f16 != 0)) return cudaErrorInvalidValue;
    std::memset(&mO, 0, sizeof(mO));
    const int tma_out = BN == BM && a.symmetric && encode_out_map(&mO, a.out, a.M, a.N, a.ldo) ? 1 : 0;
    const int mt = (a.M + BM - 1) / BM;
    const int nt = (a.N + BN - 1) / BN;
    const int grid = a.symmetric ? mt * (mt + 1) / 2 : mt * nt;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<BN, NP, GROUPED, CPS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             static_cast<int>(Cfg::SMEM));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    tc_gemm_kernel<BN, NP, GROUPED, CPS><<<grid, THREADS, Cfg::SMEM, st>>>(mA, mB, mO, a, mt, nt, tma_out);
    return cudaGetLastError();
}

}  // namespace

int tc_gemm_variants(const TcGemmArgs &a)
{
    return a.symmetric || a.grouped ? 2 : 4;
}

int tc_gemm_fill_variant(int M, int N)
{
    const int mt = (M + BM - 1) / BM, sms = sm_count();
    if (mt * ((N + 255) / 256) >= sms) return 0;
    if (mt * ((N + 127) / 128) >= sms) return 1;
    return 2;
}

cudaError_t launch_tc_gemm(const TcGemmArgs &a, cudaStream_t st, std::string *why, int variant)
{
    if (a.M <= 0 || a.N <= 0) return cudaSuccess;
    if (a.npairs < 1 || a.npairs > 8 || a.ka_pad % BK || a.ka_pad <= 0) {
        if (why) *why = "tc gemm: bad pair count or inner size";
        return cudaErrorInvalidValue;
    }
    int npa = 0, npb = 0;
    for (int i = 0; i < a.npairs; ++i) {
        npa = a.pa[i] + 1 > npa ? a.pa[i] + 1 : npa;
        npb = a.pb[i] + 1 > npb ? a.pb[i] + 1 : npb;
    }
    if (npa * a.ka_pad > a.lda || npb * a.ka_pad > a.ldb) {
        if (why) *why = "tc gemm: split part outside the operand row";
        return cudaErrorInvalidValue;
    }
    const int np = npa > npb ? npa : npb;
    if (a.symmetric && a.M != a.N) return cudaErrorInvalidValue;
    // The table (square, symmetric) uses 128 x 128 tiles with all parts of a
    // k-slice per stage; the projections use 128 x 256 tiles streamed one
    // partial product per stage (measured faster for the wide, short-K case).
    if (a.symmetric) {
        if (npa != npb) return cudaErrorInvalidValue;
        // variant 1: two CTAs per SM (one stage each); same accumulation order
        switch (np) {
        case 1: return variant == 1 ? launch_bn<128, 1, true, 2>(a, st, why) : launch_bn<128, 1, true>(a, st, why);
        case 2: return variant == 1 ? launch_bn<128, 2, true, 2>(a, st, why) : launch_bn<128, 2, true>(a, st, why);
        case 3: return variant == 1 ? launch_bn<128, 3, true, 2>(a, st, why) : launch_bn<128, 3, true>(a, st, why);
        default: break;
        }
    } else if (a.grouped) {
        // every part of a k-slice per stage: each part is read once per k-slice
        switch (np) {
        case 1: return variant == 1 ? launch_bn<128, 1, true, 2>(a, st, why) : launch_bn<128, 1, true>(a, st, why);
        case 2: return variant == 1 ? launch_bn<128, 2, true, 2>(a, st, why) : launch_bn<128, 2, true>(a, st, why);
        case 3: return variant == 1 ? launch_bn<128, 3, true, 2>(a, st, why) : launch_bn<128, 3, true>(a, st, why);
        default: break;
        }
    } else if (np <= 3) {
        // narrow products (few columns of B) fill more SMs with narrower tiles
        if (variant == 2) return launch_bn<64, 1, false>(a, st, why);
        if (variant == 3) return launch_bn<128, 1, false, 2>(a, st, why);   // two CTAs per SM
        return variant == 1 ? launch_bn<128, 1, false>(a, st, why) : launch_bn<256, 1, false>(a, st, why);
    }
    if (why) *why = "tc gemm: more than 3 split parts";
    return cudaErrorInvalidValue;
}

}  // namespace se
