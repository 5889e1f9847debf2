// se_noalloc.cu -- se_extrapolate_noalloc: the strided batch entry point for
// callers that must not allocate memory during the call.
//
// Some callers cannot call cudaMalloc (or anything that allocates) once they
// are running: real-time loops that forbid allocation after start-up, code
// that runs under an allocator it does not own, or hosts that hand the
// library only their own input and output buffers.  For them this entry
// point keeps all per-call scratch -- the block descriptors, the packed
// weighted samples and the initial projections -- in one file-scope
// __device__ array of fixed size (kScratchBytes below), which every GPU that
// loads the library holds until the process exits.  The caller still passes
// the inputs and outputs; the plan's tables live in memory the plan
// allocated when it was created.
//
// Host code cannot use the array's name as a device address (in host code it
// names a host-side stand-in).  So se_ctx_create, with the context's device
// current, looks the address up once with cudaGetSymbolAddress (through
// noalloc_scratch_address below) and keeps it in the context.  The lookup
// also makes the CUDA runtime load the module that holds the array, so the
// 16 MiB are in place from context creation on, and the calls themselves do
// no CUDA set-up of any kind.
//
// Every call shares the one array, and it keeps the last call's contents.
// Nothing in it has to start at zero (every byte a call reads was written by
// the same call's kernels), so nothing is cleared.  Calls whose work overlaps
// on the GPU (different streams, or different threads) race on the array and
// must be serialised by the caller.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "se_host.h"

namespace {

constexpr size_t kScratchBytes = 16u << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

size_t r256(size_t v) { return (v + 255) / 256 * 256; }

}  // namespace

// The device address of the static scratch on the current device; called by
// se_ctx_create with the context's device current.
se_status se::noalloc_scratch_address(void **out)
{
    *out = nullptr;
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
        return set_error(SE_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    *out = p;
    return SE_OK;
}

extern "C" se_status se_extrapolate_noalloc(se_ctx_t *ctx, const se_plan_t *plan, int n,
                                            const double *samples, double *out, int32_t *sel_idx,
                                            double *sel_coef, int iterations, void *cuda_stream)
{
    using namespace se;
    if (!ctx || !plan || n < 0) return set_error(SE_ERR_INVALID, "NULL argument or n < 0");
    if (plan->ctx != ctx) return set_error(SE_ERR_INVALID, "plan belongs to another context");
    if (iterations < 0) return set_error(SE_ERR_INVALID, "iterations < 0");
    se_plan_s *pl = const_cast<se_plan_s *>(plan);
    if (pl->cplx) return set_error(SE_ERR_INVALID, "se_extrapolate_noalloc: complex plans use se_extrapolate_strided");
    if (pl->certified)
        return set_error(SE_ERR_INVALID, "se_extrapolate_noalloc: certified plans recompute flagged blocks "
                                         "in fp64, which needs workspace; use se_extrapolate_strided");
    if (n == 0) return SE_OK;
    if (!samples || !out) return set_error(SE_ERR_INVALID, "NULL samples or out");
    if (!ctx->noalloc_scratch) return set_error(SE_ERR_CUDA, "the context has no static scratch address");
    const int I = iterations ? iterations : pl->desc.iterations;
    const bool fp64 = pl->pc.fp64;
    const int Kp = pl->Kp;

    // scratch layout: descriptors | packed samples | initial projections
    const size_t desc_b = r256(sizeof(BlockDesc) * static_cast<size_t>(n));
    const size_t xrow = fp64 ? sizeof(double) * pl->ka_pad : 2u * pl->pc.nparts * pl->ka_pad;
    const size_t x_b = pl->sep_full ? 0 : r256(xrow * n);
    const size_t r_b = r256((fp64 ? sizeof(double) : sizeof(float)) * Kp * static_cast<size_t>(n));
    const size_t log_b = fp64 ? 0 : 8 * static_cast<size_t>(n) * I;   // selection log of the fp32 form
    if (desc_b + x_b + r_b + log_b > kScratchBytes) {
        const size_t per = sizeof(BlockDesc) + (pl->sep_full ? 0 : xrow) + (fp64 ? 8 : 4) * static_cast<size_t>(Kp) +
                           (fp64 ? 0 : 8 * static_cast<size_t>(I));
        return set_error(SE_ERR_INVALID,
                         "se_extrapolate_noalloc: " + std::to_string(n) +
                             " blocks need more than the 16 MiB static scratch; at most about " +
                             std::to_string(kScratchBytes / per) + " blocks of this plan fit");
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(SE_ERR_CUDA, "cudaSetDevice failed");
    NoTuneScope no_tune;   // no timing runs (and no events) inside this call
    unsigned char *base = static_cast<unsigned char *>(ctx->noalloc_scratch);
    BlockDesc *d_desc = reinterpret_cast<BlockDesc *>(base);
    void *d_x = base + desc_b;
    void *d_r0 = base + desc_b + x_b;
    int *d_log = reinterpret_cast<int *>(base + desc_b + x_b + r_b);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);

    const StridedSpec spec{samples, out, sel_idx, sel_coef, I, 1};
    cudaError_t e = launch_fill_desc(d_desc, n, spec, pl->MN, st);
    if (e != cudaSuccess) return set_error(SE_ERR_CUDA, std::string("descriptors: ") + cudaGetErrorString(e));
    se_status s = ensure_tables(ctx, pl, st);
    if (s != SE_OK) return s;

    std::string why;
    if (pl->sep_full) {
        // the parity-class kernel applies D_k when it loads R^(0)
        e = launch_pattern_projections(ctx, pl, d_desc, n, d_r0, !pl->sym, st);
    } else if (fp64) {
        e = launch_pack_x(d_desc, n, pl->d_a_idx.as<int>(), pl->d_sqrtw.as<double>(), pl->nA,
                          pl->ka_pad, 0, pl->MN, nullptr, static_cast<double *>(d_x), st);
        if (e == cudaSuccess)
            e = launch_simt_gemm<double>(pl->d_G64.as<double>(), pl->ka_pad,
                                         static_cast<const double *>(d_x), pl->ka_pad, Kp, n,
                                         pl->ka_pad, static_cast<double *>(d_r0), Kp, 0, st);
    } else {
        e = launch_pack_x(d_desc, n, pl->d_a_idx.as<int>(), pl->d_sqrtw.as<double>(), pl->nA,
                          pl->ka_pad, pl->pc.nparts, pl->MN, static_cast<uint16_t *>(d_x), nullptr, st);
        if (e == cudaSuccess) {
            TcGemmArgs g{};
            g.A = pl->d_Gwbf.ptr;
            g.B = d_x;
            g.M = Kp;
            g.N = n;
            g.lda = g.ldb = pl->pc.nparts * pl->ka_pad;
            g.ka_pad = pl->ka_pad;
            g.npairs = pl->pc.npairs;
            for (int i = 0; i < 8; ++i) { g.pa[i] = pl->pc.pa[i]; g.pb[i] = pl->pc.pb[i]; }
            g.out = static_cast<float *>(d_r0);
            g.ldo = Kp;
            g.symmetric = 0;
            g.grouped = 1;   // the order of the batched entry points (same bits)
            g.err = ctx->ws_err.as<int>();
            g.scale = pl->d_Dk.as<float>();
            e = launch_tc_gemm(g, st, &why);
        }
    }
    if (e != cudaSuccess)
        return set_error(SE_ERR_CUDA, "se_extrapolate_noalloc projections: " + why + " " + cudaGetErrorString(e));

    IterArgs a{};
    a.blocks = d_desc;
    a.n = n;
    a.K = pl->K;
    a.Kp = Kp;
    a.R0 = d_r0;
    a.C = pl->d_C.ptr;
    a.invC = pl->d_invC.ptr;
    a.Dk = pl->d_Dk.ptr;
    a.PhiB = pl->d_PhiB.ptr;
    a.b_idx = pl->d_b_idx.as<int>();
    a.pat_support = pl->d_pattern.as<uint8_t>();
    a.nB = pl->nB;
    a.MN = pl->MN;
    a.gamma = pl->desc.gamma;
    a.I_max = I;
    a.err = ctx->ws_err.as<int>();
    if (!fp64) {   // the same model kernel as the batched entry points
        a.log_u = d_log;
        a.log_c = reinterpret_cast<float *>(d_log + static_cast<size_t>(n) * I);
    }
    int launched = 0;
    e = fp64 ? launch_iterate_full<double>(a, st, &launched) : launch_iterations_f32(ctx, pl, a, st, &launched);
    if (e == cudaSuccess && !fp64) {
        e = launch_model(pl, a, st);
        ++launched;
    }
    if (e != cudaSuccess)
        return set_error(SE_ERR_CUDA, std::string("se_extrapolate_noalloc iterations: ") + cudaGetErrorString(e));
    ctx->launches += 3 + launched;
    return SE_OK;
}
