// se_api.cpp -- the C ABI of include/se.h: contexts, plans and the batched
// extrapolation path (Alg. 2 table generation + Alg. 3 model generation).
#include <algorithm>
#include <random>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "se_host.h"

using namespace se;

namespace {

thread_local std::string g_err;

se_status fail(se_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

}  // namespace

se_status se::set_error(se_status s, const std::string &msg) { return fail(s, msg); }

namespace {

#define SE_CUDA(call)                                                                         \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(SE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    } while (0)

#define SE_TRY(expr)                      \
    do {                                  \
        se_status s_ = (expr);            \
        if (s_ != SE_OK) return s_;       \
    } while (0)

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

}  // namespace

se_status se::dev_alloc(se_ctx_s *ctx, DevBuf &b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (b.ptr && b.bytes >= bytes) return SE_OK;
    b.release();
    if (ctx->budget && ctx->used.load() + bytes > ctx->budget)
        return fail(SE_ERR_NOMEM, "HBM budget exceeded: need " + std::to_string(bytes) +
                                      " more bytes, " + std::to_string(ctx->used.load()) + " of " +
                                      std::to_string(ctx->budget) + " in use");
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(SE_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    b.ctx = ctx;
    b.ptr = p;
    b.bytes = bytes;
    ctx->used += bytes;
    return SE_OK;
}

namespace {

template <typename V>
se_status upload(se_ctx_s *ctx, DevBuf &b, const std::vector<V> &h)
{
    SE_TRY(dev_alloc(ctx, b, h.size() * sizeof(V)));
    if (!h.empty()) SE_CUDA(cudaMemcpy(b.ptr, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    return SE_OK;
}

const char *dev_err_text(int bits)
{
    if (bits & (1 << DEV_ERR_WAIT_TIMEOUT)) return "a bounded device wait (mbarrier) ran out of time";
    if (bits & (1 << DEV_ERR_BAD_INDEX)) return "no admissible atom could be selected";
    if (bits & (1 << DEV_ERR_TMEM)) return "tensor memory allocation failed";
    if (bits & (1 << DEV_ERR_LAZY_CACHE)) return "lazy column cache overflow";
    if (bits & (1 << DEV_ERR_EMPTY_SUPPORT)) return "a block's own mask leaves no admissible atom";
    return "unknown device error";
}

}  // namespace

namespace se {

int stage_begin(se_ctx_s *ctx, int stage, cudaStream_t st)
{
    if (!ctx->profiling) return -1;
    std::lock_guard<std::mutex> lk(ctx->pmu);
    cudaEvent_t ev[2];
    for (auto &e : ev) {
        if (!ctx->event_pool.empty()) {
            e = ctx->event_pool.back();
            ctx->event_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            return -1;
        }
    }
    cudaEventRecord(ev[0], st);
    ctx->pending.push_back({stage, {ev[0], ev[1]}});
    return static_cast<int>(ctx->pending.size()) - 1;
}

void stage_end(se_ctx_s *ctx, int token, cudaStream_t st)
{
    if (token < 0) return;
    std::lock_guard<std::mutex> lk(ctx->pmu);
    if (token < static_cast<int>(ctx->pending.size()))
        cudaEventRecord(ctx->pending[token].second.second, st);
}

DevBuf::~DevBuf() { release(); }

Workspace::~Workspace()
{
    if (h_desc) cudaFreeHost(h_desc);
    if (ev_staging) cudaEventDestroy(ev_staging);
    if (ev_ws) cudaEventDestroy(ev_ws);
}

cudaError_t Workspace::init()
{
    cudaError_t e = cudaEventCreateWithFlags(&ev_staging, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev_ws, cudaEventDisableTiming);
    // record once so that the first batch finds both events complete
    if (e == cudaSuccess) e = cudaEventRecord(ev_staging, 0);
    if (e == cudaSuccess) e = cudaEventRecord(ev_ws, 0);
    return e;
}

void DevBuf::release()
{
    if (ptr) {
        cudaFree(ptr);
        ctx->used -= bytes;
    }
    ptr = nullptr;
    bytes = 0;
}

PrecCfg prec_cfg(se_prec p)
{
    PrecCfg c;
    // partial products ordered from the smallest magnitude to the largest
    switch (p) {
    case SE_PREC_FP64:
        c.fp64 = true;
        break;
    case SE_PREC_CERTIFIED:
    case SE_PREC_BF16X6: {
        c.nparts = 3;
        c.npairs = 6;
        const int a[6] = {2, 1, 0, 1, 0, 0}, b[6] = {0, 1, 2, 0, 1, 0};
        for (int i = 0; i < 6; ++i) { c.pa[i] = a[i]; c.pb[i] = b[i]; }
        break;
    }
    case SE_PREC_BF16X3: {
        c.nparts = 2;
        c.npairs = 3;
        const int a[3] = {1, 0, 0}, b[3] = {0, 1, 0};
        for (int i = 0; i < 3; ++i) { c.pa[i] = a[i]; c.pb[i] = b[i]; }
        break;
    }
    case SE_PREC_BF16:
    default:
        c.nparts = 1;
        c.npairs = 1;
        break;
    }
    return c;
}

}  // namespace se

// Separable-transform products on the plan's pattern: mode 0 gives R^(0)
// (eq. 12) of every block, mode 3 the rows of C (eq. 16).  In the fp32 form
// both carry the factor D_k of the recurrence; padded atoms [K, Kp) read NaN
// there (never selected) and 0 in the fp64 form (zero criterion).
SepArgs se::pattern_sep_args(se_plan_s *pl, int mode, const BlockDesc *dd, int n, void *out, bool scaled)
{
    SepArgs s{};
    s.M = pl->M;
    s.N = pl->N;
    s.ntr = pl->sep_ntr;
    for (int t = 0; t < pl->sep_ntr; ++t) {
        s.TM[t] = pl->d_sepM[t].ptr;
        s.TN[t] = pl->d_sepN[t].ptr;
        s.koff[t] = pl->sep_koff[t];
    }
    s.mode = mode;
    s.blocks = dd;
    s.pattern = pl->d_pattern.as<uint8_t>();
    s.scale = pl->pc.fp64 || !scaled ? nullptr : pl->d_Dk.as<float>();
    s.rho = pl->d_rho.as<double>();
    s.img = pl->d_sep_img.as<float>();
    s.out = out;
    s.ldo = pl->Kp;
    s.n = n;
    s.kfill = pl->Kp;
    // the separable model kernel leaves the support pixels to this pass
    s.copy_support = mode == 0 && !pl->pc.fp64 && pl->nB > 0;
    return s;
}

// SE_GRAM_AUTO: pattern blocks go to the lazy path while that is measured to
// be cheaper than building the table (see choose_lazy_for_pattern).
void se::route_pattern_blocks(se_plan_s *pl, std::vector<BlockDesc> &full, std::vector<BlockDesc> &lazy,
                              int *I_full, int *I_lazy)
{
    if (full.empty() || !choose_lazy_for_pattern(pl, static_cast<int>(full.size()))) return;
    for (auto &x : full) {
        x.support = pl->d_pattern.as<uint8_t>();
        lazy.push_back(x);
        *I_lazy = std::max(*I_lazy, x.iterations);
    }
    full.clear();
    *I_full = 0;
}

// Parity classes (see k_sym.cu).  Enabled for the fp32 transform form with
// DCT / WHT atoms, M, N in {16, 32}, K = Kp in {512, 1024, 2048} and a
// weighting function that is exactly symmetric in m and in n; every atom is
// checked to be even or odd in each direction as its indices say, and the
// vanishing of C(k,u) across classes is checked on sampled atom pairs.
se_status se::setup_sym(se_ctx_s *ctx, se_plan_s *pl)
{
    const int M = pl->M, N = pl->N, MN = pl->MN, K = pl->K;
    const int basis = pl->desc.basis;
    if (!(pl->sep_full && !pl->pc.fp64 && !pl->certified && !pl->cplx && pl->T == 1)) return SE_OK;
    if (!(basis == SE_BASIS_DCT || basis == SE_BASIS_WHT || basis == SE_BASIS_DCT_WHT)) return SE_OK;
    if (!sym_fold_supported(M, N) || K != pl->Kp || (K != 512 && K != 1024 && K != 2048)) return SE_OK;
    if (K != pl->sep_ntr * MN || (pl->sep_ntr == 2 && pl->sep_koff[1] != MN) || pl->d_sep_img.ptr == nullptr)
        return SE_OK;
    for (int m = 0; m < M; ++m)
        for (int n = 0; n < N; ++n) {
            const double v = pl->w[static_cast<size_t>(m) * N + n];
            if (v != pl->w[static_cast<size_t>(M - 1 - m) * N + n] || v != pl->w[static_cast<size_t>(m) * N + N - 1 - n])
                return SE_OK;
        }
    auto cls = [&](int k) {
        const int kk = k >= MN ? k - MN : k;
        return (((kk / N) & 1) << 1) | ((kk % N) & 1);
    };
    std::vector<int> perm;
    perm.reserve(K);
    for (int c = 0; c < 4; ++c)
        for (int k = 0; k < K; ++k)
            if (cls(k) == c) perm.push_back(k);
    // the class order the folded transforms write: class, transform, (p / 2, q / 2)
    if (static_cast<int>(perm.size()) != K) return SE_OK;
    const int QM = M / 2, QN = N / 2, Q = K / 4;
    for (int c = 0; c < 4; ++c)
        for (int t = 0; t < pl->sep_ntr; ++t)
            for (int i = 0; i < QM; ++i)
                for (int j = 0; j < QN; ++j)
                    if (perm[static_cast<size_t>(c) * Q + t * QM * QN + i * QN + j] !=
                        t * MN + (2 * i + (c >> 1)) * N + 2 * j + (c & 1))
                        return SE_OK;
    // every atom even or odd in each direction as (p mod 2, q mod 2) says
    double amax = 0.0;
    for (size_t e = 0; e < static_cast<size_t>(K) * MN; ++e) amax = std::max(amax, std::fabs(pl->phi[e]));
    for (int k = 0; k < K; ++k) {
        const double sa = (cls(k) >> 1) ? -1.0 : 1.0, sb = (cls(k) & 1) ? -1.0 : 1.0;
        const double *f = pl->phi.data() + static_cast<size_t>(k) * MN;
        for (int m = 0; m < M; ++m)
            for (int n = 0; n < N; ++n) {
                const double v = f[m * N + n];
                if (std::fabs(f[(M - 1 - m) * N + n] - sa * v) > 1e-12 * amax ||
                    std::fabs(f[m * N + N - 1 - n] - sb * v) > 1e-12 * amax)
                    return SE_OK;
            }
    }
    // sampled check: atoms of different classes have (numerically) no weighted overlap
    std::mt19937 gen(7);
    for (int t = 0; t < 64; ++t) {
        int k = static_cast<int>(gen() % K), u = static_cast<int>(gen() % K);
        if (cls(k) == cls(u)) u = (u + 1) % K;
        if (cls(k) == cls(u)) continue;
        const double *a = pl->phi.data() + static_cast<size_t>(k) * MN, *b = pl->phi.data() + static_cast<size_t>(u) * MN;
        double x = 0.0, na = 0.0, nb = 0.0;
        for (int i = 0; i < MN; ++i) {
            x += a[i] * b[i] * pl->w[i];
            na += a[i] * a[i] * pl->w[i];
            nb += b[i] * b[i] * pl->w[i];
        }
        if (std::fabs(x) > 1e-12 * std::sqrt(na * nb) + 1e-300) return SE_OK;
    }
    // constants of the folded transforms from the transform kernels' image
    // (per transform t_p[m] at m M + p, t'_q[n] at n N + q; then rho)
    const int ntr = pl->sep_ntr;
    std::vector<float> img(static_cast<size_t>(ntr) * (M * M + N * N) + MN);
    SE_CUDA(cudaMemcpy(img.data(), pl->d_sep_img.ptr, img.size() * sizeof(float), cudaMemcpyDeviceToHost));
    std::vector<float> fimg;
    fimg.reserve(static_cast<size_t>(ntr) * (M * M + N * N) / 2 + MN);
    for (int t = 0; t < ntr; ++t) {
        const float *tm = img.data() + static_cast<size_t>(t) * (M * M + N * N), *tn = tm + M * M;
        for (int m = 0; m < QM; ++m)
            for (int a = 0; a < 2; ++a)
                for (int i = 0; i < QM; ++i) fimg.push_back(tm[m * M + 2 * i + a]);
        for (int n = 0; n < QN; ++n)
            for (int b = 0; b < 2; ++b)
                for (int j = 0; j < QN; ++j) fimg.push_back(tn[n * N + 2 * j + b]);
    }
    fimg.insert(fimg.end(), img.end() - MN, img.end());
    SE_TRY(upload(ctx, pl->d_sym_img, fimg));
    if (M == 32 && N == 32) {
        // the same constants as per-lane m16n8k8 fragments for the tensor-core R^(0)
        // kernel (g = lane / 4, q = lane mod 4); SE_R0_FFMA=1 keeps the fp32 kernels
        // TF32 parts of x: large = x rounded to 10 mantissa bits (nearest, ties away from
        // zero, on the bit pattern: the 13 dropped bits decide), small = the same rounding
        // of the exact remainder x - large
        auto tf32 = [](float x) {
            uint32_t u;
            std::memcpy(&u, &x, 4);
            u = (u + 0x1000u) & 0xffffe000u;
            float r;
            std::memcpy(&r, &u, 4);
            return r;
        };
        std::vector<float> tc;
        tc.reserve(static_cast<size_t>(ntr) * 2048 + MN);
        for (int t = 0; t < ntr; ++t)
            for (int a = 0; a < 2; ++a)
                for (int ks = 0; ks < 2; ++ks)
                    for (int part = 0; part < 2; ++part)
                        for (int l = 0; l < 32; ++l) {
                            const int g = l >> 2, q = l & 3;
                            auto At = [&](int i, int m) {
                                const float x = fimg[static_cast<size_t>(t) * 1024 + m * 32 + a * 16 + i];
                                const float xb = tf32(x);
                                return part ? tf32(x - xb) : xb;
                            };
                            tc.push_back(At(g, 8 * ks + q));
                            tc.push_back(At(g + 8, 8 * ks + q));
                            tc.push_back(At(g, 8 * ks + q + 4));
                            tc.push_back(At(g + 8, 8 * ks + q + 4));
                        }
        for (int t = 0; t < ntr; ++t)
            for (int b = 0; b < 2; ++b)
                for (int ks = 0; ks < 2; ++ks)
                    for (int nt = 0; nt < 2; ++nt)
                        for (int l = 0; l < 32; ++l) {
                            const int g = l >> 2, q = l & 3;
                            const float b0 = fimg[static_cast<size_t>(t) * 1024 + 512 + (8 * ks + q) * 32 + b * 16 + 8 * nt + g];
                            const float b1 =
                                fimg[static_cast<size_t>(t) * 1024 + 512 + (8 * ks + q + 4) * 32 + b * 16 + 8 * nt + g];
                            tc.push_back(tf32(b0));
                            tc.push_back(tf32(b1));
                            tc.push_back(tf32(b0 - tf32(b0)));
                            tc.push_back(tf32(b1 - tf32(b1)));
                        }
        tc.insert(tc.end(), img.end() - MN, img.end());
        SE_TRY(upload(ctx, pl->d_sym_tc, tc));
        const char *env = std::getenv("SE_R0_FFMA");
        pl->sym_tc = !(env && env[0] == '1');
    }

    SE_TRY(upload(ctx, pl->d_perm, perm));
    SE_TRY(dev_alloc(ctx, pl->d_Cc, sizeof(float) * static_cast<size_t>(K) * (K / 4)));
    SE_TRY(dev_alloc(ctx, pl->d_Dkp, sizeof(float) * static_cast<size_t>(K)));
    pl->sym = true;
    return SE_OK;
}

static SymSepArgs sym_sep_args(se_plan_s *pl)
{
    SymSepArgs s{};
    s.M = pl->M;
    s.N = pl->N;
    s.ntr = pl->sep_ntr;
    s.K = pl->K;
    s.img = pl->d_sym_img.as<float>();
    s.perm = pl->d_perm.as<int>();
    s.pattern = pl->d_pattern.as<uint8_t>();
    return s;
}

cudaError_t se::launch_pattern_projections(se_ctx_s *ctx, se_plan_s *pl, const BlockDesc *dd, int n, void *r0,
                                           bool scaled, cudaStream_t st)
{
    if (pl->sym) {
        SymSepArgs s = sym_sep_args(pl);
        s.blocks = dd;
        s.n = n;
        s.R0 = static_cast<float *>(r0);
        s.copy_support = pl->nB > 0;
        if (pl->sym_tc) {
            s.tc_img = pl->d_sym_tc.as<float>();
            return launch_sym_r0_tc(s, st);
        }
        const std::string key = "symr0:" + std::to_string(pl->M) + "x" + std::to_string(pl->N) + ":t" +
                                std::to_string(pl->sep_ntr);
        return tune_run(ctx, key, sym_r0_variants(pl->M, pl->N), st, [&](int v) { return launch_sym_r0(s, st, v); });
    }
    return run_sep(ctx, pl, pattern_sep_args(pl, 0, dd, n, r0, scaled), st);
}

cudaError_t se::launch_iterations_f32(se_ctx_s *ctx, se_plan_s *pl, IterArgs &a, cudaStream_t st, int *launched,
                                      bool *model_done)
{
    if (model_done) *model_done = false;
    if (pl->sym && !a.cert_flag) {
        a.perm = pl->d_perm.as<int>();
        a.Cc = pl->d_Cc.as<float>();
        a.Dkp = pl->d_Dkp.as<float>();
        // the faster shape depends on how many waves the batch fills: key by the
        // batch size rounded up to a power of two
        int nb = 1;
        while (nb < a.n) nb <<= 1;
        const std::string skey = "sym:f32:" + std::to_string(pl->Kp) + ":n" + std::to_string(nb);
        const int Mb = pl->box[1] - pl->box[0], Nb = pl->box[3] - pl->box[2];
        if (model_done && pl->Kp == 2048 && pl->sep_full && pl->nB > 0 && pl->d_model_tab.ptr &&
            sep_model_tc_box(Mb, Nb) && sym_model_box(Mb, Nb)) {
            // the iterations and the model of eq. (9) as one stage: every form followed
            // by the tensor-core model kernel, or the last-updated-class form that
            // evaluates the model itself (the same operations, so the same bits)
            FusedModel fm{};
            fm.s = pattern_sep_args(pl, 0, nullptr, 0, nullptr);
            fm.tab = pl->d_model_tab.as<float>();
            fm.m0 = pl->box[0];
            fm.Mb = Mb;
            fm.n0 = pl->box[2];
            fm.Nb = Nb;
            {
                // the tile shapes the launch takes for this box (16 MT x 8 NT)
                const int MT = Mb <= 16 ? 1 : 2, NT = Nb <= 8 ? 1 : Nb <= 16 ? 2 : 4;
                const int slots = 3 * (pl->Kp / 4), need = pl->sep_ntr * pl->M * 16 * MT + 128 + 16 * MT * (8 * NT + 1);
                fm.compact = pl->M == pl->N && fm.m0 == fm.n0 && fm.m0 + 16 * MT <= pl->M && fm.n0 + 8 * NT <= pl->N &&
                             8 * NT <= 16 * MT && need <= slots;
            }
            const int nv = iterate_sym_variants(pl->Kp);
            const std::string mkey = skey + ":model" + std::to_string(Mb) + "x" + std::to_string(Nb);
            const int pick = tune_lookup(ctx, mkey, nv + 1);
            if (pick >= 0 && pick < nv) {   // the kept form has its own model kernel: the caller runs it
                *launched = 0;
                return launch_iterate_sym(a, st, launched, pick);
            }
            *model_done = true;
            if (pick == nv) {
                *launched = 0;
                return launch_iterate_sym_model(a, fm, st, launched);
            }
            return tune_run(ctx, mkey, nv + 1, st,
                            [&](int v) {
                                *launched = 0;
                                if (v == nv) return launch_iterate_sym_model(a, fm, st, launched);
                                cudaError_t e = launch_iterate_sym(a, st, launched, v);
                                if (e == cudaSuccess) {
                                    e = launch_model(pl, a, st);
                                    ++*launched;
                                }
                                return e;
                            });
        }
        return tune_run(ctx, skey, iterate_sym_variants(pl->Kp), st, [&](int v) {
            *launched = 0;
            return launch_iterate_sym(a, st, launched, v);
        });
    }
    const std::string ikey = "iterate:f32:" + std::to_string(pl->Kp);
    return tune_run(ctx, ikey, iterate_variants(pl->Kp, false), st, [&](int v) {
        *launched = 0;
        return launch_iterate_full<float>(a, st, launched, v);
    });
}

// Relative gap between the two largest |R'| below which a certified plan
// recomputes the block in fp64 (about 10x the largest fp32 score error
// measured against the fp64 form on the benchmark workloads).
constexpr float kCertGap = 1.5e-5f;

// Model and replacement after the fp32 iteration kernel wrote its log:
// separable outer products for transform plans, gathered atom values else.
cudaError_t se::launch_model(se_plan_s *pl, const IterArgs &a, cudaStream_t st)
{
    if (pl->sep_full && pl->nB > 0)
        return launch_sep_model(a, pattern_sep_args(pl, 0, nullptr, 0, nullptr), pl->box[0], pl->box[1],
                                pl->box[2], pl->box[3], st);
    return launch_model_f32(a, st);
}

// A transform-domain launch through the autotuner (schedules with identical
// results; one key per area size and transform count).
cudaError_t se::run_sep(se_ctx_s *ctx, se_plan_s *pl, const SepArgs &sa, cudaStream_t st)
{
    const bool fp64 = pl->pc.fp64;
    const int nv = sep_variants(sa, fp64);
    const std::string key = "sep:" + std::to_string(sa.M) + "x" + std::to_string(sa.N) + ":t" +
                            std::to_string(sa.ntr) + (fp64 ? ":f64" : ":f32");
    return tune_run(ctx, key, nv, st, [&](int v) {
        return fp64 ? launch_sep<double>(sa, st, v) : launch_sep<float>(sa, st, v);
    });
}

namespace {

std::string nclass(int n)
{
    int c = 0;
    while ((1 << c) < n) ++c;
    return std::to_string(c);
}

se_status build_tables(se_ctx_s *ctx, se_plan_s *pl, cudaStream_t st)
{
    if (pl->cplx) {
        SE_TRY(build_tables_complex(ctx, pl, st));
        SE_CUDA(cudaEventRecord(pl->tables_ready, st));
        pl->tables_valid = true;
        ctx->table_builds++;
        return SE_OK;
    }
    const int Kp = pl->Kp;
    std::string why;
    if (pl->sym) {   // diagonal, D_k and the compact rows of the parity classes in one launch
        SymSepArgs s = sym_sep_args(pl);
        s.dup = pl->d_dup.as<uint8_t>();
        s.Dk = pl->d_Dk.as<float>();
        s.invC = pl->d_invC.as<float>();
        s.Cc = pl->d_Cc.as<float>();
        s.Dkp = pl->d_Dkp.as<float>();
        SE_CUDA(launch_sym_rows(s, st));
        ctx->launches += 1;
        SE_CUDA(cudaEventRecord(pl->tables_ready, st));
        pl->tables_valid = true;
        ctx->table_builds++;
        return SE_OK;
    }
    unsigned long long *dmax = reinterpret_cast<unsigned long long *>(pl->d_nadm.as<char>() + 8);
    SE_CUDA(launch_tables_diag(pl->d_G64.as<double>(), pl->ka_pad, pl->K, Kp, pl->nA,
                               pl->d_dup.as<uint8_t>(), pl->d_diag.as<double>(), dmax,
                               pl->d_nadm.as<int>(), st));
    if (pl->sep_full) {
        // C(:, i) for every atom i as a separable transform of w phi_i (Sec. VI);
        // fp32 rows carry the factor D_k of the recurrence
        if (pl->pc.fp64)
            SE_CUDA(launch_tables_finalize<double>(pl->d_diag.as<double>(), pl->d_dup.as<uint8_t>(), dmax,
                                                   pl->K, Kp, pl->d_invC.as<double>(),
                                                   pl->d_Dk.as<double>(), pl->d_nadm.as<int>(), st));
        else
            SE_CUDA(launch_tables_finalize<float>(pl->d_diag.as<double>(), pl->d_dup.as<uint8_t>(), dmax,
                                                  pl->K, Kp, pl->d_invC.as<float>(), pl->d_Dk.as<float>(),
                                                  pl->d_nadm.as<int>(), st));
        SepArgs sa = pattern_sep_args(pl, 3, nullptr, pl->K, pl->d_C.ptr);
        SE_CUDA(run_sep(ctx, pl, sa, st));
        ctx->launches += 3;
    } else if (pl->pc.fp64) {
        SE_CUDA(launch_tables_finalize<double>(pl->d_diag.as<double>(), pl->d_dup.as<uint8_t>(), dmax,
                                               pl->K, Kp, pl->d_invC.as<double>(),
                                               pl->d_Dk.as<double>(), pl->d_nadm.as<int>(), st));
        SE_CUDA(launch_simt_gemm<double>(pl->d_G64.as<double>(), pl->ka_pad, pl->d_G64.as<double>(),
                                         pl->ka_pad, Kp, Kp, pl->ka_pad, pl->d_C.as<double>(), Kp, 1,
                                         st));
        ctx->launches += 3;
    } else {
        SE_CUDA(launch_tables_finalize<float>(pl->d_diag.as<double>(), pl->d_dup.as<uint8_t>(), dmax,
                                              pl->K, Kp, pl->d_invC.as<float>(), pl->d_Dk.as<float>(),
                                              pl->d_nadm.as<int>(), st));
        TcGemmArgs g{};
        g.M = Kp;
        g.N = Kp;
        g.ka_pad = pl->ka_pad;
        if (pl->f16_table) {
            // hh, hl, lh of the fp16 parts (the small products first); both scales undone
            const int pa[3] = {1, 0, 0}, pb[3] = {0, 1, 0};
            g.A = g.B = pl->d_GH.ptr;
            g.lda = g.ldb = 2 * pl->ka_pad;
            g.npairs = 3;
            for (int i = 0; i < 3; ++i) { g.pa[i] = pa[i]; g.pb[i] = pb[i]; }
            g.f16 = 1;
            g.post = 1.0f / (pl->g_f16_scale * pl->g_f16_scale);
        } else {
            g.A = g.B = pl->d_Gbf.ptr;
            g.lda = g.ldb = pl->pc.nparts * pl->ka_pad;
            g.npairs = pl->pc.npairs;
            for (int i = 0; i < 8; ++i) { g.pa[i] = pl->pc.pa[i]; g.pb[i] = pl->pc.pb[i]; }
        }
        g.out = pl->d_C.as<float>();
        g.ldo = Kp;
        g.symmetric = 1;
        g.err = ctx->ws_err.as<int>();
        g.scale = pl->d_Dk.as<float>();
        const std::string key = "gemm_table:" + std::to_string(Kp) + ":" + std::to_string(pl->ka_pad) + ":p" +
                                std::to_string(g.npairs) + (pl->f16_table ? "h" : "");
        cudaError_t e = tune_run(ctx, key, tc_gemm_variants(g), st,
                                 [&](int v) { return launch_tc_gemm(g, st, &why, v); });
        if (e != cudaSuccess) return fail(SE_ERR_CUDA, "table GEMM: " + why + " " + cudaGetErrorString(e));
        ctx->launches += 3;
    }
    SE_CUDA(cudaEventRecord(pl->tables_ready, st));
    pl->tables_valid = true;
    ctx->table_builds++;
    return SE_OK;
}

// eq. (12) as packing of the weighted support samples and a matrix product
// with the weighted atoms (tensor cores in the bf16 forms).
se_status dense_pattern_projections(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, const BlockDesc *ddesc,
                                    int n, cudaStream_t st)
{
    const int Kp = pl->Kp;
    const bool fp64 = pl->pc.fp64;
    std::string why;
    int tok = stage_begin(ctx, 0, st);
    if (fp64)
        SE_CUDA(launch_pack_x(ddesc, n, pl->d_a_idx.as<int>(), pl->d_sqrtw.as<double>(), pl->nA,
                              pl->ka_pad, 0, pl->MN, nullptr, ws.x.as<double>(), st));
    else
        SE_CUDA(launch_pack_x(ddesc, n, pl->d_a_idx.as<int>(), pl->d_sqrtw.as<double>(), pl->nA,
                              pl->ka_pad, pl->pc.nparts, pl->MN, ws.x.as<uint16_t>(), nullptr, st));
    stage_end(ctx, tok, st);
    tok = stage_begin(ctx, 2, st);
    if (fp64) {
        SE_CUDA(launch_simt_gemm<double>(pl->d_G64.as<double>(), pl->ka_pad, ws.x.as<double>(),
                                         pl->ka_pad, Kp, n, pl->ka_pad, ws.r0.as<double>(), Kp,
                                         0, st));
    } else {
        TcGemmArgs g{};
        g.A = pl->d_Gwbf.ptr;
        g.B = ws.x.ptr;
        g.M = Kp;
        g.N = n;
        g.lda = g.ldb = pl->pc.nparts * pl->ka_pad;
        g.ka_pad = pl->ka_pad;
        g.npairs = pl->pc.npairs;
        for (int i = 0; i < 8; ++i) { g.pa[i] = pl->pc.pa[i]; g.pb[i] = pl->pc.pb[i]; }
        g.out = ws.r0.as<float>();
        g.ldo = Kp;
        g.symmetric = 0;
        g.grouped = 1;
        g.err = ctx->ws_err.as<int>();
        g.scale = pl->d_Dk.as<float>();
        const std::string key = "gemm_projg:" + std::to_string(Kp) + ":" + std::to_string(pl->ka_pad) + ":p" +
                                std::to_string(pl->pc.npairs) + ":n" + nclass(n);
        cudaError_t e = tune_run(ctx, key, tc_gemm_variants(g), st,
                                 [&](int v) { return launch_tc_gemm(g, st, &why, v); });
        if (e != cudaSuccess) return fail(SE_ERR_CUDA, "projection GEMM: " + why + " " + cudaGetErrorString(e));
    }
    stage_end(ctx, tok, st);
    ctx->launches += 2;
    return SE_OK;
}

}  // namespace

// All blocks use the plan's pattern: Alg. 2 tables (cached), eq. (12) GEMM,
// Alg. 3 iterations.
se_status se::run_batch(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, int n, const BlockDesc *hdesc,
                        int I_max, cudaStream_t st, cudaEvent_t inputs_ready, const StridedSpec *ss,
                        cudaEvent_t r0_done)
{
    const int Kp = pl->Kp;
    const bool fp64 = pl->pc.fp64;
    const size_t tsz = fp64 ? sizeof(double) : sizeof(float);
    const size_t xrow = fp64 ? static_cast<size_t>(pl->ka_pad) * sizeof(double)
                             : static_cast<size_t>(pl->pc.nparts) * pl->ka_pad * 2;

    // the workspace of the previous call must be free before it is reused
    SE_CUDA(cudaStreamWaitEvent(st, ws.ev_ws, 0));

    // The fp32 transform form computes R^(0) unscaled (the iteration kernel
    // applies D_k when it loads them), so a table build does not have to come
    // first: it runs on the context's second stream, from here on (it reads no
    // descriptor), while the descriptors are staged and R^(0) is computed, and
    // the iterations wait for it.
    const bool overlap = pl->sep_full && !fp64;
    {
        std::lock_guard<std::mutex> lk(pl->tmu);
        if (!pl->tables_valid) {
            cudaStream_t ts = st;
            if (overlap) {   // the second stream starts after the work already queued on st
                std::lock_guard<std::mutex> al(ctx->amu);
                SE_CUDA(cudaEventRecord(ctx->ev_fork, st));
                SE_CUDA(cudaStreamWaitEvent(ctx->aux, ctx->ev_fork, 0));
                ts = ctx->aux;
            }
            const int tok = stage_begin(ctx, 1, ts);
            cudaEvent_t pa = probe_begin(ctx, ts);
            SE_TRY(build_tables(ctx, pl, ts));
            probe_end(ctx, pl, 0, 0, pa, ts);
            stage_end(ctx, tok, ts);
        } else if (!overlap) {
            SE_CUDA(cudaStreamWaitEvent(st, pl->tables_ready, 0));
        }
    }

    const size_t need_desc = sizeof(BlockDesc) * n, need_x = pl->sep_full ? 16 : xrow * n,
                 need_r0 = (pl->cplx ? 2 : 1) * tsz * Kp * static_cast<size_t>(n);
    if (ws.desc.bytes < need_desc || ws.x.bytes < need_x || ws.r0.bytes < need_r0)
        SE_CUDA(cudaEventSynchronize(ws.ev_ws));
    const size_t need_logs = fp64 ? 16 : 8 * static_cast<size_t>(n) * I_max;
    if (ws.logs.bytes < need_logs) SE_CUDA(cudaEventSynchronize(ws.ev_ws));
    if (pl->certified) {
        if (ws.cert.bytes < sizeof(int) * static_cast<size_t>(n)) SE_CUDA(cudaEventSynchronize(ws.ev_ws));
        SE_TRY(dev_alloc(ctx, ws.cert, sizeof(int) * static_cast<size_t>(n)));
    }
    SE_TRY(dev_alloc(ctx, ws.desc, need_desc));
    SE_TRY(dev_alloc(ctx, ws.x, need_x));
    SE_TRY(dev_alloc(ctx, ws.r0, need_r0));
    SE_TRY(dev_alloc(ctx, ws.logs, need_logs));

    if (ss) {   // a contiguous batch: the descriptors are formed on the device
        SE_CUDA(launch_fill_desc(ws.desc.as<BlockDesc>(), n, *ss, pl->MN, st));
        ctx->launches += 1;
    } else {
        // pinned staging of the descriptors: free once the previous copy landed
        SE_CUDA(cudaEventSynchronize(ws.ev_staging));
        if (ws.h_desc_cap < static_cast<size_t>(n)) {
            if (ws.h_desc) cudaFreeHost(ws.h_desc);
            ws.h_desc = nullptr;
            ws.h_desc_cap = 0;
            SE_CUDA(cudaMallocHost(&ws.h_desc, sizeof(BlockDesc) * n));
            ws.h_desc_cap = n;
        }
        std::memcpy(ws.h_desc, hdesc, sizeof(BlockDesc) * n);
        SE_CUDA(cudaMemcpyAsync(ws.desc.ptr, ws.h_desc, sizeof(BlockDesc) * n,
                                cudaMemcpyHostToDevice, st));
        SE_CUDA(cudaEventRecord(ws.ev_staging, st));
    }
    if (inputs_ready) SE_CUDA(cudaStreamWaitEvent(st, inputs_ready, 0));   // the samples have landed

    if (pl->cplx) return run_complex(ctx, pl, ws, n, I_max, st);
    const BlockDesc *ddesc = ws.desc.as<BlockDesc>();
    cudaEvent_t probe = probe_begin(ctx, st);
    int tok;
    if (pl->sep_full) {
        // eq. (12) as a separable transform of w s per block: no packing stage
        tok = stage_begin(ctx, 2, st);
        SE_CUDA(launch_pattern_projections(ctx, pl, ddesc, n, ws.r0.ptr, !overlap, st));
        stage_end(ctx, tok, st);
        if (r0_done) SE_CUDA(cudaEventRecord(r0_done, st));
        if (overlap) SE_CUDA(cudaStreamWaitEvent(st, pl->tables_ready, 0));   // the (forked) table build
        ctx->launches += 1;
    } else {
        SE_TRY(dense_pattern_projections(ctx, pl, ws, ddesc, n, st));
        if (r0_done) SE_CUDA(cudaEventRecord(r0_done, st));
    }

    IterArgs a{};
    a.blocks = ddesc;
    a.n = n;
    a.K = pl->K;
    a.Kp = Kp;
    a.R0 = ws.r0.ptr;
    a.C = pl->d_C.ptr;
    a.invC = pl->d_invC.ptr;
    a.Dk = pl->d_Dk.ptr;
    a.PhiB = pl->d_PhiB.ptr;
    a.b_idx = pl->d_b_idx.as<int>();
    a.pat_support = pl->d_pattern.as<uint8_t>();
    a.nB = pl->nB;
    a.MN = pl->MN;
    a.gamma = pl->desc.gamma;
    a.I_max = I_max;
    a.err = ctx->ws_err.as<int>();
    if (overlap) a.r0_scale = pl->d_Dk.as<float>();
    if (!fp64) {
        a.log_u = ws.logs.as<int>();
        a.log_c = reinterpret_cast<float *>(ws.logs.as<int>() + static_cast<size_t>(n) * I_max);
    }
    if (pl->certified) {
        a.cert_flag = ws.cert.as<int>();
        a.cert_delta = kCertGap;
    }
    int launched = 0;
    bool model_done = false;   // the model of eq. (9) ran with the iterations
    tok = stage_begin(ctx, 3, st);
    cudaError_t e = fp64 ? launch_iterate_full<double>(a, st, &launched)
                         : launch_iterations_f32(ctx, pl, a, st, &launched, &model_done);
    stage_end(ctx, tok, st);
    if (e == cudaSuccess && !fp64 && !model_done) {
        tok = stage_begin(ctx, 4, st);
        e = launch_model(pl, a, st);
        stage_end(ctx, tok, st);
        ++launched;
    }
    if (e != cudaSuccess) return fail(SE_ERR_CUDA, std::string("iteration kernel: ") + cudaGetErrorString(e));
    ctx->launches += launched;
    probe_end(ctx, pl, 1, n, probe, st);
    SE_CUDA(cudaEventRecord(ws.ev_ws, st));
    if (pl->certified) {
        // blocks with a selection inside the certification gap: recompute in fp64
        std::vector<int> flag(n);
        SE_CUDA(cudaMemcpyAsync(flag.data(), ws.cert.ptr, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
        SE_CUDA(cudaStreamSynchronize(st));
        std::vector<BlockDesc> again;
        int I_again = 0;
        for (int i = 0; i < n; ++i)
            if (flag[i] >= 0) {
                BlockDesc x;
                if (hdesc) {
                    x = hdesc[i];
                } else {
                    const size_t MN = static_cast<size_t>(pl->MN);
                    x.samples = ss->samples + MN * i;
                    x.support = nullptr;
                    x.out = ss->out + MN * i;
                    x.sel_idx = ss->sel_idx ? ss->sel_idx + static_cast<size_t>(ss->I) * i : nullptr;
                    x.sel_coef = ss->sel_coef ? ss->sel_coef + static_cast<size_t>(ss->I) * ss->coef * i : nullptr;
                    x.iterations = ss->I;
                    x.pad_ = 0;
                }
                again.push_back(x);
                I_again = std::max(I_again, x.iterations);
            }
        ctx->cert_blocks += n;
        ctx->cert_recomputed += again.size();
        if (!again.empty())
            SE_TRY(run_batch(ctx, pl->shadow, ws, static_cast<int>(again.size()), again.data(), I_again, st));
    }
    return SE_OK;
}

namespace {

}  // namespace

se_status se::ensure_tables(se_ctx_s *ctx, se_plan_s *pl, cudaStream_t st)
{
    std::lock_guard<std::mutex> lk(pl->tmu);
    if (!pl->tables_valid) return build_tables(ctx, pl, st);
    SE_CUDA(cudaStreamWaitEvent(st, pl->tables_ready, 0));
    return SE_OK;
}

namespace {

se_status resolve_blocks(se_plan_s *pl, int n, const se_block *blocks, std::vector<BlockDesc> &d,
                         int *I_max, bool *any_mask)
{
    d.resize(n);
    *I_max = 0;
    *any_mask = false;
    for (int i = 0; i < n; ++i) {
        const se_block &b = blocks[i];
        if (!b.samples || !b.out) return fail(SE_ERR_INVALID, "block " + std::to_string(i) + ": NULL samples or out");
        if (b.iterations < 0) return fail(SE_ERR_INVALID, "block " + std::to_string(i) + ": iterations < 0");
        BlockDesc &x = d[i];
        x.samples = b.samples;
        x.support = b.support;
        x.out = b.out;
        x.sel_idx = b.sel_idx;
        x.sel_coef = b.sel_coef;
        x.iterations = b.iterations ? b.iterations : pl->desc.iterations;
        x.pad_ = 0;
        *I_max = std::max(*I_max, x.iterations);
        *any_mask |= b.support != nullptr;
    }
    return SE_OK;
}

}  // namespace

extern "C" {

const char *se_last_error(void) { return g_err.c_str(); }

se_status se_ctx_create(int device, size_t hbm_budget_bytes, se_ctx_t **out)
{
    if (!out) return fail(SE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    SE_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SE_ERR_INVALID, "no such CUDA device");
    SE_CUDA(cudaSetDevice(device));
    cudaDeviceProp prop;
    SE_CUDA(cudaGetDeviceProperties(&prop, device));
    if (prop.major < 10) return fail(SE_ERR_CUDA, "libse needs a Blackwell (sm_10x) GPU");
    auto *c = new se_ctx_s();
    c->device = device;
    c->budget = hbm_budget_bytes;
    c->tuner.load_env();
    cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = c->ws.init();
    if (e != cudaSuccess) {
        delete c;
        return fail(SE_ERR_CUDA, std::string("context set-up: ") + cudaGetErrorString(e));
    }
    se_status s = dev_alloc(c, c->ws_err, sizeof(int));
    if (s != SE_OK) { delete c; return s; }
    // the static scratch of se_extrapolate_noalloc: its address on this device
    // (looked up here, with the device current, so that the calls need no set-up)
    s = noalloc_scratch_address(&c->noalloc_scratch);
    if (s != SE_OK) { delete c; return s; }
    e = cudaMemset(c->ws_err.ptr, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete c;
        return fail(SE_ERR_CUDA, std::string("context set-up: ") + cudaGetErrorString(e));
    }
    *out = c;
    return SE_OK;
}

se_status se_ctx_destroy(se_ctx_t *ctx)
{
    if (!ctx) return SE_OK;
    cudaSetDevice(ctx->device);
    serve_shutdown(ctx);
    cudaDeviceSynchronize();
    for (auto &p : ctx->pending) {
        cudaEventDestroy(p.second.first);
        cudaEventDestroy(p.second.second);
    }
    for (auto e : ctx->event_pool) cudaEventDestroy(e);
    ctx->tuner.save();
    graphs_clear(ctx);
    probes_poll(ctx, true);
    for (auto e : ctx->probe_pool) cudaEventDestroy(e);
    ctx->probe_pool.clear();
    std::vector<se_plan_s *> plans = ctx->plans;
    for (auto *p : plans) se_plan_destroy(p);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    for (int i = 0; i < se_ctx_s::kPipe; ++i) {
        if (ctx->pipe_st[i]) cudaStreamDestroy(ctx->pipe_st[i]);
        if (ctx->pipe_ev_in[i]) cudaEventDestroy(ctx->pipe_ev_in[i]);
        if (ctx->pipe_ev_done[i]) cudaEventDestroy(ctx->pipe_ev_done[i]);
    }
    if (ctx->pipe_in) cudaStreamDestroy(ctx->pipe_in);
    if (ctx->pipe_out) cudaStreamDestroy(ctx->pipe_out);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
    delete ctx;
    return SE_OK;
}

se_status se_plan(se_ctx_t *ctx, const se_plan_desc *desc, se_plan_t **out)
{
    if (!ctx || !desc || !out) return fail(SE_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const se_plan_desc &d = *desc;
    if (d.M < 1 || d.N < 1 || d.M > 256 || d.N > 256) return fail(SE_ERR_INVALID, "M and N must be in [1, 256]");
    const int T = d.T == 0 ? 1 : d.T;
    if (T < 1 || T > 64) return fail(SE_ERR_INVALID, "T must be in [1, 64] (0 = 1)");
    if (static_cast<long long>(d.M) * d.N * T > 65536)
        return fail(SE_ERR_INVALID, "M N T must be at most 65536 samples");
    if (!(d.rho_hat > 0.0 && d.rho_hat <= 1.0)) return fail(SE_ERR_INVALID, "rho_hat must be in (0, 1]");
    if (!(d.gamma > 0.0 && d.gamma <= 1.0)) return fail(SE_ERR_INVALID, "gamma must be in (0, 1]");
    if (d.iterations < 1) return fail(SE_ERR_INVALID, "iterations must be >= 1");
    if (d.prec != SE_PREC_FP64 && d.prec != SE_PREC_BF16X6 && d.prec != SE_PREC_BF16X3 &&
        d.prec != SE_PREC_BF16 && d.prec != SE_PREC_CERTIFIED)
        return fail(SE_ERR_INVALID, "unknown precision");
    if (d.prec == SE_PREC_CERTIFIED && d.gram == SE_GRAM_LAZY)
        return fail(SE_ERR_INVALID, "certified plans serve the plan's pattern (gram LAZY not supported)");
    if (d.gram < SE_GRAM_AUTO || d.gram > SE_GRAM_LAZY) return fail(SE_ERR_INVALID, "unknown table mode");
    if (d.products < SE_PRODUCTS_AUTO || d.products > SE_PRODUCTS_TRANSFORM)
        return fail(SE_ERR_INVALID, "unknown product mode");
    SE_CUDA(cudaSetDevice(ctx->device));

    auto pl = std::make_unique<se_plan_s>();
    pl->ctx = ctx;
    pl->desc = d;
    pl->desc.dict = nullptr;
    pl->desc.rho = nullptr;
    pl->desc.support = nullptr;
    pl->M = d.M;
    pl->N = d.N;
    pl->T = T;
    pl->desc.T = T;
    pl->MN = d.M * d.N * T;
    pl->K = d.K;
    pl->pc = prec_cfg(d.prec);
    std::string why;
    pl->cplx = d.basis == SE_BASIS_DFT || d.basis == SE_BASIS_BDFT || d.basis == SE_BASIS_DFT_BDFT;
    if (pl->cplx) {
        if (T != 1) return fail(SE_ERR_INVALID, "complex atoms: 2-D areas only (T = 1)");
        if (d.prec != SE_PREC_FP64 && d.prec != SE_PREC_BF16X6)
            return fail(SE_ERR_INVALID, "complex atoms: precision FP64 or BF16X6");
        if (d.gram == SE_GRAM_LAZY) return fail(SE_ERR_INVALID, "complex atoms: the plan's pattern only (gram LAZY)");
        if (d.products == SE_PRODUCTS_TRANSFORM) return fail(SE_ERR_INVALID, "complex atoms use the dense products");
        if (!build_complex_dictionary(d.M, d.N, d.basis, d.K, pl->phi, pl->phi_im, &why))
            return fail(SE_ERR_INVALID, why);
    } else if (!build_dictionary(d.M, d.N, T, d.basis, d.K, d.dict, pl->phi, &why)) {
        return fail(SE_ERR_INVALID, why);
    }
    const int MN = pl->MN, K = pl->K;
    pl->Kp = iterate_kp(K, pl->pc.fp64);
    if (pl->Kp < 0) return fail(SE_ERR_INVALID, "K is larger than the iteration kernel supports (16384)");
    pl->certified = d.prec == SE_PREC_CERTIFIED;
    if (pl->certified && pl->Kp > iterate_cert_max_kp())
        return fail(SE_ERR_INVALID, "certified plans support K <= " + std::to_string(iterate_cert_max_kp()));
    if (pl->cplx) find_collinear_complex(K, MN, pl->phi.data(), pl->phi_im.data(), pl->dup);
    else find_collinear(K, MN, pl->phi.data(), pl->dup);

    pl->pattern.assign(MN, 1);
    if (d.support) {
        for (int i = 0; i < MN; ++i) pl->pattern[i] = d.support[i] ? 1 : 0;
    } else {
        // the centred loss box: M/2 x N/2 samples in frames T/4 .. T/4 + max(T/2, 1) - 1
        for (int t = T / 4; t < T / 4 + std::max(T / 2, 1); ++t)
            for (int m = d.M / 4; m < d.M / 4 + d.M / 2; ++m)
                for (int n = d.N / 4; n < d.N / 4 + d.N / 2; ++n) pl->pattern[(t * d.M + m) * d.N + n] = 0;
    }
    if (d.rho) pl->rho_map.assign(d.rho, d.rho + MN);
    weighting(d.M, d.N, T, d.rho_hat, d.rho, pl->pattern.data(), pl->w);
    for (int i = 0; i < MN; ++i) {
        if (pl->pattern[i] && !(pl->w[i] >= 0.0 && std::isfinite(pl->w[i])))
            return fail(SE_ERR_INVALID, "rho must be finite and non-negative");
        if (pl->pattern[i] && pl->w[i] > 0.0) pl->a_idx.push_back(i);
        else if (!pl->pattern[i]) pl->b_idx.push_back(i);
    }
    pl->box[0] = d.M; pl->box[1] = 0; pl->box[2] = d.N; pl->box[3] = 0;   // (2-D areas only)
    for (int m = 0; m < d.M && T == 1; ++m)
        for (int n = 0; n < d.N; ++n)
            if (!pl->pattern[m * d.N + n]) {
                pl->box[0] = std::min(pl->box[0], m); pl->box[1] = std::max(pl->box[1], m + 1);
                pl->box[2] = std::min(pl->box[2], n); pl->box[3] = std::max(pl->box[3], n + 1);
            }
    // support pixels with zero weight contribute nothing; they keep their samples
    pl->nA = static_cast<int>(pl->a_idx.size());
    pl->nB = static_cast<int>(pl->b_idx.size());
    if (pl->nA == 0) return fail(SE_ERR_EMPTY_SUPPORT, "the default pattern has no weighted support");
    {   // at least one admissible atom (same rule as the device tables)
        double mx = 0.0;
        std::vector<double> dg(K, 0.0);
        for (int k = 0; k < K; ++k) {
            const double *a = pl->phi.data() + static_cast<size_t>(k) * MN;
            const double *b = pl->cplx ? pl->phi_im.data() + static_cast<size_t>(k) * MN : nullptr;
            double s = 0.0;
            for (int i : pl->a_idx) s += (a[i] * a[i] + (b ? b[i] * b[i] : 0.0)) * pl->w[i];
            dg[k] = s;
            if (!pl->dup[k]) mx = std::max(mx, s);
        }
        int adm = 0;
        for (int k = 0; k < K; ++k) adm += !pl->dup[k] && mx > 0.0 && dg[k] > 1e-14 * mx;
        if (adm == 0) return fail(SE_ERR_EMPTY_SUPPORT, "no atom has weighted energy on the support");
    }
    pl->ka_pad = static_cast<int>(round_up(pl->nA, 64));
    const int Kp = pl->Kp, ka = pl->ka_pad;

    std::vector<double> sqw(pl->nA);
    for (int j = 0; j < pl->nA; ++j) sqw[j] = std::sqrt(pl->w[pl->a_idx[j]]);
    if (!pl->cplx) {
        std::vector<double> G(static_cast<size_t>(Kp) * ka, 0.0);
        for (int k = 0; k < K; ++k) {
            const double *a = pl->phi.data() + static_cast<size_t>(k) * MN;
            for (int j = 0; j < pl->nA; ++j) G[static_cast<size_t>(k) * ka + j] = a[pl->a_idx[j]] * sqw[j];
        }
        SE_TRY(upload(ctx, pl->d_G64, G));
    }
    std::vector<uint8_t> dupp(Kp, 1);
    for (int k = 0; k < K; ++k) dupp[k] = pl->dup[k];
    SE_TRY(upload(ctx, pl->d_sqrtw, sqw));

    SE_TRY(upload(ctx, pl->d_a_idx, pl->a_idx));
    SE_TRY(upload(ctx, pl->d_b_idx, pl->b_idx));
    SE_TRY(upload(ctx, pl->d_pattern, pl->pattern));
    SE_TRY(upload(ctx, pl->d_dup, dupp));
    const size_t nBa = std::max(pl->nB, 1);
    if (pl->cplx) {
        SE_TRY(setup_complex_plan(ctx, pl.get(), ctx->stream));
    } else if (pl->pc.fp64) {
        std::vector<double> pb(static_cast<size_t>(Kp) * nBa, 0.0);
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < pl->nB; ++j)
                pb[static_cast<size_t>(k) * nBa + j] = pl->phi[static_cast<size_t>(k) * MN + pl->b_idx[j]];
        SE_TRY(upload(ctx, pl->d_PhiB, pb));
    } else {
        std::vector<float> pb(static_cast<size_t>(Kp) * nBa, 0.0f);
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < pl->nB; ++j)
                pb[static_cast<size_t>(k) * nBa + j] =
                    static_cast<float>(pl->phi[static_cast<size_t>(k) * MN + pl->b_idx[j]]);
        SE_TRY(upload(ctx, pl->d_PhiB, pb));
        if (d.prec == SE_PREC_BF16X6) {
            // the table of eq. (16) from two fp16 parts per entry of G (11 + 11 significant
            // bits) and three products, about 2^-21 relative like the six split-bf16
            // products, for half the tensor work and two thirds of the operand bytes; G is
            // scaled by a power of two that puts its largest entry at or below 2^14 (no
            // overflow of either part, low parts normal) and the epilogue undoes it
            double gmax = 0.0;
            for (int k = 0; k < K; ++k)
                for (int j = 0; j < pl->nA; ++j)
                    gmax = std::max(gmax, std::fabs(pl->phi[static_cast<size_t>(k) * MN + pl->a_idx[j]] * sqw[j]));
            pl->g_f16_scale = gmax > 0.0 ? static_cast<float>(std::ldexp(1.0, 14 - static_cast<int>(std::ceil(std::log2(gmax)))))
                                         : 1.0f;
            SE_TRY(dev_alloc(ctx, pl->d_GH, static_cast<size_t>(Kp) * 2 * ka * 2));
            SE_CUDA(launch_split_f16(pl->d_G64.as<double>(), Kp, ka, ka, ka, pl->g_f16_scale, pl->d_GH.as<uint16_t>(),
                                     ctx->stream));
            pl->f16_table = true;
        } else {
            SE_TRY(dev_alloc(ctx, pl->d_Gbf, static_cast<size_t>(Kp) * pl->pc.nparts * ka * 2));
            SE_CUDA(launch_split_bf16(pl->d_G64.as<double>(), Kp, ka, ka, ka, pl->pc.nparts,
                                      pl->d_Gbf.as<uint16_t>(), ctx->stream));
        }
        // Phi_A w for the projections of eq. (12): the samples enter unweighted
        std::vector<double> Gw(static_cast<size_t>(Kp) * ka, 0.0);
        for (int k = 0; k < K; ++k) {
            const double *a = pl->phi.data() + static_cast<size_t>(k) * MN;
            for (int j = 0; j < pl->nA; ++j)
                Gw[static_cast<size_t>(k) * ka + j] = a[pl->a_idx[j]] * pl->w[pl->a_idx[j]];
        }
        DevBuf tmp;
        SE_TRY(upload(ctx, tmp, Gw));
        SE_TRY(dev_alloc(ctx, pl->d_Gwbf, static_cast<size_t>(Kp) * pl->pc.nparts * ka * 2));
        SE_CUDA(launch_split_bf16(tmp.as<double>(), Kp, ka, ka, ka, pl->pc.nparts,
                                  pl->d_Gwbf.as<uint16_t>(), ctx->stream));
        SE_CUDA(cudaStreamSynchronize(ctx->stream));
        ctx->launches += 2;
    }
    if (d.products != SE_PRODUCTS_DENSE) {
        SE_TRY(ensure_sep_ops(ctx, pl.get()));
        if (!pl->sep && d.products == SE_PRODUCTS_TRANSFORM)
            return fail(SE_ERR_INVALID, "transform products need a DCT / WHT dictionary whose "
                                        "transforms fit in shared memory");
        pl->sep_full = pl->sep;
    }
    SE_TRY(setup_sym(ctx, pl.get()));
    const size_t tsz = pl->pc.fp64 ? 8 : 4;
    SE_TRY(dev_alloc(ctx, pl->d_C, pl->dft_w ? 16 : (pl->cplx ? 2 : 1) * tsz * Kp * static_cast<size_t>(Kp)));
    SE_TRY(dev_alloc(ctx, pl->d_invC, tsz * Kp));
    SE_TRY(dev_alloc(ctx, pl->d_Dk, tsz * Kp));
    SE_TRY(dev_alloc(ctx, pl->d_diag, sizeof(double) * Kp));
    SE_TRY(dev_alloc(ctx, pl->d_nadm, 16));   // admissible count (int) + largest C_kk (8 bytes at +8)
    SE_CUDA(cudaEventCreateWithFlags(&pl->tables_ready, cudaEventDisableTiming));
    SE_CUDA(cudaStreamSynchronize(ctx->stream));
    if (pl->certified) {
        // the internal FP64 plan that recomputes the flagged blocks; owned by
        // this plan (not listed in the context)
        se_plan_desc d64 = d;
        d64.prec = SE_PREC_FP64;
        se_plan_s *sh = nullptr;
        SE_TRY(se_plan(ctx, &d64, &sh));
        {
            std::lock_guard<std::mutex> lk(ctx->smu);
            ctx->plans.erase(std::remove(ctx->plans.begin(), ctx->plans.end(), sh), ctx->plans.end());
        }
        pl->shadow = sh;
    }
    se_plan_s *raw = pl.release();
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->plans.push_back(raw);
    }
    *out = raw;
    return SE_OK;
}

se_status se_plan_destroy(se_plan_t *plan)
{
    if (!plan) return SE_OK;
    se_ctx_s *ctx = plan->ctx;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    probes_poll(ctx, true, plan);
    graphs_drop_plan(ctx, plan);
    if (plan->shadow) {
        probes_poll(ctx, true, plan->shadow);
        graphs_drop_plan(ctx, plan->shadow);
        if (plan->shadow->tables_ready) cudaEventDestroy(plan->shadow->tables_ready);
        delete plan->shadow;
        plan->shadow = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->plans.erase(std::remove(ctx->plans.begin(), ctx->plans.end(), plan), ctx->plans.end());
    }
    if (plan->tables_ready) cudaEventDestroy(plan->tables_ready);
    delete plan;
    return SE_OK;
}

se_status se_plan_reset_tables(se_plan_t *plan)
{
    if (!plan) return fail(SE_ERR_INVALID, "NULL plan");
    std::lock_guard<std::mutex> lk(plan->tmu);
    plan->tables_valid = false;
    return SE_OK;
}

namespace {

// Pattern blocks (routed to the table or the lazy columns) and mask blocks of
// one call, on workspace ws and stream st; ctx->mu is held by the caller.
se_status run_resolved(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, std::vector<BlockDesc> &full, int I_full,
                       std::vector<BlockDesc> &lazy, int I_lazy, cudaStream_t st,
                       cudaEvent_t inputs_ready = nullptr)
{
    probes_poll(ctx, false);
    route_pattern_blocks(pl, full, lazy, &I_full, &I_lazy);
    if (!full.empty())
        SE_TRY(run_batch(ctx, pl, ws, static_cast<int>(full.size()), full.data(), I_full, st, inputs_ready));
    if (!lazy.empty()) {
        if (inputs_ready && full.empty()) SE_CUDA(cudaStreamWaitEvent(st, inputs_ready, 0));
        SE_TRY(run_lazy(ctx, pl, ws, static_cast<int>(lazy.size()), lazy.data(), I_lazy, st));
    }
    return SE_OK;
}

// Descriptors of n contiguous pattern blocks (samples / out M x N each, logs
// [b][I], complex coefficient logs [b][I][2]).
void strided_desc(const se_plan_s *pl, int n, const double *samples, double *out, int32_t *sel_idx,
                  double *sel_coef, int I, std::vector<BlockDesc> &d)
{
    const size_t MN = static_cast<size_t>(pl->MN);
    d.resize(n);
    for (int i = 0; i < n; ++i) {
        d[i].samples = samples + MN * i;
        d[i].support = nullptr;
        d[i].out = out + MN * i;
        d[i].sel_idx = sel_idx ? sel_idx + static_cast<size_t>(I) * i : nullptr;
        d[i].sel_coef = sel_coef ? sel_coef + static_cast<size_t>(pl->cplx ? 2 : 1) * I * i : nullptr;
        d[i].iterations = I;
        d[i].pad_ = 0;
    }
}

// Streams, events and workspaces of the chunked host-buffer calls (ctx->mu held).
se_status pipe_init(se_ctx_s *ctx)
{
    if (ctx->pipe_ready) return SE_OK;
    for (int i = 0; i < se_ctx_s::kPipe; ++i) {
        SE_CUDA(cudaStreamCreateWithFlags(&ctx->pipe_st[i], cudaStreamNonBlocking));
        SE_CUDA(cudaEventCreateWithFlags(&ctx->pipe_ev_in[i], cudaEventDisableTiming));
        SE_CUDA(cudaEventCreateWithFlags(&ctx->pipe_ev_done[i], cudaEventDisableTiming));
        SE_CUDA(ctx->pipe_ws[i].init());
    }
    SE_CUDA(cudaStreamCreateWithFlags(&ctx->pipe_in, cudaStreamNonBlocking));
    SE_CUDA(cudaStreamCreateWithFlags(&ctx->pipe_out, cudaStreamNonBlocking));
    ctx->pipe_ready = true;
    return SE_OK;
}

// A contiguous batch of pattern blocks on workspace ws and stream st (ctx->mu
// held): the table path with descriptors formed on the device, or the lazy
// columns when the plan (LAZY) or the measured costs (AUTO) say so.
se_status run_strided(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, int n, const StridedSpec &ss, cudaStream_t st,
                      cudaEvent_t inputs_ready = nullptr, cudaEvent_t r0_done = nullptr)
{
    probes_poll(ctx, false);
    if (pl->desc.gram == SE_GRAM_LAZY || choose_lazy_for_pattern(pl, n)) {
        std::vector<BlockDesc> d;
        strided_desc(pl, n, ss.samples, ss.out, ss.sel_idx, ss.sel_coef, ss.I, d);
        for (auto &x : d) x.support = pl->d_pattern.as<uint8_t>();
        if (inputs_ready) SE_CUDA(cudaStreamWaitEvent(st, inputs_ready, 0));
        SE_TRY(run_lazy(ctx, pl, ws, n, d.data(), ss.I, st));
        if (r0_done) SE_CUDA(cudaEventRecord(r0_done, st));
        return SE_OK;
    }
    return run_batch(ctx, pl, ws, n, nullptr, ss.I, st, inputs_ready, &ss, r0_done);
}

}  // namespace

se_status se_extrapolate_batch(se_ctx_t *ctx, const se_plan_t *plan, int n, const se_block *blocks,
                               void *cuda_stream)
{
    if (!ctx || !plan || (n > 0 && !blocks) || n < 0) return fail(SE_ERR_INVALID, "NULL argument or n < 0");
    if (n == 0) return SE_OK;
    if (plan->ctx != ctx) return fail(SE_ERR_INVALID, "plan belongs to another context");
    SE_CUDA(cudaSetDevice(ctx->device));
    se_plan_s *pl = const_cast<se_plan_s *>(plan);
    std::vector<BlockDesc> d;
    int I_max = 0;
    bool any_mask = false;
    SE_TRY(resolve_blocks(pl, n, blocks, d, &I_max, &any_mask));
    if (any_mask && pl->desc.gram == SE_GRAM_FULL)
        return fail(SE_ERR_INVALID, "per-block support masks need the lazy table path (plan gram is FULL)");
    if (any_mask && (pl->certified || pl->cplx))
        return fail(SE_ERR_INVALID, "certified and complex plans serve blocks on the plan's pattern only");
    // blocks on the plan's pattern use the full table (unless LAZY is forced);
    // blocks with their own mask use lazily computed columns
    std::vector<BlockDesc> full, lazy;
    int I_full = 0, I_lazy = 0;
    for (auto &x : d) {
        if (!x.support && pl->desc.gram != SE_GRAM_LAZY) {
            full.push_back(x);
            I_full = std::max(I_full, x.iterations);
        } else {
            if (!x.support) x.support = pl->d_pattern.as<uint8_t>();
            lazy.push_back(x);
            I_lazy = std::max(I_lazy, x.iterations);
        }
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    return run_resolved(ctx, pl, ctx->ws, full, I_full, lazy, I_lazy, static_cast<cudaStream_t>(cuda_stream));
}

se_status se_extrapolate_strided(se_ctx_t *ctx, const se_plan_t *plan, int n, const double *samples,
                                 double *out, int32_t *sel_idx, double *sel_coef, int iterations,
                                 void *cuda_stream)
{
    if (!ctx || !plan || n < 0) return fail(SE_ERR_INVALID, "NULL argument or n < 0");
    if (n == 0) return SE_OK;
    if (!samples || !out) return fail(SE_ERR_INVALID, "NULL samples or out");
    if (iterations < 0) return fail(SE_ERR_INVALID, "iterations < 0");
    if (plan->ctx != ctx) return fail(SE_ERR_INVALID, "plan belongs to another context");
    SE_CUDA(cudaSetDevice(ctx->device));
    const int I = iterations ? iterations : plan->desc.iterations;
    const StridedSpec ss{samples, out, sel_idx, sel_coef, I, plan->cplx ? 2 : 1};
    std::lock_guard<std::mutex> lk(ctx->mu);
    return run_strided(ctx, const_cast<se_plan_s *>(plan), ctx->ws, n, ss, static_cast<cudaStream_t>(cuda_stream));
}

se_status se_check_wait_timeout(se_ctx_t *ctx, uint32_t limit_us, void *cuda_stream)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    if (limit_us < 1000 || limit_us > 2000000) return fail(SE_ERR_INVALID, "limit_us outside [1000, 2000000]");
    SE_CUDA(cudaSetDevice(ctx->device));
    SE_CUDA(launch_wait_probe(ctx->ws_err.as<int>(), 1000ull * limit_us, static_cast<cudaStream_t>(cuda_stream)));
    ctx->launches += 1;
    return SE_OK;
}

se_status se_check_sample_conversion(se_ctx_t *ctx, const double *in, float *out, double *back, int n,
                                     void *cuda_stream)
{
    if (!ctx || n < 0 || (n > 0 && (!in || !out))) return fail(SE_ERR_INVALID, "NULL argument or n < 0");
    SE_CUDA(cudaSetDevice(ctx->device));
    SE_CUDA(launch_convert_probe(in, out, back, n, static_cast<cudaStream_t>(cuda_stream)));
    ctx->launches += n > 0;
    return SE_OK;
}

se_status se_sync(se_ctx_t *ctx, void *cuda_stream)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    SE_CUDA(cudaSetDevice(ctx->device));
    SE_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    std::lock_guard<std::mutex> lk(ctx->mu);
    int bits = 0;
    SE_CUDA(cudaMemcpy(&bits, ctx->ws_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) {
        SE_CUDA(cudaMemset(ctx->ws_err.ptr, 0, sizeof(int)));
        const se_status code = bits == (1 << DEV_ERR_EMPTY_SUPPORT) ? SE_ERR_EMPTY_SUPPORT : SE_ERR_CUDA;
        return fail(code, std::string("device status: ") + dev_err_text(bits));
    }
    return SE_OK;
}

se_status se_extrapolate_host(se_ctx_t *ctx, const se_plan_t *plan, int n, const double *samples,
                              double *out, int32_t *sel_idx, double *sel_coef, int iterations)
{
    if (!ctx || !plan || n < 0) return fail(SE_ERR_INVALID, "NULL argument or n < 0");
    if (plan->cplx) return fail(SE_ERR_INVALID, "complex plans: device entry points only");
    if (n == 0) return SE_OK;
    if (!samples || !out) return fail(SE_ERR_INVALID, "NULL samples or out");
    if (iterations < 0) return fail(SE_ERR_INVALID, "iterations < 0");
    if (plan->ctx != ctx) return fail(SE_ERR_INVALID, "plan belongs to another context");
    SE_CUDA(cudaSetDevice(ctx->device));
    se_plan_s *pl = const_cast<se_plan_s *>(plan);
    const int I = iterations ? iterations : plan->desc.iterations;
    const size_t MN = static_cast<size_t>(plan->MN);
    const size_t io_bytes = 2 * MN * n * sizeof(double) +
                            (sel_idx ? sizeof(int32_t) * I * static_cast<size_t>(n) : 0) +
                            (sel_coef ? sizeof(double) * I * static_cast<size_t>(n) : 0) + 64;
    // Pinned (page-locked) caller buffers are read and written by the kernels
    // themselves over the host link (no staging copies: the transfers overlap the
    // computation); pageable ones are staged in chunks of at least 512 blocks, the
    // copies of one chunk overlapping the computation of the others.
    auto host_mapped = [](const void *p, void **dev) {
        if (!p) {
            *dev = nullptr;
            return true;
        }
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeHost || !at.devicePointer) return false;
        *dev = at.devicePointer;
        return true;
    };
    void *z_s = nullptr, *z_o = nullptr, *z_i = nullptr, *z_c = nullptr;
    const int S = std::max(1, std::min(se_ctx_s::kPipe, n / 512));
    if (host_mapped(samples, &z_s) && host_mapped(out, &z_o) && host_mapped(sel_idx, &z_i) &&
        host_mapped(sel_coef, &z_c)) {
        // chunks on their own streams; their projection passes (the readers of the
        // host samples) run one after another, so each has the link to itself
        // while the earlier chunks iterate
        std::lock_guard<std::mutex> lk(ctx->mu);
        SE_TRY(pipe_init(ctx));
        // one chunk unless SE_PINNED_CHUNKS asks for more: the iterations of the last
        // chunk take as long as a whole batch's (they are latency-bound), so chunks
        // shorten nothing and add launches (measured: 0.386 ms per 4096 blocks in
        // one chunk, 0.422 ms in four)
        const char *env = std::getenv("SE_PINNED_CHUNKS");
        const int cap = env ? std::max(1, std::min(4, std::atoi(env))) : 1;
        const int Sz = std::max(1, std::min(cap, n / 1024));
        for (int c = 0; c < Sz; ++c) {
            const int b0 = static_cast<int>(static_cast<long long>(n) * c / Sz);
            const int nc = static_cast<int>(static_cast<long long>(n) * (c + 1) / Sz) - b0;
            const size_t o = MN * b0;
            const StridedSpec ss{static_cast<const double *>(z_s) + o, static_cast<double *>(z_o) + o,
                                 z_i ? static_cast<int32_t *>(z_i) + static_cast<size_t>(I) * b0 : nullptr,
                                 z_c ? static_cast<double *>(z_c) + static_cast<size_t>(I) * b0 : nullptr, I, 1};
            SE_TRY(run_strided(ctx, pl, ctx->pipe_ws[c], nc, ss, ctx->pipe_st[c], c ? ctx->pipe_ev_in[c - 1] : nullptr,
                               ctx->pipe_ev_in[c]));
            SE_CUDA(cudaEventRecord(ctx->pipe_ev_done[c], ctx->pipe_st[c]));
            SE_CUDA(cudaStreamWaitEvent(ctx->pipe_out, ctx->pipe_ev_done[c], 0));
        }
        SE_CUDA(cudaStreamSynchronize(ctx->pipe_out));
        int bits = 0;
        SE_CUDA(cudaMemcpy(&bits, ctx->ws_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
        if (bits) {
            SE_CUDA(cudaMemset(ctx->ws_err.ptr, 0, sizeof(int)));
            const se_status code = bits == (1 << DEV_ERR_EMPTY_SUPPORT) ? SE_ERR_EMPTY_SUPPORT : SE_ERR_CUDA;
            return fail(code, std::string("device status: ") + dev_err_text(bits));
        }
        return SE_OK;
    }
    std::lock_guard<std::mutex> lk(ctx->mu);
    SE_TRY(pipe_init(ctx));
    // the previous call has finished (it synchronised), so the I/O buffer is free
    SE_TRY(dev_alloc(ctx, ctx->ws.io, io_bytes));
    double *d_s = ctx->ws.io.as<double>();
    double *d_o = d_s + MN * n;
    char *tail = reinterpret_cast<char *>(d_o + MN * n);
    int32_t *d_i = sel_idx ? reinterpret_cast<int32_t *>(tail) : nullptr;
    double *d_c = nullptr;
    if (sel_coef) {
        const size_t off = sel_idx ? round_up(sizeof(int32_t) * I * static_cast<size_t>(n), 16) : 0;
        d_c = reinterpret_cast<double *>(tail + off);
    }
    for (int c = 0; c < S; ++c) {
        const int b0 = static_cast<int>(static_cast<long long>(n) * c / S);
        const int nc = static_cast<int>(static_cast<long long>(n) * (c + 1) / S) - b0;
        const size_t o = MN * b0;
        cudaStream_t st = ctx->pipe_st[c];
        SE_CUDA(cudaMemcpyAsync(d_s + o, samples + o, MN * nc * sizeof(double), cudaMemcpyHostToDevice,
                                ctx->pipe_in));
        SE_CUDA(cudaEventRecord(ctx->pipe_ev_in[c], ctx->pipe_in));
        const StridedSpec ss{d_s + o, d_o + o, d_i ? d_i + static_cast<size_t>(I) * b0 : nullptr,
                             d_c ? d_c + static_cast<size_t>(I) * b0 : nullptr, I, 1};
        // the chunk's kernels wait for its copy; a table build (first chunk) does not
        SE_TRY(run_strided(ctx, pl, ctx->pipe_ws[c], nc, ss, st, ctx->pipe_ev_in[c]));
        SE_CUDA(cudaEventRecord(ctx->pipe_ev_done[c], st));
        SE_CUDA(cudaStreamWaitEvent(ctx->pipe_out, ctx->pipe_ev_done[c], 0));
        SE_CUDA(cudaMemcpyAsync(out + o, d_o + o, MN * nc * sizeof(double), cudaMemcpyDeviceToHost, ctx->pipe_out));
        if (sel_idx)
            SE_CUDA(cudaMemcpyAsync(sel_idx + static_cast<size_t>(I) * b0, d_i + static_cast<size_t>(I) * b0,
                                    sizeof(int32_t) * I * static_cast<size_t>(nc), cudaMemcpyDeviceToHost,
                                    ctx->pipe_out));
        if (sel_coef)
            SE_CUDA(cudaMemcpyAsync(sel_coef + static_cast<size_t>(I) * b0, d_c + static_cast<size_t>(I) * b0,
                                    sizeof(double) * I * static_cast<size_t>(nc), cudaMemcpyDeviceToHost,
                                    ctx->pipe_out));
    }
    SE_CUDA(cudaStreamSynchronize(ctx->pipe_out));
    int bits = 0;
    SE_CUDA(cudaMemcpy(&bits, ctx->ws_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) {
        SE_CUDA(cudaMemset(ctx->ws_err.ptr, 0, sizeof(int)));
        const se_status code = bits == (1 << DEV_ERR_EMPTY_SUPPORT) ? SE_ERR_EMPTY_SUPPORT : SE_ERR_CUDA;
        return fail(code, std::string("device status: ") + dev_err_text(bits));
    }
    return SE_OK;
}

namespace {

se_status host_slots_init(se_ctx_s *ctx)
{
    if (ctx->hslot_ready) return SE_OK;
    for (auto &h : ctx->hslot) {
        SE_CUDA(cudaStreamCreateWithFlags(&h.st, cudaStreamNonBlocking));
        SE_CUDA(cudaEventCreateWithFlags(&h.done, cudaEventDisableTiming));
        SE_CUDA(cudaEventCreateWithFlags(&h.computed, cudaEventDisableTiming));
        SE_CUDA(h.ws.init());
    }
    ctx->hslot_ready = true;
    return SE_OK;
}

// Read and clear the context's device status word (ctx->mu held).
se_status take_device_status(se_ctx_s *ctx)
{
    int bits = 0;
    SE_CUDA(cudaMemcpy(&bits, ctx->ws_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) {
        SE_CUDA(cudaMemset(ctx->ws_err.ptr, 0, sizeof(int)));
        const se_status code = bits == (1 << DEV_ERR_EMPTY_SUPPORT) ? SE_ERR_EMPTY_SUPPORT : SE_ERR_CUDA;
        return fail(code, std::string("device status: ") + dev_err_text(bits));
    }
    return SE_OK;
}

}  // namespace

se_status se_extrapolate_host_async(se_ctx_t *ctx, const se_plan_t *plan, int n, const double *samples,
                                    double *out, int32_t *sel_idx, double *sel_coef, int iterations,
                                    uint64_t *ticket)
{
    if (!ctx || !plan || !ticket || n < 0) return fail(SE_ERR_INVALID, "NULL argument or n < 0");
    *ticket = 0;
    if (plan->cplx) return fail(SE_ERR_INVALID, "complex plans: device entry points only");
    if (iterations < 0) return fail(SE_ERR_INVALID, "iterations < 0");
    if (plan->ctx != ctx) return fail(SE_ERR_INVALID, "plan belongs to another context");
    if (n == 0) return SE_OK;
    if (!samples || !out) return fail(SE_ERR_INVALID, "NULL samples or out");
    SE_CUDA(cudaSetDevice(ctx->device));
    se_plan_s *pl = const_cast<se_plan_s *>(plan);
    const int I = iterations ? iterations : plan->desc.iterations;
    const size_t MN = static_cast<size_t>(plan->MN), nn = static_cast<size_t>(n);
    std::lock_guard<std::mutex> lk(ctx->mu);
    SE_TRY(host_slots_init(ctx));
    const uint64_t t = ctx->host_next;
    HostSlot &h = ctx->hslot[t % se_ctx_s::kHostSlots];
    if (h.busy) {   // the oldest call in flight: its buffers are reused below
        SE_CUDA(cudaEventSynchronize(h.done));
        h.busy = false;
    }
    // device copy of the samples (computed in place), then the logs
    const size_t s_bytes = MN * nn * sizeof(double);
    const size_t i_off = round_up(s_bytes, 256), i_bytes = sel_idx ? sizeof(int32_t) * I * nn : 0;
    const size_t c_off = round_up(i_off + i_bytes, 256), c_bytes = sel_coef ? sizeof(double) * I * nn : 0;
    SE_TRY(dev_alloc(ctx, h.io, c_off + c_bytes));
    double *d_s = h.io.as<double>();
    int32_t *d_i = sel_idx ? reinterpret_cast<int32_t *>(h.io.as<char>() + i_off) : nullptr;
    double *d_c = sel_coef ? reinterpret_cast<double *>(h.io.as<char>() + c_off) : nullptr;
    // one contiguous copy in (a copy of the support alone would take one strided copy
    // per block, whose host cost outweighs the quarter of the bytes it saves)
    const int N = plan->N, m0 = pl->box[0], m1 = pl->box[1], n0 = pl->box[2], n1 = pl->box[3];
    SE_CUDA(cudaMemcpyAsync(d_s, samples, s_bytes, cudaMemcpyHostToDevice, h.st));
    {
        // a table (re)build must not overwrite the table under the kernels of the
        // calls in flight (their copies out may still run)
        std::lock_guard<std::mutex> tl(pl->tmu);
        if (!pl->tables_valid)
            for (auto &o : ctx->hslot)
                if (o.busy && &o != &h) SE_CUDA(cudaStreamWaitEvent(h.st, o.computed, 0));
    }
    const StridedSpec ss{d_s, d_s, d_i, d_c, I, 1};
    SE_TRY(run_strided(ctx, pl, h.ws, n, ss, h.st));
    SE_CUDA(cudaEventRecord(h.computed, h.st));
    if (out == samples && plan->T == 1 && m1 > m0) {
        // in place: of every block the span from the first to the last sample of its
        // loss bounding box, one strided copy (the support samples in the span are
        // the caller's own values)
        const size_t first = static_cast<size_t>(m0) * N + n0, last = static_cast<size_t>(m1 - 1) * N + n1;
        SE_CUDA(cudaMemcpy2DAsync(out + first, MN * sizeof(double), d_s + first, MN * sizeof(double),
                                  (last - first) * sizeof(double), nn, cudaMemcpyDeviceToHost, h.st));
    } else if (out != samples || plan->T > 1) {
        SE_CUDA(cudaMemcpyAsync(out, d_s, s_bytes, cudaMemcpyDeviceToHost, h.st));
    }
    if (sel_idx) SE_CUDA(cudaMemcpyAsync(sel_idx, d_i, i_bytes, cudaMemcpyDeviceToHost, h.st));
    if (sel_coef) SE_CUDA(cudaMemcpyAsync(sel_coef, d_c, c_bytes, cudaMemcpyDeviceToHost, h.st));
    SE_CUDA(cudaEventRecord(h.done, h.st));
    h.busy = true;
    h.ticket = t;
    ctx->host_next = t + 1;
    *ticket = t;
    return SE_OK;
}

se_status se_host_wait(se_ctx_t *ctx, uint64_t ticket)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    if (ticket == 0) return SE_OK;
    SE_CUDA(cudaSetDevice(ctx->device));
    cudaEvent_t done = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (ticket >= ctx->host_next) return fail(SE_ERR_UNKNOWN_TICKET, "no such host-call ticket");
        for (auto &h : ctx->hslot)
            if (h.busy && h.ticket == ticket) done = h.done;
    }
    // the wait itself does not hold the context: other threads keep enqueueing (a
    // slot is reused only after its call has completed, so the event stays this call's)
    if (done) SE_CUDA(cudaEventSynchronize(done));
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (auto &h : ctx->hslot)
        if (h.busy && h.ticket == ticket) h.busy = false;
    return take_device_status(ctx);
}

se_status se_set_profiling(se_ctx_t *ctx, int enable)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->pmu);
    ctx->profiling = enable != 0;
    return SE_OK;
}

se_status se_stage_times(se_ctx_t *ctx, double *ms, uint64_t *count, int n_stages, int reset)
{
    if (!ctx || n_stages < 0) return fail(SE_ERR_INVALID, "NULL context or n_stages < 0");
    SE_CUDA(cudaSetDevice(ctx->device));
    std::lock_guard<std::mutex> lk(ctx->pmu);
    for (auto &p : ctx->pending) {
        cudaEvent_t a = p.second.first, b = p.second.second;
        SE_CUDA(cudaEventSynchronize(b));
        float t = 0.0f;
        SE_CUDA(cudaEventElapsedTime(&t, a, b));
        ctx->stage_ms[p.first] += t;
        ctx->stage_count[p.first] += 1;
        ctx->event_pool.push_back(a);
        ctx->event_pool.push_back(b);
    }
    ctx->pending.clear();
    for (int i = 0; i < n_stages && i < se_ctx_s::kStages; ++i) {
        if (ms) ms[i] = ctx->stage_ms[i];
        if (count) count[i] = ctx->stage_count[i];
    }
    if (reset)
        for (int i = 0; i < se_ctx_s::kStages; ++i) { ctx->stage_ms[i] = 0.0; ctx->stage_count[i] = 0; }
    return SE_OK;
}

se_status se_stats(se_ctx_t *ctx, uint64_t *kernel_launches, uint64_t *table_builds,
                   uint64_t *serving_slices)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    if (kernel_launches) *kernel_launches = ctx->launches.load();
    if (table_builds) *table_builds = ctx->table_builds.load();
    if (serving_slices) *serving_slices = ctx->slices.load();
    return SE_OK;
}

se_status se_plan_autotune(se_ctx_t *ctx, se_plan_t *plan, int n_probe, void *cuda_stream)
{
    if (!ctx || !plan) return fail(SE_ERR_INVALID, "NULL context or plan");
    if (plan->ctx != ctx) return fail(SE_ERR_INVALID, "plan belongs to another context");
    if (n_probe < 1 || n_probe > 65536) return fail(SE_ERR_INVALID, "n_probe must be in [1, 65536]");
    if (plan->cplx || plan->certified)
        return fail(SE_ERR_INVALID, "complex and certified plans have no lazy path to compare");
    SE_CUDA(cudaSetDevice(ctx->device));
    se_plan_s *pl = plan;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    std::lock_guard<std::mutex> lk(ctx->mu);
    const size_t MN = static_cast<size_t>(pl->MN);
    DevBuf smp, out;
    SE_TRY(dev_alloc(ctx, smp, sizeof(double) * MN * n_probe));
    SE_TRY(dev_alloc(ctx, out, sizeof(double) * MN * n_probe));
    SE_CUDA(launch_probe_samples(smp.as<double>(), static_cast<long long>(MN) * n_probe, 0x5e1eu, st));
    const int I = pl->desc.iterations;
    std::vector<BlockDesc> full(n_probe), lazy;
    for (int i = 0; i < n_probe; ++i) {
        full[i] = BlockDesc{};
        full[i].samples = smp.as<double>() + MN * i;
        full[i].out = out.as<double>() + MN * i;
        full[i].iterations = I;
    }
    lazy = full;
    for (auto &x : lazy) x.support = pl->d_pattern.as<uint8_t>();
    // warm-up (operands, tuner choices, graph capture), then the measured pass
    for (int pass = 0; pass < 2; ++pass) {
        {
            std::lock_guard<std::mutex> tl(pl->tmu);
            pl->tables_valid = false;
        }
        SE_TRY(run_batch(ctx, pl, ctx->ws, n_probe, full.data(), I, st));
        SE_TRY(run_lazy(ctx, pl, ctx->ws, n_probe, lazy.data(), I, st));
        SE_CUDA(cudaStreamSynchronize(st));
        probes_poll(ctx, true, pl);
        if (pass == 0) {
            std::lock_guard<std::mutex> cl(pl->cmu);
            pl->t_table_ms = pl->t_full_blk_ms = pl->t_lazy_blk_ms = pl->lazy_regret_ms = 0.0;
        }
    }
    int bits = 0;
    SE_CUDA(cudaMemcpy(&bits, ctx->ws_err.ptr, sizeof(int), cudaMemcpyDeviceToHost));
    if (bits) {
        SE_CUDA(cudaMemset(ctx->ws_err.ptr, 0, sizeof(int)));
        return fail(SE_ERR_CUDA, std::string("autotune: ") + dev_err_text(bits));
    }
    return SE_OK;
}

se_status se_plan_costs(const se_plan_t *plan, double *table_ms, double *full_ms_per_block,
                        double *lazy_ms_per_block)
{
    if (!plan) return fail(SE_ERR_INVALID, "NULL plan");
    se_plan_s *pl = const_cast<se_plan_s *>(plan);
    probes_poll(pl->ctx, false, pl);
    std::lock_guard<std::mutex> lk(pl->cmu);
    if (table_ms) *table_ms = pl->t_table_ms;
    if (full_ms_per_block) *full_ms_per_block = pl->t_full_blk_ms;
    if (lazy_ms_per_block) *lazy_ms_per_block = pl->t_lazy_blk_ms;
    return SE_OK;
}

se_status se_set_graphs(se_ctx_t *ctx, int enable)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->graphs_enabled = enable != 0;
    return SE_OK;
}

se_status se_tuning_stats(se_ctx_t *ctx, uint64_t *tunings, uint64_t *graph_builds, uint64_t *graph_replays)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    if (tunings) *tunings = ctx->tunings.load();
    if (graph_builds) *graph_builds = ctx->graph_builds.load();
    if (graph_replays) *graph_replays = ctx->graph_replays.load();
    return SE_OK;
}

se_status se_cert_stats(se_ctx_t *ctx, uint64_t *blocks, uint64_t *recomputed)
{
    if (!ctx) return fail(SE_ERR_INVALID, "NULL context");
    if (blocks) *blocks = ctx->cert_blocks.load();
    if (recomputed) *recomputed = ctx->cert_recomputed.load();
    return SE_OK;
}

se_status se_plan_info(const se_plan_t *plan, char *buf, size_t len)
{
    if (!plan || !buf || len == 0) return fail(SE_ERR_INVALID, "NULL plan or buffer");
    std::string t = std::string("products=") + (plan->sep_full ? "transform" : "dense") +
                    " table=" + (plan->dft_w ? "dft-of-weights" : "table") + " iterations=" +
                    (plan->cplx ? "complex" : plan->pc.fp64 ? "fp64" : plan->sym ? "parity-classes" : "general") +
                    (plan->sym_tc ? " projections=split-tf32" : "") + (plan->certified ? " certified" : "") +
                    (plan->f16_cols ? " columns=f16x3" : "") + (plan->f16_table && !plan->sep_full ? " table_products=f16x3" : "");
    std::snprintf(buf, len, "%s", t.c_str());
    return SE_OK;
}

se_status se_tuned_variant(se_ctx_t *ctx, const char *key, int *variant)
{
    if (!ctx || !key || !variant) return fail(SE_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(ctx->tuner.mu);
    auto it = ctx->tuner.best.find(key);
    *variant = it == ctx->tuner.best.end() ? -1 : it->second;
    return SE_OK;
}

}  // extern "C"
