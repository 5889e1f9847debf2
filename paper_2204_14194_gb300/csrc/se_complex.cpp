// se_complex.cpp -- plans with complex-valued atoms (DFT, binarised DFT and
// their union; the paper's general case of Sec. II-III): the dictionary, the
// collinearity flags, the stacked real operands of the tables and
// projections, the tables and the batch.
//
// With G = phi sqrt(w) on the support (real part Gr, imaginary part Gi),
//   Re C(k,u) = Gr_k . Gr_u + Gi_k . Gi_u = [Gr|Gi]_k . [Gr|Gi]_u
//   Im C(k,u) = Gr_k . Gi_u - Gi_k . Gr_u = [Gr|Gi]_k . [Gi|-Gr]_u
// so the Hermitian table of eq. (16) is two real products of stacked rows,
// and R^(0) of eq. (12) (real samples) is one real product with the rows
// [phi_r w ; -phi_i w]; the same GEMM kernels as the real case compute them.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <random>
#include <string>
#include <vector>

#include "se_host.h"

namespace se {

namespace {

#define CX_CUDA(call)                                                                          \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return set_error(SE_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define CX_TRY(expr)                \
    do {                            \
        se_status s_ = (expr);      \
        if (s_ != SE_OK) return s_; \
    } while (0)

template <typename V>
se_status upload_cx(se_ctx_s *ctx, DevBuf &b, const std::vector<V> &h)
{
    CX_TRY(dev_alloc(ctx, b, h.size() * sizeof(V)));
    CX_CUDA(cudaMemcpy(b.ptr, h.data(), h.size() * sizeof(V), cudaMemcpyHostToDevice));
    return SE_OK;
}

}  // namespace

bool build_complex_dictionary(int M, int N, int basis, int K, std::vector<double> &re, std::vector<double> &im,
                              std::string *why)
{
    const long L = static_cast<long>(M) * N;
    const size_t V = static_cast<size_t>(L);
    const size_t expect = basis == SE_BASIS_DFT_BDFT ? 2 * V : V;
    if (static_cast<size_t>(K) != expect) {
        *why = "K does not match the basis cardinality (" + std::to_string(expect) + ")";
        return false;
    }
    re.assign(static_cast<size_t>(K) * V, 0.0);
    im.assign(static_cast<size_t>(K) * V, 0.0);
    const double pi = 3.14159265358979323846;
    auto fill = [&](size_t k0, bool binarised) {
        const double s = binarised ? 1.0 / std::sqrt(2.0 * static_cast<double>(L)) : 1.0 / std::sqrt(static_cast<double>(L));
        for (int mu = 0; mu < M; ++mu)
            for (int eta = 0; eta < N; ++eta) {
                const size_t k = k0 + static_cast<size_t>(mu) * N + eta;
                for (int m = 0; m < M; ++m)
                    for (int n = 0; n < N; ++n) {
                        // exact phase index: theta = 2 pi a / (MN)
                        const long a = (static_cast<long>(mu) * m * N + static_cast<long>(eta) * n * M) % L;
                        const size_t i = k * V + static_cast<size_t>(m) * N + n;
                        if (binarised) {
                            re[i] = (4 * a <= L || 4 * a >= 3 * L) ? s : -s;   // sgn(cos), sgn(0) = +1
                            im[i] = (2 * a <= L) ? s : -s;                     // sgn(sin)
                        } else {
                            re[i] = s * std::cos(2.0 * pi * static_cast<double>(a) / static_cast<double>(L));
                            im[i] = s * std::sin(2.0 * pi * static_cast<double>(a) / static_cast<double>(L));
                        }
                    }
            }
    };
    if (basis == SE_BASIS_DFT || basis == SE_BASIS_DFT_BDFT) fill(0, false);
    if (basis == SE_BASIS_BDFT) fill(0, true);
    if (basis == SE_BASIS_DFT_BDFT) fill(V, true);
    return true;
}

// Collinear complex atoms (|<phi_i, phi_j>| >= (1 - 1e-12) |phi_i| |phi_j|,
// <a, b> = sum conj(a) b): candidates are neighbours in the order of
// |<phi, z>| / |phi| for a fixed pseudo-random complex z (collinear unit atoms
// differ by a unit complex factor, so their keys agree to rounding), then
// the exact test.
void find_collinear_complex(int K, int MN, const double *re, const double *im, std::vector<uint8_t> &dup)
{
    dup.assign(K, 0);
    std::vector<double> zr(MN), zi(MN), nrm(K), key(K);
    std::mt19937_64 gen(0xc0ffeeull);
    std::normal_distribution<double> nd(0.0, 1.0);
    double zn = 0.0;
    for (int i = 0; i < MN; ++i) {
        zr[i] = nd(gen);
        zi[i] = nd(gen);
        zn += zr[i] * zr[i] + zi[i] * zi[i];
    }
    zn = std::sqrt(zn);
    for (int k = 0; k < K; ++k) {
        const double *a = re + static_cast<size_t>(k) * MN, *b = im + static_cast<size_t>(k) * MN;
        double s = 0.0, dr = 0.0, di = 0.0;
        for (int i = 0; i < MN; ++i) {
            s += a[i] * a[i] + b[i] * b[i];
            dr += a[i] * zr[i] + b[i] * zi[i];
            di += a[i] * zi[i] - b[i] * zr[i];
        }
        nrm[k] = std::sqrt(s);
        key[k] = nrm[k] > 0.0 ? std::sqrt(dr * dr + di * di) / nrm[k] : -1.0;
    }
    std::vector<int> ord(K);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return key[x] < key[y]; });
    const double win = 1e-5 * zn;
    for (int i = 0; i < K; ++i) {
        const int ki = ord[i];
        if (nrm[ki] == 0.0) continue;
        for (int j = i + 1; j < K && key[ord[j]] - key[ki] <= win; ++j) {
            const int kj = ord[j];
            if (nrm[kj] == 0.0) continue;
            const double *ar = re + static_cast<size_t>(ki) * MN, *ai = im + static_cast<size_t>(ki) * MN;
            const double *br = re + static_cast<size_t>(kj) * MN, *bi = im + static_cast<size_t>(kj) * MN;
            double dr = 0.0, di = 0.0;
            for (int t = 0; t < MN; ++t) {
                dr += ar[t] * br[t] + ai[t] * bi[t];
                di += ar[t] * bi[t] - ai[t] * br[t];
            }
            if (std::sqrt(dr * dr + di * di) >= (1.0 - 1e-12) * nrm[ki] * nrm[kj]) dup[std::max(ki, kj)] = 1;
        }
    }
}

// The 2-D DFT of the weighting function, What[a][b] = sum w[m][n]
// exp(-j 2 pi (a m / M + b n / N)) / MN (exact phase reduction, fp64): for DFT
// atoms C(k,u) = What[(mu_k - mu_u) mod M][(eta_k - eta_u) mod N] (Sec. VI, the
// product of an atom and a conjugated atom is the atom of the frequency
// difference).
static void dft_of_weights(int M, int N, const std::vector<double> &w, std::vector<double> &re,
                           std::vector<double> &im)
{
    const long L = static_cast<long>(M) * N;
    const double pi = 3.14159265358979323846;
    re.assign(L, 0.0);
    im.assign(L, 0.0);
    for (int a = 0; a < M; ++a)
        for (int b = 0; b < N; ++b) {
            double sr = 0.0, si = 0.0;
            for (int m = 0; m < M; ++m)
                for (int n = 0; n < N; ++n) {
                    const double v = w[static_cast<size_t>(m) * N + n];
                    if (v == 0.0) continue;
                    const long ph = (static_cast<long>(a) * m * N + static_cast<long>(b) * n * M) % L;
                    const double t = 2.0 * pi * static_cast<double>(ph) / static_cast<double>(L);
                    sr += v * std::cos(t);
                    si -= v * std::sin(t);
                }
            re[static_cast<size_t>(a) * N + b] = sr / static_cast<double>(L);
            im[static_cast<size_t>(a) * N + b] = si / static_cast<double>(L);
        }
}

se_status setup_complex_plan(se_ctx_s *ctx, se_plan_s *pl, cudaStream_t st)
{
    const int K = pl->K, Kp = pl->Kp, ka = pl->ka_pad, MN = pl->MN, nA = pl->nA, nB = pl->nB;
    const int ka2 = 2 * ka;
    const double *re = pl->phi.data(), *im = pl->phi_im.data();
    const bool fp64 = pl->pc.fp64;
    pl->dft_w = pl->desc.basis == SE_BASIS_DFT;
    if (pl->dft_w) {
        std::vector<double> wr, wi;
        dft_of_weights(pl->M, pl->N, pl->w, wr, wi);
        std::vector<double> planes(wr);
        planes.insert(planes.end(), wi.begin(), wi.end());
        if (fp64) CX_TRY(upload_cx(ctx, pl->d_What, planes));
        else CX_TRY(upload_cx(ctx, pl->d_What, std::vector<float>(planes.begin(), planes.end())));
        pl->dft_invC.assign(Kp, 0.0);
        for (int k = 0; k < K; ++k) pl->dft_invC[k] = wr[0] > 0.0 ? 1.0 / wr[0] : 0.0;
    }
    std::vector<double> G(static_cast<size_t>(Kp) * ka2, 0.0), Gc(static_cast<size_t>(Kp) * ka2, 0.0),
        P(static_cast<size_t>(2) * Kp * ka, 0.0);
    for (int k = 0; k < K; ++k)
        for (int j = 0; j < nA; ++j) {
            const size_t src = static_cast<size_t>(k) * MN + pl->a_idx[j];
            const double w = pl->w[pl->a_idx[j]], sw = std::sqrt(w);
            const double gr = re[src] * sw, gi = im[src] * sw;
            G[static_cast<size_t>(k) * ka2 + j] = gr;
            G[static_cast<size_t>(k) * ka2 + ka + j] = gi;
            Gc[static_cast<size_t>(k) * ka2 + j] = gi;
            Gc[static_cast<size_t>(k) * ka2 + ka + j] = -gr;
            // eq. (12) rows: the fp64 form packs sqrt(w) s, the split forms pack s
            const double f = fp64 ? sw : w;
            P[static_cast<size_t>(k) * ka + j] = re[src] * f;
            P[static_cast<size_t>(Kp + k) * ka + j] = -im[src] * f;
        }
    if (!pl->dft_w) CX_TRY(upload_cx(ctx, pl->d_G64, G));   // the diagonal of eq. (16) is read from it
    if (fp64) {
        if (!pl->dft_w) CX_TRY(upload_cx(ctx, pl->d_Gc64, Gc));
        CX_TRY(upload_cx(ctx, pl->d_P64, P));
    } else {
        if (!pl->dft_w) {
            DevBuf tmp;
            CX_TRY(dev_alloc(ctx, pl->d_Gbf, static_cast<size_t>(Kp) * pl->pc.nparts * ka2 * 2));
            CX_CUDA(launch_split_bf16(pl->d_G64.as<double>(), Kp, ka2, ka2, ka2, pl->pc.nparts,
                                      pl->d_Gbf.as<uint16_t>(), st));
            CX_TRY(upload_cx(ctx, tmp, Gc));
            CX_TRY(dev_alloc(ctx, pl->d_Gcbf, static_cast<size_t>(Kp) * pl->pc.nparts * ka2 * 2));
            CX_CUDA(launch_split_bf16(tmp.as<double>(), Kp, ka2, ka2, ka2, pl->pc.nparts,
                                      pl->d_Gcbf.as<uint16_t>(), st));
            CX_CUDA(cudaStreamSynchronize(st));
        }
        DevBuf tp;
        CX_TRY(upload_cx(ctx, tp, P));
        CX_TRY(dev_alloc(ctx, pl->d_Gwbf, static_cast<size_t>(2) * Kp * pl->pc.nparts * ka * 2));
        CX_CUDA(launch_split_bf16(tp.as<double>(), 2 * Kp, ka, ka, ka, pl->pc.nparts, pl->d_Gwbf.as<uint16_t>(), st));
        CX_CUDA(cudaStreamSynchronize(st));
        ctx->launches += 3;
    }
    // atoms on the loss pixels, [Kp][2][nB]
    const size_t nBa = std::max(nB, 1);
    if (fp64) {
        std::vector<double> pb(static_cast<size_t>(Kp) * 2 * nBa, 0.0);
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < nB; ++j) {
                pb[static_cast<size_t>(k) * 2 * nBa + j] = re[static_cast<size_t>(k) * MN + pl->b_idx[j]];
                pb[static_cast<size_t>(k) * 2 * nBa + nBa + j] = im[static_cast<size_t>(k) * MN + pl->b_idx[j]];
            }
        CX_TRY(upload_cx(ctx, pl->d_PhiB, pb));
    } else {
        std::vector<float> pb(static_cast<size_t>(Kp) * 2 * nBa, 0.0f);
        for (int k = 0; k < K; ++k)
            for (int j = 0; j < nB; ++j) {
                pb[static_cast<size_t>(k) * 2 * nBa + j] = static_cast<float>(re[static_cast<size_t>(k) * MN + pl->b_idx[j]]);
                pb[static_cast<size_t>(k) * 2 * nBa + nBa + j] =
                    static_cast<float>(im[static_cast<size_t>(k) * MN + pl->b_idx[j]]);
            }
        CX_TRY(upload_cx(ctx, pl->d_PhiB, pb));
    }
    return SE_OK;
}

// Alg. 2 for complex atoms: C_kk from the stacked rows, 1/C_kk, then the real
// and imaginary planes of every row u of the table, C(., u).
se_status build_tables_complex(se_ctx_s *ctx, se_plan_s *pl, cudaStream_t st)
{
    const int K = pl->K, Kp = pl->Kp, ka2 = 2 * pl->ka_pad;
    if (pl->dft_w) {   // no table: the DFT of w is uploaded with the plan; 1/C_kk is uniform
        if (pl->pc.fp64) {
            CX_CUDA(cudaMemcpyAsync(pl->d_invC.ptr, pl->dft_invC.data(), sizeof(double) * Kp,
                                    cudaMemcpyHostToDevice, st));
        } else {
            static thread_local std::vector<float> f;
            f.assign(pl->dft_invC.begin(), pl->dft_invC.end());
            CX_CUDA(cudaMemcpyAsync(pl->d_invC.ptr, f.data(), sizeof(float) * Kp, cudaMemcpyHostToDevice, st));
            CX_CUDA(cudaStreamSynchronize(st));
        }
        return SE_OK;
    }
    unsigned long long *dmax = reinterpret_cast<unsigned long long *>(pl->d_nadm.as<char>() + 8);
    CX_CUDA(launch_tables_diag(pl->d_G64.as<double>(), ka2, K, Kp, ka2, pl->d_dup.as<uint8_t>(),
                               pl->d_diag.as<double>(), dmax, pl->d_nadm.as<int>(), st));
    std::string why;
    if (pl->pc.fp64) {
        CX_CUDA(launch_tables_finalize<double>(pl->d_diag.as<double>(), pl->d_dup.as<uint8_t>(), dmax, K, Kp,
                                               pl->d_invC.as<double>(), pl->d_Dk.as<double>(), pl->d_nadm.as<int>(),
                                               st));
        double *C = pl->d_C.as<double>();
        CX_CUDA(launch_simt_gemm<double>(pl->d_G64.as<double>(), ka2, pl->d_G64.as<double>(), ka2, Kp, Kp, ka2, C,
                                         2 * Kp, 0, st));
        CX_CUDA(launch_simt_gemm<double>(pl->d_G64.as<double>(), ka2, pl->d_Gc64.as<double>(), ka2, Kp, Kp, ka2,
                                         C + Kp, 2 * Kp, 0, st));
    } else {
        CX_CUDA(launch_tables_finalize<float>(pl->d_diag.as<double>(), pl->d_dup.as<uint8_t>(), dmax, K, Kp,
                                              pl->d_invC.as<float>(), pl->d_Dk.as<float>(), pl->d_nadm.as<int>(), st));
        for (int part = 0; part < 2; ++part) {
            TcGemmArgs g{};
            g.A = pl->d_Gbf.ptr;
            g.B = part == 0 ? pl->d_Gbf.ptr : pl->d_Gcbf.ptr;
            g.M = Kp;
            g.N = Kp;
            g.lda = g.ldb = pl->pc.nparts * ka2;
            g.ka_pad = ka2;
            g.npairs = pl->pc.npairs;
            for (int i = 0; i < 8; ++i) { g.pa[i] = pl->pc.pa[i]; g.pb[i] = pl->pc.pb[i]; }
            g.out = pl->d_C.as<float>() + part * Kp;
            g.ldo = 2 * Kp;
            g.symmetric = 0;
            g.err = ctx->ws_err.as<int>();
            cudaError_t e = launch_tc_gemm(g, st, &why);
            if (e != cudaSuccess) return set_error(SE_ERR_CUDA, "complex table GEMM: " + why + " " + cudaGetErrorString(e));
        }
    }
    ctx->launches += 4;
    return SE_OK;
}

// eq. (12) and the iterations for a batch whose descriptors are staged in
// ws.desc and whose tables are built (run_batch does both).
se_status run_complex(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, int n, int I_max, cudaStream_t st)
{
    const int Kp = pl->Kp, ka = pl->ka_pad;
    const bool fp64 = pl->pc.fp64;
    const BlockDesc *ddesc = ws.desc.as<BlockDesc>();
    std::string why;
    int tok = stage_begin(ctx, 0, st);
    if (fp64)
        CX_CUDA(launch_pack_x(ddesc, n, pl->d_a_idx.as<int>(), pl->d_sqrtw.as<double>(), pl->nA, ka, 0, pl->MN,
                              nullptr, ws.x.as<double>(), st));
    else
        CX_CUDA(launch_pack_x(ddesc, n, pl->d_a_idx.as<int>(), pl->d_sqrtw.as<double>(), pl->nA, ka, pl->pc.nparts,
                              pl->MN, ws.x.as<uint16_t>(), nullptr, st));
    stage_end(ctx, tok, st);
    tok = stage_begin(ctx, 2, st);
    if (fp64) {
        CX_CUDA(launch_simt_gemm<double>(pl->d_P64.as<double>(), ka, ws.x.as<double>(), ka, 2 * Kp, n, ka,
                                         ws.r0.as<double>(), 2 * Kp, 0, st));
    } else {
        TcGemmArgs g{};
        g.A = pl->d_Gwbf.ptr;
        g.B = ws.x.ptr;
        g.M = 2 * Kp;
        g.N = n;
        g.lda = g.ldb = pl->pc.nparts * ka;
        g.ka_pad = ka;
        g.npairs = pl->pc.npairs;
        for (int i = 0; i < 8; ++i) { g.pa[i] = pl->pc.pa[i]; g.pb[i] = pl->pc.pb[i]; }
        g.out = ws.r0.as<float>();
        g.ldo = 2 * Kp;
        g.symmetric = 0;
        g.err = ctx->ws_err.as<int>();
        cudaError_t e = launch_tc_gemm(g, st, &why);
        if (e != cudaSuccess) return set_error(SE_ERR_CUDA, "complex projection GEMM: " + why + " " + cudaGetErrorString(e));
    }
    stage_end(ctx, tok, st);
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
    if (pl->dft_w) {
        a.What = pl->d_What.ptr;
        a.Mdft = pl->M;
        a.Ndft = pl->N;
    }
    tok = stage_begin(ctx, 3, st);
    cudaError_t e = fp64 ? launch_iterate_cplx<double>(a, st) : launch_iterate_cplx<float>(a, st);
    stage_end(ctx, tok, st);
    if (e != cudaSuccess) return set_error(SE_ERR_CUDA, std::string("complex iterations: ") + cudaGetErrorString(e));
    ctx->launches += 3;
    CX_CUDA(cudaEventRecord(ws.ev_ws, st));
    return SE_OK;
}

}  // namespace se
