// se_internal.h -- types shared by the host runtime and the kernel launchers
// of libse.so.  Not part of the public ABI (include/se.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace se {

// Per-block descriptor as the kernels read it (device copy of se_block,
// resolved: iterations filled in, support == nullptr means the batch's
// shared pattern).
struct BlockDesc {
    const double *samples;
    const uint8_t *support;
    double *out;
    int32_t *sel_idx;
    double *sel_coef;
    int iterations;
    int pad_;
};

// Device-side error codes written to the batch status word.
enum DevErr : int {
    DEV_OK = 0,
    DEV_ERR_WAIT_TIMEOUT = 1,     // an mbarrier wait ran out of time
    DEV_ERR_BAD_INDEX = 2,        // a selected index fell outside [0, K)
    DEV_ERR_TMEM = 3,             // tensor-memory allocation returned an unusable address
    DEV_ERR_LAZY_CACHE = 4,       // lazy column cache overflowed
    DEV_ERR_EMPTY_SUPPORT = 5     // a block's own mask leaves no admissible atom
};

// Argmax candidate exchanged between warps: score, index, value.
template <typename T> struct Cand { T s; int k; T r; };

// ----------------------------------------------------------------- GEMMs
// D[m][n] = sum_pairs sum_k A[m][pa*ka_pad + k] * B[n][pb*ka_pad + k]
// with bf16 A (rows M) and B (rows N), fp32 accumulation on tcgen05.
struct TcGemmArgs {
    const void *A;       // bf16 [M_rows][lda] (lda in elements)
    const void *B;       // bf16 [N_rows][ldb]
    int M, N;            // logical sizes (rows of A, rows of B)
    int lda, ldb;        // row pitch in elements (multiple of 8)
    int ka_pad;          // columns of one split part (multiple of 64)
    int npairs;
    int pa[8], pb[8];    // split part of A / B for each partial product
    float *out;          // output
    long long ldo;       // output row pitch (elements)
    int symmetric;       // 1: Gram mode (M == N, upper tiles, mirrored store)
    const float *scale;  // optional per-atom factors: out[n][m] = D[m][n] * scale[m]; in Gram
                         // mode also out[m][n] = D[m][n] * scale[n] (NULL: no scaling)
    const long long *out_rows;  // optional (non-symmetric): element (n, m) goes to out[out_rows[n] + m]
    const int *n_dev;    // optional device count: only rows n < min(N, *n_dev) of B are used
    int *err;            // device status word
    int f16;             // 1: the parts are fp16 (kind::f16 with f16 operands), else bf16
    float post;          // factor applied to every sum before the scale above (0: none); a power
                         //   of two undoes the scaling of fp16 parts exactly
    int grouped;         // non-symmetric products: 1 = 128 x 128 tiles holding every split part
                         //   of a k-slice per stage (each part read once per k-slice), else one
                         //   partial product per stage; the two orders give different roundings
};
// variant: non-symmetric products 0 = 128 x 256 tiles, 1 = 128 x 128, 2 =
// 128 x 64, 3 = 128 x 128 with two CTAs per SM (all stream one partial
// product per stage, so they accumulate in the same order and give identical
// results); symmetric and grouped products 0 = one CTA
// per SM with a two-stage ring, 1 = two CTAs per SM of one stage each (the
// same kernel and order, identical results).
cudaError_t launch_tc_gemm(const TcGemmArgs &a, cudaStream_t st, std::string *why, int variant = 0);
int tc_gemm_variants(const TcGemmArgs &a);
// The tile variant that fills the GPU for an M x N product: the widest tile
// whose grid covers every SM at least once (128 x 64 if none does).
int tc_gemm_fill_variant(int M, int N);

// fp64 (or fp32) CUDA-core GEMM, same contraction with a single part:
// D[m][n] = sum_k A[m][k] B[n][k]; output mode as above.
template <typename T>
cudaError_t launch_simt_gemm(const T *A, int lda, const T *B, int ldb, int M, int N, int Kd,
                             T *out, long long ldo, int symmetric, cudaStream_t st);
// With optional output row offsets and device-side row count (as TcGemmArgs).
template <typename T>
cudaError_t launch_simt_gemm_ex(const T *A, int lda, const T *B, int ldb, int M, int N, int Kd,
                                T *out, long long ldo, const long long *out_rows, const int *n_dev,
                                cudaStream_t st);

// ------------------------------------------------------------- prep / tables
// Pack the samples of the shared pattern's support pixels: for block b and
// support pixel j, the raw sample s_b[a_idx[j]] as nparts exact bf16 split
// parts ([part][ka_pad] per row; the weights are in the dictionary operand)
// and/or sqrtw[j] * s_b[a_idx[j]] in fp64; zero for j >= nA.
cudaError_t launch_pack_x(const BlockDesc *blocks, int n, const int *a_idx, const double *sqrtw,
                          int nA, int ka_pad, int nparts, int MN, uint16_t *x_bf16, double *x_f64,
                          cudaStream_t st);

// diag[k] = sum_j G64[k][j]^2 (fp64) and the largest admissible diagonal
// entry (dmax, 8 bytes); then invC / D / admissibility (n_admissible).
cudaError_t launch_tables_diag(const double *G64, int ldg, int K, int Kp, int nA, const uint8_t *dup,
                               double *diag, unsigned long long *dmax, int *n_admissible,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_tables_finalize(const double *diag, const uint8_t *dup,
                                   const unsigned long long *dmax, int K, int Kp, T *invC, T *Dk,
                                   int *n_admissible, cudaStream_t st);

// A contiguous batch: block b has samples / out at b MN, sel_idx at b I and
// sel_coef at b I coef (coef = 2 for complex plans); NULL logs stay NULL.
struct StridedSpec {
    const double *samples;
    double *out;
    int32_t *sel_idx;
    double *sel_coef;
    int I;
    int coef;
};
// Descriptors of such a batch, written on the device.
cudaError_t launch_fill_desc(BlockDesc *d, int n, const StridedSpec &s, int MN, cudaStream_t st);

// One CTA that waits on an mbarrier nothing arrives at, bounded by limit_ns;
// it sets DEV_ERR_WAIT_TIMEOUT in *err and returns (the failure path, on purpose).
cudaError_t launch_wait_probe(int *err, unsigned long long limit_ns, cudaStream_t st);
// The fp64 -> fp32 sample conversion of the projection kernels, on n values,
// and (back != NULL) the fp32 -> fp64 output conversion of the model kernels.
cudaError_t launch_convert_probe(const double *in, float *out, double *back, int n, cudaStream_t st);

// Grid of a persistent launch: min(want, SMs x resident CTAs per SM) for
// kernel kern at this block size and dynamic shared memory; the first call for
// a kernel raises its dynamic shared memory limit (and, with max_shared,
// prefers the largest shared-memory carveout).  Cached per device.
cudaError_t launch_grid(const void *kern, int threads, size_t smem, int want, int *grid, bool max_shared = false);
// SMs of the current device (cached).
int sm_count();
// Ask for the largest shared-memory carveout for a kernel (once per device):
// kernels launched side by side on several streams share SMs only when their
// carveouts agree.
cudaError_t prefer_max_shared(const void *kern);

// ------------------------------------------------------------------ iterate
struct IterArgs {
    const BlockDesc *blocks;
    int n;
    int K, Kp;              // dictionary size and padded size (row pitch of C, R0)
    const void *R0;         // [n][Kp] initial projections (eq. 12); fp32 form: scaled by D_k
    const void *C;          // [Kp][Kp] table (eq. 16); fp32 form: rows scaled, T[u][k] = C(k,u) D_k
    const void *invC;       // [Kp] 1 / C_kk (0 for inadmissible)
    const void *Dk;         // [Kp] 1 / sqrt(C_kk) (NaN for inadmissible)
    const void *PhiB;       // [Kp][nB] atoms on the pattern's loss pixels
    const int *b_idx;       // [nB] loss pixel indices of the pattern
    const uint8_t *pat_support;   // [MN] the pattern (1 = A)
    int nB;
    int MN;
    double gamma;
    int I_max;              // largest iteration count in the batch
    int *err;
    int *log_u;             // fp32 form: [n][I_max] selection log (workspace) read by the
    float *log_c;           //   model kernel (required); the fp64 form evaluates the model itself
    // symmetric weighting with parity-structured atoms (the fp32 class kernel): atoms permuted
    // so that the 4 parity classes are contiguous (perm[new] = original index), each row of the
    // compact table holds only its class (Kp/4 entries), D in the permuted order
    const int *perm;
    const float *Cc;
    const float *Dkp;
    const float *r0_scale;  // fp32 form: if set, R0 holds unscaled R_k and the kernel forms
                            //   R'_k = R_k * r0_scale[k] (D_k) when it loads them
    const void *What;       // complex DFT plans: [2][M*N] planes of the 2-D DFT of w (scaled by
                            //   1/MN); C(k,u) = What[(mu_k - mu_u) mod M][(eta_k - eta_u) mod N]
                            //   replaces the table (Sec. VI); NULL: the table C is used
    int Mdft, Ndft;
    int *cert_flag;         // certified fp32 form: [n] first iteration whose two best |R'| lie
                            //   within cert_delta (relative) of each other, -1 if none; NULL: off
    float cert_delta;
};
// variant < iterate_variants(Kp, fp64): launch shapes with identical results
// (see launch_iterate_full<float>).
template <typename T>
cudaError_t launch_iterate_full(const IterArgs &a, cudaStream_t st, int *launches, int variant = 0);
int iterate_variants(int Kp, bool fp64);
// Largest padded K of the certified fp32 form (one warp per block).
int iterate_cert_max_kp();
// The parity-class form of the fp32 iterations (a.perm, a.Cc, a.Dkp set; Kp = K
// in {512, 1024, 2048}): each update touches only the selected atom's class.
// variant < iterate_sym_variants(Kp): 0 projections in registers, 1 in shared
// memory (more blocks per SM), 2 (Kp = 2048) in tensor memory, 3 (Kp = 2048) the
// last-updated class in registers and the rest in shared memory; identical results.
cudaError_t launch_iterate_sym(const IterArgs &a, cudaStream_t st, int *launches, int variant = 0);
struct FusedModel;
// The last-updated-class form (K = 2048) with the model of eq. (9) evaluated in
// the same kernel, for loss boxes that sym_model_box accepts (up to 16 x 16 or
// 32 x 8: one or two 16 x 8 output tiles).
bool sym_model_box(int Mb, int Nb);
cudaError_t launch_iterate_sym_model(const IterArgs &a, const FusedModel &fm, cudaStream_t st, int *launches);
int iterate_sym_variants(int Kp);
// Folded separable transforms of the parity-class form (M, N in {16, 32};
// K = ntr M N, atoms k = t M N + p N + q; class c = 2 (p mod 2) + (q mod 2);
// class order perm: class, then transform, then (p, q)).
struct SymSepArgs {
    int M, N, ntr, K;
    const float *img;           // per transform A_t[M/2][2][M/2] (t_{2i+a}[m] at (m, a, i)),
                                //   B_t[N/2][2][N/2]; then rho [MN] (unmasked weights)
    const float *tc_img;        // 32 x 32 only: the same constants as m16n8k8 fragments per lane,
                                //   split into TF32 parts x_b + x_s: AF[t][a][ks][part][lane] (4 words:
                                //   A^T rows g, g + 8, columns 8 ks + q, + 4), BF[t][b][ks][nt][lane]
                                //   (b0, b1 large, b0, b1 small), then rho (fp32)
    const int *perm;            // [K] class order -> original atom
    const uint8_t *pattern;     // [MN] 1 = support
    // table: the diagonal of eq. (16) and D_k, 1/C_kk of eq. (17) (written to Dk, invC in
    // atom order; dup marks collinear duplicates), the compact rows
    // Cc[u][j] = C(perm[c Q + j], perm[u]) D_{perm[c Q + j]} (Q = K/4, c = u / Q), Dkp[u] = D_{perm[u]}
    const uint8_t *dup;
    float *Dk;
    float *invC;
    float *Cc;
    float *Dkp;
    // projections: R0[b][c Q + t (MN/4) + i (N/2) + j] = R_k of atom (t, 2i + a, 2j + b),
    // unscaled; with copy_support the support samples go to the block's out
    const BlockDesc *blocks;
    int n;
    float *R0;
    int copy_support;
};
bool sym_fold_supported(int M, int N);
cudaError_t launch_sym_rows(const SymSepArgs &a, cudaStream_t st);
// variant < sym_r0_variants(M, N): identical results (0 generic, 1 the 32 x 32 kernel)
cudaError_t launch_sym_r0(const SymSepArgs &a, cudaStream_t st, int variant = 0);
int sym_r0_variants(int M, int N);
// R^(0) of 32 x 32 parity-class blocks with split-TF32 tensor-core products (a.tc_img set);
// accurate like the fp32 transforms but not bitwise equal to them.
cudaError_t launch_sym_r0_tc(const SymSepArgs &a, cudaStream_t st);
// Iterations, model and replacement for complex-valued atoms (k_complex.cu):
// R0 [n][2][Kp], C [Kp][2][Kp] (row u = C(., u)), invC [Kp], PhiB [Kp][2][nB];
// sel_coef receives (Re, Im) pairs.
template <typename T> cudaError_t launch_iterate_cplx(const IterArgs &a, cudaStream_t st);

// ------------------------------------------------------------ lazy columns
struct LazyArgs {
    const BlockDesc *blocks;   // device; support = the block's own mask
    int n, K, Kp, MN, I_max;
    const uint8_t *dup;        // [Kp] inadmissible-by-duplication flags (padding = 1)
    const void *Phi;           // [Kp][MN] atoms (T) for the model
    void *R;                   // [n][Kp] projections; unscaled R0 before init, then D-scaled
    void *Dk;                  // [n][Kp] D_b,k
    const void *diag;          // [n][Kp] C_b(k, k)
    int *slot_of;              // [n][Kp] cache slot of atom k or -1
    int *n_slots;              // [n] slots used (-1: block skipped)
    void *cache;               // [n][slots][Kp] columns C_b(:, u) (unscaled)
    int slots;
    int *u_log;                // [n][I_max]
    void *c_log;               // [n][I_max] (T)
    int *cur_u;                // [n]
    void *cur_c;               // [n] (T)
    int *miss_n;               // [2] column requests; round nu counts in miss_n[nu & 1]
                               // and clears miss_n[(nu + 1) & 1] for the next round
    int *miss_blk;             // [n]
    long long *miss_rows;      // [n] element offset of the requested cache row
    double gamma;
    int *err;
    // fp32 form with a compensated running recurrence (long iteration counts):
    // R' = hi + lo with hi the fp32 R' in R and lo [n][Kp] in Rlo as fp16 in
    // units of 2^(e(hi) - 24) (e(hi) the exponent of hi; |lo| <= ulp(hi) / 2, so
    // the unit value lies in [-1, 1]), the current coefficient as a float pair
    // [n] in cur_c64 and the logged coefficients in fp64 [n][I_max] in c_log64;
    // the columns, D, the diagonal and the float log of the model stay fp32.
    // NULL: off.
    uint16_t *Rlo;
    double *cur_c64;
    double *c_log64;
};
cudaError_t launch_lazy_pack(const BlockDesc *blocks, int n, int MN, int MN_pad, uint16_t *xb,
                             double *xd, uint16_t *mb, double *md, cudaStream_t st);
cudaError_t launch_lazy_pack_cols(const BlockDesc *blocks, int n, const int *miss_n, const int *miss_blk,
                                  const int *cur_u, const double *Phi64, int MN, int MN_pad,
                                  uint16_t *vb, double *vd, cudaStream_t st, uint16_t *vh = nullptr,
                                  float hscale = 1.0f);
// Rows of a plan operand (fp64 [rows][ld_in]) as two fp16 parts of x * scale:
// out[r][part][ka_pad], zero past cols.
cudaError_t launch_split_f16(const double *in, int rows, int cols, int ld_in, int ka_pad, float scale,
                             uint16_t *out, cudaStream_t st);
template <typename T> cudaError_t launch_lazy_init(const LazyArgs &a, cudaStream_t st);
template <typename T> cudaError_t launch_lazy_round(const LazyArgs &a, int nu, cudaStream_t st);
template <typename T> cudaError_t launch_lazy_model(const LazyArgs &a, cudaStream_t st);

// Separable transform-domain scalar products (DCT / WHT dictionaries).
struct SepArgs {
    int M, N;
    int ntr;                    // 1 or 2 transforms (DCT u WHT)
    const void *TM[2];          // [M][M] 1-D basis rows of transform t (T)
    const void *TN[2];          // [N][N]
    int koff[2];                // first atom index of transform t
    int mode;                   // 0: R0, 1: diagonal, 2: column of the current atom,
                                // 3: column of atom i (item i) on the pattern
    const BlockDesc *blocks;    // support = the block's mask (NULL: pattern)
    const uint8_t *pattern;     // mask used when a block's support is NULL, and by mode 3
    const float *scale;         // optional per-atom factor applied to every output (fp32 form)
    const double *rho;          // [MN] weights of eq. (5) without the mask
    const int *n_dev;           // optional live item count
    const int *item_blk;        // optional block of item i (mode 2), else i
    const int *cur_u;           // mode 2: atom of block b
    void *out;                  // T output
    long long ldo;              // row pitch for row b when out_rows is NULL
    const long long *out_rows;  // optional element offset of item i's row
    int n;
    int kfill;                  // entries [K, kfill) of each row are set to the padding
                                // value (NaN with scale, else 0); 0 = none
    int copy_support;           // mode 0: also write the samples on the item's support to its
                                // out (the replacement of Alg. 3 on A, fused with the read)
    const float *img;           // fp32 shared-memory image of the constants: per transform
                                // TmT [M][M] (t_p[m] at m M + p), TnT [N][N]; then rho [MN]
};
// variant < sep_variants(a, fp64): schedules with identical results (fp32:
// 0 = one warp per item, 1 = one 64-thread group per item, where both exist).
template <typename T> cudaError_t launch_sep(const SepArgs &a, cudaStream_t st, int variant = 0);
int sep_variants(const SepArgs &a, bool fp64);

// Model on the loss pixels and replacement from the selection log written by
// the fp32 iteration kernel (eq. 9 and the last step of Alg. 3).
cudaError_t launch_model_f32(const IterArgs &a, cudaStream_t st);

// The same for separable dictionaries: g[m][n] = sum_nu c_nu t_p[m] t'_q[n]
// over the log, from the 1-D rows held in shared memory (no gather of atom
// values); evaluated on the bounding box [m0, m1) x [n0, n1) of B and
// written on its loss pixels.  The support pixels are not written here: the
// projection pass (mode 0 with copy_support) has copied them.  Uses s.M,
// s.N, s.ntr, s.TM, s.TN, s.koff.
cudaError_t launch_sep_model(const IterArgs &a, const SepArgs &s, int m0, int m1, int n0, int n1,
                             cudaStream_t st);
// True when launch_sep_model takes the tensor-core form for an Mb x Nb box.
bool sep_model_tc_box(int Mb, int Nb);

// The same model evaluated by the parity-class iteration kernel itself once a
// block's iterations are done (same operations as the tensor-core model kernel,
// so the same bits): the pattern's transforms, their 1-D rows in the model
// kernel's layout and the loss box [m0, m0 + Mb) x [n0, n0 + Nb).
struct FusedModel {
    SepArgs s;
    const float *tab;   // ntr (M M + N N) floats: T_t[p][m] at t (M M + N N) + p M + m,
                        // then T'_t[q][n] at t (M M + N N) + M M + q N + n
    int m0, Mb, n0, Nb;
    int compact;        // 1: M = N, m0 = n0, no clamped box row or column, and the rows
                        //   t_p[m0 .. m0 + 16 MT) of every transform fit the block's slots
                        //   beside the log table and output tile (staged there, serving
                        //   both factors); 0: the rows are read from tab
};

// Seeded synthetic samples in [0, 255) for the probe batches of the tuner.
cudaError_t launch_probe_samples(double *s, long long total, uint32_t seed, cudaStream_t st);

// Padded dictionary size the iteration kernel uses for K atoms (-1: too large).
int iterate_kp(int K, bool fp64);

// Split fp64 rows into bf16 parts: out[r][p * ka_pad + j] for j < cols
// (zero for cols <= j < ka_pad).
cudaError_t launch_split_bf16(const double *in, int rows, int cols, int ld_in, int ka_pad,
                              int nparts, uint16_t *out, cudaStream_t st);

}  // namespace se
