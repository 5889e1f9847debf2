// se_host.h -- host-side structures of libse.so (contexts, plans, buffers).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "../../include/se.h"
#include "se_internal.h"

struct se_ctx_s;

namespace se {

bool build_dictionary(int M, int N, int T, int basis, int K, const double *numeric,
                      std::vector<double> &phi, std::string *why);
void find_collinear(int K, int MN, const double *phi, std::vector<uint8_t> &dup);
// 1-D bases: orthonormal DCT-II rows and +-1 Walsh rows in sequency order (L x L).
void dct_rows(int L, std::vector<double> &T);
void walsh_seq_rows(int L, std::vector<double> &T);
void weighting(int M, int N, int T, double rho_hat, const double *rho, const uint8_t *support,
               std::vector<double> &w);

// A device allocation charged against the context's HBM budget.
struct DevBuf {
    se_ctx_s *ctx = nullptr;
    void *ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf();
    void release();
    template <typename T> T *as() const { return static_cast<T *>(ptr); }
};

// Device workspace of one in-flight batch (descriptors, packed operands,
// initial projections, host-call I/O) with its pinned descriptor staging.
struct Workspace {
    DevBuf desc, x, r0, io, logs, cert;
    // per-block-mask (lazy) path
    DevBuf lz_R, lz_D, lz_diag, lz_slot, lz_nslots, lz_cache, lz_ulog, lz_clog, lz_cur, lz_miss,
        lz_x, lz_mk, lz_v;
    DevBuf lz_R64, lz_c64;   // fp64 running recurrence of long fp32 runs: R', current and logged c
    BlockDesc *h_desc = nullptr;
    size_t h_desc_cap = 0;
    cudaEvent_t ev_staging = nullptr;     // the staging copy of the last batch has landed
    cudaEvent_t ev_ws = nullptr;          // the last batch no longer uses the workspace
    ~Workspace();
    cudaError_t init();
};

// Record a failure for se_last_error() and return the status.
se_status set_error(se_status s, const std::string &msg);

// Device address (on the current device) of the static array that
// se_extrapolate_noalloc uses as scratch (se_noalloc.cu).
se_status noalloc_scratch_address(void **out);

// Precision set-up derived from se_prec.
struct PrecCfg {
    bool fp64 = false;
    int nparts = 1;
    int npairs = 1;
    int pa[8] = {0}, pb[8] = {0};
};
PrecCfg prec_cfg(se_prec p);

// Autotuner state of a context (se_tune.cpp): the chosen variant per shape
// key, the candidates' measured times, the persistence file and forced choices.
struct Tuner {
    std::mutex mu;
    std::map<std::string, int> best;
    std::map<std::string, std::vector<float>> ms;
    std::string file;
    std::vector<std::pair<std::string, int>> force;
    void load_env();
    void save() const;
};

}  // namespace se

struct se_plan_s;

namespace se {
// Identity of a captured lazy round loop: plan, wave size, iteration count
// and the workspace addresses baked into its kernel arguments.
struct GraphKey {
    const se_plan_s *plan = nullptr;
    int nw = 0, I_max = 0;
    const void *ptr[10] = {};
    bool operator==(const GraphKey &o) const
    {
        if (plan != o.plan || nw != o.nw || I_max != o.I_max) return false;
        for (int i = 0; i < 10; ++i)
            if (ptr[i] != o.ptr[i]) return false;
        return true;
    }
};
struct CachedGraph {
    GraphKey key;
    cudaGraphExec_t exec = nullptr;
    uint64_t last = 0;
};
// Cost probe: events around a table build (which 0), a shared-pattern batch
// without the table (1) or a lazy batch (2) of n blocks, read once complete.
struct CostProbe {
    se_plan_s *plan = nullptr;
    int which = 0, n = 0;
    cudaEvent_t a = nullptr, b = nullptr;
};
}  // namespace se

// Serving request as queued by se_submit.
struct ServeReq {
    uint64_t ticket = 0;
    se_plan_s *plan = nullptr;
    std::vector<double> samples;
    std::vector<uint8_t> support;      // empty: plan pattern
    double *out = nullptr;
    int32_t *sel_idx = nullptr;
    double *sel_coef = nullptr;
    int iterations = 0;
    double t_submit = 0.0;
    double t_done = 0.0;
    int state = 0;                     // 0 queued, 1 running, 2 done, 3 failed, 4 cancelled
    se_status status = SE_OK;
};

// One serving lane: a stream with its own batch workspace and I/O buffers.
struct ServeLane {
    cudaStream_t st = nullptr;
    se::Workspace ws;
    se::DevBuf d_io;
    char *h_io = nullptr;
    size_t h_io_cap = 0;
    cudaEvent_t done = nullptr;
    bool busy = false;
    se_plan_s *plan = nullptr;
    int I_max = 0;
    std::vector<std::shared_ptr<ServeReq>> batch;
    ~ServeLane()
    {
        if (h_io) cudaFreeHost(h_io);
        if (done) cudaEventDestroy(done);
        if (st) cudaStreamDestroy(st);
    }
};

// One slot of the asynchronous host-buffer calls: a stream, a batch workspace,
// the device copy of the call's samples (computed in place) and its logs.
struct HostSlot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;           // the call's copies out have landed
    cudaEvent_t computed = nullptr;       // its kernels are done (the table is no longer read)
    se::Workspace ws;
    se::DevBuf io;
    uint64_t ticket = 0;
    bool busy = false;
    ~HostSlot()
    {
        if (done) cudaEventDestroy(done);
        if (computed) cudaEventDestroy(computed);
        if (st) cudaStreamDestroy(st);
    }
};

struct se_ctx_s {
    int device = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    cudaStream_t stream = nullptr;        // internal stream (host-buffer calls, serving)
    cudaStream_t aux = nullptr;           // table builds that overlap a batch's projections
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::mutex amu;                       // orders the fork onto the second stream
    std::mutex mu;                        // serialises batch calls (shared workspace)

    // workspace of the batch entry points (grown on demand, reused)
    se::Workspace ws;
    // host-buffer calls in chunks: copies in on pipe_in, each chunk on its own stream
    // and workspace (chunks overlap on the device), copies out on pipe_out
    static constexpr int kPipe = 8;
    se::Workspace pipe_ws[kPipe];
    cudaStream_t pipe_st[kPipe] = {};
    cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
    cudaEvent_t pipe_ev_in[kPipe] = {}, pipe_ev_done[kPipe] = {};
    bool pipe_ready = false;
    // asynchronous host-buffer calls (se_extrapolate_host_async): round-robin slots
    static constexpr int kHostSlots = 3;
    HostSlot hslot[kHostSlots];
    bool hslot_ready = false;
    uint64_t host_next = 1;               // the next ticket
    se::DevBuf ws_err;                    // device status word shared by all kernels
    void *noalloc_scratch = nullptr;      // device address of se_extrapolate_noalloc's static array

    // per-stage timing (se_set_profiling)
    static constexpr int kStages = 5;
    bool profiling = false;
    std::mutex pmu;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;   // stage, (start, stop)
    std::vector<cudaEvent_t> event_pool;
    double stage_ms[kStages] = {0, 0, 0, 0, 0};
    uint64_t stage_count[kStages] = {0, 0, 0, 0, 0};

    std::atomic<uint64_t> launches{0};
    std::atomic<uint64_t> table_builds{0};
    std::atomic<uint64_t> slices{0};

    // autotuner, measured costs and graph cache (se_tune.cpp)
    se::Tuner tuner;
    std::atomic<uint64_t> tunings{0};
    std::mutex cpmu;
    std::vector<se::CostProbe> probes;
    std::vector<cudaEvent_t> probe_pool;
    bool graphs_enabled = true;
    static constexpr size_t kGraphCache = 32;
    std::mutex gmu;
    std::vector<se::CachedGraph> graphs;
    std::vector<se::GraphKey> graph_seen;   // shapes run once without a graph
    uint64_t graph_clock = 0;
    std::atomic<uint64_t> graph_builds{0}, graph_replays{0};
    std::atomic<uint64_t> cert_blocks{0}, cert_recomputed{0};

    // serving
    std::mutex smu;
    std::condition_variable scv;
    std::deque<std::shared_ptr<ServeReq>> queue;
    std::map<uint64_t, std::shared_ptr<ServeReq>> tickets;
    std::thread server;
    bool stop = false;
    bool server_started = false;
    std::vector<std::unique_ptr<ServeLane>> lanes;
    uint64_t next_ticket = 1;
    std::vector<se_plan_s *> plans;
};

struct se_plan_s {
    se_ctx_s *ctx = nullptr;
    se_plan_desc desc{};
    int M = 0, N = 0, MN = 0, K = 0, Kp = 0;
    int T = 1;                            // frames of a 3-D (video) area; MN = M N T samples
    se::PrecCfg pc;
    bool certified = false;               // SE_PREC_CERTIFIED: fp32 path + fp64 recomputation
    se_plan_s *shadow = nullptr;          //   the internal FP64 plan of a certified plan (owned)
    std::vector<double> phi;              // host K x MN atoms (fp64; real part for complex atoms)
    std::vector<double> phi_im;           // host K x MN imaginary part (complex atoms only)
    bool cplx = false;                    // complex-valued atoms (DFT, binarised DFT)
    std::vector<uint8_t> dup;             // host K flags
    std::vector<uint8_t> pattern;         // host MN default support
    std::vector<double> w;                // host MN weights of the default pattern
    std::vector<double> rho_map;          // host MN user weights replacing eq. (5), or empty
    std::vector<int> a_idx, b_idx;
    int nA = 0, nB = 0, ka_pad = 0;

    // device copies
    se::DevBuf d_a_idx, d_b_idx, d_sqrtw, d_pattern, d_dup;
    se::DevBuf d_G64;                     // Kp x ka_pad fp64, G = phi_A sqrt(w)
    se::DevBuf d_Gbf;                     // Kp x nparts*ka_pad bf16 split of G (tables)
    se::DevBuf d_GH;                      // Kp x 2*ka_pad fp16 split of g_f16_scale * G (tables, f16_table)
    bool f16_table = false;               // the table of eq. (16) from two-part fp16 splits (3 products)
    float g_f16_scale = 1.0f;             // power of two putting the largest |G| at or below 2^14
    se::DevBuf d_Gwbf;                    // Kp x nparts*ka_pad bf16 split of Phi_A w (projections)
    se::DevBuf d_PhiB;                    // Kp x nB (T) atoms on the loss pixels ([Kp][2][nB] complex)
    // complex atoms: [Gi|-Gr] rows for Im C (fp64 / bf16 split), [phi_r w; -phi_i w] rows of eq. 12 (fp64)
    se::DevBuf d_Gc64, d_Gcbf, d_P64;
    // DFT atoms: the table is replaced by the 2-D DFT of w ([2][MN], scaled by 1/MN, Sec. VI);
    // every atom has C_kk = What[0][0], so 1/C_kk is uniform (host copy for the table stage)
    bool dft_w = false;
    // symmetric weighting with DCT / WHT atoms: parity classes (k_sym.cu)
    // (class order perm, compact table Cc [K][K/4], D in class order, constants of the folded
    // transforms); R^(0) of such plans is stored in class order
    bool sym = false;
    se::DevBuf d_perm, d_Cc, d_Dkp, d_sym_img;
    se::DevBuf d_sym_tc;         // 32 x 32: the folded constants as tensor-core fragments
    bool sym_tc = false;         // R^(0) by split-TF32 tensor-core products
    se::DevBuf d_What;
    std::vector<double> dft_invC;
    // tables (eqs. 16-17)
    se::DevBuf d_C, d_invC, d_Dk, d_diag, d_nadm;
    bool tables_valid = false;
    // per-block-mask (lazy) operands, built on first use: Phi (fp64 and the
    // plan precision), Phi rho and Phi^2 rho over all MN pixels (bf16 parts or fp64)
    bool lazy_ready = false;
    int MN_pad = 0;
    se::DevBuf d_Phi64, d_PhiT, d_ArBf, d_AdBf, d_Ar64, d_Ad64;
    // lazy columns of numeric dictionaries in the fp32 form: Phi rho as two
    // fp16 parts scaled by f16_a_scale, the packed m_b phi_u by f16_v_scale
    se::DevBuf d_ArH;
    bool f16_cols = false;
    float f16_a_scale = 1.0f, f16_v_scale = 1.0f;
    // transform-domain form for DCT / WHT dictionaries: 1-D bases and rho
    bool sep = false, sep_checked = false;
    bool sep_full = false;       // shared-pattern tables and projections by transforms
    int box[4] = {0, 0, 0, 0};   // bounding box [m0, m1) x [n0, n1) of the pattern's B
    int sep_ntr = 0, sep_koff[2] = {0, 0};
    se::DevBuf d_sepM[2], d_sepN[2], d_rho;
    se::DevBuf d_sep_img;        // fp32 constants in the transform kernels' shared-memory layout
    se::DevBuf d_model_tab;      // fp32 1-D rows in the model kernel's layout (T_t, then T'_t, per t)
    cudaEvent_t tables_ready = nullptr;
    std::mutex tmu;
    // measured costs (ms) for the full-versus-lazy choice: one table build, one
    // block with the table built, one block with lazy columns; and the extra
    // cost of the pattern blocks served lazily since the table was last needed
    std::mutex cmu;
    double t_table_ms = 0.0, t_full_blk_ms = 0.0, t_lazy_blk_ms = 0.0, lazy_regret_ms = 0.0;
};

namespace se {
// One batch of blocks of one plan, all on the plan's pattern: tables of
// Alg. 2 if not cached, eq. (12) GEMM, Alg. 3 iterations, on stream st.  The
// descriptors come from hdesc (host) or, for a contiguous batch, from ss
// (formed on the device; hdesc may then be NULL); the kernels that read the
// samples wait for inputs_ready when it is given, and r0_done (if given) is
// recorded once they are done (before the iterations).
se_status run_batch(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, int n, const BlockDesc *hdesc,
                    int I_max, cudaStream_t st, cudaEvent_t inputs_ready = nullptr,
                    const StridedSpec *ss = nullptr, cudaEvent_t r0_done = nullptr);
// Blocks with their own masks (desc.support set for every block): lazy columns.
// Upload the transform-domain operands (weights without mask, 1-D basis
// rows) when the plan's dictionary is separable; sets pl->sep.  Idempotent;
// the caller holds pl->tmu or owns the plan exclusively.
se_status ensure_sep_ops(se_ctx_s *ctx, se_plan_s *pl);
// Transform-domain products on the plan's pattern (needs pl->sep): mode 0
// R^(0) of n blocks, mode 3 the first n rows of C, written to out with row
// pitch Kp.
SepArgs pattern_sep_args(se_plan_s *pl, int mode, const BlockDesc *dd, int n, void *out, bool scaled = true);
// Model (eq. 9) and replacement from the log of the fp32 iteration kernel
// (a.log_u / a.log_c set), for blocks on the plan's pattern.
cudaError_t launch_model(se_plan_s *pl, const IterArgs &a, cudaStream_t st);
se_status run_lazy(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, int n, const BlockDesc *hdesc,
                   int I_max, cudaStream_t st);
// Device bytes one block of a lazy (per-block mask) wave needs at I_max iterations.
size_t lazy_bytes_per_block(const se_plan_s *pl, int I_max);
se_status dev_alloc(se_ctx_s *ctx, DevBuf &b, size_t bytes);
// Build the plan's tables on stream st if they are not cached (plan memory
// only, nothing is allocated), else make st wait for the cached build.
se_status ensure_tables(se_ctx_s *ctx, se_plan_s *pl, cudaStream_t st);
// Stage timing: stage_begin returns a token (or -1 when profiling is off).
int stage_begin(se_ctx_s *ctx, int stage, cudaStream_t st);
void stage_end(se_ctx_s *ctx, int token, cudaStream_t st);
void serve_shutdown(se_ctx_s *ctx);

// While an object of this type lives, the calling thread's tune_run calls do
// not time candidates (they take the cached choice or the first candidate);
// used by the allocation-free entry point.
struct NoTuneScope {
    NoTuneScope();
    ~NoTuneScope();
};
// Complex-valued atoms (se_complex.cpp).
bool build_complex_dictionary(int M, int N, int basis, int K, std::vector<double> &re, std::vector<double> &im,
                              std::string *why);
void find_collinear_complex(int K, int MN, const double *re, const double *im, std::vector<uint8_t> &dup);
se_status setup_complex_plan(se_ctx_s *ctx, se_plan_s *pl, cudaStream_t st);
se_status build_tables_complex(se_ctx_s *ctx, se_plan_s *pl, cudaStream_t st);
se_status run_complex(se_ctx_s *ctx, se_plan_s *pl, Workspace &ws, int n, int I_max, cudaStream_t st);
// Detect the parity-class structure (symmetric w, DCT / WHT atoms) and set up
// the permutation and the compact table buffers; sets pl->sym.
se_status setup_sym(se_ctx_s *ctx, se_plan_s *pl);
// The fp32 iterations: the parity-class kernel when pl->sym, else the tuned shapes.
// With model_done given, a parity-class plan of the transform form may also run
// the model (eq. 9) in the same tuned stage; *model_done then says so.
cudaError_t launch_iterations_f32(se_ctx_s *ctx, se_plan_s *pl, IterArgs &a, cudaStream_t st, int *launched,
                                  bool *model_done = nullptr);
// A transform-domain launch with the schedule chosen by the autotuner.
cudaError_t run_sep(se_ctx_s *ctx, se_plan_s *pl, const SepArgs &sa, cudaStream_t st);
// R^(0) of n pattern blocks in the transform form (needs pl->sep_full): the
// folded class-order kernel for parity-class plans (unscaled), else the
// separable transform (scaled by D_k when scaled); support samples copied to out.
cudaError_t launch_pattern_projections(se_ctx_s *ctx, se_plan_s *pl, const BlockDesc *dd, int n, void *r0,
                                       bool scaled, cudaStream_t st);
// Move pattern blocks to the lazy list when the measured costs favour it.
void route_pattern_blocks(se_plan_s *pl, std::vector<BlockDesc> &full, std::vector<BlockDesc> &lazy,
                          int *I_full, int *I_lazy);
// Autotuner: run the fastest of n_cand interchangeable launches (identical
// results) for this shape key, timing all of them on first use.
// The forced or kept variant of a shape key (-1: none yet; the next tune_run times them).
int tune_lookup(se_ctx_s *ctx, const std::string &key, int n_cand);
cudaError_t tune_run(se_ctx_s *ctx, const std::string &key, int n_cand, cudaStream_t st,
                     const std::function<cudaError_t(int)> &run);
// SE_GRAM_AUTO, table not built: serve n pattern blocks lazily (true) or
// build the table (false), from the plan's measured costs.
bool choose_lazy_for_pattern(se_plan_s *pl, int n);
void record_cost(se_plan_s *pl, int which, double ms, int n);
// Cost probes around a stage (events from a pool; read when complete).
cudaEvent_t probe_begin(se_ctx_s *ctx, cudaStream_t st);
void probe_end(se_ctx_s *ctx, se_plan_s *pl, int which, int n, cudaEvent_t a, cudaStream_t st);
void probes_poll(se_ctx_s *ctx, bool wait, const se_plan_s *only = nullptr);
// Replay (or capture, then replay) the launches that record() issues.
cudaError_t graph_run(se_ctx_s *ctx, const GraphKey &key, cudaStream_t st,
                      const std::function<cudaError_t(cudaStream_t)> &record);
void graphs_clear(se_ctx_s *ctx);
void graphs_drop_plan(se_ctx_s *ctx, const se_plan_s *pl);
}  // namespace se
