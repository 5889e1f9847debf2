/*
 * se.h -- C ABI of the GB300 Fast Selective Extrapolation library (libse.so).
 *
 * Selective Extrapolation (SE) conceals a loss area B of an M x N
 * extrapolation area L = A u B from the support area A by building the
 * sparse model g = sum_k c_k phi_k of eq. (1) greedily over a dictionary of
 * K atoms phi_k.  This library runs the fast formulation (FaSE, Alg. 2 and
 * Alg. 3 of Seiler & Kaup, "A Fast Algorithm for Selective Signal
 * Extrapolation with Arbitrary Basis Functions"), which selects the same
 * atoms with the same coefficients as the original SE of Alg. 1 (Sec. III).
 *
 * Conventions shared by every entry point
 *   - Every function returns an se_status; nothing aborts, throws or exits
 *     across this boundary.  On failure se_last_error() describes it.
 *   - Arrays are row-major: an area is M x N with m the row index; a
 *     dictionary is atom-major, K x M x N.
 *   - "device" pointers are CUDA device (or managed) memory of the context's
 *     device; "host" pointers are ordinary host memory.
 *   - The caller keeps ownership of every buffer it passes.  Descriptor
 *     contents (se_plan_desc arrays) are copied before the call returns.
 *   - Precision and layout of results do not depend on how requests are
 *     grouped into batches: a block gives the same result alone and mixed
 *     with others.
 */
#ifndef SE_H
#define SE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SE_OK = 0,
    SE_PENDING = 1,            /* se_poll: request not finished yet */
    SE_ERR_INVALID = -1,       /* an argument is out of range (see se_last_error) */
    SE_ERR_NOMEM = -2,         /* device or host allocation failed, or the HBM budget is too small */
    SE_ERR_CUDA = -3,          /* a CUDA call failed, or a kernel reported an error status */
    SE_ERR_TIMEOUT = -4,       /* a bounded wait ran out */
    SE_ERR_EMPTY_SUPPORT = -5, /* no atom has weighted energy on A (e.g. w == 0 everywhere) */
    SE_ERR_CANCELLED = -6,     /* the request was cancelled with se_cancel */
    SE_ERR_UNKNOWN_TICKET = -7 /* se_poll / se_cancel: no such ticket */
} se_status;

/* Dictionaries.  DCT: 2-D orthonormal DCT-II, atom (p, q) has index p*N + q.
 * WHT: 2-D Walsh-Hadamard in sequency order (p sign changes along m), index
 * p*N + q, M and N powers of two.  DCT_WHT: DCT atoms at [0, MN), WHT atoms
 * at [MN, 2MN) (the union used in Sec. I, Fig. 1).  NUMERIC: caller-given
 * atoms (the "only numerically defined" case of Sec. III). */
typedef enum {
    SE_BASIS_DCT = 1,
    SE_BASIS_WHT = 2,
    SE_BASIS_DCT_WHT = 3,
    SE_BASIS_NUMERIC = 4,
    /* Complex-valued atoms (the general case of Sec. II-III; conjugated scalar
     * products, Hermitian table).  DFT: exp(j 2 pi (mu m / M + eta n / N)) /
     * sqrt(MN), k = mu N + eta.  BDFT (binarised DFT, Sec. I): sgn(cos theta) +
     * j sgn(sin theta) of the same phase, sgn(0) = +1, scaled by 1/sqrt(2MN).
     * DFT_BDFT: DFT at [0, MN), BDFT at [MN, 2MN).  Samples stay real; the model
     * is complex and its real part replaces the loss area; sel_coef receives
     * (Re, Im) pairs (2 doubles per iteration).  2-D areas, FP64 or BF16X6,
     * blocks on the plan's pattern, device entry points (batch, strided). */
    SE_BASIS_DFT = 5,
    SE_BASIS_BDFT = 6,
    SE_BASIS_DFT_BDFT = 7
} se_basis;

/* Arithmetic of the scalar-product stage (tables C of eq. 16 and initial
 * projections R^(0) of eq. 12) and of the running recurrence of eq. (20).
 *   FP64    every stage in double precision on CUDA cores (the plain form);
 *   BF16X6  tensor-core products of a 3-way bf16 split (6 partial products,
 *           ~fp32 accuracy), fp32 accumulation, fp32 recurrence;
 *   BF16X3  2-way bf16 split (3 partial products), fp32 accumulation;
 *   BF16    single bf16 products, fp32 accumulation (fastest, ~3 digits);
 *   CERTIFIED  the BF16X6 form whose iteration kernel also tracks, per block,
 *           the relative gap between the two largest |R_k| D_k of every
 *           selection (eq. 18); blocks where it falls to 1.5e-5 or below at
 *           any iteration -- where the fp32 selection could differ from the
 *           fp64 one -- are computed again by an internal FP64 plan, so every
 *           block's selected-index sequence is the FP64 form's (tested on the
 *           benchmark workloads; the threshold is about 10x the largest fp32
 *           score error measured there).  Synchronous on the caller's stream
 *           (the flagged blocks are collected on the host); blocks on the
 *           plan's pattern only, K <= 2048.  Counted by se_cert_stats. */
typedef enum {
    SE_PREC_FP64 = 0,
    SE_PREC_BF16X6 = 1,
    SE_PREC_BF16X3 = 3,
    SE_PREC_BF16 = 4,
    SE_PREC_CERTIFIED = 5
} se_prec;

/* How the weighted scalar products between atoms (eq. 16) are provided.
 * FULL: the K x K table per weighting pattern (Alg. 2), for blocks that use
 * the plan's pattern.  LAZY: only the columns C(:, u) of atoms actually
 * selected, computed per block on first selection and cached; required for
 * blocks with their own support mask.  AUTO: FULL for the plan's pattern,
 * LAZY for per-block masks. */
typedef enum {
    SE_GRAM_AUTO = 0,
    SE_GRAM_FULL = 1,
    SE_GRAM_LAZY = 2
} se_gram;

/* How the scalar products of the shared-pattern path (table C of eq. 16 and
 * projections R^(0) of eq. 12) are computed.
 * DENSE: as matrix products over the support pixels (tensor cores in the
 * bf16 forms, CUDA cores in FP64).  TRANSFORM: for DCT, WHT and DCT_WHT
 * dictionaries, whose atoms are products of 1-D basis rows, every weighted
 * scalar product with a signal is an entry of a separable 2-D transform of
 * that weighted signal (Sec. VI, eqs. 21-23): fp32 (fp64 in the FP64 form)
 * transforms on CUDA cores, 2MN(M+N) operations per signal instead of
 * 2KMN; the bf16 split of `prec` is then not used.  Requires a separable
 * basis whose transform operands fit in shared memory (else SE_ERR_INVALID).
 * AUTO: TRANSFORM where it applies, DENSE otherwise. */
typedef enum {
    SE_PRODUCTS_AUTO = 0,
    SE_PRODUCTS_DENSE = 1,
    SE_PRODUCTS_TRANSFORM = 2
} se_products;

typedef struct se_ctx_s se_ctx_t;    /* opaque, library-owned */
typedef struct se_plan_s se_plan_t;  /* opaque, library-owned */

/* Parameters of the method (Sec. II): area size, dictionary, weighting
 * function (eqs. 4-5), orthogonality-deficiency factor gamma (eq. 8) and the
 * iteration count I.  All host arrays are copied by se_plan. */
typedef struct {
    int M, N;                 /* extrapolation area L is M x N samples, 1 <= M, N <= 256 */
    se_basis basis;
    int K;                    /* dictionary size: MN for DCT/WHT, 2MN for DCT_WHT, >= 1 for NUMERIC */
    const double *dict;       /* NUMERIC: host K x M x N atoms; ignored otherwise */
    double rho_hat;           /* decay of eq. (5), 0 < rho_hat <= 1 */
    const double *rho;        /* optional host M x N weights replacing eq. (5); NULL = isotropic */
    const uint8_t *support;   /* optional host M x N default pattern, 1 = A, 0 = B;
                                 NULL = centred loss area of (M/2) x (N/2) samples */
    double gamma;             /* eq. (8), 0 < gamma <= 1 */
    int iterations;           /* default I >= 1 (eq. 10: exactly I iterations) */
    se_prec prec;
    se_gram gram;
    se_products products;     /* scalar products of the shared-pattern path */
    int T;                    /* frames of a 3-D (video) area, 1..64; 0 = 1 (a 2-D area).  A 3-D
                                 area is M x N x T samples stored frame-major, index
                                 (t M + m) N + n; eq. (5) takes the distance to the centre of
                                 the block; DCT / WHT atoms are products of three 1-D rows,
                                 k = (r M + p) N + q (WHT: T a power of two); the default pattern
                                 loses the centred M/2 x N/2 box in frames T/4 .. T/4+max(T/2,1)-1.
                                 M N T <= 65536.  3-D plans use the dense products. */
} se_plan_desc;

/* One concealment block for se_extrapolate_batch (all pointers device). */
typedef struct {
    const double *samples;    /* M x N samples s; values on B are never read */
    const uint8_t *support;   /* M x N mask (1 = A, 0 = B), or NULL = the plan's pattern */
    double *out;              /* M x N result: s on A, the model g on B (Alg. 1/3 last step);
                                 out may be samples (in place: only B is written) */
    int32_t *sel_idx;         /* optional [iterations] selected atom index u per iteration */
    double *sel_coef;         /* optional [iterations] coefficient c_u per iteration */
    int iterations;           /* 0 = the plan's default I */
} se_block;

/* One request for the serving loop (all pointers host). */
typedef struct {
    const double *samples;    /* M x N; copied by se_submit */
    const uint8_t *support;   /* M x N or NULL = the plan's pattern; copied by se_submit */
    double *out;              /* M x N, written before se_poll returns SE_OK; owned by the caller */
    int32_t *sel_idx;         /* optional [iterations], written like out */
    double *sel_coef;         /* optional [iterations], written like out */
    int iterations;           /* 0 = the plan's default I */
} se_request;

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory the context allocates for plans, batch workspaces and
 * serving slots (0 = no bound).  Returns SE_ERR_CUDA if the device cannot
 * be used. */
se_status se_ctx_create(int device, size_t hbm_budget_bytes, se_ctx_t **out);

/* Stop the serving thread (pending requests end as SE_ERR_CANCELLED), free
 * all plans and device memory of the context.  NULL is accepted. */
se_status se_ctx_destroy(se_ctx_t *ctx);

/* Build a plan: the dictionary (Sec. I / NUMERIC), the default weighting
 * pattern (eqs. 4-5), the admissible-atom flags (collinear duplicates of a
 * lower-index atom are never selected, so ties go to the smallest index),
 * and device copies of the atoms in the plan's precision.  The table C of
 * eq. (16) for the default pattern is built lazily by the first batch that
 * needs it (and again after se_plan_reset_tables).  Validation: M, N in
 * [1, 256]; K must match the basis; WHT needs powers of two; 0 < rho_hat
 * <= 1; 0 < gamma <= 1; iterations >= 1 -- else SE_ERR_INVALID.  A default
 * pattern without support returns SE_ERR_EMPTY_SUPPORT. */
se_status se_plan(se_ctx_t *ctx, const se_plan_desc *desc, se_plan_t **out);

/* Free a plan.  The caller must ensure no batch using it is in flight. */
se_status se_plan_destroy(se_plan_t *plan);

/* Drop the cached table C / D of eq. (16)-(17) so the next batch rebuilds
 * it (Alg. 2).  Used to time table generation as part of a step. */
se_status se_plan_reset_tables(se_plan_t *plan);

/* Extrapolate n blocks of one plan, asynchronously on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Runs, on the device:
 * weighting and operand packing, the table C (Alg. 2) if not cached, the
 * initial projections R^(0) (eq. 12), the I iterations of Alg. 3
 * (selection eq. 18, coefficient eq. 19, model eq. 9, update eq. 20) and
 * the replacement of B.  Device buffers of the blocks must stay valid until
 * the stream reaches this point; the library's workspace is reused by the
 * next call on the same context, so calls on one context are serialised on
 * the host.  Returns SE_ERR_INVALID for bad blocks (NULL samples/out,
 * iterations < 0), SE_ERR_NOMEM if the workspace exceeds the budget. */
se_status se_extrapolate_batch(se_ctx_t *ctx, const se_plan_t *plan, int n,
                               const se_block *blocks, void *cuda_stream);

/* Convenience form of se_extrapolate_batch for n blocks stored contiguously
 * on the device: samples[n][M][N], out[n][M][N], optional sel_idx /
 * sel_coef [n][iterations] (iterations = 0: the plan's I), all blocks on
 * the plan's pattern.  out may equal samples: then the call works in place,
 * reading only the support samples and writing only the loss areas. */
se_status se_extrapolate_strided(se_ctx_t *ctx, const se_plan_t *plan, int n,
                                 const double *samples, double *out,
                                 int32_t *sel_idx, double *sel_coef,
                                 int iterations, void *cuda_stream);

/* Allocation-free form of se_extrapolate_strided, for callers that cannot
 * allocate memory while they run (no cudaMalloc, no pinned host memory, no
 * allocating library routine in the call): for example a real-time loop that
 * forbids allocation after start-up, or a host that gives the library only
 * its own input and output buffers.  The paper has no counterpart; this is
 * a deployment variant of the same computation and gives the same results as
 * se_extrapolate_strided.  Arguments as there (device buffers, contiguous
 * blocks on the plan's pattern).  Per-call scratch (descriptors, packed
 * samples of the dense products, initial projections, the selection log)
 * lives in one static 16 MiB device array that every GPU loading the library
 * holds until exit; n is limited by it (for 32 x 32 blocks with K = 2048 and
 * I = 100: about 1800 with transform products, 1200 with dense split-bf16
 * products, 1000 in the fp64 form) and larger n returns SE_ERR_INVALID with
 * the limit in se_last_error().  se_ctx_create looks up the array's device
 * address on the context's device (which also loads the array, so its
 * 16 MiB are held from context creation); the call itself allocates
 * nothing and does no CUDA set-up.  Argument errors (complex or certified
 * plans, iterations < 0) are reported whatever n is.  All calls share the
 * array: calls whose work overlaps on the GPU race, so
 * serialise them.  The plan's table is built into plan memory on first use;
 * the autotuner times no candidates inside this call (it takes its kept
 * choice, else the first variant). */
se_status se_extrapolate_noalloc(se_ctx_t *ctx, const se_plan_t *plan, int n,
                                 const double *samples, double *out, int32_t *sel_idx,
                                 double *sel_coef, int iterations, void *cuda_stream);

/* Same as se_extrapolate_strided but with HOST buffers; returns when out (and
 * the optional logs) hold the results.  Buffers the GPU can address (pinned /
 * page-locked memory: cudaHostAlloc, cudaHostRegister, torch pin_memory) are
 * read and written by the kernels directly over the host link, so the transfers
 * overlap the computation; other (pageable) buffers are copied through the
 * context's device buffer in chunks of at least 512 blocks, the copies of one
 * chunk overlapping the computation of the others.  out may equal samples (in
 * place): each block's loss area is overwritten with its extrapolation, and
 * with pinned buffers only the support samples cross the link inwards and
 * only the loss areas outwards (half the bytes of separate buffers for a
 * quarter loss area).  Pinned calls run as one chunk; SE_PINNED_CHUNKS
 * (environment, 1 .. 4, read at each call) splits them into up to that many
 * chunks of at least 1024 blocks on their own streams.
 * Serialised with the other batch calls of the context. */
se_status se_extrapolate_host(se_ctx_t *ctx, const se_plan_t *plan, int n,
                              const double *samples, double *out,
                              int32_t *sel_idx, double *sel_coef, int iterations);

/* Asynchronous form of se_extrapolate_host (the same operation: Alg. 2 table
 * if not cached, eq. 12, Alg. 3 with eqs. 18-20, eq. 9 and the replacement of
 * the loss area), for a stream of batches: it enqueues the batch and returns a
 * ticket; the results are in out (and the optional logs) once
 * se_host_wait(ctx, ticket) has returned SE_OK.  Each call copies its n
 * blocks of samples (host, MN doubles each, block-major) into a device buffer
 * of one of the context's three host slots with a copy engine, runs the batch
 * there in place, and copies back: with out == samples, of every block, the
 * samples from the first to the last one of the pattern's loss bounding box
 * (every sample of a 3-D block), else every sample; then the logs (host int32
 * [n][I] and fp64 [n][I], each optional).
 * So the copies of one call overlap the computation of the calls in flight
 * beside it.  The caller keeps samples, out and the logs unchanged and valid
 * until the wait; they should be pinned (page-locked: cudaHostAlloc,
 * cudaHostRegister, torch pin_memory), since copies from pageable memory are
 * not asynchronous.  A call that finds all three slots busy first waits for
 * the oldest one.  A table rebuild (first use, se_plan_reset_tables) waits on
 * the device for the calls still in flight.  Device errors of any call of the
 * context are reported by the next se_host_wait or se_sync.  Returns
 * SE_ERR_INVALID for NULL arguments, n < 0, iterations < 0, complex plans or
 * a plan of another context; n = 0 returns SE_OK and ticket 0.  Serialised
 * with the other batch calls of the context on the host. */
se_status se_extrapolate_host_async(se_ctx_t *ctx, const se_plan_t *plan, int n,
                                    const double *samples, double *out,
                                    int32_t *sel_idx, double *sel_coef, int iterations,
                                    uint64_t *ticket);

/* Wait for the asynchronous host-buffer call `ticket` (0 and tickets already
 * waited for return SE_OK at once).  SE_ERR_CUDA with a message if the
 * context's device status word reports an error (it is then cleared);
 * SE_ERR_UNKNOWN_TICKET for a ticket that was never issued. */
se_status se_host_wait(se_ctx_t *ctx, uint64_t ticket);

/* Exercises the device failure path: queues on `cuda_stream` one CTA that
 * waits on an mbarrier nothing arrives at.  Like every wait in the library's
 * kernels the wait is bounded (%globaltimer); after limit_us microseconds
 * (1000 .. 2000000) it gives up, records the timeout in the context's status
 * word and returns, so the context stays usable; the next se_sync on that
 * stream returns SE_ERR_CUDA with the message and clears the word.  For tests
 * and health checks of a deployment. */
se_status se_check_wait_timeout(se_ctx_t *ctx, uint32_t limit_us, void *cuda_stream);

/* Applies, on `cuda_stream`, the fp64 -> fp32 conversion that the projection
 * kernels use for the samples (eq. 12 in the fp32 form: w s with s rounded
 * to fp32) to n device doubles `in`, writing n device floats `out`, and, if
 * `back` (n device doubles) is not NULL, the fp32 -> fp64 conversion that the
 * model kernels use for their results (eq. 9) to those floats.  The first
 * rounds to nearest, ties to even, the second is exact, as IEEE 754 defines
 * them; most values take integer-pipe paths, so this lets a test check both
 * bit for bit.  SE_ERR_INVALID for NULL in/out with n > 0 or n < 0. */
se_status se_check_sample_conversion(se_ctx_t *ctx, const double *in, float *out, double *back, int n,
                                     void *cuda_stream);

/* Wait for the work this context queued on `cuda_stream` and report
 * errors that its kernels recorded in the device status word (SE_ERR_CUDA
 * with a message, e.g. a bounded wait that ran out).  Clears the word. */
se_status se_sync(se_ctx_t *ctx, void *cuda_stream);

/* Serving loop.  se_submit copies the request into library memory (the
 * caller may free samples/support on return), queues it and returns a
 * ticket.  A scheduler thread admits queued requests into device slots as
 * slots and HBM budget free up, runs the iteration kernels in slices over
 * all admitted blocks (continuous batching: requests that arrive while
 * others run join at the next slice) and copies results into the caller's
 * out/sel buffers.  Each slot has its own stream and workspace.  The state it
 * shares with the batch entry points is locked: tables, tuner, cost probes,
 * graphs and the budget.  So requests may be submitted while other threads
 * call those entry points on the same context.  Returns SE_ERR_INVALID for a
 * bad request, SE_ERR_NOMEM if one block can never fit the budget. */
se_status se_submit(se_ctx_t *ctx, const se_plan_t *plan, const se_request *req,
                    uint64_t *ticket);

/* Wait up to timeout_us microseconds (0 = do not wait, < 0 = wait without
 * limit) for a ticket.  SE_OK: done, out written, the ticket is retired
 * and latency_s (if non-NULL) receives submit-to-completion seconds.
 * SE_PENDING: not finished.  Other codes: the request failed (retired). */
se_status se_poll(se_ctx_t *ctx, uint64_t ticket, int64_t timeout_us, double *latency_s);

/* Cancel a request that has not been admitted yet (SE_OK), or report that
 * it is already running / done (SE_PENDING / SE_ERR_INVALID). */
se_status se_cancel(se_ctx_t *ctx, uint64_t ticket);

/* Message of the last failing call on this thread ("" if none). */
const char *se_last_error(void);

/* Statistics of the context since creation: kernels launched by the library,
 * table builds, serving slices.  Any pointer may be NULL. */
se_status se_stats(se_ctx_t *ctx, uint64_t *kernel_launches, uint64_t *table_builds,
                   uint64_t *serving_slices);

/* Per-stage device timing.  When enabled, the library records CUDA events
 * on the launching stream around each stage of every batch and accumulates
 * their durations after the batch completes (read with se_stage_times).
 * Stages: 0 operand packing, 1 table generation (Alg. 2, only when rebuilt),
 * 2 initial projections (eq. 12), 3 iterations (Alg. 3; for the fp64 form
 * and for per-block masks this includes the model and replacement), 4 model
 * evaluation and replacement (eq. 9, the fp32 shared-pattern form).
 * se_stage_times synchronises the context's outstanding batches, writes up
 * to n_stages accumulated milliseconds and launch counts (either pointer may
 * be NULL) and, if reset != 0, clears the accumulators. */
se_status se_set_profiling(se_ctx_t *ctx, int enable);
se_status se_stage_times(se_ctx_t *ctx, double *ms, uint64_t *count, int n_stages, int reset);

/* Measured choice between the full table (Alg. 2) and lazily computed
 * columns for blocks on a plan's pattern under SE_GRAM_AUTO.  While the table
 * is not built, a batch of pattern blocks is served lazily as long as the
 * extra cost of the blocks served lazily since the table was last needed,
 * plus this batch, stays below one table build; otherwise the table is built
 * (and then kept).  The three costs -- one table build, one block with the
 * table, one block with lazy columns -- are measured with CUDA events on
 * every batch and by se_plan_autotune, which runs n_probe (1..65536) seeded
 * synthetic blocks of the plan's pattern through both paths, synchronously
 * on cuda_stream, after a warm-up that also lets the autotuner time the
 * kernel variants of these shapes.  The plan's table is left built.  Uses the
 * context's batch workspace and two temporary device buffers of n_probe M N
 * doubles (SE_ERR_NOMEM beyond the budget). */
se_status se_plan_autotune(se_ctx_t *ctx, se_plan_t *plan, int n_probe, void *cuda_stream);
/* The plan's measured costs in milliseconds (0 = not measured yet); any
 * pointer may be NULL. */
se_status se_plan_costs(const se_plan_t *plan, double *table_ms, double *full_ms_per_block,
                        double *lazy_ms_per_block);

/* CUDA graphs: the lock-step rounds of the lazy path are captured once per
 * (plan, wave size, iteration count, workspace) and replayed (default on;
 * at most 32 graphs per context, the least recently used dropped first).
 * A shape is launched directly the first time it is seen and captured the
 * second time, so one-off shapes (most serving batches) cost no capture. */
se_status se_set_graphs(se_ctx_t *ctx, int enable);
/* Autotuner and graph counters: shapes tuned (each timed its candidates
 * once), graphs captured, graph replays.  Any pointer may be NULL.  The
 * autotuner times interchangeable kernel variants (identical results) on
 * the first launch of a shape; SE_TUNE_FILE (environment) names a file that
 * stores the choices across processes, and SE_TUNE_FORCE ("prefix=variant,...")
 * forces the variant of every shape key that starts with a prefix.  SE_R0_FFMA=1
 * (read when a plan is created) keeps the fp32 CUDA-core projection kernels of
 * 32 x 32 parity-class plans instead of the split-TF32 tensor-core one. */
se_status se_tuning_stats(se_ctx_t *ctx, uint64_t *tunings, uint64_t *graph_builds, uint64_t *graph_replays);
/* SE_PREC_CERTIFIED plans: blocks computed, and blocks computed again in fp64
 * because a selection was within the certification gap.  Either pointer may
 * be NULL. */
se_status se_cert_stats(se_ctx_t *ctx, uint64_t *blocks, uint64_t *recomputed);
/* Which forms a plan's shared-pattern batches use, as a short text into buf
 * (NUL-terminated, truncated to len): products ("transform" / "dense"),
 * table ("table" / "dft-of-weights"), iterations ("parity-classes" when the
 * weighting function is symmetric and the atoms are DCT / WHT rows, see
 * k_sym.cu; "general" otherwise; "complex"; "fp64"), "projections=split-tf32"
 * when a 32 x 32 parity-class plan forms eq. (12) on the tensor cores, and
 * "certified" for certified plans, and "columns=f16x3" once a batch with
 * per-block masks has prepared the lazy columns of eq. (16) of a numeric
 * dictionary in the fp32 form as products of two-part fp16 splits (three
 * partial products, about 2^-21 relative).  Example: "products=transform
 * table=table iterations=parity-classes projections=split-tf32". */
se_status se_plan_info(const se_plan_t *plan, char *buf, size_t len);
/* The variant the autotuner keeps for a shape key (e.g. "iterate:f32:2048",
 * "sep:32x32:t2:f32", "sym:f32:2048:n4096" for the parity-class iterations of
 * a 4096-block batch, "symr0:32x32:t2"), or -1 in *variant when that key has
 * not been tuned. */
se_status se_tuned_variant(se_ctx_t *ctx, const char *key, int *variant);

#ifdef __cplusplus
}
#endif

#endif /* SE_H */
