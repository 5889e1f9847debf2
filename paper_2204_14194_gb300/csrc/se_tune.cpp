// se_tune.cpp -- the library's autotuner, the measured choice between the
// full table and lazily computed columns, and the CUDA-graph cache of the
// lazy round loop.
//
// Autotuner.  Where a stage has several kernels or launch shapes that give
// identical results (transform schedules, GEMM tile widths, warps per block of
// the iteration kernel), the first launch of a shape key times every candidate
// on the caller's stream with CUDA events (one warm-up and two timed runs
// each) and keeps the fastest for the context.  Choices can be persisted:
// SE_TUNE_FILE names a text file of "key variant" lines that is read when a
// context is created and rewritten when it is destroyed.  SE_TUNE_FORCE
// ("prefix=variant,...") forces the variant of every key that starts with a
// prefix (used by the tests to run each candidate).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <sstream>

#include "se_host.h"

namespace se {

namespace {

thread_local int tl_no_tune = 0;

bool capturing(cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

}  // namespace

NoTuneScope::NoTuneScope() { ++tl_no_tune; }
NoTuneScope::~NoTuneScope() { --tl_no_tune; }

void Tuner::load_env()
{
    if (const char *f = std::getenv("SE_TUNE_FILE")) {
        file = f;
        std::ifstream in(file);
        std::string key;
        int v;
        while (in >> key >> v) best[key] = v;
    }
    if (const char *f = std::getenv("SE_TUNE_FORCE")) {
        std::stringstream ss(f);
        std::string item;
        while (std::getline(ss, item, ',')) {
            const auto eq = item.find('=');
            if (eq != std::string::npos) force.emplace_back(item.substr(0, eq), std::atoi(item.c_str() + eq + 1));
        }
    }
}

void Tuner::save() const
{
    if (file.empty()) return;
    std::ofstream out(file);
    for (const auto &kv : best) out << kv.first << ' ' << kv.second << '\n';
}

int tune_lookup(se_ctx_s *ctx, const std::string &key, int n_cand)
{
    Tuner &t = ctx->tuner;
    int pick = -1;
    std::lock_guard<std::mutex> lk(t.mu);
    for (const auto &f : t.force)
        if (key.compare(0, f.first.size(), f.first) == 0) pick = std::min(std::max(f.second, 0), n_cand - 1);
    if (pick < 0) {
        auto it = t.best.find(key);
        if (it != t.best.end() && it->second < n_cand) pick = it->second;
    }
    return pick;
}

cudaError_t tune_run(se_ctx_s *ctx, const std::string &key, int n_cand, cudaStream_t st,
                     const std::function<cudaError_t(int)> &run)
{
    Tuner &t = ctx->tuner;
    int pick = tune_lookup(ctx, key, n_cand);
    if (pick < 0 && (n_cand <= 1 || tl_no_tune || capturing(st))) pick = 0;
    if (pick >= 0) return run(pick);

    // first use of this key: time every candidate (they write the same output)
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    std::vector<float> ms(n_cand, 0.0f);
    for (int c = 0; c < n_cand && e == cudaSuccess; ++c) {
        e = run(c);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = run(c);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[c], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    pick = static_cast<int>(std::min_element(ms.begin(), ms.end()) - ms.begin());
    {
        std::lock_guard<std::mutex> lk(t.mu);
        t.best[key] = pick;
        t.ms[key] = ms;
    }
    ctx->tunings++;
    return run(pick);
}

// ---------------------------------------------------------------------------
// Full table versus lazy columns for blocks on the plan's pattern.
//
// The table costs t_table once per pattern (Alg. 2) and makes each block
// cheaper by (t_lazy - t_full) per block.  With the table not built, a batch
// of n pattern blocks under SE_GRAM_AUTO runs lazily while the lazy blocks
// served so far plus this batch have cost less extra than one table build,
// and builds the table otherwise (the ski-rental rule: never more than twice
// the cost of the best choice made in hindsight).  The three costs come from
// measurement: se_plan_autotune times them on a probe batch, and every batch
// timed with events updates them.
bool choose_lazy_for_pattern(se_plan_s *pl, int n)
{
    std::lock_guard<std::mutex> lk(pl->cmu);
    if (pl->tables_valid || pl->desc.gram != SE_GRAM_AUTO || pl->certified || pl->cplx) return false;
    if (!(pl->t_table_ms > 0.0 && pl->t_full_blk_ms > 0.0 && pl->t_lazy_blk_ms > 0.0)) return false;
    const double extra = pl->t_lazy_blk_ms - pl->t_full_blk_ms;
    if (extra <= 0.0) return true;
    if (pl->lazy_regret_ms + n * extra < pl->t_table_ms) {
        pl->lazy_regret_ms += n * extra;
        return true;
    }
    pl->lazy_regret_ms = 0.0;
    return false;
}

void record_cost(se_plan_s *pl, int which, double ms, int n)
{
    if (!(ms > 0.0)) return;
    std::lock_guard<std::mutex> lk(pl->cmu);
    auto ema = [](double &v, double x) { v = v > 0.0 ? 0.75 * v + 0.25 * x : x; };
    if (which == 0) ema(pl->t_table_ms, ms);
    else if (which == 1 && n > 0) ema(pl->t_full_blk_ms, ms / n);
    else if (which == 2 && n > 0) ema(pl->t_lazy_blk_ms, ms / n);
}

cudaEvent_t probe_begin(se_ctx_s *ctx, cudaStream_t st)
{
    if (capturing(st)) return nullptr;
    cudaEvent_t e = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->cpmu);
        if (!ctx->probe_pool.empty()) {
            e = ctx->probe_pool.back();
            ctx->probe_pool.pop_back();
        }
    }
    if (!e && cudaEventCreate(&e) != cudaSuccess) return nullptr;
    if (cudaEventRecord(e, st) != cudaSuccess) {
        cudaEventDestroy(e);
        return nullptr;
    }
    return e;
}

void probe_end(se_ctx_s *ctx, se_plan_s *pl, int which, int n, cudaEvent_t a, cudaStream_t st)
{
    if (!a) return;
    cudaEvent_t b = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->cpmu);
        if (!ctx->probe_pool.empty()) {
            b = ctx->probe_pool.back();
            ctx->probe_pool.pop_back();
        }
    }
    if ((!b && cudaEventCreate(&b) != cudaSuccess) || cudaEventRecord(b, st) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(ctx->cpmu);
        ctx->probe_pool.push_back(a);
        if (b) ctx->probe_pool.push_back(b);
        return;
    }
    std::lock_guard<std::mutex> lk(ctx->cpmu);
    ctx->probes.push_back(CostProbe{pl, which, n, a, b});
}

void probes_poll(se_ctx_s *ctx, bool wait, const se_plan_s *only)
{
    std::vector<CostProbe> done;
    {
        std::lock_guard<std::mutex> lk(ctx->cpmu);
        for (auto it = ctx->probes.begin(); it != ctx->probes.end();) {
            if (only && it->plan != only) { ++it; continue; }
            const bool ready = wait ? cudaEventSynchronize(it->b) == cudaSuccess
                                    : cudaEventQuery(it->b) == cudaSuccess;
            if (!ready && !wait) { ++it; continue; }
            done.push_back(*it);
            it = ctx->probes.erase(it);
        }
    }
    cudaGetLastError();   // a not-ready query is not an error
    for (auto &p : done) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) record_cost(p.plan, p.which, ms, p.n);
        std::lock_guard<std::mutex> lk(ctx->cpmu);
        ctx->probe_pool.push_back(p.a);
        ctx->probe_pool.push_back(p.b);
    }
}

// ---------------------------------------------------------------------------
// CUDA graphs of the lazy round loop: the I_max - 1 rounds of a wave (round
// kernel and column computation per iteration, all arguments fixed by the
// plan, the wave size and the workspace addresses) are captured once and
// replayed.  A small cache per context; the oldest graph is dropped first.
cudaError_t graph_run(se_ctx_s *ctx, const GraphKey &key, cudaStream_t st,
                      const std::function<cudaError_t(cudaStream_t)> &record)
{
    if (!ctx->graphs_enabled || capturing(st)) return record(st);
    {
        std::lock_guard<std::mutex> lk(ctx->gmu);
        for (auto &g : ctx->graphs)
            if (g.key == key) {
                g.last = ++ctx->graph_clock;
                ctx->graph_replays++;
                return cudaGraphLaunch(g.exec, st);
            }
        // A shape seen for the first time runs directly; only a shape that comes
        // back is captured.  Serving batches rarely repeat their shape, and a
        // capture that is never replayed costs more than the launches it holds.
        auto seen = std::find(ctx->graph_seen.begin(), ctx->graph_seen.end(), key);
        if (seen == ctx->graph_seen.end()) {
            if (ctx->graph_seen.size() >= 4 * se_ctx_s::kGraphCache) ctx->graph_seen.erase(ctx->graph_seen.begin());
            ctx->graph_seen.push_back(key);
            return record(st);
        }
        ctx->graph_seen.erase(seen);
    }
    // capture on a private stream ordered after the caller's work
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        cudaError_t er = record(cs);
        e = cudaStreamEndCapture(cs, &graph);
        if (er != cudaSuccess) e = er;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        if (exec) cudaGraphExecDestroy(exec);
        cudaGetLastError();
        return record(st);   // capture failed: launch the rounds directly
    }
    e = cudaGraphLaunch(exec, st);
    std::lock_guard<std::mutex> lk(ctx->gmu);
    if (ctx->graphs.size() >= se_ctx_s::kGraphCache) {
        auto old = std::min_element(ctx->graphs.begin(), ctx->graphs.end(),
                                    [](const CachedGraph &a, const CachedGraph &b) { return a.last < b.last; });
        cudaGraphExecDestroy(old->exec);
        ctx->graphs.erase(old);
    }
    ctx->graphs.push_back(CachedGraph{key, exec, ++ctx->graph_clock});
    ctx->graph_builds++;
    return e;
}

void graphs_clear(se_ctx_s *ctx)
{
    std::lock_guard<std::mutex> lk(ctx->gmu);
    for (auto &g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    ctx->graph_seen.clear();
}

void graphs_drop_plan(se_ctx_s *ctx, const se_plan_s *pl)
{
    std::lock_guard<std::mutex> lk(ctx->gmu);
    for (auto it = ctx->graphs.begin(); it != ctx->graphs.end();) {
        if (it->key.plan == pl) {
            cudaGraphExecDestroy(it->exec);
            it = ctx->graphs.erase(it);
        } else {
            ++it;
        }
    }
}

}  // namespace se
