// se_serve.cpp -- the serving loop behind se_submit / se_poll / se_cancel.
//
// Continuous batching over "lanes": each lane owns a CUDA stream, a batch
// workspace and device/pinned I/O buffers.  A scheduler thread admits queued
// requests into any free lane as soon as one is free (and the context's HBM
// budget allows the lane's buffers), so requests that arrive while other
// batches run start immediately on another stream and their work overlaps on
// the device.  A batch holds requests of one plan (any mix of per-request
// iteration counts).  Completion is detected with events; results are
// copied into the caller's buffers by the scheduler, and se_poll waits on a
// condition variable.  Requests with their own support mask go through the
// per-block-mask (lazy column) path inside the same lane.  Every result is
// computed by the same kernels with the same per-block arithmetic as
// se_extrapolate_batch, so it does not depend on which other requests shared
// its batch.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "se_host.h"

using namespace se;

namespace {

constexpr int kLanes = 4;
constexpr int kMaxBatch = 2048;

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

namespace {

// Byte offsets of one lane batch inside its I/O buffer.
struct IoLayout {
    size_t samples, masks, out, idx, coef, total;
};

// samples | masks (requests with their own support) | out | logs; the H2D copy
// covers [samples, out), the D2H copy [out, total).
IoLayout io_layout(int n, int MN, int I)
{
    auto r16 = [](size_t v) { return (v + 15) / 16 * 16; };
    IoLayout L;
    L.samples = 0;
    L.masks = r16(sizeof(double) * MN * static_cast<size_t>(n));
    L.out = L.masks + r16(static_cast<size_t>(MN) * n);
    L.idx = L.out + r16(sizeof(double) * MN * static_cast<size_t>(n));
    L.coef = L.idx + r16(sizeof(int32_t) * I * static_cast<size_t>(n));
    L.total = L.coef + r16(sizeof(double) * I * static_cast<size_t>(n));
    return L;
}

void finish(se_ctx_s *ctx, ServeLane &lane, se_status st, const std::string &why)
{
    const int MN = lane.plan ? lane.plan->MN : 0;
    const IoLayout L = io_layout(static_cast<int>(lane.batch.size()), MN, lane.I_max);
    const double t = now_s();
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        for (size_t i = 0; i < lane.batch.size(); ++i) {
            ServeReq &r = *lane.batch[i];
            if (st == SE_OK) {
                std::memcpy(r.out, lane.h_io + L.out + sizeof(double) * MN * i, sizeof(double) * MN);
                if (r.sel_idx)
                    std::memcpy(r.sel_idx, lane.h_io + L.idx + sizeof(int32_t) * lane.I_max * i,
                                sizeof(int32_t) * r.iterations);
                if (r.sel_coef)
                    std::memcpy(r.sel_coef, lane.h_io + L.coef + sizeof(double) * lane.I_max * i,
                                sizeof(double) * r.iterations);
                r.state = 2;
            } else {
                r.state = 3;
                r.status = st;
            }
            r.t_done = t;
            (void)why;
        }
    }
    lane.batch.clear();
    lane.busy = false;
    ctx->scv.notify_all();
}

// Launch one batch on a free lane.  Returns false (requests put back) if the
// HBM budget cannot hold the lane's buffers right now.
bool launch(se_ctx_s *ctx, ServeLane &lane, std::vector<std::shared_ptr<ServeReq>> &&reqs,
            bool others_busy)
{
    se_plan_s *pl = reqs.front()->plan;
    const int n = static_cast<int>(reqs.size());
    int I_max = 0;
    for (auto &r : reqs) I_max = std::max(I_max, r->iterations);
    const int MN = pl->MN;
    const IoLayout L = io_layout(n, MN, I_max);

    se_status s = SE_OK;
    std::string why;
    if (lane.d_io.bytes < L.total) {
        cudaStreamSynchronize(lane.st);
        s = dev_alloc(ctx, lane.d_io, L.total);
    }
    if (s == SE_OK && lane.h_io_cap < L.total) {
        if (lane.h_io) cudaFreeHost(lane.h_io);
        lane.h_io = nullptr;
        lane.h_io_cap = 0;
        if (cudaMallocHost(&lane.h_io, L.total) != cudaSuccess) s = SE_ERR_NOMEM;
        else lane.h_io_cap = L.total;
    }
    if (s == SE_ERR_NOMEM && others_busy) {
        std::lock_guard<std::mutex> lk(ctx->smu);
        for (auto it = reqs.rbegin(); it != reqs.rend(); ++it) {
            (*it)->state = 0;
            ctx->queue.push_front(*it);
        }
        return false;
    }
    lane.plan = pl;
    lane.I_max = I_max;
    lane.batch = std::move(reqs);
    lane.busy = true;
    if (s != SE_OK) {
        finish(ctx, lane, s, "serving buffers do not fit the HBM budget");
        return true;
    }
    char *d = static_cast<char *>(lane.d_io.ptr);
    // requests on the plan's pattern use the full table, requests with their
    // own mask (or every request when the plan forces LAZY) lazy columns
    std::vector<BlockDesc> full, lazy;
    int I_full = 0, I_lazy = 0;
    for (int i = 0; i < n; ++i) {
        ServeReq &r = *lane.batch[i];
        std::memcpy(lane.h_io + L.samples + sizeof(double) * MN * i, r.samples.data(),
                    sizeof(double) * MN);
        BlockDesc x;
        x.samples = reinterpret_cast<const double *>(d + L.samples) + static_cast<size_t>(MN) * i;
        x.support = nullptr;
        if (!r.support.empty()) {
            std::memcpy(lane.h_io + L.masks + static_cast<size_t>(MN) * i, r.support.data(), MN);
            x.support = reinterpret_cast<const uint8_t *>(d + L.masks) + static_cast<size_t>(MN) * i;
        } else if (pl->desc.gram == SE_GRAM_LAZY) {
            x.support = pl->d_pattern.as<uint8_t>();
        }
        x.out = reinterpret_cast<double *>(d + L.out) + static_cast<size_t>(MN) * i;
        x.sel_idx = reinterpret_cast<int32_t *>(d + L.idx) + static_cast<size_t>(I_max) * i;
        x.sel_coef = reinterpret_cast<double *>(d + L.coef) + static_cast<size_t>(I_max) * i;
        x.iterations = r.iterations;
        x.pad_ = 0;
        if (x.support) {
            lazy.push_back(x);
            I_lazy = std::max(I_lazy, x.iterations);
        } else {
            full.push_back(x);
            I_full = std::max(I_full, x.iterations);
        }
    }
    probes_poll(ctx, false);
    route_pattern_blocks(pl, full, lazy, &I_full, &I_lazy);
    cudaError_t e = cudaMemcpyAsync(d + L.samples, lane.h_io + L.samples, L.out - L.samples,
                                    cudaMemcpyHostToDevice, lane.st);
    if (e == cudaSuccess) {
        if (!full.empty())
            s = run_batch(ctx, pl, lane.ws, static_cast<int>(full.size()), full.data(), I_full, lane.st);
        if (s == SE_OK && !lazy.empty())
            s = run_lazy(ctx, pl, lane.ws, static_cast<int>(lazy.size()), lazy.data(), I_lazy, lane.st);
        if (s == SE_OK) {
            e = cudaMemcpyAsync(lane.h_io + L.out, d + L.out, L.total - L.out, cudaMemcpyDeviceToHost,
                                lane.st);
            if (e == cudaSuccess) e = cudaEventRecord(lane.done, lane.st);
        }
    }
    if (e != cudaSuccess) s = SE_ERR_CUDA;
    if (s != SE_OK) finish(ctx, lane, s, "batch launch failed");
    else ctx->slices++;
    return true;
}

void serve_loop(se_ctx_s *ctx)
{
    cudaSetDevice(ctx->device);
    for (;;) {
        bool any_busy = false;
        for (auto &lp : ctx->lanes) {
            ServeLane &lane = *lp;
            if (!lane.busy) continue;
            cudaError_t q = cudaEventQuery(lane.done);
            if (q == cudaSuccess) finish(ctx, lane, SE_OK, "");
            else if (q != cudaErrorNotReady) finish(ctx, lane, SE_ERR_CUDA, cudaGetErrorString(q));
            else any_busy = true;
        }
        ServeLane *free_lane = nullptr;
        for (auto &lp : ctx->lanes)
            if (!lp->busy) { free_lane = lp.get(); break; }

        std::vector<std::shared_ptr<ServeReq>> take;
        {
            std::unique_lock<std::mutex> lk(ctx->smu);
            if (ctx->stop) {
                for (auto &r : ctx->queue) { r->state = 4; r->status = SE_ERR_CANCELLED; }
                ctx->queue.clear();
                if (!any_busy) break;
            } else if (free_lane && !ctx->queue.empty()) {
                se_plan_s *pl = ctx->queue.front()->plan;
                // a slice fits one lazy wave within a lane's share of the budget: a larger
                // one would run as several waves in a row, each repeating every round, and
                // the requests queued meanwhile would form ever larger slices
                int cap = kMaxBatch;
                if (ctx->budget) {
                    const size_t per = lazy_bytes_per_block(pl, std::max(1, pl->desc.iterations));
                    cap = static_cast<int>(std::max<size_t>(1, std::min<size_t>(kMaxBatch, ctx->budget / kLanes / per)));
                }
                for (auto it = ctx->queue.begin();
                     it != ctx->queue.end() && static_cast<int>(take.size()) < cap;) {
                    if ((*it)->plan == pl) {
                        (*it)->state = 1;
                        take.push_back(*it);
                        it = ctx->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
            } else if (!any_busy) {
                ctx->scv.wait_for(lk, std::chrono::milliseconds(50));
                continue;
            }
        }
        if (!take.empty()) {
            launch(ctx, *free_lane, std::move(take), any_busy);
            continue;
        }
        if (any_busy) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    ctx->scv.notify_all();
}

se_status ensure_server(se_ctx_s *ctx)
{
    std::lock_guard<std::mutex> lk(ctx->smu);
    if (ctx->server_started) return SE_OK;
    for (int i = 0; i < kLanes; ++i) {
        auto lane = std::make_unique<ServeLane>();
        cudaError_t e = cudaStreamCreateWithFlags(&lane->st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&lane->done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = lane->ws.init();
        if (e != cudaSuccess) return set_error(SE_ERR_CUDA, std::string("serving lane: ") + cudaGetErrorString(e));
        ctx->lanes.push_back(std::move(lane));
    }
    ctx->server = std::thread(serve_loop, ctx);
    ctx->server_started = true;
    return SE_OK;
}

}  // namespace

void se::serve_shutdown(se_ctx_s *ctx)
{
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        ctx->stop = true;
    }
    ctx->scv.notify_all();
    if (ctx->server.joinable()) ctx->server.join();
    ctx->lanes.clear();
}

extern "C" {

se_status se_submit(se_ctx_t *ctx, const se_plan_t *plan, const se_request *req, uint64_t *ticket)
{
    if (!ctx || !plan || !req || !ticket) return set_error(SE_ERR_INVALID, "NULL argument");
    if (plan->ctx != ctx) return set_error(SE_ERR_INVALID, "plan belongs to another context");
    if (!req->samples || !req->out) return set_error(SE_ERR_INVALID, "NULL samples or out");
    if (req->iterations < 0) return set_error(SE_ERR_INVALID, "iterations < 0");
    if (plan->cplx) return set_error(SE_ERR_INVALID, "complex plans: device entry points only");
    if (req->support && plan->desc.gram == SE_GRAM_FULL)
        return set_error(SE_ERR_INVALID, "per-request support masks need the lazy table path (plan gram is FULL)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return set_error(SE_ERR_CUDA, "cudaSetDevice failed");
    se_status s = ensure_server(ctx);
    if (s != SE_OK) return s;
    auto r = std::make_shared<ServeReq>();
    r->plan = const_cast<se_plan_s *>(plan);
    r->samples.assign(req->samples, req->samples + plan->MN);
    if (req->support) r->support.assign(req->support, req->support + plan->MN);
    r->out = req->out;
    r->sel_idx = req->sel_idx;
    r->sel_coef = req->sel_coef;
    r->iterations = req->iterations ? req->iterations : plan->desc.iterations;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(ctx->smu);
        if (ctx->stop) return set_error(SE_ERR_CANCELLED, "context is shutting down");
        r->ticket = ctx->next_ticket++;
        ctx->tickets[r->ticket] = r;
        ctx->queue.push_back(r);
        *ticket = r->ticket;
    }
    ctx->scv.notify_all();
    return SE_OK;
}

se_status se_poll(se_ctx_t *ctx, uint64_t ticket, int64_t timeout_us, double *latency_s)
{
    if (!ctx) return set_error(SE_ERR_INVALID, "NULL context");
    std::unique_lock<std::mutex> lk(ctx->smu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return set_error(SE_ERR_UNKNOWN_TICKET, "no such ticket");
    std::shared_ptr<ServeReq> r = it->second;
    auto finished = [&] { return r->state >= 2; };
    if (!finished() && timeout_us != 0) {
        if (timeout_us < 0) ctx->scv.wait(lk, finished);
        else ctx->scv.wait_for(lk, std::chrono::microseconds(timeout_us), finished);
    }
    if (!finished()) return SE_PENDING;
    ctx->tickets.erase(ticket);
    if (latency_s) *latency_s = r->t_done - r->t_submit;
    if (r->state == 2) return SE_OK;
    return set_error(r->status, r->state == 4 ? "request cancelled" : "request failed");
}

se_status se_cancel(se_ctx_t *ctx, uint64_t ticket)
{
    if (!ctx) return set_error(SE_ERR_INVALID, "NULL context");
    std::lock_guard<std::mutex> lk(ctx->smu);
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return set_error(SE_ERR_UNKNOWN_TICKET, "no such ticket");
    std::shared_ptr<ServeReq> r = it->second;
    if (r->state == 0) {
        ctx->queue.erase(std::remove(ctx->queue.begin(), ctx->queue.end(), r), ctx->queue.end());
        r->state = 4;
        r->status = SE_ERR_CANCELLED;
        r->t_done = now_s();
        ctx->scv.notify_all();
        return SE_OK;
    }
    if (r->state == 1) return SE_PENDING;
    return set_error(SE_ERR_INVALID, "request already finished");
}

}  // extern "C"
