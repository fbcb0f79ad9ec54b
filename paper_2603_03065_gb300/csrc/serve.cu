// Serving loop (continuous batching) for audit-commit requests.
//
// A scheduler thread admits queued requests while their footprint fits the
// HBM budget minus what is resident.  Requests are batched by size class
// (LDE elements): each scheduler pass takes the class whose oldest request
// arrived first, fuses that class's queued requests (in arrival order) into
// one batched launch (one launch per stage over all of them) and runs it on
// a free slot, on the slot's stream for that class.  Small requests thus
// never wait for the stages of large ones admitted beside them, and their
// streams have the higher priority.  Up to max_inflight batches overlap on
// the device; a class takes the last free slot only when no other class is
// waiting.  Finished requests keep their LDE and tree resident until
// v3c_release, for the later FRI and opening phases.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <stdexcept>

#include "serve.h"

using namespace v3c;
using namespace v3c::detail;
using serve::Request;
using serve::Server;
using serve::Slot;

int v3c::serve::size_class(const v3c_commit_desc& d)
{
    const u64 e = (u64)d.c << (d.log_n + d.rate_bits);
    return e <= (16ull << 20) ? 0 : e <= (128ull << 20) ? 1 : 2;
}

namespace {

size_t lde_scratch_words_s(u32 c, u32 log_n, u32 r)
{
    u32 l1, l2;
    plan_split(log_n, r, l1, l2);
    if (!l1) return 0;
    return (size_t)c * (((size_t)1 << log_n) + ((size_t)1 << (log_n + r)));
}

void fail_all_pending(Server* S, v3c_status st)
{
    for (auto& kv : S->reqs) {
        Request& r = kv.second;
        if (r.state == V3C_REQ_QUEUED || r.state == V3C_REQ_ADMITTED) {
            r.state = V3C_REQ_FAILED;
            r.status = st;
            r.times.t_done = now_s();
        }
    }
    S->queue.clear();
}

// Marks finished batches DONE.  Caller holds S->mu.
void reap(Server* S, bool wait)
{
    for (auto& sl : S->slots) {
        if (!sl.busy) continue;
        cudaError_t e = wait ? cudaEventSynchronize(sl.done) : cudaEventQuery(sl.done);
        if (e == cudaErrorNotReady) continue;
        double t = now_s();
        for (u64 tk : sl.tickets) {
            auto it = S->reqs.find(tk);
            if (it == S->reqs.end()) continue;
            Request& r = it->second;
            r.state = e == cudaSuccess ? V3C_REQ_DONE : V3C_REQ_FAILED;
            r.status = e == cudaSuccess ? V3C_OK : V3C_ECUDA;
            r.times.t_done = t;
        }
        sl.tickets.clear();
        sl.busy = false;
    }
}

// Stages the batch's inputs and launches it on `slot`, on the slot's stream
// of size class k.  Caller holds S->mu.
void launch_batch_on(Server* S, Slot* slot, int k, const std::vector<u64>& batch, size_t scratch, size_t staged,
                     size_t copied)
{
    double t = now_s();
    // Slot buffers grow on demand while the slot is idle.
    size_t need = scratch + staged;
    v3c_status st = V3C_OK;
    if (need > slot->arena_words) {
        if (slot->arena) cudaFree(slot->arena);
        slot->arena = nullptr;
        slot->arena_words = 0;
        if (cudaMalloc(&slot->arena, need * 8) != cudaSuccess) {
            cudaGetLastError();
            st = V3C_ENOMEM;
        } else {
            slot->arena_words = need;
        }
    }
    if (!st && copied > slot->pinned_words) {
        if (slot->pinned) cudaFreeHost(slot->pinned);
        slot->pinned = nullptr;
        slot->pinned_words = 0;
        if (cudaMallocHost(&slot->pinned, copied * 8) != cudaSuccess) {
            cudaGetLastError();
            st = V3C_ENOMEM;
        } else {
            slot->pinned_words = copied;
        }
    }
    std::vector<v3c_commit_desc> descs;
    size_t poff = 0;
    for (u64 tk : batch) {
        Request& r = S->reqs[tk];
        r.state = V3C_REQ_ADMITTED;
        r.times.t_admit = t;
        v3c_commit_desc d = r.desc;
        if (!st && d.on_device == V3C_INPUT_HOST_COPY) {
            // Copied at submit: stage through the slot's pinned buffer.
            size_t w = (size_t)d.c << d.log_n;
            memcpy(slot->pinned + poff, r.host_copy.data(), w * 8);
            d.cols = slot->pinned + poff;
            poff += w;
        }
        if (d.on_device == V3C_INPUT_HOST_BORROW) d.on_device = V3C_INPUT_HOST_COPY;  // caller's pinned memory
        descs.push_back(d);
    }
    cudaStream_t stream = slot->streams[k];
    if (!st) {
        std::vector<u64> ids(batch.size());
        std::lock_guard<std::mutex> g(ctx_mutex(S->ctx));
        st = commit_locked(S->ctx, descs.data(), (u32)descs.size(), ids.data(), stream, slot->arena,
                           slot->arena_words, batch.data(), /*allow_graph=*/false);  // mixes rarely repeat
        if (!st && cudaEventRecord(slot->done, stream) != cudaSuccess) st = V3C_ECUDA;
    }
    double t2 = now_s();
    for (u64 tk : batch) {
        Request& r = S->reqs[tk];
        if (st) {
            r.state = V3C_REQ_FAILED;
            r.status = st;
            r.times.t_done = t2;
        } else {
            r.state = V3C_REQ_RUNNING;
            r.times.t_start = t2;
            r.host_copy.clear();
            r.host_copy.shrink_to_fit();
        }
    }
    if (!st) {
        // Footprint is counted as resident by the context from here on.
        slot->busy = true;
        slot->stream = stream;
        slot->cls = k;
        slot->tickets = batch;
    }
}

// A request older than this that does not fit the budget stops the
// admission of newer requests of the other classes, so that a stream of
// small requests cannot keep a large one waiting for memory forever.
constexpr double kStarveS = 0.25;

// One scheduler pass: admit one batch into a free slot.  Returns true if a
// batch was launched.  Caller holds S->mu.
bool admit_and_launch(Server* S)
{
    int nfree = 0;
    Slot* slot = nullptr;
    for (auto& sl : S->slots)
        if (!sl.busy) {
            nfree++;
            if (!slot) slot = &sl;
        }
    if (!slot || S->queue.empty()) return false;
    const v3c_config& cfg = ctx_config(S->ctx);
    const u64 budget = cfg.hbm_budget_bytes;
    const u64 resident = ctx_resident(S->ctx);
    // Classes in the order of their oldest queued request.
    int order[serve::kSizeClasses], norder = 0;
    bool seen[serve::kSizeClasses] = {false, false, false};
    for (u64 tk : S->queue) {
        const int k = serve::size_class(S->reqs[tk].desc);
        if (!seen[k]) {
            seen[k] = true;
            order[norder++] = k;
            if (norder == serve::kSizeClasses) break;
        }
    }
    const Request& head = S->reqs[S->queue.front()];
    const int head_cls = serve::size_class(head.desc);
    const bool head_starved = resident + head.footprint > budget &&
                              now_s() - head.times.t_submit > kStarveS;
    const u32 max_batch = S->cfg.max_batch ? S->cfg.max_batch : 32;
    const u64 slot_cap = S->cfg.slot_scratch_bytes ? S->cfg.slot_scratch_bytes : (16ull << 30);
    const u64 elem_cap = S->cfg.batch_elems ? S->cfg.batch_elems : (1ull << 28);
    for (int oi = 0; oi < norder; oi++) {
        const int k = order[oi];
        if (head_starved && k != head_cls) continue;
        // The last free slot goes to the class that has waited longest.
        if (nfree == 1 && oi > 0) continue;
        std::vector<u64> batch;
        size_t scratch = 0, staged = 0, copied = 0;
        u64 reserve = 0, elems = 0;
        for (u64 tk : S->queue) {
            if (batch.size() >= max_batch) break;
            Request& r = S->reqs[tk];
            if (serve::size_class(r.desc) != k) continue;
            if (resident + reserve + r.footprint > budget) break;  // FIFO within the class
            size_t sw = lde_scratch_words_s(r.desc.c, r.desc.log_n, r.desc.rate_bits);
            size_t iw = r.desc.on_device == V3C_INPUT_DEVICE ? 0 : (size_t)r.desc.c << r.desc.log_n;
            // A pass takes at least one request; more only while its scratch
            // and staged inputs stay within the slot cap.
            if (!batch.empty() && (scratch + staged + sw + iw) * 8 > slot_cap) break;
            const u64 re = (u64)r.desc.c << (r.desc.log_n + r.desc.rate_bits);
            if (!batch.empty() && elems + re > elem_cap) break;  // the batch's work stays bounded
            elems += re;
            reserve += r.footprint;
            scratch += sw;
            staged += iw;
            if (r.desc.on_device == V3C_INPUT_HOST_COPY) copied += iw;
            batch.push_back(tk);
        }
        if (batch.empty()) continue;
        {   // take the batch out of the queue, keeping the rest in order
            std::deque<u64> rest;
            size_t bi = 0;
            for (u64 tk : S->queue) {
                if (bi < batch.size() && tk == batch[bi]) bi++;
                else rest.push_back(tk);
            }
            S->queue.swap(rest);
        }
        launch_batch_on(S, slot, k, batch, scratch + arena_padding((u32)batch.size()), staged, copied);
        return true;
    }
    return false;
}

void run(Server* S)
{
    cudaSetDevice(ctx_device(S->ctx));
    std::unique_lock<std::mutex> lk(S->mu);
    try {
        while (!S->stop) {
            if (S->inject_after >= 0 && S->inject_after-- == 0) throw std::runtime_error("injected scheduler failure");
            reap(S, false);
            bool launched = admit_and_launch(S);
            bool busy = false;
            for (auto& sl : S->slots) busy |= sl.busy;
            if (launched) continue;
            if (busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                S->cv.wait_for(lk, std::chrono::milliseconds(5));
            }
        }
        reap(S, true);
        fail_all_pending(S, V3C_ECANCELED);
    } catch (...) {
        log_msg(S->ctx, 0, "serving: the scheduler thread failed; queued requests are cancelled");
        // The scheduler cannot go on: batches already on the device finish
        // (their requests become DONE), everything still queued fails.
        S->crashed = true;
        try {
            reap(S, true);
        } catch (...) {
        }
        fail_all_pending(S, V3C_ECANCELED);
    }
}

}  // namespace

extern "C" {

v3c_status v3c_serve_start(v3c_ctx* ctx, const v3c_serve_cfg* cfg)
{
    if (!ctx) return V3C_EINVAL;
    Server*& S = ctx_server(ctx);
    if (S) return ctx_fail(ctx, V3C_EINVAL, "serving already started");
    v3c_status st = lock_and_select(ctx);
    if (st) return st;
    Server* srv = new Server();
    srv->ctx = ctx;
    if (cfg) srv->cfg = *cfg;
    if (!srv->cfg.queue_capacity) srv->cfg.queue_capacity = 4096;
    if (!srv->cfg.max_batch) srv->cfg.max_batch = 32;
    u32 inflight = srv->cfg.max_inflight ? srv->cfg.max_inflight : ctx_config(ctx).max_inflight;
    srv->slots.resize(std::max(inflight, 1u));
    // Stream priorities by size class: class 0 (small) the greatest, class 2
    // the least (numerically larger is lower priority).
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    const int prio[serve::kSizeClasses] = {greatest, (least + greatest) / 2, least};
    bool ok = true;
    for (auto& sl : srv->slots) {
        for (int k = 0; k < serve::kSizeClasses; k++)
            ok = ok && cudaStreamCreateWithPriority(&sl.streams[k], cudaStreamNonBlocking, prio[k]) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        for (auto& sl : srv->slots) {
            for (auto st : sl.streams)
                if (st) cudaStreamDestroy(st);
            if (sl.done) cudaEventDestroy(sl.done);
        }
        delete srv;
        return ctx_fail(ctx, V3C_ECUDA, "serve: stream creation failed");
    }
    S = srv;
    srv->th = std::thread(run, srv);
    log_msg(ctx, 1, "serving started: %u slots, batches up to %u requests", (unsigned)srv->slots.size(),
            (unsigned)srv->cfg.max_batch);
    return V3C_OK;
}

v3c_status v3c_serve_submit(v3c_ctx* ctx, const v3c_commit_desc* desc, uint64_t* ticket)
{
    if (!ctx || !desc || !ticket) return V3C_EINVAL;
    Server* S = ctx_server(ctx);
    if (!S) return V3C_ECANCELED;
    const v3c_commit_desc& d = *desc;
    if (!d.cols || d.c < 1 || d.log_n > V3C_MAX_LOG_N || d.rate_bits > V3C_MAX_RATE_BITS ||
        d.log_n + d.rate_bits > V3C_MAX_LOG_LDE || d.cap_height > d.log_n + d.rate_bits)
        return V3C_EINVAL;
    u64 fp = v3c_commit_footprint(d.c, d.log_n, d.rate_bits, d.cap_height);
    if (fp > ctx_config(ctx).hbm_budget_bytes) return V3C_ENOMEM;
    if (d.on_device != V3C_INPUT_HOST_COPY && d.on_device != V3C_INPUT_DEVICE && d.on_device != V3C_INPUT_HOST_BORROW)
        return V3C_EINVAL;
    if ((S->cfg.flags & V3C_FLAG_VALIDATE) && d.on_device != V3C_INPUT_DEVICE) {
        size_t w = (size_t)d.c << d.log_n;
        for (size_t i = 0; i < w; i++)
            if (d.cols[i] >= 0xFFFFFFFF00000001ull) return V3C_EINVAL;
    }
    Request r;
    r.desc = d;
    r.footprint = fp;
    if (d.on_device == V3C_INPUT_HOST_COPY) r.host_copy.assign(d.cols, d.cols + ((size_t)d.c << d.log_n));
    r.times.t_submit = now_s();
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop || S->crashed) return V3C_ECANCELED;
    if (S->queue.size() >= S->cfg.queue_capacity) return V3C_EAGAIN;
    {
        std::lock_guard<std::mutex> g2(ctx_mutex(ctx));
        r.ticket = ctx_next_id(ctx);
    }
    *ticket = r.ticket;
    u64 tk = r.ticket;
    S->reqs.emplace(tk, std::move(r));
    S->queue.push_back(tk);
    S->cv.notify_one();
    return V3C_OK;
}

v3c_status v3c_serve_poll(v3c_ctx* ctx, uint64_t ticket, v3c_req_state* state, uint64_t* h_cap,
                          v3c_req_times* times)
{
    if (!ctx) return V3C_EINVAL;
    Server* S = ctx_server(ctx);
    if (!S) return V3C_ECANCELED;
    v3c_req_state stt;
    v3c_status status;
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->reqs.find(ticket);
        if (it == S->reqs.end()) return V3C_ENOTFOUND;
        stt = it->second.state;
        status = it->second.status;
        if (state) *state = stt;
        if (times) *times = it->second.times;
    }
    if (stt == V3C_REQ_DONE) {
        if (h_cap) return v3c_commit_cap(ctx, ticket, h_cap);
        return V3C_OK;
    }
    if (stt == V3C_REQ_FAILED) return status;
    return V3C_EAGAIN;
}

v3c_status v3c_serve_inject_failure(v3c_ctx* ctx, uint32_t after_passes)
{
    if (!ctx) return V3C_EINVAL;
    Server* S = ctx_server(ctx);
    if (!S) return ctx_fail(ctx, V3C_EINVAL, "v3c_serve_inject_failure: not serving");
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop || S->crashed) return V3C_ECANCELED;
    S->inject_after = (long)after_passes;
    S->cv.notify_all();
    return V3C_OK;
}

v3c_status v3c_serve_stop(v3c_ctx* ctx)
{
    if (!ctx) return V3C_EINVAL;
    Server*& S = ctx_server(ctx);
    if (!S) return V3C_OK;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->th.joinable()) S->th.join();
    for (auto& sl : S->slots) {
        for (auto st : sl.streams)
            if (st) cudaStreamSynchronize(st);
        if (sl.arena) cudaFree(sl.arena);
        if (sl.pinned) cudaFreeHost(sl.pinned);
        if (sl.done) cudaEventDestroy(sl.done);
        for (auto st : sl.streams)
            if (st) cudaStreamDestroy(st);
    }
    delete S;
    S = nullptr;
    log_msg(ctx, 1, "serving stopped");
    return V3C_OK;
}

}  // extern "C"
