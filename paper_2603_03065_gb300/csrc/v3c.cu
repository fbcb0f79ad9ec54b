// C ABI of the commitment library: context, plan cache, scratch arena,
// resident commit objects and the batched (one launch per stage) commit.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/v3c.h"
#include "ctx.h"
#include "gl.cuh"
#include "internal.h"
#include "serve.h"

namespace v3c {

thread_local int g_dev_cache = -1;

int num_sms()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

int max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

Tiles default_tiles()
{
    Tiles t;
    t.a_threads = 256;
    t.a_cols = 8;
    t.b_threads = 256;
    t.c_threads = 256;
    t.c_q = 4;
    t.h_threads = 128;
    t.m_threads = 128;
    return t;
}

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace v3c

using namespace v3c;

static thread_local std::string g_err_copy;

// The callback and its level, read under the log lock; called without it.
static bool log_target(v3c_ctx* ctx, int level, v3c_log_fn* fn, void** user)
{
    std::lock_guard<std::mutex> g(ctx->log_mu);
    if (!ctx->log_fn || level > ctx->log_level) return false;
    *fn = ctx->log_fn;
    *user = ctx->log_user;
    return true;
}

v3c_status fail(v3c_ctx* ctx, v3c_status s, const char* fmt, ...)
{
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        {
            std::lock_guard<std::mutex> g(ctx->err_mu);
            ctx->err = buf;
        }
        v3c_log_fn fn;
        void* user;
        if (log_target(ctx, 0, &fn, &user)) fn(user, 0, buf);
    }
    return s;
}

void log_msg(v3c_ctx* ctx, int level, const char* fmt, ...)
{
    v3c_log_fn fn;
    void* user;
    if (!ctx || !log_target(ctx, level, &fn, &user)) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    fn(user, level, buf);
}

v3c_status v3c_set_log(v3c_ctx* ctx, v3c_log_fn fn, void* user, int max_level)
{
    if (!ctx) return V3C_EINVAL;
    std::lock_guard<std::mutex> g(ctx->log_mu);
    ctx->log_fn = fn;
    ctx->log_user = user;
    ctx->log_level = fn ? max_level : -1;
    return V3C_OK;
}


v3c_status use_device(v3c_ctx* ctx)
{
    if (g_dev_cache != ctx->device) {
        CK(cudaSetDevice(ctx->device));
        g_dev_cache = ctx->device;
    }
    return V3C_OK;
}

namespace v3c {
namespace detail {

cudaEvent_t pool_event(v3c_ctx* ctx)
{
    std::lock_guard<std::mutex> g(ctx->tmu);
    if (!ctx->ev_pool.empty()) {
        cudaEvent_t e = ctx->ev_pool.back();
        ctx->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Plan tables of a shape, built once and kept.  The coset is 7 * gshift *
// <w_N> and the scale table carries sfac (0 = n^-1, the LDE of columns).
// Caller holds ctx->mu.
v3c_status get_plan(v3c_ctx* ctx, u32 log_n, u32 r, cudaStream_t s, Plan* out, u64 gshift = 1, u64 sfac = 0)
{
    if (!sfac) sfac = gl::h_inv(((u64)1 << log_n) % gl::P);
    auto key = std::make_tuple(log_n, r, gshift, sfac);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) {
        *out = it->second.plan;
        return V3C_OK;
    }
    PlanEntry pe;
    size_t words = plan_table_words(log_n, r);
    CK(cudaMalloc(&pe.mem, words * sizeof(u64)));
    pe.plan.log_n = log_n;
    pe.plan.r = r;
    pe.plan.gshift = gshift;
    pe.plan.sfac = sfac;
    cudaError_t e = build_plan_tables(pe.plan, pe.mem, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(pe.mem);
        return fail(ctx, V3C_ECUDA, "plan tables: %s", cudaGetErrorString(e));
    }
    ctx->launches++;
    ctx->plans[key] = pe;
    *out = pe.plan;
    log_msg(ctx, 1, "plan tables for log_n %u, rate_bits %u: %zu bytes", log_n, r, words * sizeof(u64));
    return V3C_OK;
}

// Scratch words for the arena; orders `s` after the arena's previous user.
// Caller holds ctx->mu.
v3c_status arena_acquire(v3c_ctx* ctx, size_t words, cudaStream_t s, u64** out)
{
    Arena& a = ctx->arena;
    if (!a.ev) CK(cudaEventCreateWithFlags(&a.ev, cudaEventDisableTiming));
    if (words > a.words) {
        if (a.used) CK(cudaEventSynchronize(a.ev));
        if (a.mem) CK(cudaFree(a.mem));
        a.mem = nullptr;
        a.words = 0;
        size_t want = std::max(words, (size_t)1 << 16);
        cudaError_t e = cudaMalloc(&a.mem, want * sizeof(u64));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, V3C_ENOMEM, "scratch arena of %zu bytes: %s", want * 8, cudaGetErrorString(e));
        }
        a.words = want;
        log_msg(ctx, 1, "scratch arena grown to %zu bytes", want * sizeof(u64));
        a.used = false;
    }
    if (a.used && a.last != s) CK(cudaStreamWaitEvent(s, a.ev, 0));
    *out = a.mem;
    return V3C_OK;
}

v3c_status arena_release(v3c_ctx* ctx, cudaStream_t s)
{
    Arena& a = ctx->arena;
    CK(cudaEventRecord(a.ev, s));
    a.used = true;
    a.last = s;
    return V3C_OK;
}

// Copies `bytes` from host `src` to a device buffer that stays valid until
// the work enqueued on `s` after this call completes (call upload_done).
v3c_status upload(v3c_ctx* ctx, const void* src, size_t bytes, cudaStream_t s, void** d_out, u32* slot_out)
{
    if (ctx->ring.empty()) ctx->ring.resize(8);
    u32 k = ctx->ring_next++ % (u32)ctx->ring.size();
    UploadSlot& u = ctx->ring[k];
    if (!u.ev) CK(cudaEventCreateWithFlags(&u.ev, cudaEventDisableTiming));
    CK(cudaEventSynchronize(u.ev));
    if (bytes > u.cap) {
        if (u.h) CK(cudaFreeHost(u.h));
        if (u.d) CK(cudaFree(u.d));
        u.h = u.d = nullptr;
        size_t want = std::max(bytes, (size_t)1 << 16);
        CK(cudaMallocHost(&u.h, want));
        CK(cudaMalloc(&u.d, want));
        u.cap = want;
    }
    memcpy(u.h, src, bytes);
    CK(cudaMemcpyAsync(u.d, u.h, bytes, cudaMemcpyHostToDevice, s));
    *d_out = u.d;
    *slot_out = k;
    return V3C_OK;
}

v3c_status upload_done(v3c_ctx* ctx, u32 slot, cudaStream_t s)
{
    CK(cudaEventRecord(ctx->ring[slot].ev, s));
    return V3C_OK;
}

static void job_tiles(LdeJob& j) { lde_job_tiles(j); }

static size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Job table + stage item lists of a batch, packed into one upload.
// Layout: LdeJob[], TreeJob[], fa, fb, fc, fl, fm[...], 16-byte aligned parts.
static void build_blob(Batch& b, std::vector<char>& blob, std::vector<size_t>& off)
{
    std::vector<std::pair<const void*, size_t>> parts;
    parts.push_back({b.lde.data(), b.lde.size() * sizeof(LdeJob)});
    parts.push_back({b.tree.data(), b.tree.size() * sizeof(TreeJob)});
    parts.push_back({b.fa.data(), b.fa.size() * 4});
    parts.push_back({b.fb.data(), b.fb.size() * 4});
    parts.push_back({b.fc.data(), b.fc.size() * 4});
    parts.push_back({b.fl.data(), b.fl.size() * 4});
    for (auto& f : b.fm) parts.push_back({f.data(), f.size() * 4});
    for (auto& f : b.fac) parts.push_back({f.data(), f.size() * 4});
    for (auto& f : b.fbc) parts.push_back({f.data(), f.size() * 4});
    off.clear();
    size_t total = 0;
    for (auto& p : parts) {
        off.push_back(total);
        total = align16(total + p.second);
    }
    blob.assign(total, 0);
    for (size_t i = 0; i < parts.size(); i++)
        if (parts[i].second) memcpy(blob.data() + off[i], parts[i].first, parts[i].second);
}

// Enqueues every stage of a finalised batch whose blob sits at device
// address dc.  timed = record per-stage events (not inside graph capture).
static v3c_status enqueue_stages(v3c_ctx* ctx, const Batch& b, const Tiles& t, char* dc,
                                 const std::vector<size_t>& off, cudaStream_t s, bool timed)
{
    const LdeJob* dl = (const LdeJob*)(dc + off[0]);
    const TreeJob* dt = (const TreeJob*)(dc + off[1]);
    auto list = [&](size_t part, const std::vector<u32>& f, u32 njobs) {
        StageList l;
        l.first = (const u32*)(dc + off[part]);
        l.njobs = njobs;
        l.total = f.back();
        return l;
    };
    u32 nl = (u32)b.lde.size(), nt = (u32)b.tree.size();
    // The specialised stage kernels when every job of the launch has the
    // large commit's plan and the default tiles.
    auto all_spec = [&](u32 first, u32 count) {
        for (u32 k = first; k < first + count; k++)
            if (!lde_job_spec(b.lde[k])) return false;
        return count > 0;
    };
    auto stage = [&](int id, cudaError_t (*fn)(const Batch&, const Tiles&, StageList, const LdeJob*,
                                               const TreeJob*, size_t, cudaStream_t),
                     StageList l, size_t g) -> v3c_status {
        if (!l.total) return V3C_OK;
        StageTimer tm(ctx, timed ? id : -1, s, id);
        CK(fn(b, t, l, dl, dt, g, s));
        tm.done();
        ctx->launches++;
        return V3C_OK;
    };
    v3c_status st;
    if (nl && !b.chunks.empty()) {
        // Per column chunk: wait for its input copy, then stages A and B.
        const size_t base = 6 + b.fm.size();
        for (size_t g = 0; g < b.chunks.size(); g++) {
            CK(cudaStreamWaitEvent(s, b.chunk_ready[g], 0));
            const LdeJob* dj = dl + b.chunks[g].first;
            const u32 nj = b.chunks[g].second;
            StageList la = list(base + g, b.fac[g], nj), lb = list(base + b.chunks.size() + g, b.fbc[g], nj);
            if (la.total) {
                StageTimer tm(ctx, timed ? 0 : -1, s, 0);
                CK(launch_stage_a(dj, la, b.smem_a, t, 0, s));
                tm.done();
                ctx->launches++;
            }
            if (lb.total) {
                StageTimer tm(ctx, timed ? 1 : -1, s, 1);
                CK(launch_stage_b(dj, lb, b.smem_b, t, 0, s, all_spec(b.chunks[g].first, nj)));
                tm.done();
                ctx->launches++;
            }
        }
    } else if (nl) {
        st = stage(0, [](const Batch& b, const Tiles& t, StageList l, const LdeJob* dl, const TreeJob*, size_t,
                         cudaStream_t s) { return launch_stage_a(dl, l, b.smem_a, t, 0, s); },
                   list(2, b.fa, nl), 0);
        if (st) return st;
        const bool spec_b = all_spec(0, nl);
        st = stage(1, [](const Batch& b, const Tiles& t, StageList l, const LdeJob* dl, const TreeJob*, size_t g,
                         cudaStream_t s) { return launch_stage_b(dl, l, b.smem_b, t, 0, s, g != 0); },
                   list(3, b.fb, nl), spec_b ? 1 : 0);
        if (st) return st;
    }
    if (nl) {
        st = stage(2, [](const Batch& b, const Tiles& t, StageList l, const LdeJob* dl, const TreeJob*, size_t,
                         cudaStream_t s) { return launch_stage_c(dl, l, b.smem_c, t, 0, s); },
                   list(4, b.fc, nl), 0);
        if (st) return st;
    }
    if (nt && !b.leaves_ready) {
        st = stage(3, [](const Batch&, const Tiles& t, StageList l, const LdeJob*, const TreeJob* dt, size_t,
                         cudaStream_t s) { return launch_leaf_hash(dt, l, t, 0, s); },
                   list(5, b.fl, nt), 0);
        if (st) return st;
    }
    if (nt) {
        for (size_t g = 0; g < b.fm.size(); g++) {
            st = stage(4, [](const Batch& b, const Tiles& t, StageList l, const LdeJob*, const TreeJob* dt,
                             size_t g, cudaStream_t s) {
                if (b.mwarp[g]) return launch_merkle_warp(dt, l, b.mgroups[g].first, b.mgroups[g].second, 0, s);
                return launch_merkle(dt, l, b.mgroups[g].first, b.mgroups[g].second, t, 0, s);
            }, list(6 + g, b.fm[g], nt), g);
            if (st) return st;
        }
    }
    return V3C_OK;
}

// Direct path: upload the blob through the ring and launch every stage.
v3c_status launch_batch(v3c_ctx* ctx, Batch& b, cudaStream_t s)
{
    Tiles t = ctx->tiles;
    if (b.h_threads) t.h_threads = b.h_threads;
    b.finalize(t);
    std::vector<char> blob;
    std::vector<size_t> off;
    build_blob(b, blob, off);
    void* d = nullptr;
    u32 slot = 0;
    v3c_status st = upload(ctx, blob.data(), blob.size(), s, &d, &slot);
    if (st) return st;
    st = enqueue_stages(ctx, b, t, (char*)d, off, s, true);
    if (st) return st;
    return upload_done(ctx, slot, s);
}

// Graph path: every distinct batch signature (shapes, tiles, launch
// configuration) is captured once as [job-table copy, stage launches] on a
// ring of kGraphRing instances, each with its own pinned host and device
// table.  A call rewrites the table of the next instance (after that
// instance's previous replay has finished) and replays the graph.
static std::string batch_signature(const Batch& b, const Tiles& t)
{
    std::string k;
    char buf[96];
    snprintf(buf, sizeof buf, "t%u.%u.%u.%u.%u.%d|", t.a_threads, t.b_threads, t.c_threads,
             b.h_threads ? b.h_threads : t.h_threads, t.m_threads, (int)b.leaves_ready);
    k += buf;
    for (auto& j : b.lde) {
        snprintf(buf, sizeof buf, "L%u.%u.%u.%u.%u.%u.%u.%u.%u.%u|", j.c, j.ld, j.plan.log_n, j.plan.r, j.vec_ok,
                 j.a_cols, j.c_q, j.c_qc, j.kcap, j.mode);
        k += buf;
    }
    for (auto& j : b.tree) {
        snprintf(buf, sizeof buf, "T%u.%u.%u.%u.%u|", j.ld, j.width, j.log_N, j.h, j.vec_ok);
        k += buf;
    }
    return k;
}

v3c_status launch_batch_graph(v3c_ctx* ctx, Batch& b, cudaStream_t s)
{
    Tiles t = ctx->tiles;
    if (b.h_threads) t.h_threads = b.h_threads;
    b.finalize(t);
    std::string key = batch_signature(b, t);
    // A signature is captured on its second appearance (one-off batch mixes
    // launch directly), and at most kMaxGraphSets signatures are kept.
    auto seen = ctx->graph_seen.find(key);
    bool repeat = seen != ctx->graph_seen.end();
    if (!repeat && ctx->graph_seen.size() < 4 * kMaxGraphSets) ctx->graph_seen.emplace(key, 1);
    if (!repeat || (!ctx->graphs.count(key) && ctx->graphs.size() >= kMaxGraphSets)) return launch_batch(ctx, b, s);
    std::vector<char> blob;
    std::vector<size_t> off;
    build_blob(b, blob, off);
    GraphSet& gs = ctx->graphs[key];
    if (gs.inst.empty()) gs.inst.resize(kGraphRing);
    GraphInst& gi = gs.inst[gs.next++ % kGraphRing];
    if (!gi.exec) {
        gi.bytes = blob.size();
        CK(cudaMallocHost(&gi.h_blob, gi.bytes));
        CK(cudaMalloc(&gi.d_blob, gi.bytes));
        CK(cudaEventCreateWithFlags(&gi.done, cudaEventDisableTiming));
        if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaStream_t cs = ctx->capture_stream;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        cudaError_t e = cudaMemcpyAsync(gi.d_blob, gi.h_blob, gi.bytes, cudaMemcpyHostToDevice, cs);
        u64 before = ctx->launches.load();
        v3c_status st = e == cudaSuccess ? enqueue_stages(ctx, b, t, (char*)gi.d_blob, off, cs, false) : V3C_ECUDA;
        ctx->launches = before;  // captured launches are counted when replayed
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (st || e != cudaSuccess || e2 != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            return st ? st : fail(ctx, V3C_ECUDA, "graph capture failed: %s", cudaGetErrorString(e ? e : e2));
        }
        size_t nnodes = 0;
        cudaGraphGetNodes(g, nullptr, &nnodes);
        gi.kernels = (u32)(nnodes ? nnodes - 1 : 0);
        e = cudaGraphInstantiate(&gi.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        log_msg(ctx, 2, "captured a CUDA graph of %u kernels for a batch of %zu commits", gi.kernels, b.lde.size());
    }
    if (blob.size() != gi.bytes) return fail(ctx, V3C_ECUDA, "graph table size mismatch");
    CK(cudaEventSynchronize(gi.done));  // the previous replay of this instance read h_blob/d_blob
    memcpy(gi.h_blob, blob.data(), gi.bytes);
    CK(cudaStreamWaitEvent(s, gi.done, 0));
    CK(cudaGraphLaunch(gi.exec, s));
    CK(cudaEventRecord(gi.done, s));
    ctx->launches += gi.kernels;
    ctx->graph_replays++;
    return V3C_OK;
}

static bool shape_ok(u32 c, u32 log_n, u32 r)
{
    return c >= 1 && log_n <= V3C_MAX_LOG_N && r <= V3C_MAX_RATE_BITS && log_n + r <= V3C_MAX_LOG_LDE;
}

constexpr size_t kArenaAlign = 32;  // words (256 bytes)
static size_t align_words(size_t w) { return (w + kArenaAlign - 1) & ~(kArenaAlign - 1); }

}  // namespace detail
}  // namespace v3c

// Alignment slack of a batch's arena: each desc takes at most two blocks
// per column chunk (staged input, scratch) plus two unchunked.
size_t arena_padding(v3c::u32 nb) { return (size_t)nb * (2 * kCopyChunks + 2) * v3c::detail::kArenaAlign; }

namespace v3c {
namespace detail {

static size_t lde_scratch_words(u32 c, u32 log_n, u32 r)
{
    u32 l1, l2;
    plan_split(log_n, r, l1, l2);
    if (!l1) return 0;
    return (size_t)c * (((size_t)1 << log_n) + ((size_t)1 << (log_n + r)));
}

static v3c_status make_lde_job(v3c_ctx* ctx, const u64* x, u32 c, u32 log_n, u32 r, u64* lde, u32 ld,
                               u64* scratch, cudaStream_t s, LdeJob* out)
{
    LdeJob j;
    memset(&j, 0, sizeof j);
    v3c_status st = get_plan(ctx, log_n, r, s, &j.plan);
    if (st) return st;
    j.x = x;
    j.c = c;
    j.ld = ld;
    j.wcols = ld;
    j.lde = lde;
    j.vec_ok = ((uintptr_t)lde % 16 == 0) && (ld % 2 == 0);
    if (j.plan.log_n1) {
        j.Y = scratch;
        j.Z = scratch + ((size_t)c << log_n);
    }
    job_tiles(j);
    auto it = ctx->tuned.find(std::make_pair(log_n, r));
    if (it != ctx->tuned.end()) lde_job_apply_tune(j, it->second);
    *out = j;
    return V3C_OK;
}

static TreeJob make_tree_job(const u64* rows, u32 ld, u32 width, u32 log_N, u32 h, u64* tree, u64* cap);

// Autotuner.  For one (log_n, rate_bits) shape it times candidate tile
// choices on a synthetic 32-column problem of that shape, once, and keeps
// the fastest.  The candidates are the in-register radix cap, the Z
// blocking / stage-C q values, the stage-A column tile, and the leaf-hash
// CTA size (hash-lane mapping: one state per thread, 64 or 128 threads per
// CTA).  Coordinate descent in that order, best of 2 runs per candidate
// after a warm-up.  Synchronous; caller holds ctx->mu.
static v3c_status autotune_shape(v3c_ctx* ctx, u32 log_n, u32 r)
{
    auto key = std::make_pair(log_n, r);
    if (ctx->tuned.count(key)) return V3C_OK;
    const u32 c = 32, ld = 32;
    const size_t n = (size_t)1 << log_n, N = n << r;
    const size_t sw = lde_scratch_words(c, log_n, r);
    cudaStream_t ts = nullptr;
    u64 *x = nullptr, *lde = nullptr, *scr = nullptr, *leaves = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    v3c_status st = V3C_OK;
    TuneEntry best{};
    auto cleanup = [&]() {
        if (ts) cudaStreamSynchronize(ts);
        cudaFree(x);
        cudaFree(lde);
        cudaFree(scr);
        cudaFree(leaves);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ts) cudaStreamDestroy(ts);
    };
    auto ck = [&](cudaError_t e) {
        if (e != cudaSuccess && !st) st = fail(ctx, V3C_ECUDA, "autotune: %s", cudaGetErrorString(e));
        return e == cudaSuccess;
    };
    if (!ck(cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking)) || !ck(cudaMalloc(&x, c * n * 8)) ||
        !ck(cudaMalloc(&lde, N * ld * 8)) || (sw && !ck(cudaMalloc(&scr, sw * 8))) ||
        !ck(cudaMalloc(&leaves, N * 32)) || !ck(cudaEventCreate(&e0)) || !ck(cudaEventCreate(&e1)) ||
        !ck(cudaMemsetAsync(x, 0x11, c * n * 8, ts))) {  // 0x1111... is a canonical field element
        cleanup();
        return st;
    }
    LdeJob base;
    memset(&base, 0, sizeof base);
    st = get_plan(ctx, log_n, r, ts, &base.plan);
    if (st) {
        cleanup();
        return st;
    }
    base.x = x;
    base.c = c;
    base.ld = ld;
    base.lde = lde;
    base.vec_ok = 1;
    if (base.plan.log_n1) {
        base.Y = scr;
        base.Z = scr + (size_t)c * n;
    }
    lde_job_tiles(base);
    const u32 saved_flags = ctx->cfg.flags;
    ctx->cfg.flags &= ~V3C_FLAG_TIMING;
    auto time_lde = [&](const TuneEntry& t, float* ms) -> bool {
        LdeJob j = base;
        if (!lde_job_apply_tune(j, t)) return false;
        float bestms = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            Batch b;
            b.lde.push_back(j);
            if (!ck(cudaEventRecord(e0, ts))) return false;
            if (launch_batch(ctx, b, ts)) return false;
            if (!ck(cudaEventRecord(e1, ts)) || !ck(cudaEventSynchronize(e1))) return false;
            float m = 0;
            cudaEventElapsedTime(&m, e0, e1);
            if (rep) bestms = std::min(bestms, m);
        }
        *ms = bestms;
        return true;
    };
    best = TuneEntry{base.a_cols, base.c_q, base.c_qc, base.kcap, ctx->tiles.h_threads};
    float best_ms = 1e30f;
    time_lde(best, &best_ms);
    auto consider = [&](TuneEntry t) {
        float m;
        if (!st && time_lde(t, &m) && m < best_ms) {
            best_ms = m;
            best = t;
        }
    };
    for (u32 k : {3u, 4u}) {
        TuneEntry t = best;
        t.kcap = k;
        consider(t);
    }
    const u32 qz[][2] = {{2, 2}, {4, 2}, {4, 4}, {8, 2}, {8, 4}, {8, 8}, {1, 1}};
    for (auto& q : qz) {
        TuneEntry t = best;
        t.c_q = q[0];
        t.c_qc = q[1];
        consider(t);
    }
    for (u32 a : {2u, 4u, 8u, 16u}) {
        TuneEntry t = best;
        t.a_cols = a;
        consider(t);
    }
    // Leaf hash CTA size on the trial LDE (cap = leaves, no tree levels).
    float leaf_best = 1e30f;
    for (u32 ht : {64u, 128u}) {
        if (st) break;
        float bestms = 1e30f;
        for (int rep = 0; rep < 3; rep++) {
            Batch b;
            b.h_threads = ht;
            b.tree.push_back(make_tree_job(lde, ld, c, log_n + r, log_n + r, nullptr, leaves));
            if (!ck(cudaEventRecord(e0, ts)) || launch_batch(ctx, b, ts) || !ck(cudaEventRecord(e1, ts)) ||
                !ck(cudaEventSynchronize(e1)))
                break;
            float m = 0;
            cudaEventElapsedTime(&m, e0, e1);
            if (rep) bestms = std::min(bestms, m);
        }
        if (bestms < leaf_best) {
            leaf_best = bestms;
            best.h_threads = ht;
        }
    }
    ctx->cfg.flags = saved_flags;
    cleanup();
    if (st) return st;
    ctx->tuned[key] = best;
    log_msg(ctx, 1, "autotuned log_n %u, rate_bits %u: stage A %u columns, stage C %u/%u q, radix cap 2^%u, hash %u threads",
            log_n, r, best.a_cols, best.c_q, best.c_qc, best.kcap, best.h_threads);
    return V3C_OK;
}

static TreeJob make_tree_job(const u64* rows, u32 ld, u32 width, u32 log_N, u32 h, u64* tree, u64* cap)
{
    TreeJob t;
    memset(&t, 0, sizeof t);
    t.rows = rows;
    t.ld = ld;
    t.width = width;
    t.log_N = log_N;
    t.h = h;
    t.tree = tree;
    t.cap = cap;
    t.vec_ok = ((uintptr_t)rows % 16 == 0) && (ld % 2 == 0);
    return t;
}

}  // namespace detail
}  // namespace v3c

using namespace v3c::detail;

// ---------------------------------------------------------------- ABI

extern "C" {

const char* v3c_strerror(v3c_status s)
{
    switch (s) {
    case V3C_OK: return "ok";
    case V3C_EINVAL: return "invalid argument";
    case V3C_ENOMEM: return "out of device memory or HBM budget";
    case V3C_ECUDA: return "CUDA runtime error";
    case V3C_EAGAIN: return "not ready / queue full";
    case V3C_ETIMEDOUT: return "timed out";
    case V3C_ENOTFOUND: return "unknown id";
    case V3C_ECANCELED: return "cancelled";
    }
    return "unknown status";
}

const char* v3c_last_error_detail(v3c_ctx* ctx)
{
    if (!ctx) return "";
    std::lock_guard<std::mutex> g(ctx->err_mu);
    g_err_copy = ctx->err;
    return g_err_copy.c_str();
}

v3c_status v3c_create(int device, const v3c_config* cfg, v3c_ctx** out)
{
    if (!out) return V3C_EINVAL;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return V3C_EINVAL;
    }
    v3c_ctx* ctx = new (std::nothrow) v3c_ctx();
    if (!ctx) return V3C_ENOMEM;
    ctx->device = device;
    if (cfg) ctx->cfg = *cfg;
    if (!ctx->cfg.max_inflight) ctx->cfg.max_inflight = 4;
    if (!ctx->cfg.timeout_ms) ctx->cfg.timeout_ms = 60000;
    ctx->tiles = default_tiles();
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return V3C_ECUDA;
    }
    g_dev_cache = device;
    if (!ctx->cfg.hbm_budget_bytes) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        ctx->cfg.hbm_budget_bytes = (uint64_t)(fr * 0.9);
    }
    // Resident objects come from the device's default stream-ordered pool.
    // Keep freed blocks in this process's pool instead of returning them to
    // the driver at every synchronisation, so a commit/release cycle reuses
    // the same memory.  The pool belongs to this process.
    cudaMemPool_t pool = nullptr;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
    if (cudaMalloc(&ctx->d_flag, 16) != cudaSuccess) {
        delete ctx;
        return V3C_ENOMEM;
    }
    *out = ctx;
    return V3C_OK;
}

v3c_status v3c_destroy(v3c_ctx* ctx)
{
    if (!ctx) return V3C_EINVAL;
    v3c_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    fri_free_all(ctx);
    snap_free_all(ctx);
    for (auto& kv : ctx->objects) {
        cudaFree(kv.second.lde);
        cudaFree(kv.second.tree);
        cudaFree(kv.second.cap);
        if (kv.second.done) cudaEventDestroy(kv.second.done);
    }
    for (auto& kv : ctx->plans) cudaFree(kv.second.mem);
    for (auto& u : ctx->ring) {
        if (u.h) cudaFreeHost(u.h);
        if (u.d) cudaFree(u.d);
        if (u.ev) cudaEventDestroy(u.ev);
    }
    for (auto& p : ctx->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    if (ctx->arena.mem) cudaFree(ctx->arena.mem);
    if (ctx->arena.ev) cudaEventDestroy(ctx->arena.ev);
    if (ctx->d_flag) cudaFree(ctx->d_flag);
    if (ctx->release_stream) cudaStreamDestroy(ctx->release_stream);
    if (ctx->readback_stream) cudaStreamDestroy(ctx->readback_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->copy_fork) cudaEventDestroy(ctx->copy_fork);
    for (auto e : ctx->copy_events) cudaEventDestroy(e);
    for (auto& kv : ctx->graphs)
        for (auto& gi : kv.second.inst) {
            if (gi.exec) cudaGraphExecDestroy(gi.exec);
            if (gi.h_blob) cudaFreeHost(gi.h_blob);
            if (gi.d_blob) cudaFree(gi.d_blob);
            if (gi.done) cudaEventDestroy(gi.done);
        }
    if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
    delete ctx;
    return V3C_OK;
}

v3c_status v3c_lde(v3c_ctx* ctx, const uint64_t* d_cols, uint32_t c, uint32_t log_n, uint32_t rate_bits,
                   uint64_t* d_lde, uint32_t ld, void* stream)
{
    NvtxScope range("v3c_lde");
    if (!ctx) return V3C_EINVAL;
    if (!d_cols || !d_lde) return fail(ctx, V3C_EINVAL, "v3c_lde: NULL pointer");
    if (!shape_ok(c, log_n, rate_bits) || ld < c)
        return fail(ctx, V3C_EINVAL, "v3c_lde: bad shape c=%u log_n=%u r=%u ld=%u", c, log_n, rate_bits, ld);
    v3c_status st = use_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    size_t words = lde_scratch_words(c, log_n, rate_bits);
    u64* scratch = nullptr;
    if (words) {
        st = arena_acquire(ctx, words, s, &scratch);
        if (st) return st;
    }
    Batch b;
    LdeJob j;
    st = make_lde_job(ctx, d_cols, c, log_n, rate_bits, d_lde, ld, scratch, s, &j);
    if (st) return st;
    b.lde.push_back(j);
    u32 done_cols = c + (c & 1);
    if (ld > done_cols) {
        size_t N = (size_t)1 << (log_n + rate_bits);
        CK(cudaMemset2DAsync(d_lde + done_cols, (size_t)ld * 8, 0, (size_t)(ld - done_cols) * 8, N, s));
    }
    st = launch_batch(ctx, b, s);
    if (st) return st;
    if (words) return arena_release(ctx, s);
    return V3C_OK;
}

v3c_status v3c_merkle(v3c_ctx* ctx, const uint64_t* d_rows, uint32_t ld, uint32_t width, uint32_t log_rows,
                      uint32_t cap_height, uint64_t* d_tree, uint64_t* d_cap, void* stream)
{
    NvtxScope range("v3c_merkle");
    if (!ctx) return V3C_EINVAL;
    if (!d_rows || !d_cap || (!d_tree && cap_height != log_rows))
        return fail(ctx, V3C_EINVAL, "v3c_merkle: NULL pointer");
    if (cap_height > log_rows || width > ld || width == 0 || log_rows > V3C_MAX_LOG_LDE)
        return fail(ctx, V3C_EINVAL, "v3c_merkle: bad shape width=%u ld=%u log_rows=%u h=%u", width, ld,
                    log_rows, cap_height);
    if ((uintptr_t)d_tree % 16 || (uintptr_t)d_cap % 16)
        return fail(ctx, V3C_EINVAL, "v3c_merkle: tree and cap must be 16-byte aligned");
    v3c_status st = use_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    Batch b;
    b.tree.push_back(make_tree_job(d_rows, ld, width, log_rows, cap_height, d_tree, d_cap));
    return launch_batch(ctx, b, s);
}

uint64_t v3c_commit_footprint(uint32_t c, uint32_t log_n, uint32_t rate_bits, uint32_t cap_height)
{
    u32 ld = c + (c & 1);
    uint64_t N = (uint64_t)1 << (log_n + rate_bits);
    uint64_t tree_words = cap_height <= log_n + rate_bits ? (2 * N - ((uint64_t)2 << cap_height)) * 4 : 0;
    return (N * ld + tree_words + ((uint64_t)4 << cap_height)) * 8;
}

}  // extern "C"

namespace v3c {
namespace detail {

// Allocates the resident objects for descs (all or nothing), stages host
// inputs in the arena, and launches the batch.  Caller holds ctx->mu and
// has selected the device.  Shared by v3c_commit and the serving loop.
v3c_status commit_locked(v3c_ctx* ctx, const v3c_commit_desc* descs, u32 nb, u64* ids, cudaStream_t s,
                         u64* arena_override, size_t arena_words, const u64* preassigned_ids, bool allow_graph)
{
    // Large host inputs on the direct commit path are copied in column chunks
    // on the context's copy stream into a buffer of their own (not the shared
    // arena), so the copies need not wait for earlier work on the stream and
    // overlap the previous commit's kernels; stages A and B of a chunk start
    // when its copy lands.
    const bool may_chunk = !arena_override && allow_graph && !(ctx->cfg.flags & V3C_FLAG_VALIDATE);
    auto chunked = [&](const v3c_commit_desc& d) {
        return may_chunk && d.on_device != V3C_INPUT_DEVICE && d.c >= 16 &&
               ((size_t)d.c << d.log_n) >= ((size_t)1 << 22);
    };
    size_t need = 0, scratch = 0, staged = 0;
    for (u32 i = 0; i < nb; i++) {
        const v3c_commit_desc& d = descs[i];
        if (!d.cols || !shape_ok(d.c, d.log_n, d.rate_bits) || d.cap_height > d.log_n + d.rate_bits)
            return fail(ctx, V3C_EINVAL, "v3c_commit: bad desc %u (c=%u log_n=%u r=%u h=%u)", i, d.c, d.log_n,
                        d.rate_bits, d.cap_height);
        need += v3c_commit_footprint(d.c, d.log_n, d.rate_bits, d.cap_height);
        scratch += lde_scratch_words(d.c, d.log_n, d.rate_bits);
        if (d.on_device != V3C_INPUT_DEVICE && !chunked(d)) staged += (size_t)d.c << d.log_n;
    }
    if (!arena_override && ctx->resident + need > ctx->cfg.hbm_budget_bytes)
        return fail(ctx, V3C_ENOMEM, "v3c_commit: %zu bytes requested, %zu resident, budget %llu", need,
                    ctx->resident, (unsigned long long)ctx->cfg.hbm_budget_bytes);
    u32 h_threads = 0, biggest = 0;
    if (ctx->cfg.autotune) {
        for (u32 i = 0; i < nb; i++) {
            v3c_status st = autotune_shape(ctx, descs[i].log_n, descs[i].rate_bits);
            if (st) return st;
            u32 logN = descs[i].log_n + descs[i].rate_bits;
            if (logN >= biggest) {
                biggest = logN;
                h_threads = ctx->tuned[std::make_pair(descs[i].log_n, descs[i].rate_bits)].h_threads;
            }
        }
    }
    u64* arena = nullptr;
    // Every staged input and scratch block starts on a 256-byte boundary
    // (kArenaAlign words), so the kernels' vector accesses stay aligned.
    size_t arena_need = scratch + staged + arena_padding(nb);
    v3c_status st;
    if (arena_need) {
        if (arena_override) {
            if (arena_need > arena_words) return fail(ctx, V3C_ENOMEM, "slot arena too small");
            arena = arena_override;
        } else {
            st = arena_acquire(ctx, arena_need, s, &arena);
            if (st) return st;
        }
    }
    std::vector<Object> objs(nb);
    auto rollback = [&](u32 upto) {
        for (u32 k = 0; k < upto; k++) {
            if (objs[k].lde) cudaFreeAsync(objs[k].lde, s);
            if (objs[k].tree) cudaFreeAsync(objs[k].tree, s);
            if (objs[k].cap) cudaFreeAsync(objs[k].cap, s);
            if (objs[k].done) cudaEventDestroy(objs[k].done);
        }
    };
    for (u32 i = 0; i < nb; i++) {
        const v3c_commit_desc& d = descs[i];
        Object& o = objs[i];
        o.c = d.c;
        o.ld = d.c + (d.c & 1);
        o.log_n = d.log_n;
        o.r = d.rate_bits;
        o.h = d.cap_height;
        size_t N = (size_t)1 << (d.log_n + d.rate_bits);
        size_t tw = (2 * N - ((size_t)2 << d.cap_height)) * 4;
        o.bytes = v3c_commit_footprint(d.c, d.log_n, d.rate_bits, d.cap_height);
        cudaError_t e = cudaMallocAsync((void**)&o.lde, N * o.ld * 8, s);
        if (e == cudaSuccess && tw) e = cudaMallocAsync((void**)&o.tree, tw * 8, s);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&o.cap, ((size_t)4 << d.cap_height) * 8, s);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rollback(i + 1);
            return fail(ctx, V3C_ENOMEM, "v3c_commit: allocation of %zu bytes failed: %s", o.bytes,
                        cudaGetErrorString(e));
        }
    }
    Batch b;
    size_t aoff = 0;
    std::vector<u64*> staged_bufs;  // per-commit input buffers, freed on s after the stages
    auto rollback_all = [&](u32 upto) {
        for (u64* p : staged_bufs) cudaFreeAsync(p, ctx->copy_stream);
        staged_bufs.clear();
        rollback(upto);
    };
    if (!ctx->copy_fork) CK(cudaEventCreateWithFlags(&ctx->copy_fork, cudaEventDisableTiming));
    CK(cudaEventRecord(ctx->copy_fork, s));  // "ready at once" for the groups that wait on no copy
    for (u32 i = 0; i < nb; i++) {
        const v3c_commit_desc& d = descs[i];
        Object& o = objs[i];
        const u64* x = d.cols;
        size_t n = (size_t)1 << d.log_n;
        if (chunked(d)) {
            if (!ctx->copy_stream) CK(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
            u64* in = nullptr;
            cudaError_t ea = cudaMallocAsync((void**)&in, ((size_t)d.c << d.log_n) * 8, ctx->copy_stream);
            if (ea != cudaSuccess) {
                cudaGetLastError();
                rollback_all(nb);
                return fail(ctx, V3C_ENOMEM, "v3c_commit: input staging buffer: %s", cudaGetErrorString(ea));
            }
            staged_bufs.push_back(in);
            const u32 per = ((d.c + kCopyChunks - 1) / kCopyChunks + 3) & ~3u;  // columns per chunk, multiple of 4
            for (u32 c0 = 0; c0 < d.c; c0 += per) {
                const u32 ck = std::min(per, d.c - c0);
                u64* dst = in + (size_t)c0 * n;
                size_t sw = lde_scratch_words(ck, d.log_n, d.rate_bits);
                u64* scr = sw ? arena + aoff : nullptr;
                aoff = align_words(aoff + sw);
                cudaError_t e = cudaMemcpyAsync(dst, d.cols + (size_t)c0 * n, (size_t)ck * n * 8,
                                                cudaMemcpyHostToDevice, ctx->copy_stream);
                const size_t g = b.chunks.size();
                while (ctx->copy_events.size() <= g) {
                    cudaEvent_t ev = nullptr;
                    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
                    if (e != cudaSuccess) break;
                    ctx->copy_events.push_back(ev);
                }
                if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_events[g], ctx->copy_stream);
                if (e != cudaSuccess) {
                    rollback_all(nb);
                    return fail(ctx, V3C_ECUDA, "input copy: %s", cudaGetErrorString(e));
                }
                LdeJob j;
                st = make_lde_job(ctx, dst, ck, d.log_n, d.rate_bits, o.lde + c0, o.ld, scr, s, &j);
                if (st) {
                    rollback_all(nb);
                    return st;
                }
                j.wcols = o.ld - c0;
                j.vec_ok = j.vec_ok && (c0 % 2 == 0);
                b.chunks.push_back({(u32)b.lde.size(), 1});
                b.chunk_ready.push_back(ctx->copy_events[g]);
                b.lde.push_back(j);
            }
            b.tree.push_back(make_tree_job(o.lde, o.ld, d.c, d.log_n + d.rate_bits, d.cap_height, o.tree, o.cap));
            continue;
        }
        if (!b.chunks.empty()) {
            // Jobs outside the chunked inputs form one more group, ready at once.
            b.chunks.push_back({(u32)b.lde.size(), 1});
            b.chunk_ready.push_back(ctx->copy_fork);
        }
        if (d.on_device != V3C_INPUT_DEVICE) {
            u64* dst = arena + aoff;
            aoff = align_words(aoff + d.c * n);
            cudaError_t e = cudaMemcpyAsync(dst, d.cols, d.c * n * 8, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) {
                rollback_all(nb);
                return fail(ctx, V3C_ECUDA, "input copy: %s", cudaGetErrorString(e));
            }
            x = dst;
        }
        size_t sw = lde_scratch_words(d.c, d.log_n, d.rate_bits);
        u64* scr = sw ? arena + aoff : nullptr;
        aoff = align_words(aoff + sw);
        LdeJob j;
        st = make_lde_job(ctx, x, d.c, d.log_n, d.rate_bits, o.lde, o.ld, scr, s, &j);
        if (st) {
            rollback_all(nb);
            return st;
        }
        b.lde.push_back(j);
        b.tree.push_back(make_tree_job(o.lde, o.ld, d.c, d.log_n + d.rate_bits, d.cap_height, o.tree, o.cap));
    }
    if ((ctx->cfg.flags & V3C_FLAG_VALIDATE)) {
        cudaMemsetAsync(ctx->d_flag, 0, 4, s);
        for (auto& j : b.lde) {
            cudaError_t e = launch_validate(j.x, (u64)j.c << j.plan.log_n, ctx->d_flag, s);
            if (e != cudaSuccess) {
                rollback_all(nb);
                return fail(ctx, V3C_ECUDA, "validate: %s", cudaGetErrorString(e));
            }
            ctx->launches++;
        }
        u32 flag = 0;
        cudaError_t e = cudaMemcpyAsync(&flag, ctx->d_flag, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess || flag) {
            rollback_all(nb);
            return e != cudaSuccess ? fail(ctx, V3C_ECUDA, "validate: %s", cudaGetErrorString(e))
                                    : fail(ctx, V3C_EINVAL, "v3c_commit: input not canonical (>= p)");
        }
    }
    b.h_threads = h_threads;
    if (!b.chunks.empty()) {
        // Jobs before the first chunked input form a group of their own, ready at once.
        if (b.chunks.front().first > 0) {
            b.chunks.insert(b.chunks.begin(), {0u, b.chunks.front().first});
            b.chunk_ready.insert(b.chunk_ready.begin(), ctx->copy_fork);
        }
    }
    // Replay a captured graph of this batch signature unless graphs are off,
    // per-stage timing (events around each launch) is requested, or inputs
    // arrive in chunks on the copy stream.
    if (!allow_graph || !b.chunks.empty() || (ctx->cfg.flags & (V3C_FLAG_NO_GRAPH | V3C_FLAG_TIMING)))
        st = launch_batch(ctx, b, s);
    else st = launch_batch_graph(ctx, b, s);
    if (st) {
        rollback_all(nb);
        return st;
    }
    // The staged inputs are read only by stages A and B, enqueued above.
    for (u64* p : staged_bufs) CK(cudaFreeAsync(p, s));
    if (arena_need && !arena_override) {
        st = arena_release(ctx, s);
        if (st) return st;
    }
    for (u32 i = 0; i < nb; i++) {
        Object& o = objs[i];
        CK(cudaEventRecord(o.done, s));
        o.stream = s;
        o.id = preassigned_ids ? preassigned_ids[i] : ctx->next_id++;
        ctx->resident += o.bytes;
        ids[i] = o.id;
        ctx->objects[o.id] = o;
    }
    return V3C_OK;
}

v3c_status lock_and_select(v3c_ctx* ctx) { return use_device(ctx); }
std::mutex& ctx_mutex(v3c_ctx* ctx) { return ctx->mu; }
u64 ctx_next_id(v3c_ctx* ctx) { return ctx->next_id++; }
const v3c_config& ctx_config(v3c_ctx* ctx) { return ctx->cfg; }
size_t ctx_resident(v3c_ctx* ctx) { return ctx->resident; }
serve::Server*& ctx_server(v3c_ctx* ctx) { return ctx->server; }
int ctx_device(v3c_ctx* ctx) { return ctx->device; }
v3c_status ctx_fail(v3c_ctx* ctx, v3c_status s, const char* msg) { return fail(ctx, s, "%s", msg); }

}  // namespace detail
}  // namespace v3c

extern "C" {

v3c_status v3c_commit(v3c_ctx* ctx, const v3c_commit_desc* descs, uint32_t nb, v3c_commit_id* ids, void* stream)
{
    NvtxScope range("v3c_commit");
    if (!ctx) return V3C_EINVAL;
    if (!descs || !ids || nb == 0) return fail(ctx, V3C_EINVAL, "v3c_commit: empty batch or NULL");
    v3c_status st = use_device(ctx);
    if (st) return st;
    std::lock_guard<std::mutex> g(ctx->mu);
    return commit_locked(ctx, descs, nb, ids, (cudaStream_t)stream, nullptr, 0, nullptr);
}

v3c_status v3c_coeffs(v3c_ctx* ctx, const uint64_t* d_cols, uint32_t c, uint32_t log_n, uint64_t* d_coeffs,
                      void* stream)
{
    if (!ctx) return V3C_EINVAL;
    if (!d_cols || !d_coeffs) return fail(ctx, V3C_EINVAL, "v3c_coeffs: NULL pointer");
    if (!shape_ok(c, log_n, 0)) return fail(ctx, V3C_EINVAL, "v3c_coeffs: bad shape c=%u log_n=%u", c, log_n);
    v3c_status st = use_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    // The inverse stages of the rate-3 plan of this size (its split keeps
    // stage B's inverse transform at n2 <= 2^10).
    const u32 r = std::min(3u, (u32)V3C_MAX_LOG_LDE - log_n);
    u32 l1, l2;
    plan_split(log_n, r, l1, l2);
    const size_t words = l1 ? (size_t)c << log_n : 0;  // Y only
    u64* scratch = nullptr;
    if (words) {
        st = arena_acquire(ctx, words, s, &scratch);
        if (st) return st;
    }
    LdeJob j;
    memset(&j, 0, sizeof j);
    st = get_plan(ctx, log_n, r, s, &j.plan);
    if (st) return st;
    j.x = d_cols;
    j.c = c;
    j.ld = c;
    j.wcols = c;
    j.lde = d_coeffs;
    j.Y = scratch;
    j.mode = kCoeffsOut;
    j.cscale = gl::h_inv(((u64)1 << log_n) % gl::P);
    job_tiles(j);
    Batch b;
    b.lde.push_back(j);
    st = launch_batch(ctx, b, s);
    if (st) return st;
    if (words) return arena_release(ctx, s);
    return V3C_OK;
}

v3c_status v3c_commit_part(v3c_ctx* ctx, const v3c_part_desc* d, v3c_commit_id* id, void* stream)
{
    if (!ctx) return V3C_EINVAL;
    if (!d || !id || !d->coeffs) return fail(ctx, V3C_EINVAL, "v3c_commit_part: NULL pointer");
    if (!shape_ok(d->c, d->log_n, d->rate_bits) || d->log_parts > d->rate_bits || d->log_parts > d->cap_height ||
        (d->part >> d->log_parts) || d->cap_height > d->log_n + d->rate_bits)
        return fail(ctx, V3C_EINVAL, "v3c_commit_part: bad desc (c=%u log_n=%u r=%u h=%u log_parts=%u part=%u)", d->c,
                    d->log_n, d->rate_bits, d->cap_height, d->log_parts, d->part);
    v3c_status st = use_device(ctx);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    // Part q holds rows [q N/G, (q+1) N/G): the evaluations on the coset
    // 7 w_N^kappa <w_{N/G}>, kappa = bitrev_{log G}(q), in bit-reversed order.
    const u32 rp = d->rate_bits - d->log_parts, hp = d->cap_height - d->log_parts;
    const u32 logN = d->log_n + d->rate_bits, logNp = d->log_n + rp;
    const u64 kappa = gl::bitrev(d->part, d->log_parts);
    const u64 gshift = gl::h_pow(gl::h_root(logN), kappa);
    const size_t need = v3c_commit_footprint(d->c, d->log_n, rp, hp);
    if (ctx->resident + need > ctx->cfg.hbm_budget_bytes)
        return fail(ctx, V3C_ENOMEM, "v3c_commit_part: %zu bytes requested, %zu resident, budget %llu", need,
                    ctx->resident, (unsigned long long)ctx->cfg.hbm_budget_bytes);
    u32 l1, l2;
    plan_split(d->log_n, rp, l1, l2);
    const size_t words = l1 ? (size_t)d->c << logNp : 0;  // Z only
    u64* scratch = nullptr;
    if (words) {
        st = arena_acquire(ctx, words, s, &scratch);
        if (st) return st;
    }
    Object o;
    o.c = d->c;
    o.ld = d->c + (d->c & 1);
    o.log_n = d->log_n;
    o.r = rp;
    o.h = hp;
    o.bytes = need;
    const size_t Np = (size_t)1 << logNp;
    const size_t tw = (2 * Np - ((size_t)2 << hp)) * 4;
    cudaError_t e = cudaMallocAsync((void**)&o.lde, Np * o.ld * 8, s);
    if (e == cudaSuccess && tw) e = cudaMallocAsync((void**)&o.tree, tw * 8, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&o.cap, ((size_t)4 << hp) * 8, s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&o.done, cudaEventDisableTiming);
    auto rollback = [&]() {
        if (o.lde) cudaFreeAsync(o.lde, s);
        if (o.tree) cudaFreeAsync(o.tree, s);
        if (o.cap) cudaFreeAsync(o.cap, s);
        if (o.done) cudaEventDestroy(o.done);
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        rollback();
        return fail(ctx, V3C_ENOMEM, "v3c_commit_part: allocation of %zu bytes failed: %s", need,
                    cudaGetErrorString(e));
    }
    LdeJob j;
    memset(&j, 0, sizeof j);
    st = get_plan(ctx, d->log_n, rp, s, &j.plan, gshift, 1);
    if (st) {
        rollback();
        return st;
    }
    j.x = d->coeffs;
    j.c = d->c;
    j.ld = o.ld;
    j.wcols = o.ld;
    j.lde = o.lde;
    j.vec_ok = 1;
    j.Z = scratch;
    j.mode = kLdeFromCoeffs;
    job_tiles(j);
    auto it = ctx->tuned.find(std::make_pair(d->log_n, rp));
    if (it != ctx->tuned.end()) lde_job_apply_tune(j, it->second);
    Batch b;
    b.lde.push_back(j);
    b.tree.push_back(make_tree_job(o.lde, o.ld, d->c, logNp, hp, o.tree, o.cap));
    st = launch_batch(ctx, b, s);
    if (st) {
        rollback();
        return st;
    }
    if (words) {
        st = arena_release(ctx, s);
        if (st) return st;
    }
    CK(cudaEventRecord(o.done, s));
    o.stream = s;
    o.id = ctx->next_id++;
    ctx->resident += o.bytes;
    *id = o.id;
    ctx->objects[o.id] = o;
    return V3C_OK;
}

v3c_status v3c_commit_buffers(v3c_ctx* ctx, v3c_commit_id id, uint64_t** d_lde, uint32_t* ld, uint64_t** d_tree,
                              uint64_t** d_cap, uint32_t* log_rows, uint32_t* cap_height)
{
    if (!ctx) return V3C_EINVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->objects.find(id);
    if (it == ctx->objects.end()) return fail(ctx, V3C_ENOTFOUND, "commit id %llu", (unsigned long long)id);
    const Object& o = it->second;
    if (d_lde) *d_lde = o.lde;
    if (ld) *ld = o.ld;
    if (d_tree) *d_tree = o.tree;
    if (d_cap) *d_cap = o.cap;
    if (log_rows) *log_rows = o.log_n + o.r;
    if (cap_height) *cap_height = o.h;
    return V3C_OK;
}

v3c_status v3c_commit_cap(v3c_ctx* ctx, v3c_commit_id id, uint64_t* h_cap)
{
    if (!ctx || !h_cap) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    Object o;
    cudaStream_t rb = nullptr;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->objects.find(id);
        if (it == ctx->objects.end()) return fail(ctx, V3C_ENOTFOUND, "commit id %llu", (unsigned long long)id);
        o = it->second;
        if (!ctx->readback_stream) CK(cudaStreamCreateWithFlags(&ctx->readback_stream, cudaStreamNonBlocking));
        rb = ctx->readback_stream;
    }
    // The copy waits for this object's work only (not for later work the
    // caller has already enqueued on the producing stream).
    CK(cudaStreamWaitEvent(rb, o.done, 0));
    CK(cudaMemcpyAsync(h_cap, o.cap, ((size_t)4 << o.h) * 8, cudaMemcpyDeviceToHost, rb));
    CK(cudaStreamSynchronize(rb));
    return V3C_OK;
}

v3c_status v3c_open(v3c_ctx* ctx, v3c_commit_id id, uint64_t leaf, uint64_t* h_row, uint64_t* h_path)
{
    if (!ctx) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    Object o;
    {
        std::lock_guard<std::mutex> g(ctx->mu);
        auto it = ctx->objects.find(id);
        if (it == ctx->objects.end()) return fail(ctx, V3C_ENOTFOUND, "commit id %llu", (unsigned long long)id);
        o = it->second;
    }
    u32 logN = o.log_n + o.r;
    if (leaf >> logN) return fail(ctx, V3C_EINVAL, "v3c_open: leaf %llu out of range", (unsigned long long)leaf);
    CK(cudaEventSynchronize(o.done));
    if (h_row) CK(cudaMemcpy(h_row, o.lde + leaf * o.ld, (size_t)o.c * 8, cudaMemcpyDeviceToHost));
    if (h_path) {
        size_t N = (size_t)1 << logN;
        for (u32 k = 0; k < logN - o.h; k++) {
            size_t off = 8 * N - ((8 * N) >> k);
            size_t sib = (size_t)((leaf >> k) ^ 1);
            CK(cudaMemcpy(h_path + 4 * k, o.tree + off + 4 * sib, 32, cudaMemcpyDeviceToHost));
        }
    }
    return V3C_OK;
}

v3c_status v3c_release(v3c_ctx* ctx, v3c_commit_id id)
{
    if (!ctx) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->objects.find(id);
    if (it == ctx->objects.end()) return fail(ctx, V3C_ENOTFOUND, "commit id %llu", (unsigned long long)id);
    Object o = it->second;
    ctx->objects.erase(it);
    // Stream-ordered free after the producing work, on the context's own
    // release stream: the producing stream may belong to the caller or to a
    // serving slot that no longer exists.
    if (!ctx->release_stream) CK(cudaStreamCreateWithFlags(&ctx->release_stream, cudaStreamNonBlocking));
    CK(cudaStreamWaitEvent(ctx->release_stream, o.done, 0));
    CK(cudaFreeAsync(o.lde, ctx->release_stream));
    if (o.tree) CK(cudaFreeAsync(o.tree, ctx->release_stream));
    CK(cudaFreeAsync(o.cap, ctx->release_stream));
    CK(cudaEventDestroy(o.done));
    ctx->resident -= o.bytes;
    return V3C_OK;
}

uint64_t v3c_kernel_launches(v3c_ctx* ctx) { return ctx ? ctx->launches.load() : 0; }

uint64_t v3c_graph_replays(v3c_ctx* ctx) { return ctx ? ctx->graph_replays.load() : 0; }

// Value of the non-negative integer field "key" inside [b, e), or -1.
static long long tune_field(const char* b, const char* e, const char* key)
{
    const std::string pat = std::string("\"") + key + "\"";
    const char* p = std::search(b, e, pat.begin(), pat.end());
    if (p == e) return -1;
    p += pat.size();
    while (p < e && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) p++;
    if (p == e || *p != ':') return -1;
    p++;
    while (p < e && (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r')) p++;
    if (p == e || *p < '0' || *p > '9') return -1;
    long long v = 0;
    while (p < e && *p >= '0' && *p <= '9' && v < (1ll << 40)) v = v * 10 + (*p++ - '0');
    return v;
}

v3c_status v3c_tune_export(v3c_ctx* ctx, char* buf, size_t cap, size_t* len)
{
    if (!ctx || !len || (cap && !buf)) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    std::lock_guard<std::mutex> g(ctx->mu);
    std::string t = "{\"sm_count\": " + std::to_string(num_sms()) + ", \"entries\": [";
    bool first = true;
    for (const auto& kv : ctx->tuned) {
        const TuneEntry& e = kv.second;
        char row[256];
        snprintf(row, sizeof row,
                 "%s{\"log_n\": %u, \"rate_bits\": %u, \"a_cols\": %u, \"c_q\": %u, \"c_qc\": %u, \"kcap\": %u, "
                 "\"h_threads\": %u}",
                 first ? "" : ", ", kv.first.first, kv.first.second, e.a_cols, e.c_q, e.c_qc, e.kcap, e.h_threads);
        t += row;
        first = false;
    }
    t += "]}";
    *len = t.size();
    if (cap < t.size() + 1)  // a size query (cap 0) is not logged as a failure
        return cap ? fail(ctx, V3C_EINVAL, "v3c_tune_export: %zu bytes needed", t.size() + 1) : V3C_EINVAL;
    memcpy(buf, t.c_str(), t.size() + 1);
    return V3C_OK;
}

v3c_status v3c_tune_import(v3c_ctx* ctx, const char* text)
{
    if (!ctx || !text) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    const char* end = text + strlen(text);
    const char* ent = strstr(text, "\"entries\"");
    if (!ent) return fail(ctx, V3C_EINVAL, "v3c_tune_import: no \"entries\"");
    const long long sms = tune_field(text, ent, "sm_count");
    if (sms != (long long)num_sms())
        return fail(ctx, V3C_EINVAL, "v3c_tune_import: tuned for %lld SMs, this device has %d", sms, num_sms());
    const char* p = strchr(ent, '[');
    if (!p) return fail(ctx, V3C_EINVAL, "v3c_tune_import: \"entries\" is not a list");
    auto pow2 = [](long long x) { return x > 0 && !(x & (x - 1)); };
    std::vector<std::pair<std::pair<u32, u32>, TuneEntry>> got;
    for (p++;;) {
        const char* ob = strchr(p, '{');
        const char* rb = strchr(p, ']');
        if (!rb) return fail(ctx, V3C_EINVAL, "v3c_tune_import: unterminated \"entries\"");
        if (!ob || rb < ob) break;
        const char* oe = strchr(ob, '}');
        if (!oe || oe > end) return fail(ctx, V3C_EINVAL, "v3c_tune_import: unterminated entry");
        const char* names[7] = {"log_n", "rate_bits", "a_cols", "c_q", "c_qc", "kcap", "h_threads"};
        long long f[7];
        for (int i = 0; i < 7; i++) {
            f[i] = tune_field(ob, oe, names[i]);
            if (f[i] < 0) return fail(ctx, V3C_EINVAL, "v3c_tune_import: entry %zu has no \"%s\"", got.size(), names[i]);
        }
        if (f[0] > V3C_MAX_LOG_N || f[1] > V3C_MAX_RATE_BITS || f[0] + f[1] > V3C_MAX_LOG_LDE || !pow2(f[2]) ||
            !pow2(f[3]) || !pow2(f[4]) || f[2] > 16384 || f[3] > 16384 || f[4] > f[3] || f[5] < 1 || f[5] > 4 ||
            (f[6] != 64 && f[6] != 128))
            return fail(ctx, V3C_EINVAL, "v3c_tune_import: entry %zu is out of range", got.size());
        got.push_back({{(u32)f[0], (u32)f[1]}, TuneEntry{(u32)f[2], (u32)f[3], (u32)f[4], (u32)f[5], (u32)f[6]}});
        p = oe + 1;
    }
    std::lock_guard<std::mutex> g(ctx->mu);
    for (const auto& kv : got) ctx->tuned[kv.first] = kv.second;
    log_msg(ctx, 1, "imported the tuned tiles of %zu shapes", got.size());
    return V3C_OK;
}

v3c_status v3c_mem_stats(v3c_ctx* ctx, uint64_t* out)
{
    if (!ctx || !out) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    std::lock_guard<std::mutex> g(ctx->mu);
    cudaMemPool_t pool = nullptr;
    uint64_t used = 0;
    CK(cudaDeviceGetDefaultMemPool(&pool, ctx->device));
    CK(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used));
    out[0] = ctx->resident;
    out[1] = used;
    out[2] = (uint64_t)ctx->arena.words * sizeof(u64);
    return V3C_OK;
}

v3c_status v3c_stage_stats(v3c_ctx* ctx, v3c_stage_stats_t* out, int reset)
{
    if (!ctx || !out) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    std::vector<v3c_ctx::Pending> pend;
    {
        std::lock_guard<std::mutex> g(ctx->tmu);
        pend.swap(ctx->pending);
    }
    for (auto& p : pend) {
        float ms = 0;
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "stage timing: %s", cudaGetErrorString(e));
        std::lock_guard<std::mutex> g(ctx->tmu);
        ctx->stage_ms[p.stage] += ms;
        ctx->stage_n[p.stage] += 1;
        ctx->ev_pool.push_back(p.a);
        ctx->ev_pool.push_back(p.b);
    }
    std::lock_guard<std::mutex> g(ctx->tmu);
    for (int i = 0; i < V3C_NUM_STAGES; i++) {
        out->ms[i] = ctx->stage_ms[i];
        out->launches[i] = ctx->stage_n[i];
        if (reset) {
            ctx->stage_ms[i] = 0;
            ctx->stage_n[i] = 0;
        }
    }
    return V3C_OK;
}

v3c_status v3c_int_pipe_rate(v3c_ctx* ctx, uint32_t kind, uint32_t reps, double* rate, double* mhz)
{
    if (!ctx || !rate || kind > 1) return V3C_EINVAL;
    v3c_status st = use_device(ctx);
    if (st) return st;
    int sms = num_sms();
    int grid = sms * 8, threads = 256;
    u32 iters = 4096;
    u64* out = nullptr;
    CK(cudaMalloc(&out, (size_t)(grid + 1) * 8));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    double best = 0, best_mhz = 0;
    for (u32 r = 0; r < std::max(reps, 1u) + 1; r++) {
        CK(cudaEventRecord(a, 0));
        CK(launch_int_peak(out, grid, threads, iters, kind == 0, 0));
        ctx->launches++;
        CK(cudaEventRecord(b, 0));
        CK(cudaEventSynchronize(b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, a, b));
        u64 rate20 = 0;  // SM cycles per 2^20 ns, seen by block 0
        CK(cudaMemcpy(&rate20, out, 8, cudaMemcpyDeviceToHost));
        double ops = (double)grid * threads * iters * 8 * 4;
        if (r > 0 && ops / (ms * 1e-3) > best) {
            best = ops / (ms * 1e-3);
            best_mhz = (double)rate20 / (double)(1u << 20) * 1e3;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(out);
    *rate = best;
    if (mhz) *mhz = best_mhz;
    return V3C_OK;
}

v3c_status v3c_int_peak(v3c_ctx* ctx, uint32_t reps, double* rate, double* mhz)
{
    return v3c_int_pipe_rate(ctx, 0, reps, rate, mhz);
}

}  // extern "C"
