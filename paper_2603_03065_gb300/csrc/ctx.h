// Library context, resident objects and the batch descriptor, shared by
// the translation units that implement the C ABI (v3c.cu, fri.cu).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "../../include/v3c.h"
#include "internal.h"

namespace v3c {
namespace serve {
struct Server;
}
struct FriState;
struct SnapState;
struct SnapCbCache;
extern thread_local int g_dev_cache;
}  // namespace v3c

using namespace v3c;

// Column chunks per large host input on the direct commit path.
constexpr v3c::u32 kCopyChunks = 4;

// ---------------------------------------------------------------- context

struct PlanEntry {
    Plan plan;
    u64* mem = nullptr;
};

// One captured instance of a batch signature (see launch_batch_graph).
struct GraphInst {
    cudaGraphExec_t exec = nullptr;
    void* h_blob = nullptr;
    void* d_blob = nullptr;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
    uint32_t kernels = 0;
};
struct GraphSet {
    std::vector<GraphInst> inst;
    uint32_t next = 0;
};
constexpr uint32_t kGraphRing = 3;
constexpr size_t kMaxGraphSets = 64;

struct UploadSlot {
    void* h = nullptr;
    void* d = nullptr;
    size_t cap = 0;
    cudaEvent_t ev = nullptr;
};

struct Arena {
    u64* mem = nullptr;
    size_t words = 0;
    cudaEvent_t ev = nullptr;
    cudaStream_t last = nullptr;
    bool used = false;
};

struct Object {
    u64 id = 0;
    u64* lde = nullptr;
    u64* tree = nullptr;
    u64* cap = nullptr;
    u32 c = 0, ld = 0, log_n = 0, r = 0, h = 0;
    size_t bytes = 0;
    cudaEvent_t done = nullptr;
    cudaStream_t stream = nullptr;
};

struct v3c_ctx {
    int device = 0;
    v3c_config cfg{};
    std::mutex mu;
    // Plan tables by (log_n, rate_bits, coset multiplier, scale factor).
    std::map<std::tuple<u32, u32, u64, u64>, PlanEntry> plans;
    Arena arena;
    std::vector<UploadSlot> ring;
    u32 ring_next = 0;
    std::unordered_map<u64, Object> objects;
    u64 next_id = 1;
    size_t resident = 0;
    std::atomic<u64> launches{0};
    std::mutex err_mu;
    std::string err;
    // Log callback (v3c_set_log); silent while log_fn is null.
    std::mutex log_mu;
    v3c_log_fn log_fn = nullptr;
    void* log_user = nullptr;
    int log_level = -1;
    Tiles tiles;
    u32* d_flag = nullptr;
    serve::Server* server = nullptr;
    std::unordered_map<u64, FriState*> fri;      // FRI commit-phase states (fri.cu)
    std::unordered_map<u64, SnapState*> snaps;   // snapshot commitments (snapshot.cu)
    SnapCbCache* snap_cb = nullptr;              // codebook-digest cache (snapshot.cu)
    cudaStream_t release_stream = nullptr;  // orders frees of resident objects
    cudaStream_t readback_stream = nullptr; // cap reads: waits on one object's event only
    // Chunked input copies of large host inputs (commit_locked).
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_fork = nullptr;
    std::vector<cudaEvent_t> copy_events;
    // CUDA graphs of batch signatures, and the autotuner's per-shape choices
    std::unordered_map<std::string, GraphSet> graphs;
    std::unordered_map<std::string, int> graph_seen;
    cudaStream_t capture_stream = nullptr;
    std::atomic<u64> graph_replays{0};
    std::map<std::pair<u32, u32>, TuneEntry> tuned;
    // per-stage timing (V3C_FLAG_TIMING)
    std::mutex tmu;
    struct Pending {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
    double stage_ms[V3C_NUM_STAGES] = {0};
    uint64_t stage_n[V3C_NUM_STAGES] = {0};
};


// Records the error text of the last failing call (and logs it at level 0)
// and returns s.
v3c_status fail(v3c_ctx* ctx, v3c_status s, const char* fmt, ...);
// Sends a message to the context's log callback if one is set for `level`.
void log_msg(v3c_ctx* ctx, int level, const char* fmt, ...);
// Makes the context's device current for this thread.
v3c_status use_device(v3c_ctx* ctx);
// Frees every FRI state of the context (fri.cu).
void fri_free_all(v3c_ctx* ctx);
// Frees every snapshot object of the context (snapshot.cu).
void snap_free_all(v3c_ctx* ctx);

#define CK(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, V3C_ECUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                                       \
    } while (0)

namespace v3c {
namespace detail {

// A batch of LDE jobs and tree jobs, launched as one persistent launch per
// stage.  Builds the upload blob (jobs + stage item lists).
struct Batch {
    std::vector<LdeJob> lde;
    std::vector<TreeJob> tree;
    std::vector<u32> fa, fb, fc, fl;
    std::vector<std::vector<u32>> fm;
    size_t smem_a = 0, smem_b = 0, smem_c = 0;
    u32 max_top = 0;

    void finalize(const Tiles& t)
    {
        fa.assign(1, 0);
        fb.assign(1, 0);
        fc.assign(1, 0);
        for (auto& j : lde) {
            fa.push_back(fa.back() + stage_a_items(j, t));
            fb.push_back(fb.back() + stage_b_items(j));
            fc.push_back(fc.back() + stage_c_items(j, t));
            smem_a = std::max(smem_a, stage_a_smem(j, t));
            smem_b = std::max(smem_b, stage_b_smem(j));
            smem_c = std::max(smem_c, stage_c_smem(j, t));
        }
        fl.assign(1, 0);
        max_top = 0;
        for (auto& j : tree) {
            fl.push_back(fl.back() + leaf_items(j, t));
            max_top = std::max(max_top, j.log_N - j.h);
        }
        // Merkle launches: one per level while the level has enough nodes to
        // fill the GPU with one compression per thread, then one launch that
        // folds up to 8 levels per CTA in shared memory.
        fac.clear();
        fbc.clear();
        for (auto& g : chunks) {
            std::vector<u32> a(1, 0), b(1, 0);
            for (u32 k = g.first; k < g.first + g.second; k++) {
                a.push_back(a.back() + stage_a_items(lde[k], t));
                b.push_back(b.back() + stage_b_items(lde[k]));
            }
            fac.push_back(a);
            fbc.push_back(b);
        }
        // Levels with at most kMerkleWarpMaxNodes nodes take the warp-per-node
        // form (the latency of one compression sets their time); thread-per-node
        // launches fold levels until a level is that small.
        fm.clear();
        mgroups.clear();
        mwarp.clear();
        for (u32 lev0 = 0; lev0 < max_top;) {
            u64 nodes = 0;
            for (auto& j : tree)
                if (j.log_N - j.h > lev0) nodes += (u64)1 << (j.log_N - lev0 - 1);
            const bool warp = nodes <= kMerkleWarpMaxNodes;
            u32 nlev = 1;
            if (warp) {
                nlev = kMerkleWarpLevels;
            } else if (nodes < ((u64)1 << 17)) {
                nlev = 0;
                for (u64 n = nodes; n > kMerkleWarpMaxNodes && nlev < 8; n >>= 1) nlev++;
            }
            std::vector<u32> f(1, 0);
            for (auto& j : tree) f.push_back(f.back() + (warp ? merkle_warp_items(j, lev0) : merkle_items(j, lev0, t)));
            fm.push_back(f);
            mgroups.push_back({lev0, nlev});
            mwarp.push_back(warp);
            lev0 += nlev;
        }
    }
    std::vector<std::pair<u32, u32>> mgroups;  // (first level, levels) of each Merkle launch
    std::vector<bool> mwarp;                   // warp-per-node form for that launch
    u32 h_threads = 0;                          // leaf-hash CTA size (0 = context default)
    bool leaves_ready = false;                  // level 0 of every tree is already written: no leaf hash
    // Column chunks whose inputs arrive by separate copies: stages A and B
    // run per chunk, each after its copy's event; stage C and the trees run
    // once over all jobs.  Empty: one launch per stage over all jobs.
    std::vector<std::pair<u32, u32>> chunks;    // (first LDE job, job count)
    std::vector<cudaEvent_t> chunk_ready;       // one per chunk, recorded after its copy
    std::vector<std::vector<u32>> fac, fbc;     // per-chunk stage A / B item prefixes
};


// An event from the context's pool (timing events are recycled).
cudaEvent_t pool_event(v3c_ctx* ctx);

// Brackets one stage launch with events on its stream when timing is on.
// NVTX range over a scope.  On the host it spans the enqueue of the work it
// names; a profiler lines it up with the kernels launched inside it.  With
// no profiler attached the calls return at once.
struct NvtxScope {
    explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
    ~NvtxScope() { nvtxRangePop(); }
    NvtxScope(const NvtxScope&) = delete;
    NvtxScope& operator=(const NvtxScope&) = delete;
};

// NVTX names of the stages, in v3c_stage_stats order.
inline const char* stage_range_name(int id)
{
    static const char* const names[V3C_NUM_STAGES] = {
        "v3c stage A", "v3c stage B", "v3c stage C", "v3c leaf hash", "v3c Merkle", "v3c FRI combination",
        "v3c FRI fold", "v3c openings", "v3c SetEq", "v3c snapshot slots", "v3c snapshot codebook"};
    return id >= 0 && id < V3C_NUM_STAGES ? names[id] : "v3c";
}

// Events around one stage launch (V3C_FLAG_TIMING, stage >= 0) and an NVTX
// range named after `name_id` (the stage itself when not given).
struct StageTimer {
    v3c_ctx* ctx;
    int stage;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    StageTimer(v3c_ctx* c, int st, cudaStream_t str, int name_id = -2) : ctx(c), stage(st), s(str)
    {
        nvtxRangePushA(stage_range_name(name_id == -2 ? st : name_id));
        if ((ctx->cfg.flags & V3C_FLAG_TIMING) && st >= 0) {
            a = pool_event(ctx);
            if (a) cudaEventRecord(a, s);
        }
    }
    ~StageTimer() { nvtxRangePop(); }
    StageTimer(const StageTimer&) = delete;
    StageTimer& operator=(const StageTimer&) = delete;
    void done()
    {
        if (!a) return;
        cudaEvent_t b = pool_event(ctx);
        if (!b) return;
        cudaEventRecord(b, s);
        std::lock_guard<std::mutex> g(ctx->tmu);
        ctx->pending.push_back({stage, a, b});
        a = nullptr;
    }
};

// Staged upload of a small host table through the context's pinned ring.
v3c_status upload(v3c_ctx* ctx, const void* src, size_t bytes, cudaStream_t s, void** d_out, u32* slot_out);
v3c_status upload_done(v3c_ctx* ctx, u32 slot, cudaStream_t s);

// Direct launch of a finalised batch (upload of its job tables, then one
// launch per stage).
v3c_status launch_batch(v3c_ctx* ctx, Batch& b, cudaStream_t s);

}  // namespace detail
}  // namespace v3c
