// Serving loop: continuous batching of commit requests.  Requests that
// arrive while others run on the device join the next scheduler pass.
#pragma once
#include <cuda_runtime.h>

#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/v3c.h"
#include "internal.h"

namespace v3c {

double now_s();

namespace serve {

struct Request {
    u64 ticket = 0;
    v3c_commit_desc desc{};
    std::vector<u64> host_copy;  // input copied at submit (host requests)
    v3c_req_state state = V3C_REQ_QUEUED;
    v3c_status status = V3C_EAGAIN;
    v3c_req_times times{};
    u64 footprint = 0;
};

// Requests are batched within size classes (LDE elements c * 2^(log_n + r):
// class 0 up to 2^24, class 1 up to 2^27, class 2 above), so that a batch of
// small requests completes apart from the large ones admitted beside it.
constexpr int kSizeClasses = 3;
int size_class(const v3c_commit_desc& d);

struct Slot {
    // One stream per size class, with the class's priority (small requests
    // highest); a batch runs on the stream of its class.
    cudaStream_t streams[kSizeClasses] = {nullptr, nullptr, nullptr};
    cudaStream_t stream = nullptr;  // stream of the batch in flight
    int cls = -1;                   // its size class
    cudaEvent_t done = nullptr;
    u64* arena = nullptr;        // device scratch + staged inputs of the batch
    size_t arena_words = 0;
    u64* pinned = nullptr;       // pinned staging of host inputs
    size_t pinned_words = 0;
    bool busy = false;
    std::vector<u64> tickets;
};

struct Server {
    v3c_ctx* ctx = nullptr;
    v3c_serve_cfg cfg{};
    std::thread th;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<u64> queue;
    std::unordered_map<u64, Request> reqs;
    std::vector<Slot> slots;
    bool stop = false;
    bool crashed = false;
    long inject_after = -1;  // scheduler passes before an injected failure (-1: none)
};

}  // namespace serve

namespace detail {
}  // namespace detail
}  // namespace v3c

// Arena words a batched commit of nb descs adds for block alignment.
size_t arena_padding(v3c::u32 nb);
// The context's log callback (v3c_set_log), if set for `level`.
void log_msg(v3c_ctx* ctx, int level, const char* fmt, ...);

namespace v3c {
namespace detail {
v3c_status commit_locked(v3c_ctx* ctx, const v3c_commit_desc* descs, u32 nb, u64* ids, cudaStream_t s,
                         u64* arena_override, size_t arena_words, const u64* preassigned_ids,
                         bool allow_graph = true);
v3c_status lock_and_select(v3c_ctx* ctx);
std::mutex& ctx_mutex(v3c_ctx* ctx);
u64 ctx_next_id(v3c_ctx* ctx);
const v3c_config& ctx_config(v3c_ctx* ctx);
size_t ctx_resident(v3c_ctx* ctx);
serve::Server*& ctx_server(v3c_ctx* ctx);
int ctx_device(v3c_ctx* ctx);
v3c_status ctx_fail(v3c_ctx* ctx, v3c_status s, const char* msg);
}  // namespace detail

}  // namespace v3c
