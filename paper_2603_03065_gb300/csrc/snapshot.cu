// Snapshot commitment of a fixed-shape IVF-PQ index (Sec. 4.3, Snapshot
// Commitments): slot digests Hash(i, j, f, item, v), per-list Merkle roots,
// centroid binding Hash(i, mu_i, root_i), the top-level root root_mk and the
// codebook digest root_cb.
//
// GB300 mapping: one thread per slot sponges its record in registers and
// writes level 0 of one Merkle tree over all nlist * n slots.  List i owns
// the contiguous leaves [i n, (i+1) n), so the list roots are the cap of
// that tree at height log2(nlist), and the batched Merkle-level launches of
// the polynomial commitment build every list tree at once.  One thread per
// list binds the centroid; the top-level tree reuses the same launches.
// The codebook digest is one sequential sponge (M K d / 8 permutations): it
// runs on a side stream, overlapped with the trees, and is reused when a
// later commit's codebooks are equal word for word (checked on the device).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/v3c_snapshot.h"
#include "ctx.h"
#include "gl.cuh"
#include "internal.h"
#include "poseidon.cuh"
#include "poseidon_warp.cuh"

namespace v3c {

using gl::u32;
using gl::u64;
typedef pos::Default SPC;

struct SnapState {
    u64 id = 0;
    u32 log_nlist = 0;
    u64* mem = nullptr;   // list roots, top tree, root_mk, root_cb
    size_t bytes = 0;
    u64* list_roots = nullptr;  // [nlist][4]
    u64* top_tree = nullptr;    // level-major, levels 0 .. log_nlist - 1 (level 0 = centroid digests)
    u64* root_mk = nullptr;     // [4]
    u64* root_cb = nullptr;     // [4]
    cudaEvent_t ev = nullptr;
};

// The context's codebook-digest cache: the last committed codebooks and their
// digest.  PQ codebooks are static once trained (Sec. 4.3), so successive
// snapshot versions usually share them; a commit compares its codebooks
// with the cached copy on the device and reuses the digest only if every
// word is equal.  Layout of mem: [diff flag, digest (4), codebooks (count)].
struct SnapCbCache {
    u64* mem = nullptr;
    u32 count = 0;
    cudaEvent_t ev = nullptr;
};

// Poseidon sponge over len words produced by get(e): overwrite lanes 0..7
// with each chunk of 8 and permute; digest = lanes 0..3.  Inputs of at most
// 4 words are their own zero-padded digest.
template <typename Get>
__device__ __forceinline__ void sponge_digest(u32 len, Get get, u64* dst)
{
    u64 s[12];
#pragma unroll
    for (int i = 0; i < 12; i++) s[i] = 0;
    if (len <= 4) {
#pragma unroll
        for (u32 i = 0; i < 4; i++)
            if (i < len) s[i] = get(i);
    } else {
        for (u32 st = 0; st < len; st += 8) {
            const u32 l = min(8u, len - st);
#pragma unroll
            for (u32 k = 0; k < 8; k++)
                if (k < l) s[k] = get(st + k);
            pos::permute<SPC>(s);
        }
    }
    *reinterpret_cast<ulonglong2*>(dst) = make_ulonglong2(gl::canon(s[0]), gl::canon(s[1]));
    *reinterpret_cast<ulonglong2*>(dst + 2) = make_ulonglong2(gl::canon(s[2]), gl::canon(s[3]));
}

// hash_{i,j} for every slot t = i n + j: input (i, j, rec[t][0 .. 2+M)).
__global__ void __launch_bounds__(128, 8) k_snap_slots(const u64* __restrict__ rec, u32 M, u32 log_n, u64 N,
                                                       u64* __restrict__ out)
{
    const u32 w = 2 + M;
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < N; t += (u64)gridDim.x * blockDim.x) {
        const u64* r = rec + t * w;
        const u64 i = t >> log_n, j = t & (((u64)1 << log_n) - 1);
        sponge_digest(4 + M, [&](u32 e) -> u64 { return e == 0 ? i : e == 1 ? j : __ldg(r + e - 2); },
                      out + 4 * t);
    }
}

// hash_i = Hash(i, mu_i[0..D), root_i[0..4)) for every list i.
__global__ void __launch_bounds__(128) k_snap_centroids(const u64* __restrict__ mu, u32 D,
                                                        const u64* __restrict__ roots, u32 nlist,
                                                        u64* __restrict__ out)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < nlist; i += gridDim.x * blockDim.x) {
        const u64* m = mu + (u64)i * D;
        const u64* rt = roots + 4 * (u64)i;
        auto get = [&](u32 e) -> u64 {
            return e == 0 ? (u64)i : e <= D ? __ldg(m + e - 1) : __ldg(rt + e - 1 - D);
        };
        sponge_digest(1 + D + 4, get, out + 4 * (u64)i);
    }
}

// root_cb = Hash of the flattened codebooks.  The sponge is sequential
// (count / 8 permutations, each on the previous state), so its time is the
// latency of one permutation times their number.  One warp shares each
// permutation (poseidon_warp.cuh): lane l < 12 holds state word s_l.
// With `same` non-null, *same == 0 means the codebooks equal the cached ones
// (k_snap_cb_compare) and the cached digest is copied instead.
__global__ void __launch_bounds__(32) k_snap_codebook(const u64* __restrict__ cb, u32 count, u64* __restrict__ out,
                                                     const u64* __restrict__ same, const u64* __restrict__ cached)
{
    __shared__ pos::WarpRc s_rc;
    const u32 l = threadIdx.x;
    if (same && *same == 0) {
        if (l < 4) out[l] = cached[l];
        return;
    }
    pos::warp_rc_init(s_rc, l, 32);
    __syncwarp();
    u32 m[12];
    pos::warp_mds_row(m, l);
    u64 x = 0;  // s_l, non-canonical in [0, 2^64) between permutations
    if (count <= 4) {
        if (l < count) x = __ldg(cb + l);
    } else {
        u64 next = l < 8 && l < count ? __ldg(cb + l) : 0;
        for (u32 st = 0; st < count; st += 8) {
            const u32 len = min(8u, count - st);
            if (l < len) x = next;  // overwrite lanes 0 .. len-1
            if (st + 8 < count)     // prefetch the next chunk during the permutation
                next = l < 8 && st + 8 + l < count ? __ldg(cb + st + 8 + l) : 0;
            x = pos::permute_warp(x, s_rc, m, l);
        }
    }
    if (l < 4) out[l] = gl::canon(x);
}

// *diff = 1 if a[i] != b[i] for some i < count (diff cleared beforehand).
__global__ void k_snap_cb_compare(const u64* __restrict__ a, const u64* __restrict__ b, u32 count, u64* diff)
{
    bool d = false;
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) d |= a[i] != b[i];
    if (__any_sync(0xffffffffu, d) && (threadIdx.x & 31) == 0) *diff = 1;
}

// Top-level paths: for query q and word o < 4 log_nlist, sibling digest of
// level o / 4 (level k starts at word 8 nl - 8 nl / 2^k).
__global__ void k_snap_paths(const u64* __restrict__ tree, u32 log_nlist, const u32* __restrict__ lists, u32 nq,
                             u64* __restrict__ out)
{
    const u32 per = 4 * log_nlist;
    const u64 total = (u64)per * nq;
    for (u64 g = blockIdx.x * (u64)blockDim.x + threadIdx.x; g < total; g += (u64)gridDim.x * blockDim.x) {
        u64 q = g / per, o = g - q * per;
        u32 lvl = (u32)(o >> 2), comp = (u32)(o & 3);
        u64 eight = (u64)8 << log_nlist;
        out[g] = tree[(eight - (eight >> lvl)) + 4 * (((u64)lists[q] >> lvl) ^ 1) + comp];
    }
}

}  // namespace v3c

using namespace v3c::detail;

namespace {

int sgrid(u64 work, int threads)
{
    u64 g = (work + threads - 1) / threads;
    return (int)std::max<u64>(1, std::min<u64>(g, (u64)num_sms() * 16));
}

TreeJob digest_tree(u64* tree, u64* cap, u32 log_leaves, u32 h)
{
    TreeJob t;
    memset(&t, 0, sizeof t);
    t.ld = t.width = 4;
    t.log_N = log_leaves;
    t.h = h;
    t.tree = tree;
    t.cap = cap;
    return t;
}

SnapState* find_snap(v3c_ctx* ctx, v3c_snapshot_id id)
{
    auto it = ctx->snaps.find(id);
    return it == ctx->snaps.end() ? nullptr : it->second;
}

}  // namespace

void snap_free_all(v3c_ctx* ctx)
{
    for (auto& kv : ctx->snaps) {
        if (kv.second->mem) cudaFree(kv.second->mem);
        if (kv.second->ev) cudaEventDestroy(kv.second->ev);
        delete kv.second;
    }
    ctx->snaps.clear();
    if (ctx->snap_cb) {
        if (ctx->snap_cb->mem) cudaFree(ctx->snap_cb->mem);
        if (ctx->snap_cb->ev) cudaEventDestroy(ctx->snap_cb->ev);
        delete ctx->snap_cb;
        ctx->snap_cb = nullptr;
    }
}

extern "C" {

v3c_status v3c_snapshot_commit(v3c_ctx* ctx, const v3c_snapshot_desc* d, v3c_snapshot_id* out, void* stream)
{
    if (!ctx) return V3C_EINVAL;
    if (!d || !out || !d->records || !d->centroids || !d->codebooks)
        return fail(ctx, V3C_EINVAL, "v3c_snapshot_commit: NULL argument");
    if (d->log_nlist > 20 || d->log_nlist + d->log_n > 26 || d->M < 1 || d->M > 64 || d->D < 1 || d->D > 65536 ||
        d->K < 1 || d->d < 1 || (u64)d->M * d->K * d->d >= ((u64)1 << 31))
        return fail(ctx, V3C_EINVAL, "v3c_snapshot_commit: shape out of range (log_nlist %u, log_n %u, M %u, D %u)",
                    d->log_nlist, d->log_n, d->M, d->D);
    v3c_status r = use_device(ctx);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    const u32 ln = d->log_nlist, lN = d->log_nlist + d->log_n;
    const u64 nlist = (u64)1 << ln, N = (u64)1 << lN;
    const u64 w = 2 + d->M, cbw = (u64)d->M * d->K * d->d;
    // Resident part: list roots, top tree below its root, root_mk, root_cb.
    const size_t top_words = ln ? (2 * nlist - 2) * 4 : 0;
    const size_t res_words = nlist * 4 + top_words + 8;
    // Scratch: slot tree below the list roots, and host inputs if copied.
    const size_t slot_words = (2 * N - 2 * nlist) * 4;
    const bool host = d->on_device != V3C_INPUT_DEVICE;
    const size_t in_words = host ? N * w + nlist * d->D + cbw : 0;
    SnapState* st = new SnapState();
    st->log_nlist = ln;
    st->bytes = res_words * 8;
    if (ctx->resident + st->bytes > ctx->cfg.hbm_budget_bytes) {
        delete st;
        return fail(ctx, V3C_ENOMEM, "v3c_snapshot_commit: over the HBM budget");
    }
    u64* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&st->mem, st->bytes, s);
    if (e == cudaSuccess && slot_words + in_words)
        e = cudaMallocAsync((void**)&scratch, (slot_words + in_words) * 8, s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (st->mem) cudaFreeAsync(st->mem, s);
        if (scratch) cudaFreeAsync(scratch, s);
        delete st;
        return fail(ctx, V3C_ENOMEM, "v3c_snapshot_commit: allocation failed: %s", cudaGetErrorString(e));
    }
    st->list_roots = st->mem;
    st->top_tree = st->mem + nlist * 4;
    st->root_mk = st->top_tree + top_words;
    st->root_cb = st->root_mk + 4;
    u64* slot_tree = scratch;
    const u64* rec = d->records;
    const u64* mu = d->centroids;
    const u64* cb = d->codebooks;
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    auto cleanup = [&](v3c_status code) {
        if (side) cudaStreamDestroy(side);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        return code;
    };
    auto bail = [&](v3c_status code) {
        cudaFreeAsync(st->mem, s);
        if (scratch) cudaFreeAsync(scratch, s);
        cudaEventDestroy(st->ev);
        delete st;
        return cleanup(code);
    };
#define CKS(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bail(fail(ctx, V3C_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)));     \
    } while (0)
    if (host) {
        u64* in = scratch + slot_words;
        CKS(cudaMemcpyAsync(in, rec, N * w * 8, cudaMemcpyHostToDevice, s));
        CKS(cudaMemcpyAsync(in + N * w, mu, nlist * d->D * 8, cudaMemcpyHostToDevice, s));
        CKS(cudaMemcpyAsync(in + N * w + nlist * d->D, cb, cbw * 8, cudaMemcpyHostToDevice, s));
        rec = in;
        mu = in + N * w;
        cb = in + N * w + nlist * d->D;
        CKS(cudaStreamSynchronize(s));  // host buffers may be reused after return
    }
    // Codebook digest on a side stream, joined before the object is done.
    CKS(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    CKS(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    CKS(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
    CKS(cudaEventRecord(fork, s));
    CKS(cudaStreamWaitEvent(side, fork, 0));
    {
        SnapCbCache*& cc = ctx->snap_cb;
        if (!cc) cc = new SnapCbCache();
        const bool usable = cc->mem && cc->count == (u32)cbw;
        StageTimer tm(ctx, 10, side);
        if (usable) {
            CKS(cudaStreamWaitEvent(side, cc->ev, 0));
            CKS(cudaMemsetAsync(cc->mem, 0, 8, side));
            k_snap_cb_compare<<<sgrid(cbw, 256), 256, 0, side>>>(cc->mem + 5, cb, (u32)cbw, cc->mem);
            CKS(cudaGetLastError());
            k_snap_codebook<<<1, 32, 0, side>>>(cb, (u32)cbw, st->root_cb, cc->mem, cc->mem + 1);
            ctx->launches += 2;
        } else {
            k_snap_codebook<<<1, 32, 0, side>>>(cb, (u32)cbw, st->root_cb, nullptr, nullptr);
            ctx->launches++;
        }
        CKS(cudaGetLastError());
        tm.done();
        // Refresh the cache with this commit's codebooks and digest.
        // The cache counts as filled (count set) only once its copies are queued.
        if (!usable) {
            cc->count = 0;
            if (cc->mem) {
                CKS(cudaStreamWaitEvent(side, cc->ev, 0));
                CKS(cudaFreeAsync(cc->mem, side));
                cc->mem = nullptr;
            }
            CKS(cudaMallocAsync((void**)&cc->mem, (5 + cbw) * 8, side));
            if (!cc->ev) CKS(cudaEventCreateWithFlags(&cc->ev, cudaEventDisableTiming));
        }
        CKS(cudaMemcpyAsync(cc->mem + 1, st->root_cb, 32, cudaMemcpyDeviceToDevice, side));
        CKS(cudaMemcpyAsync(cc->mem + 5, cb, cbw * 8, cudaMemcpyDeviceToDevice, side));
        CKS(cudaEventRecord(cc->ev, side));
        cc->count = (u32)cbw;
    }
    CKS(cudaEventRecord(join, side));
    // Slot digests: level 0 of the slot tree, or the list roots when n = 1.
    {
        StageTimer tm(ctx, 9, s);
        k_snap_slots<<<sgrid(N, 128), 128, 0, s>>>(rec, d->M, d->log_n, N, d->log_n ? slot_tree : st->list_roots);
        CKS(cudaGetLastError());
        tm.done();
        ctx->launches++;
    }
    if (d->log_n) {
        Batch b;
        b.leaves_ready = true;
        b.tree.push_back(digest_tree(slot_tree, st->list_roots, lN, ln));
        r = launch_batch(ctx, b, s);
        if (r) return bail(r);
    }
    // Centroid binding: level 0 of the top tree, or root_mk when nlist = 1.
    k_snap_centroids<<<sgrid(nlist, 128), 128, 0, s>>>(mu, d->D, st->list_roots, (u32)nlist,
                                                       ln ? st->top_tree : st->root_mk);
    CKS(cudaGetLastError());
    ctx->launches++;
    if (ln) {
        Batch b;
        b.leaves_ready = true;
        b.tree.push_back(digest_tree(st->top_tree, st->root_mk, ln, 0));
        r = launch_batch(ctx, b, s);
        if (r) return bail(r);
    }
    CKS(cudaStreamWaitEvent(s, join, 0));
    if (scratch) CKS(cudaFreeAsync(scratch, s));
    scratch = nullptr;
    CKS(cudaEventRecord(st->ev, s));
#undef CKS
    st->id = ctx->next_id++;
    ctx->resident += st->bytes;
    ctx->snaps[st->id] = st;
    *out = st->id;
    return cleanup(V3C_OK);
}

v3c_status v3c_snapshot_roots(v3c_ctx* ctx, v3c_snapshot_id id, uint64_t* h_root_mk, uint64_t* h_root_cb)
{
    if (!ctx) return V3C_EINVAL;
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    SnapState* st = find_snap(ctx, id);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "snapshot id %llu", (unsigned long long)id);
    CK(cudaEventSynchronize(st->ev));
    if (h_root_mk) CK(cudaMemcpy(h_root_mk, st->root_mk, 32, cudaMemcpyDeviceToHost));
    if (h_root_cb) CK(cudaMemcpy(h_root_cb, st->root_cb, 32, cudaMemcpyDeviceToHost));
    return V3C_OK;
}

v3c_status v3c_snapshot_list_roots(v3c_ctx* ctx, v3c_snapshot_id id, uint64_t* h_roots)
{
    if (!ctx || !h_roots) return V3C_EINVAL;
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    SnapState* st = find_snap(ctx, id);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "snapshot id %llu", (unsigned long long)id);
    CK(cudaEventSynchronize(st->ev));
    CK(cudaMemcpy(h_roots, st->list_roots, ((size_t)4 << st->log_nlist) * 8, cudaMemcpyDeviceToHost));
    return V3C_OK;
}

v3c_status v3c_snapshot_open_lists(v3c_ctx* ctx, v3c_snapshot_id id, const uint32_t* h_lists, uint32_t nq,
                                   uint64_t* h_paths)
{
    if (!ctx) return V3C_EINVAL;
    if (nq && (!h_lists || !h_paths)) return fail(ctx, V3C_EINVAL, "v3c_snapshot_open_lists: NULL argument");
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    SnapState* st = find_snap(ctx, id);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "snapshot id %llu", (unsigned long long)id);
    for (u32 q = 0; q < nq; q++)
        if (h_lists[q] >> st->log_nlist) return fail(ctx, V3C_EINVAL, "v3c_snapshot_open_lists: list %u out of range", q);
    if (!nq || !st->log_nlist) return V3C_OK;
    if (!ctx->release_stream) CK(cudaStreamCreateWithFlags(&ctx->release_stream, cudaStreamNonBlocking));
    cudaStream_t s = ctx->release_stream;
    const size_t words = (size_t)nq * 4 * st->log_nlist;
    u64* dmem = nullptr;
    CK(cudaMallocAsync((void**)&dmem, words * 8 + ((size_t)nq * 4 + 7) / 8 * 8, s));
    u32* d_lists = reinterpret_cast<u32*>(dmem + words);
    CK(cudaStreamWaitEvent(s, st->ev, 0));
    cudaError_t e = cudaMemcpyAsync(d_lists, h_lists, (size_t)nq * 4, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        StageTimer tm(ctx, 7, s);
        k_snap_paths<<<sgrid(words, 256), 256, 0, s>>>(st->top_tree, st->log_nlist, d_lists, nq, dmem);
        e = cudaGetLastError();
        tm.done();
        ctx->launches++;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_paths, dmem, words * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(dmem, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "v3c_snapshot_open_lists: %s", cudaGetErrorString(e));
    return V3C_OK;
}

v3c_status v3c_snapshot_release(v3c_ctx* ctx, v3c_snapshot_id id)
{
    if (!ctx) return V3C_EINVAL;
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    SnapState* st = find_snap(ctx, id);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "snapshot id %llu", (unsigned long long)id);
    ctx->snaps.erase(id);
    if (!ctx->release_stream) CK(cudaStreamCreateWithFlags(&ctx->release_stream, cudaStreamNonBlocking));
    CK(cudaStreamWaitEvent(ctx->release_stream, st->ev, 0));
    CK(cudaFreeAsync(st->mem, ctx->release_stream));
    CK(cudaEventDestroy(st->ev));
    ctx->resident -= st->bytes;
    delete st;
    return V3C_OK;
}

}  // extern "C"
