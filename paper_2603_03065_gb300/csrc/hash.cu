// Poseidon-w12 leaf hashing and Merkle levels.
//
// The paper commits with Poseidon (Sec. 4.3) in balanced Merkle trees
// opened by the bits of the leaf index (Sec. 4.3; Sec. 4.4, MerkleOpen).
// Here the tree is built over the rows of the LDE and cut at a cap.
//
// GB300 mapping: this is 64-bit modular integer work with no dense
// contraction, so it runs on the integer pipes.  One thread owns one 12-lane
// state in registers (poseidon.cuh).  The leaf kernel reads each LDE row
// once, in 16-byte loads.  Large tree levels get one launch each with one
// compression per thread; middle levels are folded several per CTA in
// shared memory.  Levels of at most a few thousand nodes, whose time is the
// latency of one compression, take one warp per compression
// (poseidon_warp.cuh) and fold six levels per CTA.
#include <cuda_runtime.h>
#include <algorithm>

#include "gl.cuh"
#include "internal.h"
#include "poseidon.cuh"
#include "poseidon_warp.cuh"

namespace v3c {

using gl::u32;
using gl::u64;
typedef pos::Default PC;

__device__ __forceinline__ u32 find_job_t(const u32* first, u32 njobs, u32 item)
{
    u32 lo = 0, hi = njobs;
    while (hi - lo > 1) {
        u32 mid = (lo + hi) >> 1;
        if (first[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Tree level k below the cap, or the cap itself for k = log N - h.
// Level k starts at word 8N - 8N / 2^k of the level-major tree.
__device__ __forceinline__ u64* level_ptr(const TreeJob& J, u32 k)
{
    u32 top = J.log_N - J.h;
    if (k == top) return J.cap;
    u64 eightN = (u64)8 << J.log_N;
    return J.tree + (eightN - (eightN >> k));
}

__device__ __forceinline__ void store_digest(u64* dst, const u64 (&s)[12])
{
    *reinterpret_cast<ulonglong2*>(dst) = make_ulonglong2(gl::canon(s[0]), gl::canon(s[1]));
    *reinterpret_cast<ulonglong2*>(dst + 2) = make_ulonglong2(gl::canon(s[2]), gl::canon(s[3]));
}

// ---------------------------------------------------------------- leaf hash

u32 leaf_items(const TreeJob& j, const Tiles& t)
{
    u64 N = (u64)1 << j.log_N;
    return (u32)((N + t.h_threads - 1) / t.h_threads);
}

// One thread per row: sponge over the first `width` entries in chunks of 8
// (overwrite mode), digest = lanes 0..3.
__global__ void __launch_bounds__(128, 8) k_leaf_hash(const TreeJob* __restrict__ jobs, StageList L)
{
    for (u32 item = blockIdx.x; item < L.total; item += gridDim.x) {
        u32 jid = find_job_t(L.first, L.njobs, item);
        const TreeJob& J = jobs[jid];
        u64 row = (u64)(item - L.first[jid]) * blockDim.x + threadIdx.x;
        if (row >> J.log_N) continue;
        const u64* src = J.rows + row * J.ld;
        u64* dst = level_ptr(J, 0) + row * 4;
        const u32 width = J.width;
        u64 s[12];
#pragma unroll
        for (int i = 0; i < 12; i++) s[i] = 0;
        if (width <= 4) {
#pragma unroll
            for (u32 i = 0; i < 4; i++) s[i] = i < width ? src[i] : 0;
            store_digest(dst, s);
            continue;
        }
        const bool vec = J.vec_ok;
        for (u32 st = 0; st < width; st += 8) {
            // Overwrite lanes 0..len-1 with the next chunk of the row.
            const u32 len = min(8u, width - st);
            const u64* p = src + st;
            if (vec) {
#pragma unroll
                for (u32 k = 0; k < 4; k++) {
                    if (2 * k < len) {
                        // With len odd, 2k+1 = len <= width - st - 1 + 1 <= ld - st - 1:
                        // width is odd then and ld is even, so the pair stays in the row.
                        ulonglong2 q = __ldg(reinterpret_cast<const ulonglong2*>(p + 2 * k));
                        s[2 * k] = q.x;
                        if (2 * k + 1 < len) s[2 * k + 1] = q.y;
                    }
                }
            } else {
#pragma unroll
                for (u32 k = 0; k < 8; k++)
                    if (k < len) s[k] = __ldg(p + k);
            }
            pos::permute<PC>(s);
        }
        store_digest(dst, s);
    }
}

cudaError_t launch_leaf_hash(const TreeJob* d_jobs, StageList l, const Tiles& t, int grid, cudaStream_t s)
{
    if (l.total == 0) return cudaSuccess;
    if (grid <= 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_leaf_hash, t.h_threads, 0);
        if (e != cudaSuccess) return e;
        grid = std::max(nb, 1) * num_sms();
    }
    grid = (int)std::min<u32>((u32)grid, l.total);
    k_leaf_hash<<<grid, t.h_threads, 0, s>>>(d_jobs, l);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Merkle levels

u32 merkle_items(const TreeJob& j, u32 lev0, const Tiles& t)
{
    u32 top = j.log_N - j.h;
    if (top <= lev0) return 0;
    u64 cnt = (u64)1 << (j.log_N - lev0 - 1);  // nodes at level lev0 + 1
    return (u32)std::max<u64>(1, cnt / t.m_threads);
}

// Each CTA of T threads takes 2T digests of level lev0 and compresses them
// to T digests of level lev0+1.  With nlev > 1 it keeps halving in shared
// memory for up to nlev levels.  Every level is written to its place in
// the level-major tree, or to the cap for the top level.
__global__ void __launch_bounds__(128) k_merkle(const TreeJob* __restrict__ jobs, StageList L, u32 lev0, u32 nlev)
{
    __shared__ ulonglong2 sm[128 * 2];
    const u32 T = blockDim.x;
    const u32 tid = threadIdx.x;
    for (u32 item = blockIdx.x; item < L.total; item += gridDim.x) {
        u32 jid = find_job_t(L.first, L.njobs, item);
        const TreeJob& J = jobs[jid];
        u32 top = J.log_N - J.h;
        u64 cnt_out = (u64)1 << (J.log_N - lev0 - 1);
        u32 cnt1 = (u32)min((u64)T, cnt_out);
        u64 base = (u64)(item - L.first[jid]) * T;
        u32 levels = min(nlev, top - lev0);
        levels = min(levels, (u32)(__ffs(cnt1) - 1) + 1);
        const u64* in = level_ptr(J, lev0);
        u64 s[12];
        if (tid < cnt1) {
            const ulonglong2* src = reinterpret_cast<const ulonglong2*>(in + (base + tid) * 8);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                ulonglong2 p = __ldg(src + k);
                s[2 * k] = p.x;
                s[2 * k + 1] = p.y;
            }
#pragma unroll
            for (int k = 8; k < 12; k++) s[k] = 0;
            pos::permute<PC>(s);
            u64* dst = level_ptr(J, lev0 + 1) + (base + tid) * 4;
            store_digest(dst, s);
            if (levels > 1) {
                sm[2 * tid] = make_ulonglong2(gl::canon(s[0]), gl::canon(s[1]));
                sm[2 * tid + 1] = make_ulonglong2(gl::canon(s[2]), gl::canon(s[3]));
            }
        }
        for (u32 l = 2; l <= levels; l++) {
            __syncthreads();
            u32 cnt = cnt1 >> (l - 1);
            if (tid < cnt) {
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    ulonglong2 p = sm[4 * tid + k];
                    s[2 * k] = p.x;
                    s[2 * k + 1] = p.y;
                }
#pragma unroll
                for (int k = 8; k < 12; k++) s[k] = 0;
                pos::permute<PC>(s);
            }
            __syncthreads();
            if (tid < cnt) {
                u64* dst = level_ptr(J, lev0 + l) + ((base >> (l - 1)) + tid) * 4;
                store_digest(dst, s);
                sm[2 * tid] = make_ulonglong2(gl::canon(s[0]), gl::canon(s[1]));
                sm[2 * tid + 1] = make_ulonglong2(gl::canon(s[2]), gl::canon(s[3]));
            }
        }
        __syncthreads();
    }
}

cudaError_t launch_merkle(const TreeJob* d_jobs, StageList l, u32 lev0, u32 nlev, const Tiles& t, int grid,
                          cudaStream_t s)
{
    if (l.total == 0) return cudaSuccess;
    if (grid <= 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_merkle, t.m_threads, 0);
        if (e != cudaSuccess) return e;
        grid = std::max(nb, 1) * num_sms();
    }
    grid = (int)std::min<u32>((u32)grid, l.total);
    k_merkle<<<grid, t.m_threads, 0, s>>>(d_jobs, l, lev0, nlev);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- small levels

u32 merkle_warp_items(const TreeJob& j, u32 lev0)
{
    u32 top = j.log_N - j.h;
    if (top <= lev0) return 0;
    u64 cnt = (u64)1 << (j.log_N - lev0 - 1);  // nodes at level lev0 + 1
    return (u32)std::max<u64>(1, cnt / kMerkleWarps);
}

// Each CTA takes kMerkleWarps nodes of level lev0+1 (fewer at the top of a
// tree); warp w computes node w, the warp sharing the permutation
// (poseidon_warp.cuh), and the CTA keeps halving in shared memory.  Every
// level is written to its place in the level-major tree, or to the cap.
__global__ void __launch_bounds__(kMerkleWarps * 32) k_merkle_warp(const TreeJob* __restrict__ jobs, StageList L,
                                                                   u32 lev0, u32 nlev)
{
    __shared__ pos::WarpRc s_rc;
    __shared__ u64 s_dig[kMerkleWarps * 4];
    pos::warp_rc_init(s_rc, threadIdx.x, blockDim.x);
    __syncthreads();
    const u32 w = threadIdx.x >> 5, l = threadIdx.x & 31;
    u32 m[12];
    pos::warp_mds_row(m, l);
    for (u32 item = blockIdx.x; item < L.total; item += gridDim.x) {
        const u32 jid = find_job_t(L.first, L.njobs, item);
        const TreeJob& J = jobs[jid];
        const u32 top = J.log_N - J.h;
        const u64 cnt_out = (u64)1 << (J.log_N - lev0 - 1);
        const u32 cnt1 = (u32)min((u64)kMerkleWarps, cnt_out);
        const u64 base = (u64)(item - L.first[jid]) * kMerkleWarps;
        u32 levels = min(nlev, top - lev0);
        levels = min(levels, (u32)(__ffs(cnt1) - 1) + 1);
        const u64* in = level_ptr(J, lev0);
        for (u32 lv = 1; lv <= levels; lv++) {
            const u32 cnt = cnt1 >> (lv - 1);
            const bool act = w < cnt;  // warp-uniform
            u64 x = 0;                 // lanes 0-7: the two child digests; 8-11: zero
            if (act && l < 8) x = lv == 1 ? __ldg(in + (base + w) * 8 + l) : s_dig[8 * w + l];
            if (act) x = pos::permute_warp(x, s_rc, m, l);
            __syncthreads();  // every read of s_dig for this level is done
            if (act && l < 4) {
                const u64 d = gl::canon(x);
                level_ptr(J, lev0 + lv)[((base >> (lv - 1)) + w) * 4 + l] = d;
                s_dig[4 * w + l] = d;
            }
            __syncthreads();
        }
    }
}

cudaError_t launch_merkle_warp(const TreeJob* d_jobs, StageList l, u32 lev0, u32 nlev, int grid, cudaStream_t s)
{
    if (l.total == 0) return cudaSuccess;
    if (grid <= 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_merkle_warp, kMerkleWarps * 32, 0);
        if (e != cudaSuccess) return e;
        grid = std::max(nb, 1) * num_sms();
    }
    grid = (int)std::min<u32>((u32)grid, l.total);
    k_merkle_warp<<<grid, kMerkleWarps * 32, 0, s>>>(d_jobs, l, lev0, nlev);
    return cudaGetLastError();
}

}  // namespace v3c
