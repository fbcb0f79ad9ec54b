// Poseidon-w12 leaf hashing and Merkle levels.
//
// The paper commits with Poseidon (Sec. 4.3) in balanced Merkle trees
// opened by the bits of the leaf index (Sec. 4.3; Sec. 4.4, MerkleOpen).
// Here the tree is built over the rows of the LDE and cut at a cap.
//
// GB300 mapping: this is 64-bit modular integer work with no dense
// contraction, so it runs on the integer pipes: one thread owns one 12-lane
// state in registers.  The MDS row has entries below 64, so every MDS
// product is two 32x32->64 multiply-adds into 42-bit accumulators, with one
// special-form fold per output lane.  Inside the permutation values stay
// non-canonical in [0, 2^64); digests are made canonical on output.  The
// round loop is not unrolled, which keeps the kernel's code small enough to
// stay resident in the instruction cache.  Round constants come from
// constant memory as uniform loads.
#include <cuda_runtime.h>
#include <algorithm>

#include "gl.cuh"
#include "internal.h"
#include "poseidon_params.h"  // generated at build time by gen_params.cpp

namespace v3c {

using gl::u32;
using gl::u64;

__constant__ u64 c_rc[30][12] = V3C_RC_INIT;

__host__ __device__ constexpr u32 mds_coef(int k)
{
    constexpr u32 row[12] = V3C_MDS_ROW_INIT;
    return row[k];
}

// L + H * 2^32 for L, H < 2^42, folded to a value in [0, 2^64).
__device__ __forceinline__ u64 mds_fold(u64 L, u64 H)
{
    u32 hl = (u32)H, hh = (u32)(H >> 32);
    u64 v = L + ((u64)hl << 32);
    u32 c = v < L;
    u32 x = hh + c;              // < 2^11: the multiple of 2^64 still to fold
    u64 t = ((u64)x << 32) - x;  // x * (2^64 mod p)
    u64 r = v + t;
    if (r < t) r += gl::EPS;
    return r;
}

// s <- M s with M[i][j] = m[(j - i) mod 12].
__device__ __forceinline__ void mds(u64 (&s)[12])
{
    u32 lo[12], hi[12];
#pragma unroll
    for (int j = 0; j < 12; j++) {
        lo[j] = (u32)s[j];
        hi[j] = (u32)(s[j] >> 32);
    }
#pragma unroll
    for (int i = 0; i < 12; i++) {
        u64 L = 0, H = 0;
#pragma unroll
        for (int j = 0; j < 12; j++) {
            const u32 m = mds_coef((j - i + 12) % 12);
            L += (u64)lo[j] * m;
            H += (u64)hi[j] * m;
        }
        s[i] = mds_fold(L, H);
    }
}

__device__ __forceinline__ u64 sbox(u64 x)
{
    u64 x2 = gl::mul_nc(x, x);
    u64 x3 = gl::mul_nc(x2, x);
    u64 x4 = gl::mul_nc(x2, x2);
    return gl::mul_nc(x3, x4);
}

__device__ __forceinline__ void full_round(u64 (&s)[12], int r)
{
#pragma unroll
    for (int i = 0; i < 12; i++) s[i] = sbox(gl::add_nc_small(s[i], c_rc[r][i]));
    mds(s);
}

__device__ __forceinline__ void partial_round(u64 (&s)[12], int r)
{
#pragma unroll
    for (int i = 0; i < 12; i++) s[i] = gl::add_nc_small(s[i], c_rc[r][i]);
    s[0] = sbox(s[0]);
    mds(s);
}

// Rounds 0-3 and 26-29 full, 4-25 partial.
__device__ __forceinline__ void permute(u64 (&s)[12])
{
#pragma unroll 1
    for (int r = 0; r < 4; r++) full_round(s, r);
#pragma unroll 1
    for (int r = 4; r < 26; r++) partial_round(s, r);
#pragma unroll 1
    for (int r = 26; r < 30; r++) full_round(s, r);
}

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

// Offset (in u64) of tree level k below the cap, or the cap itself.
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
__global__ void __launch_bounds__(128) k_leaf_hash(const TreeJob* __restrict__ jobs, StageList L)
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
        for (u32 st = 0; st < width; st += 8) {
            u32 len = min(8u, width - st);
            u64 v[8];
            if (J.vec_ok) {
#pragma unroll
                for (u32 k = 0; k < 4; k++) {
                    if (2 * k < len) {
                        ulonglong2 p = __ldg(reinterpret_cast<const ulonglong2*>(src + st + 2 * k));
                        v[2 * k] = p.x;
                        v[2 * k + 1] = p.y;
                    }
                }
            } else {
#pragma unroll
                for (u32 k = 0; k < 8; k++)
                    if (k < len) v[k] = __ldg(src + st + k);
            }
#pragma unroll
            for (u32 k = 0; k < 8; k++)
                if (k < len) s[k] = v[k];
            permute(s);
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
// to T digests of level lev0+1, then keeps halving in shared memory for up
// to nlev levels.  Every level is written to its place in the level-major
// tree, or to the cap for the top level.
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
            permute(s);
            u64* dst = level_ptr(J, lev0 + 1) + (base + tid) * 4;
            store_digest(dst, s);
            sm[2 * tid] = make_ulonglong2(gl::canon(s[0]), gl::canon(s[1]));
            sm[2 * tid + 1] = make_ulonglong2(gl::canon(s[2]), gl::canon(s[3]));
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
                permute(s);
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

}  // namespace v3c
