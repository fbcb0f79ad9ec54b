// FRI commit phase on resident commitments, and batched Merkle openings.
//
// The prover of the paper runs Plonky2 with its default FRI setup (Sec. 5,
// evaluation environment); the commitments it opens are the Merkle trees of
// Sec. 4.3, opened by the bits of the leaf index (Sec. 4.4, MerkleOpen).
// The FRI steps are the textbook commit phase (Ben-Sasson et al., ICALP
// 2018): a random linear combination of the committed columns, then folds
// f -> sum_i beta^i f_i of f = sum_i X^i f_i(X^(2^a)), each layer committed
// with the same Poseidon Merkle kernels as the LDE.
//
// GB300 mapping: the combination streams the whole resident LDE once (the
// only HBM-heavy step): the tensor-memory accelerator copies tiles of 256
// rows x 16 words into a ring of shared-memory stages and each thread sums
// one row into an unreduced 192-bit accumulator (register loads, one row per
// thread, where a shape does not fit a tensor map).  A fold reads each coset (2^a
// contiguous values) into registers and applies a arity-2 steps there, one
// output per thread.  The layer
// trees go through the batched leaf-hash and Merkle launches.  Openings are
// one gather launch per call over every (query, word) pair.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/v3c_fri.h"
#include "ctx.h"
#include "gl.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace v3c {

using gl::u32;
using gl::u64;

struct FriState {
    u64 id = 0;
    u32 rounds = 0, done = 0, log_N = 0, ncols = 0;
    u32 ext = 1;  // extension degree of the layers: 1 (F_p) or 2 (F_p[u]/(u^2 - 7))
    u32 arity[V3C_FRI_MAX_ROUNDS] = {0};
    u32 log_size[V3C_FRI_MAX_ROUNDS + 1] = {0};
    u32 h[V3C_FRI_MAX_ROUNDS] = {0};
    u64 shift[V3C_FRI_MAX_ROUNDS + 1] = {0};  // s_k
    u64* mem = nullptr;
    size_t bytes = 0;
    u64* f[V3C_FRI_MAX_ROUNDS + 1] = {nullptr};
    u64* tree[V3C_FRI_MAX_ROUNDS] = {nullptr};
    u64* cap[V3C_FRI_MAX_ROUNDS] = {nullptr};
    u64* final_coef = nullptr;
    u64* pw_inv = nullptr;  // [3][512] powers of w_N^-1
    u64* alpha_pw = nullptr;
    u32* err = nullptr;  // set by a combine whose bounded wait expired
    bool err_checked = false;
    u32 committed = 0;  // layers [0, committed) have trees
    u64 query_words = 0;
    cudaEvent_t ev = nullptr;
};

// ---------------------------------------------------------------- kernels

// out[i] = alpha^i.
__global__ void k_fri_powers(u64 alpha, u32 count, u64* out)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        out[i] = gl::pow(alpha, i);
}

// (a0 + a1 u)(b0 + b1 u) in F_p[u] / (u^2 - 7); canonical in and out.
__device__ __forceinline__ void ext_mul_d(u64 a0, u64 a1, u64 b0, u64 b1, u64& r0, u64& r1)
{
    const u64 x = gl::add(gl::mul(a0, b0), gl::mul(7, gl::mul(a1, b1)));
    r1 = gl::add(gl::mul(a0, b1), gl::mul(a1, b0));
    r0 = x;
}

// out[2i], out[2i+1] = alpha^i in the quadratic extension.
__global__ void k_fri_powers_ext(u64 a0, u64 a1, u32 count, u64* out)
{
    for (u32 i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        u64 r0 = 1, r1 = 0, x0 = a0, x1 = a1;
        for (u32 e = i; e; e >>= 1) {
            if (e & 1) ext_mul_d(r0, r1, x0, x1, r0, r1);
            ext_mul_d(x0, x1, x0, x1, x0, x1);
        }
        out[2 * i] = r0;
        out[2 * i + 1] = r1;
    }
}

// pw[512 l + j] = winv^((j << 9 l) mod N): w_N^-e for e < 2^27 is then the
// product of pw[e mod 2^9], pw[512 + (e >> 9) mod 2^9], pw[1024 + (e >> 18)].
__global__ void k_fri_root_tables(u64 winv, u32 log_N, u64* pw)
{
    u32 i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 1536) return;
    u64 e = ((u64)(i & 511) << (9 * (i >> 9))) & (((u64)1 << log_N) - 1);
    pw[i] = gl::pow(winv, e);
}

__device__ __forceinline__ u64 pow3(const u64* __restrict__ pw, u64 e)
{
    u64 r = gl::mul(__ldg(pw + (e & 511)), __ldg(pw + 512 + ((e >> 9) & 511)));
    return gl::mul(r, __ldg(pw + 1024 + (e >> 18)));
}

using gl::fold192;
using gl::mac192;

// Column pairs loaded per iteration of the combine: 4 pairs are one 64-byte
// run (two whole sectors) per thread; 8 measured no faster.
constexpr int kCombPairs = 4;

// f[t] (+)= sum_{i<c} pw[i] row_t[i].  One thread per row: 16-byte loads of
// column pairs, kCombPairs pairs per iteration, products summed unreduced
// and reduced once per row.  The powers pw[i] are the same for every thread
// of a warp (broadcast loads).
// Rows are 16-byte aligned (ld even); c < 2^31.
__global__ void __launch_bounds__(256) k_fri_combine(const u64* __restrict__ rows, u32 ld, u32 c,
                                                     const u64* __restrict__ pw, u64 nrows, int acc,
                                                     u64* __restrict__ f)
{
    const u32 pairs = c >> 1;
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < nrows; t += (u64)gridDim.x * blockDim.x) {
        const ulonglong2* row = reinterpret_cast<const ulonglong2*>(rows + t * ld);
        u64 lo = 0, mid = 0;
        u32 hi = 0;
        u32 k = 0;
        for (; k + kCombPairs <= pairs; k += kCombPairs) {
            ulonglong2 v[kCombPairs];
#pragma unroll
            for (int j = 0; j < kCombPairs; j++) v[j] = __ldg(row + k + j);
#pragma unroll
            for (int j = 0; j < kCombPairs; j++) {
                mac192(lo, mid, hi, v[j].x, __ldg(pw + 2 * (k + j)));
                mac192(lo, mid, hi, v[j].y, __ldg(pw + 2 * (k + j) + 1));
            }
        }
        for (; k < pairs; k++) {
            ulonglong2 v = __ldg(row + k);
            mac192(lo, mid, hi, v.x, __ldg(pw + 2 * k));
            mac192(lo, mid, hi, v.y, __ldg(pw + 2 * k + 1));
        }
        if (c & 1) mac192(lo, mid, hi, __ldg(rows + t * ld + c - 1), __ldg(pw + c - 1));
        u64 r = fold192(lo, mid, hi);
        f[t] = acc ? gl::add(f[t], r) : r;
    }
}

// f[t] (+)= sum_{i<c} alpha^i row_t[i] with alpha^i in the extension (pw
// holds (re, im) pairs): the same row walk as k_fri_combine with two
// unreduced sums, one per component.  Two 64x64 products per element make
// it IMAD-bound rather than HBM-bound (two lanes per row measured slower).
__global__ void __launch_bounds__(256) k_fri_combine_ext(const u64* __restrict__ rows, u32 ld, u32 c,
                                                         const u64* __restrict__ pw, u64 nrows, int acc,
                                                         u64* __restrict__ f)
{
    const u32 pairs = c >> 1;
    const ulonglong2* pw2 = reinterpret_cast<const ulonglong2*>(pw);
    for (u64 t = blockIdx.x * (u64)blockDim.x + threadIdx.x; t < nrows; t += (u64)gridDim.x * blockDim.x) {
        const ulonglong2* row = reinterpret_cast<const ulonglong2*>(rows + t * ld);
        u64 lo0 = 0, mid0 = 0, lo1 = 0, mid1 = 0;
        u32 hi0 = 0, hi1 = 0;
        u32 k = 0;
        for (; k + kCombPairs <= pairs; k += kCombPairs) {
            ulonglong2 v[kCombPairs];
#pragma unroll
            for (int j = 0; j < kCombPairs; j++) v[j] = __ldg(row + k + j);
#pragma unroll
            for (int j = 0; j < kCombPairs; j++) {
                const ulonglong2 p0 = __ldg(pw2 + 2 * (k + j)), p1 = __ldg(pw2 + 2 * (k + j) + 1);
                mac192(lo0, mid0, hi0, v[j].x, p0.x);
                mac192(lo1, mid1, hi1, v[j].x, p0.y);
                mac192(lo0, mid0, hi0, v[j].y, p1.x);
                mac192(lo1, mid1, hi1, v[j].y, p1.y);
            }
        }
        for (; k < pairs; k++) {
            const ulonglong2 v = __ldg(row + k);
            const ulonglong2 p0 = __ldg(pw2 + 2 * k), p1 = __ldg(pw2 + 2 * k + 1);
            mac192(lo0, mid0, hi0, v.x, p0.x);
            mac192(lo1, mid1, hi1, v.x, p0.y);
            mac192(lo0, mid0, hi0, v.y, p1.x);
            mac192(lo1, mid1, hi1, v.y, p1.y);
        }
        if (c & 1) {
            const u64 x = __ldg(rows + t * ld + c - 1);
            const ulonglong2 p0 = __ldg(pw2 + c - 1);
            mac192(lo0, mid0, hi0, x, p0.x);
            mac192(lo1, mid1, hi1, x, p0.y);
        }
        u64 r0 = fold192(lo0, mid0, hi0), r1 = fold192(lo1, mid1, hi1);
        if (acc) {
            r0 = gl::add(f[2 * t], r0);
            r1 = gl::add(f[2 * t + 1], r1);
        }
        reinterpret_cast<ulonglong2*>(f)[t] = make_ulonglong2(r0, r1);
    }
}

// Column pairs per iteration of the two-row combine (2.26 ms on 135 x 2^20
// against 2.38 ms with 4 and 2.37 ms with 8).
constexpr int kCombPairs2 = 2;

// The same combination with two adjacent rows per thread: each 16-byte load
// of alpha powers serves both rows, and the two rows' accumulator chains are
// independent work for the same instructions' latencies.
__global__ void __launch_bounds__(256, 2) k_fri_combine_ext2(const u64* __restrict__ rows, u32 ld, u32 c,
                                                             const u64* __restrict__ pw, u64 nrows, int acc,
                                                             u64* __restrict__ f)
{
    const u32 pairs = c >> 1;
    const ulonglong2* pw2 = reinterpret_cast<const ulonglong2*>(pw);
    for (u64 t = 2 * (blockIdx.x * (u64)blockDim.x + threadIdx.x); t < nrows; t += 2 * (u64)gridDim.x * blockDim.x) {
        const bool two = t + 1 < nrows;
        const ulonglong2* ra = reinterpret_cast<const ulonglong2*>(rows + t * ld);
        const ulonglong2* rb = reinterpret_cast<const ulonglong2*>(rows + (two ? t + 1 : t) * ld);
        u64 la0 = 0, ma0 = 0, la1 = 0, ma1 = 0, lb0 = 0, mb0 = 0, lb1 = 0, mb1 = 0;
        u32 ha0 = 0, ha1 = 0, hb0 = 0, hb1 = 0;
        u32 k = 0;
        for (; k + kCombPairs2 <= pairs; k += kCombPairs2) {
            ulonglong2 va[kCombPairs2], vb[kCombPairs2];
#pragma unroll
            for (int j = 0; j < kCombPairs2; j++) {
                va[j] = __ldg(ra + k + j);
                vb[j] = __ldg(rb + k + j);
            }
#pragma unroll
            for (int j = 0; j < kCombPairs2; j++) {
                const ulonglong2 p0 = __ldg(pw2 + 2 * (k + j)), p1 = __ldg(pw2 + 2 * (k + j) + 1);
                mac192(la0, ma0, ha0, va[j].x, p0.x);
                mac192(la1, ma1, ha1, va[j].x, p0.y);
                mac192(la0, ma0, ha0, va[j].y, p1.x);
                mac192(la1, ma1, ha1, va[j].y, p1.y);
                mac192(lb0, mb0, hb0, vb[j].x, p0.x);
                mac192(lb1, mb1, hb1, vb[j].x, p0.y);
                mac192(lb0, mb0, hb0, vb[j].y, p1.x);
                mac192(lb1, mb1, hb1, vb[j].y, p1.y);
            }
        }
        for (; k < pairs; k++) {
            const ulonglong2 a = __ldg(ra + k), b = __ldg(rb + k);
            const ulonglong2 p0 = __ldg(pw2 + 2 * k), p1 = __ldg(pw2 + 2 * k + 1);
            mac192(la0, ma0, ha0, a.x, p0.x);
            mac192(la1, ma1, ha1, a.x, p0.y);
            mac192(la0, ma0, ha0, a.y, p1.x);
            mac192(la1, ma1, ha1, a.y, p1.y);
            mac192(lb0, mb0, hb0, b.x, p0.x);
            mac192(lb1, mb1, hb1, b.x, p0.y);
            mac192(lb0, mb0, hb0, b.y, p1.x);
            mac192(lb1, mb1, hb1, b.y, p1.y);
        }
        if (c & 1) {
            const u64 xa = __ldg(rows + t * ld + c - 1), xb = __ldg(rows + (two ? t + 1 : t) * ld + c - 1);
            const ulonglong2 p0 = __ldg(pw2 + c - 1);
            mac192(la0, ma0, ha0, xa, p0.x);
            mac192(la1, ma1, ha1, xa, p0.y);
            mac192(lb0, mb0, hb0, xb, p0.x);
            mac192(lb1, mb1, hb1, xb, p0.y);
        }
        u64 r0 = fold192(la0, ma0, ha0), r1 = fold192(la1, ma1, ha1);
        u64 s0 = fold192(lb0, mb0, hb0), s1 = fold192(lb1, mb1, hb1);
        if (acc) {
            r0 = gl::add(f[2 * t], r0);
            r1 = gl::add(f[2 * t + 1], r1);
            if (two) {
                s0 = gl::add(f[2 * t + 2], s0);
                s1 = gl::add(f[2 * t + 3], s1);
            }
        }
        reinterpret_cast<ulonglong2*>(f)[t] = make_ulonglong2(r0, r1);
        if (two) reinterpret_cast<ulonglong2*>(f)[t + 1] = make_ulonglong2(s0, s1);
    }
}

// ------------------------------------------- combination fed by TMA tiles
//
// The register-load kernels above give each thread its own row, so one warp
// load touches 32 rows (32 cache lines) and the L1's per-line throughput,
// not DRAM, bounds them.  Here the tensor-memory accelerator copies tiles of
// kTmaRows rows x kTmaCols words (one 128-byte line per row) from the LDE
// into a ring of shared-memory stages, with the 128-byte swizzle: 16-byte
// unit u of tile row r lands at unit u ^ (r mod 8) of that row's line, so the
// eight threads of each quarter-warp phase (rows r..r+7, same unit) read
// eight different bank groups.  One producer thread issues the copies;
// consumer thread t owns tile row t and sums its words into the same
// unreduced 192-bit accumulators as the register-load kernels.  Every wait
// is bounded in time: on expiry the CTA records an error and stops, and the
// producer waits (bounded) for the copies it issued before the CTA exits.
constexpr u32 kTmaCols = 16;                        // words per tile row (128 bytes)
constexpr u32 kTmaRows = 256;                       // tile rows = consumer threads
constexpr u32 kTmaStages = 3;
constexpr u32 kTmaBytes = kTmaCols * kTmaRows * 8;  // 32 KB per stage
constexpr u32 kTmaThreads = kTmaRows + 32;          // consumers + one producer warp
constexpr size_t kTmaSmem = (size_t)kTmaStages * kTmaBytes + 1024 + 128;
constexpr u64 kTmaWaitNs = 1000000000ull;           // 1 s per wait

struct TmaRing {
    u64 full[kTmaStages];   // copy landed (producer's expect_tx + the copy's bytes)
    u64 empty[kTmaStages];  // every consumer has read the stage
    u32 abort;
    u32 issued;
};

// f[t] (+)= sum_{i<c} alpha^i row_t[i] (EXT words per alpha power and per
// output) over tiles of kTmaRows rows; requires c >= kTmaCols and
// nrows >= kTmaRows (the host takes the register-load kernels otherwise).
template <int EXT>
__global__ void __launch_bounds__(kTmaThreads, 2) k_fri_combine_tma(const __grid_constant__ CUtensorMap map, u32 c,
                                                                   const u64* __restrict__ pw, u64 nrows, int acc,
                                                                   u64* __restrict__ f, u32* __restrict__ err)
{
    extern __shared__ unsigned char tma_raw[];
    unsigned char* stage0 =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tma_raw) + 1023) & ~(uintptr_t)1023);
    TmaRing* ring = reinterpret_cast<TmaRing*>(stage0 + (size_t)kTmaStages * kTmaBytes);
    const u32 tiles = (u32)((nrows + kTmaRows - 1) / kTmaRows);
    const u32 chunks = (c + kTmaCols - 1) / kTmaCols;
    const u32 my_tiles = blockIdx.x < tiles ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const u32 items = my_tiles * chunks;
    if (threadIdx.x == 0) {
        for (u32 s = 0; s < kTmaStages; s++) {
            mbar_init(&ring->full[s], 1);
            mbar_init(&ring->empty[s], kTmaRows);
        }
        ring->abort = 0;
        ring->issued = 0;
        mbar_init_fence();
    }
    __syncthreads();
    volatile u32* abort = &ring->abort;
    if (threadIdx.x >= kTmaRows) {
        // Producer: one thread issues every copy of this CTA, in item order.
        if (threadIdx.x == kTmaRows) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<u64>(&map)) : "memory");
            u32 issued = 0;
            for (u32 it = 0; it < items; it++) {
                const u32 s = it % kTmaStages;
                if (it >= kTmaStages && !mbar_wait(&ring->empty[s], ((it / kTmaStages) - 1) & 1, kTmaWaitNs)) {
                    *abort = 1;
                    break;
                }
                if (*abort) break;
                const u32 tile = blockIdx.x + (it / chunks) * gridDim.x;
                mbar_expect_tx(&ring->full[s], kTmaBytes);
                tma_load_2d(stage0 + (size_t)s * kTmaBytes, &map, (it % chunks) * kTmaCols, tile * kTmaRows,
                            &ring->full[s]);
                issued = it + 1;
            }
            ring->issued = issued;
        }
    } else {
        const u32 t = threadIdx.x, sw = t & 7;
        u32 it = 0;
        for (u32 ti = 0; ti < my_tiles && !*abort; ti++) {
            const u64 row = (u64)(blockIdx.x + ti * gridDim.x) * kTmaRows + t;
            u64 l0 = 0, m0 = 0, l1 = 0, m1 = 0;
            u32 h0 = 0, h1 = 0;
            bool ok = true;
            for (u32 ch = 0; ch < chunks; ch++, it++) {
                const u32 s = it % kTmaStages;
                if (!mbar_wait(&ring->full[s], (it / kTmaStages) & 1, kTmaWaitNs)) {
                    *abort = 1;
                    ok = false;
                    break;
                }
                const ulonglong2* line = reinterpret_cast<const ulonglong2*>(stage0 + (size_t)s * kTmaBytes + t * 128);
                const u32 c0 = ch * kTmaCols;
                if (c0 + kTmaCols <= c) {
#pragma unroll
                    for (u32 u = 0; u < kTmaCols / 2; u++) {
                        const ulonglong2 v = line[u ^ sw];
                        if (EXT == 2) {
                            const ulonglong2* pw2 = reinterpret_cast<const ulonglong2*>(pw) + c0 + 2 * u;
                            const ulonglong2 p0 = __ldg(pw2), p1 = __ldg(pw2 + 1);
                            mac192(l0, m0, h0, v.x, p0.x);
                            mac192(l1, m1, h1, v.x, p0.y);
                            mac192(l0, m0, h0, v.y, p1.x);
                            mac192(l1, m1, h1, v.y, p1.y);
                        } else {
                            // pw + c0 may be 8-byte aligned only (an odd column offset).
                            mac192(l0, m0, h0, v.x, __ldg(pw + c0 + 2 * u));
                            mac192(l1, m1, h1, v.y, __ldg(pw + c0 + 2 * u + 1));
                        }
                    }
                } else {
                    // The last, partial chunk (words past c are the copy's zero fill).
                    for (u32 w = 0; c0 + w < c; w++) {
                        const u64 x = reinterpret_cast<const u64*>(line + ((w >> 1) ^ sw))[w & 1];
                        if (EXT == 2) {
                            const ulonglong2 p = __ldg(reinterpret_cast<const ulonglong2*>(pw) + c0 + w);
                            mac192(l0, m0, h0, x, p.x);
                            mac192(l1, m1, h1, x, p.y);
                        } else {
                            mac192(l0, m0, h0, x, __ldg(pw + c0 + w));
                        }
                    }
                }
                mbar_arrive(&ring->empty[s]);
            }
            if (!ok) break;
            if (row < nrows) {
                if (EXT == 2) {
                    u64 r0 = fold192(l0, m0, h0), r1 = fold192(l1, m1, h1);
                    if (acc) {
                        r0 = gl::add(f[2 * row], r0);
                        r1 = gl::add(f[2 * row + 1], r1);
                    }
                    reinterpret_cast<ulonglong2*>(f)[row] = make_ulonglong2(r0, r1);
                } else {
                    u64 r = gl::add(fold192(l0, m0, h0), fold192(l1, m1, h1));
                    f[row] = acc ? gl::add(f[row], r) : r;
                }
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == kTmaRows && *abort) {
        // Wait (bounded) for this CTA's copies still in flight: the last
        // issued copy of each stage is that stage's latest full phase.
        const u32 issued = ring->issued;
        for (u32 it = issued > kTmaStages ? issued - kTmaStages : 0; it < issued; it++)
            mbar_wait(&ring->full[it % kTmaStages], (it / kTmaStages) & 1, kTmaWaitNs);
        atomicOr(err, 1u);
    }
}

// Per-round fold constants.  Step m of a round pairs positions (2u, 2u+1) of
// the intermediate layer; with u = w 2^b + v' (b = a-1-m) the point of
// position 2u is x = s^(2^m) w_{2^(b+1)}^bitrev_b(v') (w_{N_k}^e)^(2^m),
// e = bitrev_{log N_{k+1}}(w).  K holds beta^(2^m) (2 s^(2^m))^-1
// w_{2^(b+1)}^-bitrev_b(v') for every (m, v'), steps in order.
struct FoldArgs {
    const u64* in;
    u64* out;
    const u64* pw_inv;
    u32 log_out;    // log2 N_{k+1}
    u32 exp_shift;  // log2 (N_0 / N_k)
    u64 inv2;
    u64 K[15][2];  // (re, im); im = 0 in the base field
};

// g(x^2) = (f(x) + f(-x)) / 2 + beta (f(x) - f(-x)) / (2x), applied a times
// in registers to one coset of 2^a values (EXT words each; x is in F_p).
template <int A_BITS, int EXT>
__global__ void __launch_bounds__(256) k_fri_fold(FoldArgs p)
{
    constexpr int A = 1 << A_BITS;
    const u64 nout = (u64)1 << p.log_out;
    for (u64 w = blockIdx.x * (u64)blockDim.x + threadIdx.x; w < nout; w += (u64)gridDim.x * blockDim.x) {
        u64 v[A][EXT];
        const ulonglong2* src = reinterpret_cast<const ulonglong2*>(p.in + ((w << A_BITS) * EXT));
#pragma unroll
        for (int k = 0; k < A * EXT / 2; k++) {
            ulonglong2 q = __ldg(src + k);
            v[(2 * k) / EXT][(2 * k) % EXT] = q.x;
            v[(2 * k + 1) / EXT][(2 * k + 1) % EXT] = q.y;
        }
        u64 e = (u64)gl::bitrev((u32)w, p.log_out) << p.exp_shift;
        u64 z = pow3(p.pw_inv, e);  // 1 / (w_{N_k}^e)
        int kidx = 0;
#pragma unroll
        for (int m = 0; m < A_BITS; m++) {
            const int half = A >> (m + 1);
#pragma unroll
            for (int u = 0; u < half; u++) {
                if (EXT == 1) {
                    u64 a0 = v[2 * u][0], a1 = v[2 * u + 1][0];
                    u64 t = gl::mul(p.K[kidx + u][0], z);
                    v[u][0] = gl::add(gl::mul(gl::add(a0, a1), p.inv2), gl::mul(gl::sub(a0, a1), t));
                } else {
                    const u64 t0 = gl::mul(p.K[kidx + u][0], z), t1 = gl::mul(p.K[kidx + u][EXT - 1], z);
                    const u64 s0 = gl::add(v[2 * u][0], v[2 * u + 1][0]);
                    const u64 s1 = gl::add(v[2 * u][EXT - 1], v[2 * u + 1][EXT - 1]);
                    const u64 d0 = gl::sub(v[2 * u][0], v[2 * u + 1][0]);
                    const u64 d1 = gl::sub(v[2 * u][EXT - 1], v[2 * u + 1][EXT - 1]);
                    u64 q0, q1;
                    ext_mul_d(d0, d1, t0, t1, q0, q1);
                    v[u][0] = gl::add(gl::mul(s0, p.inv2), q0);
                    v[u][EXT - 1] = gl::add(gl::mul(s1, p.inv2), q1);
                }
            }
            kidx += half;
            z = gl::mul(z, z);
        }
#pragma unroll
        for (int x = 0; x < EXT; x++) p.out[w * EXT + x] = v[0][x];
    }
}

// c_i = m^-1 s^-i sum_j E_j w_m^-ij with E_j = f[bitrev(j)]: the inverse DFT
// of the natural-order values, unshifted.  One CTA, m <= 1024.
// Extension values are interpolated componentwise (the DFT is linear over
// F_p): component `comp` of element j sits at f[ext j + comp].
__global__ void __launch_bounds__(256) k_fri_final(const u64* __restrict__ f, u32 logm, u64 winv, u64 sinv,
                                                   u64 minv, u64* __restrict__ out, u32 ext, u32 comp)
{
    __shared__ u64 E[1024];
    const u32 m = 1u << logm;
    for (u32 j = threadIdx.x; j < m; j += blockDim.x) E[j] = f[(size_t)ext * gl::bitrev(j, logm) + comp];
    __syncthreads();
    for (u32 i = threadIdx.x; i < m; i += blockDim.x) {
        u64 wi = gl::pow(winv, i), wij = 1, acc = 0;
        for (u32 j = 0; j < m; j++) {
            acc = gl::add(acc, gl::mul(E[j], wij));
            wij = gl::mul(wij, wi);
        }
        out[(size_t)ext * i + comp] = gl::mul(acc, gl::mul(gl::pow(sinv, i), minv));
    }
}

struct QueryLayer {
    const u64* f;
    const u64* tree;
    u64 word0;  // first word of this layer in a query's record
    u32 a, logL, h, tshift;  // arity bits, log2 leaves, cap height, sum of earlier arities
};
struct QueryArgs {
    QueryLayer L[V3C_FRI_MAX_ROUNDS];
    u32 R;
    u32 ext;
    u32 nq;
    u64 words;
    const u64* idx;
    u64* out;
};

// One thread per (query, word): the coset values of each layer's leaf, then
// the leaf's siblings up to the cap (level j starts at word 8L - 8L/2^j).
__global__ void k_fri_query(QueryArgs p)
{
    const u64 total = (u64)p.nq * p.words;
    for (u64 g = blockIdx.x * (u64)blockDim.x + threadIdx.x; g < total; g += (u64)gridDim.x * blockDim.x) {
        u64 q = g / p.words, o = g - q * p.words;
        u32 k = 0;
        while (k + 1 < p.R && p.L[k + 1].word0 <= o) k++;
        const QueryLayer& L = p.L[k];
        u64 off = o - L.word0;
        u64 leaf = (p.idx[q] >> L.tshift) >> L.a;
        u64 val;
        const u64 vw = ((u64)1 << L.a) * p.ext;  // value words of one leaf
        if (off < vw) {
            val = L.f[(leaf << L.a) * p.ext + off];
        } else {
            off -= vw;
            u32 lvl = (u32)(off >> 2), comp = (u32)(off & 3);
            u64 eightL = (u64)8 << L.logL;
            val = L.tree[(eightL - (eightL >> lvl)) + 4 * ((leaf >> lvl) ^ 1) + comp];
        }
        p.out[g] = val;
    }
}

// Rows and authentication paths of a list of leaves of one commitment.
__global__ void k_open_rows(const u64* __restrict__ lde, u32 ld, u32 c, const u64* __restrict__ tree, u32 log_N,
                            u32 h, const u64* __restrict__ idx, u32 nq, u64* __restrict__ rows_out,
                            u64* __restrict__ paths_out)
{
    const u32 plen = 4 * (log_N - h);
    const u64 per = (u64)c + plen;
    const u64 total = per * nq;
    for (u64 g = blockIdx.x * (u64)blockDim.x + threadIdx.x; g < total; g += (u64)gridDim.x * blockDim.x) {
        u64 q = g / per, o = g - q * per;
        u64 t = idx[q];
        if (o < c) {
            if (rows_out) rows_out[q * c + o] = lde[t * ld + o];
        } else if (paths_out) {
            o -= c;
            u32 lvl = (u32)(o >> 2), comp = (u32)(o & 3);
            u64 eightN = (u64)8 << log_N;
            paths_out[q * plen + o] = tree[(eightN - (eightN >> lvl)) + 4 * ((t >> lvl) ^ 1) + comp];
        }
    }
}

}  // namespace v3c

using namespace v3c::detail;

namespace {

// Host arithmetic in F_p[u] / (u^2 - 7).  The sums of two values below p
// are taken in 128 bits (they can exceed 2^64).
u64 h_add(u64 a, u64 b) { return (u64)(((unsigned __int128)a + b) % gl::P); }
void h_ext_mul(const u64* a, const u64* b, u64* r)
{
    const u64 r0 = h_add(gl::h_mul(a[0], b[0]), gl::h_mul(7, gl::h_mul(a[1], b[1])));
    const u64 r1 = h_add(gl::h_mul(a[0], b[1]), gl::h_mul(a[1], b[0]));
    r[0] = r0;
    r[1] = r1;
}

int grid_for(u64 work, int threads)
{
    u64 g = (work + threads - 1) / threads;
    return (int)std::max<u64>(1, std::min<u64>(g, (u64)num_sms() * 16));
}

// Enqueues round k's fold: f_{k+1} from f_k with challenge beta (st.ext words).
// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against the driver library).
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// The tensor map of an object's LDE for the TMA combination: c x N words,
// rows ld words apart, tiles of kTmaRows x kTmaCols with the 128-byte
// swizzle.  False when the shape or the buffer does not meet the copy
// engine's rules (16-byte aligned base and row pitch) or is smaller than one
// tile; the caller then takes the register-load kernel.
bool combine_map(const Object& o, u64 N, CUtensorMap* map)
{
    // Item counters are 32-bit: tiles x column chunks must stay below 2^32.
    const u64 items = ((N + kTmaRows - 1) / kTmaRows) * (((u64)o.c + kTmaCols - 1) / kTmaCols);
    if (o.c < kTmaCols || N < kTmaRows || N > 0xFFFFFFFFull || items >= (1ull << 32) || ((size_t)o.ld * 8) % 16 ||
        (reinterpret_cast<uintptr_t>(o.lde) & 15))
        return false;
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {o.c, N};
    const cuuint64_t pitch[1] = {(cuuint64_t)o.ld * 8};
    const cuuint32_t box[2] = {kTmaCols, kTmaRows};
    const cuuint32_t step[2] = {1, 1};
    if (fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, (void*)o.lde, dims, pitch, box, step, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    return cudaFuncSetAttribute(k_fri_combine_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem) ==
               cudaSuccess &&
           cudaFuncSetAttribute(k_fri_combine_tma<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTmaSmem) ==
               cudaSuccess;
}

v3c_status launch_fold(v3c_ctx* ctx, FriState& st, u32 k, const u64* beta, cudaStream_t s)
{
    const u32 a = st.arity[k];
    FoldArgs p;
    memset(&p, 0, sizeof p);
    p.in = st.f[k];
    p.out = st.f[k + 1];
    p.pw_inv = st.pw_inv;
    p.log_out = st.log_size[k + 1];
    p.exp_shift = st.log_N - st.log_size[k];
    p.inv2 = gl::h_inv(2);
    int kidx = 0;
    u64 bm[2] = {beta[0], st.ext == 2 ? beta[1] : 0}, sm = st.shift[k];
    for (u32 m = 0; m < a; m++) {
        const u32 b = a - 1 - m;
        const u64 scale = gl::h_inv(gl::h_mul(2, sm));
        const u64 rinv = gl::h_inv(gl::h_root(b + 1));
        for (u32 vp = 0; vp < (1u << b); vp++) {
            const u64 c = gl::h_mul(scale, gl::h_pow(rinv, gl::bitrev(vp, b)));
            p.K[kidx + vp][0] = gl::h_mul(bm[0], c);
            p.K[kidx + vp][1] = gl::h_mul(bm[1], c);
        }
        kidx += 1 << b;
        if (st.ext == 2) h_ext_mul(bm, bm, bm);
        else bm[0] = gl::h_mul(bm[0], bm[0]);
        sm = gl::h_mul(sm, sm);
    }
    const int threads = 256;
    const int grid = grid_for((u64)1 << p.log_out, threads);
    StageTimer tm(ctx, 6, s);
    if (st.ext == 2) {
        switch (a) {
        case 1: k_fri_fold<1, 2><<<grid, threads, 0, s>>>(p); break;
        case 2: k_fri_fold<2, 2><<<grid, threads, 0, s>>>(p); break;
        case 3: k_fri_fold<3, 2><<<grid, threads, 0, s>>>(p); break;
        default: k_fri_fold<4, 2><<<grid, threads, 0, s>>>(p); break;
        }
    } else {
        switch (a) {
        case 1: k_fri_fold<1, 1><<<grid, threads, 0, s>>>(p); break;
        case 2: k_fri_fold<2, 1><<<grid, threads, 0, s>>>(p); break;
        case 3: k_fri_fold<3, 1><<<grid, threads, 0, s>>>(p); break;
        default: k_fri_fold<4, 1><<<grid, threads, 0, s>>>(p); break;
        }
    }
    CK(cudaGetLastError());
    tm.done();
    ctx->launches++;
    return V3C_OK;
}

v3c_status launch_final(v3c_ctx* ctx, FriState& st, cudaStream_t s)
{
    const u32 logm = st.log_size[st.rounds];
    const u64 winv = gl::h_inv(gl::h_root(logm));
    const u64 sinv = gl::h_inv(st.shift[st.rounds]);
    const u64 minv = gl::h_inv((u64)1 << logm);
    StageTimer tm(ctx, 6, s);
    for (u32 comp = 0; comp < st.ext; comp++) {
        k_fri_final<<<1, 256, 0, s>>>(st.f[st.rounds], logm, winv, sinv, minv, st.final_coef, st.ext, comp);
        CK(cudaGetLastError());
    }
    tm.done();
    ctx->launches++;
    return V3C_OK;
}

// Tree of every layer that exists and is below R but not committed yet, in
// one batched leaf-hash / Merkle launch sequence.
v3c_status commit_layers(v3c_ctx* ctx, FriState& st, cudaStream_t s)
{
    Batch b;
    u32 upto = std::min(st.done + 1, st.rounds);
    for (u32 k = st.committed; k < upto; k++) {
        TreeJob t;
        memset(&t, 0, sizeof t);
        t.rows = st.f[k];
        t.ld = t.width = (1u << st.arity[k]) * st.ext;
        t.log_N = st.log_size[k] - st.arity[k];
        t.h = st.h[k];
        t.tree = st.tree[k];
        t.cap = st.cap[k];
        t.vec_ok = ((uintptr_t)t.rows % 16 == 0) && (t.ld % 2 == 0);
        b.tree.push_back(t);
    }
    if (b.tree.empty()) return V3C_OK;
    v3c_status r = launch_batch(ctx, b, s);
    if (r) return r;
    st.committed = upto;
    return V3C_OK;
}

// Applies the next n rounds, commits the new layers, and the final
// coefficients once every round is done.  Caller holds ctx->mu.
v3c_status advance(v3c_ctx* ctx, FriState& st, const uint64_t* betas, u32 n, cudaStream_t s)
{
    for (u32 i = 0; i < n * st.ext; i++) {
        if (betas[i] >= gl::P) return fail(ctx, V3C_EINVAL, "v3c_fri: beta word %u not canonical", i);
    }
    for (u32 i = 0; i < n; i++) {
        v3c_status r = launch_fold(ctx, st, st.done, betas + (size_t)i * st.ext, s);
        if (r) return r;
        st.done++;
    }
    v3c_status r = commit_layers(ctx, st, s);
    if (r) return r;
    if (st.done == st.rounds && n + (st.rounds == 0) > 0) {
        r = launch_final(ctx, st, s);
        if (r) return r;
    }
    CK(cudaEventRecord(st.ev, s));
    return V3C_OK;
}

FriState* find_fri(v3c_ctx* ctx, v3c_fri_id id)
{
    auto it = ctx->fri.find(id);
    return it == ctx->fri.end() ? nullptr : it->second;
}

cudaStream_t aux_stream(v3c_ctx* ctx)
{
    if (!ctx->release_stream) cudaStreamCreateWithFlags(&ctx->release_stream, cudaStreamNonBlocking);
    return ctx->release_stream;
}

}  // namespace

void fri_free_all(v3c_ctx* ctx)
{
    for (auto& kv : ctx->fri) {
        FriState* st = kv.second;
        if (st->mem) cudaFree(st->mem);
        if (st->ev) cudaEventDestroy(st->ev);
        delete st;
    }
    ctx->fri.clear();
}

extern "C" {

v3c_status v3c_fri_begin(v3c_ctx* ctx, const v3c_commit_id* ids, uint32_t n_ids, const uint64_t* alpha,
                         const v3c_fri_cfg* cfg, const uint64_t* h_betas, uint32_t n_betas, v3c_fri_id* out,
                         void* stream)
{
    NvtxScope range("v3c_fri_begin");
    if (!ctx) return V3C_EINVAL;
    if (!ids || !n_ids || !cfg || !out || !alpha || (n_betas && !h_betas))
        return fail(ctx, V3C_EINVAL, "v3c_fri_begin: NULL argument or no commitments");
    const u32 ext = cfg->ext_degree ? cfg->ext_degree : 1;
    if (cfg->arity_bits < 1 || cfg->arity_bits > 4 || cfg->final_log > 10 || ext > 2 || alpha[0] >= gl::P ||
        (ext == 2 && alpha[1] >= gl::P))
        return fail(ctx, V3C_EINVAL, "v3c_fri_begin: arity_bits %u, final_log %u, ext_degree %u or alpha out of range",
                    cfg->arity_bits, cfg->final_log, cfg->ext_degree);
    v3c_status r = use_device(ctx);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    std::vector<Object> objs;
    for (u32 i = 0; i < n_ids; i++) {
        auto it = ctx->objects.find(ids[i]);
        if (it == ctx->objects.end())
            return fail(ctx, V3C_ENOTFOUND, "commit id %llu", (unsigned long long)ids[i]);
        objs.push_back(it->second);
    }
    const u32 log_N = objs[0].log_n + objs[0].r;
    u32 ncols = 0;
    for (auto& o : objs) {
        if (o.log_n + o.r != log_N) return fail(ctx, V3C_EINVAL, "v3c_fri_begin: commitments differ in row count");
        ncols += o.c;
    }
    FriState* st = new FriState();
    st->log_N = log_N;
    st->ncols = ncols;
    st->ext = ext;
    st->log_size[0] = log_N;
    st->shift[0] = 7;
    for (u32 m = log_N; m > cfg->final_log;) {
        u32 a = std::min(cfg->arity_bits, m - cfg->final_log);
        u32 k = st->rounds++;
        st->arity[k] = a;
        st->h[k] = std::min(cfg->cap_height, m - a);
        m -= a;
        st->log_size[k + 1] = m;
        st->shift[k + 1] = gl::h_pow(st->shift[k], (u64)1 << a);
    }
    if (n_betas > st->rounds) {
        delete st;
        return fail(ctx, V3C_EINVAL, "v3c_fri_begin: %u betas for %u rounds", n_betas, st->rounds);
    }
    // One allocation: root tables, alpha powers, layers, trees, caps, final.
    auto even = [](size_t w) { return (w + 1) & ~(size_t)1; };
    size_t words = 1536 + even((size_t)ncols * ext);
    size_t off_f[V3C_FRI_MAX_ROUNDS + 1], off_t[V3C_FRI_MAX_ROUNDS], off_c[V3C_FRI_MAX_ROUNDS];
    for (u32 k = 0; k <= st->rounds; k++) {
        off_f[k] = words;
        words += even(((size_t)1 << st->log_size[k]) * ext);
    }
    st->query_words = 0;
    for (u32 k = 0; k < st->rounds; k++) {
        size_t L = (size_t)1 << (st->log_size[k] - st->arity[k]);
        off_t[k] = words;
        words += (2 * L - ((size_t)2 << st->h[k])) * 4;
        off_c[k] = words;
        words += (size_t)4 << st->h[k];
        st->query_words += ((u64)1 << st->arity[k]) * ext + 4 * (st->log_size[k] - st->arity[k] - st->h[k]);
    }
    size_t off_final = words;
    words += even(((size_t)1 << st->log_size[st->rounds]) * ext);
    const size_t off_err = words;
    words += 2;
    st->bytes = words * 8;
    if (ctx->resident + st->bytes > ctx->cfg.hbm_budget_bytes) {
        size_t need = st->bytes;
        delete st;
        return fail(ctx, V3C_ENOMEM, "v3c_fri_begin: %zu bytes over the HBM budget", need);
    }
    cudaError_t e = cudaMallocAsync((void**)&st->mem, st->bytes, s);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st->ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (st->mem) cudaFreeAsync(st->mem, s);
        delete st;
        return fail(ctx, V3C_ENOMEM, "v3c_fri_begin: allocation failed: %s", cudaGetErrorString(e));
    }
    u64* base = st->mem;
    st->pw_inv = base;
    st->alpha_pw = base + 1536;
    for (u32 k = 0; k <= st->rounds; k++) st->f[k] = base + off_f[k];
    for (u32 k = 0; k < st->rounds; k++) {
        st->tree[k] = base + off_t[k];
        st->cap[k] = base + off_c[k];
    }
    st->final_coef = base + off_final;
    st->err = reinterpret_cast<u32*>(base + off_err);
    auto bail = [&](v3c_status code) {
        cudaFreeAsync(st->mem, s);
        cudaEventDestroy(st->ev);
        delete st;
        return code;
    };
#define CKB(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return bail(fail(ctx, V3C_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)));     \
    } while (0)
    for (auto& o : objs) CKB(cudaStreamWaitEvent(s, o.done, 0));
    CKB(cudaMemsetAsync(st->err, 0, 8, s));
    k_fri_root_tables<<<6, 256, 0, s>>>(gl::h_inv(gl::h_root(log_N)), log_N, st->pw_inv);
    CKB(cudaGetLastError());
    if (ext == 2) k_fri_powers_ext<<<grid_for(ncols, 256), 256, 0, s>>>(alpha[0], alpha[1], ncols, st->alpha_pw);
    else k_fri_powers<<<grid_for(ncols, 256), 256, 0, s>>>(alpha[0], ncols, st->alpha_pw);
    CKB(cudaGetLastError());
    ctx->launches += 2;
    u32 e0 = 0;
    const u64 N = (u64)1 << log_N;
    for (size_t i = 0; i < objs.size(); i++) {
        const Object& o = objs[i];
        const u64* pw = st->alpha_pw + (size_t)ext * e0;
        CUtensorMap map;
        const bool tiled = combine_map(o, N, &map);
        log_msg(ctx, 2, "FRI combination of a %u x 2^%u object: %s", o.c, log_N,
                tiled ? "tensor-map tiles" : "register loads");
        if (tiled) {
            StageTimer tm(ctx, 5, s);
            const int grid = (int)std::min<u64>((u64)2 * num_sms(), (N + kTmaRows - 1) / kTmaRows);
            if (ext == 2)
                k_fri_combine_tma<2><<<grid, kTmaThreads, kTmaSmem, s>>>(map, o.c, pw, N, i > 0, st->f[0], st->err);
            else
                k_fri_combine_tma<1><<<grid, kTmaThreads, kTmaSmem, s>>>(map, o.c, pw, N, i > 0, st->f[0], st->err);
            CKB(cudaGetLastError());
            tm.done();
            ctx->launches++;
            e0 += o.c;
            continue;
        }
        int nb = 0;
        CKB(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fri_combine, 256, 0));
        int grid = (int)std::min<u64>((u64)std::max(nb, 1) * num_sms(), (N + 255) / 256);
        StageTimer tm(ctx, 5, s);
        if (ext == 2)
            k_fri_combine_ext2<<<std::max(grid, 1), 256, 0, s>>>(o.lde, o.ld, o.c, pw, N, i > 0, st->f[0]);
        else
            k_fri_combine<<<std::max(grid, 1), 256, 0, s>>>(o.lde, o.ld, o.c, pw, N, i > 0, st->f[0]);
        CKB(cudaGetLastError());
        tm.done();
        ctx->launches++;
        e0 += o.c;
    }
#undef CKB
    st->id = ctx->next_id++;
    r = advance(ctx, *st, h_betas, n_betas, s);
    if (r) return bail(r);
    ctx->resident += st->bytes;
    ctx->fri[st->id] = st;
    *out = st->id;
    return V3C_OK;
}

v3c_status v3c_fri_fold(v3c_ctx* ctx, v3c_fri_id fri, const uint64_t* h_betas, uint32_t n_betas, void* stream)
{
    if (!ctx) return V3C_EINVAL;
    if (n_betas && !h_betas) return fail(ctx, V3C_EINVAL, "v3c_fri_fold: NULL betas");
    v3c_status r = use_device(ctx);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    FriState* st = find_fri(ctx, fri);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "fri id %llu", (unsigned long long)fri);
    if (n_betas > st->rounds - st->done)
        return fail(ctx, V3C_EINVAL, "v3c_fri_fold: %u betas, %u rounds left", n_betas, st->rounds - st->done);
    if (!n_betas) return V3C_OK;
    CK(cudaStreamWaitEvent(s, st->ev, 0));
    return advance(ctx, *st, h_betas, n_betas, s);
}

v3c_status v3c_fri_info(v3c_ctx* ctx, v3c_fri_id fri, v3c_fri_info_t* out)
{
    if (!ctx || !out) return V3C_EINVAL;
    std::lock_guard<std::mutex> g(ctx->mu);
    FriState* st = find_fri(ctx, fri);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "fri id %llu", (unsigned long long)fri);
    memset(out, 0, sizeof *out);
    out->rounds = st->rounds;
    out->rounds_done = st->done;
    out->log_N = st->log_N;
    out->n_columns = st->ncols;
    for (u32 k = 0; k < st->rounds; k++) {
        out->arity_bits[k] = st->arity[k];
        out->cap_height[k] = st->h[k];
    }
    for (u32 k = 0; k <= st->rounds; k++) out->log_size[k] = st->log_size[k];
    out->query_words = st->query_words;
    out->bytes = st->bytes;
    out->ext_degree = st->ext;
    return V3C_OK;
}

// The combination runs once, at v3c_fri_begin; the first call that reads a
// result back (after waiting for the state's work) also reads its error word.
v3c_status check_combine(v3c_ctx* ctx, FriState& st)
{
    if (st.err_checked) return V3C_OK;
    u32 e = 0;
    CK(cudaMemcpy(&e, st.err, 4, cudaMemcpyDeviceToHost));
    if (e) return fail(ctx, V3C_ETIMEDOUT, "FRI combination: a wait of the copy pipeline timed out");
    st.err_checked = true;
    return V3C_OK;
}

v3c_status v3c_fri_cap(v3c_ctx* ctx, v3c_fri_id fri, uint32_t layer, uint64_t* h_cap)
{
    if (!ctx || !h_cap) return V3C_EINVAL;
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    FriState* st = find_fri(ctx, fri);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "fri id %llu", (unsigned long long)fri);
    if (layer >= st->committed) return fail(ctx, V3C_EINVAL, "v3c_fri_cap: layer %u is not committed", layer);
    CK(cudaEventSynchronize(st->ev));
    r = check_combine(ctx, *st);
    if (r) return r;
    CK(cudaMemcpy(h_cap, st->cap[layer], ((size_t)4 << st->h[layer]) * 8, cudaMemcpyDeviceToHost));
    return V3C_OK;
}

v3c_status v3c_fri_final(v3c_ctx* ctx, v3c_fri_id fri, uint64_t* h_coeffs)
{
    if (!ctx || !h_coeffs) return V3C_EINVAL;
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    FriState* st = find_fri(ctx, fri);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "fri id %llu", (unsigned long long)fri);
    if (st->done != st->rounds) return fail(ctx, V3C_EINVAL, "v3c_fri_final: %u of %u rounds done", st->done, st->rounds);
    CK(cudaEventSynchronize(st->ev));
    r = check_combine(ctx, *st);
    if (r) return r;
    CK(cudaMemcpy(h_coeffs, st->final_coef, ((size_t)1 << st->log_size[st->rounds]) * st->ext * 8,
                  cudaMemcpyDeviceToHost));
    return V3C_OK;
}

v3c_status v3c_fri_query(v3c_ctx* ctx, v3c_fri_id fri, const uint64_t* h_idx, uint32_t nq, uint64_t* h_out)
{
    if (!ctx) return V3C_EINVAL;
    if (nq && (!h_idx || !h_out)) return fail(ctx, V3C_EINVAL, "v3c_fri_query: NULL argument");
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    FriState* st = find_fri(ctx, fri);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "fri id %llu", (unsigned long long)fri);
    if (st->done != st->rounds) return fail(ctx, V3C_EINVAL, "v3c_fri_query: %u of %u rounds done", st->done, st->rounds);
    for (u32 q = 0; q < nq; q++)
        if (h_idx[q] >> st->log_N) return fail(ctx, V3C_EINVAL, "v3c_fri_query: index %u out of range", q);
    if (!nq || !st->rounds) return V3C_OK;
    cudaStream_t s = aux_stream(ctx);
    if (!s) return fail(ctx, V3C_ECUDA, "v3c_fri_query: no stream");
    QueryArgs p;
    memset(&p, 0, sizeof p);
    u64 w0 = 0;
    u32 tsh = 0;
    for (u32 k = 0; k < st->rounds; k++) {
        QueryLayer& L = p.L[k];
        L.f = st->f[k];
        L.tree = st->tree[k];
        L.word0 = w0;
        L.a = st->arity[k];
        L.logL = st->log_size[k] - st->arity[k];
        L.h = st->h[k];
        L.tshift = tsh;
        w0 += ((u64)1 << L.a) * st->ext + 4 * (L.logL - L.h);
        tsh += L.a;
    }
    p.R = st->rounds;
    p.ext = st->ext;
    p.nq = nq;
    p.words = st->query_words;
    size_t out_words = (size_t)nq * st->query_words;
    u64* d = nullptr;
    CK(cudaMallocAsync((void**)&d, (nq + out_words) * 8, s));
    p.idx = d;
    p.out = d + nq;
    CK(cudaStreamWaitEvent(s, st->ev, 0));
    cudaError_t e = cudaMemcpyAsync(d, h_idx, (size_t)nq * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        StageTimer tm(ctx, 7, s);
        k_fri_query<<<grid_for(out_words, 256), 256, 0, s>>>(p);
        e = cudaGetLastError();
        tm.done();
        ctx->launches++;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_out, p.out, out_words * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "v3c_fri_query: %s", cudaGetErrorString(e));
    return check_combine(ctx, *st);
}

v3c_status v3c_fri_release(v3c_ctx* ctx, v3c_fri_id fri)
{
    if (!ctx) return V3C_EINVAL;
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    FriState* st = find_fri(ctx, fri);
    if (!st) return fail(ctx, V3C_ENOTFOUND, "fri id %llu", (unsigned long long)fri);
    ctx->fri.erase(fri);
    cudaStream_t s = aux_stream(ctx);
    if (!s) return fail(ctx, V3C_ECUDA, "v3c_fri_release: no stream");
    CK(cudaStreamWaitEvent(s, st->ev, 0));
    CK(cudaFreeAsync(st->mem, s));
    CK(cudaEventDestroy(st->ev));
    ctx->resident -= st->bytes;
    delete st;
    return V3C_OK;
}

v3c_status v3c_open_batch(v3c_ctx* ctx, v3c_commit_id id, const uint64_t* h_leaves, uint32_t nq, uint64_t* h_rows,
                          uint64_t* h_paths)
{
    if (!ctx) return V3C_EINVAL;
    if (nq && !h_leaves) return fail(ctx, V3C_EINVAL, "v3c_open_batch: NULL leaves");
    v3c_status r = use_device(ctx);
    if (r) return r;
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->objects.find(id);
    if (it == ctx->objects.end()) return fail(ctx, V3C_ENOTFOUND, "commit id %llu", (unsigned long long)id);
    const Object o = it->second;
    const u32 log_N = o.log_n + o.r;
    for (u32 q = 0; q < nq; q++)
        if (h_leaves[q] >> log_N) return fail(ctx, V3C_EINVAL, "v3c_open_batch: leaf %u out of range", q);
    if (!nq || (!h_rows && !h_paths)) return V3C_OK;
    cudaStream_t s = aux_stream(ctx);
    if (!s) return fail(ctx, V3C_ECUDA, "v3c_open_batch: no stream");
    const size_t plen = 4 * (size_t)(log_N - o.h);
    const size_t rows_w = (size_t)nq * o.c, paths_w = (size_t)nq * plen;
    u64* d = nullptr;
    CK(cudaMallocAsync((void**)&d, (nq + rows_w + paths_w) * 8, s));
    u64* d_rows = d + nq;
    u64* d_paths = d_rows + rows_w;
    CK(cudaStreamWaitEvent(s, o.done, 0));
    cudaError_t e = cudaMemcpyAsync(d, h_leaves, (size_t)nq * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        StageTimer tm(ctx, 7, s);
        k_open_rows<<<grid_for(rows_w + paths_w, 256), 256, 0, s>>>(o.lde, o.ld, o.c, o.tree, log_N, o.h, d, nq,
                                                                    d_rows, plen ? d_paths : nullptr);
        e = cudaGetLastError();
        tm.done();
        ctx->launches++;
    }
    if (e == cudaSuccess && h_rows) e = cudaMemcpyAsync(h_rows, d_rows, rows_w * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && h_paths && plen)
        e = cudaMemcpyAsync(h_paths, d_paths, paths_w * 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "v3c_open_batch: %s", cudaGetErrorString(e));
    return V3C_OK;
}

}  // extern "C"
