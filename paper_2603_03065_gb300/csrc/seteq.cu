// Multiset-equality gadget (Sec. 4.5, Gadgets and Cost Model): the SetEq
// grand-product column Z_{i+1} = Z_i (alpha - x_i) / (alpha - y_i) over
// tuples compressed by Compress(t; beta) = sum_k t_k beta^k.
//
// GB300 mapping: one persistent launch scans every instance in tiles of
// 2048 elements (8 per thread), in the order a global counter hands the
// tiles out.  A tile reads its tuples once (coalesced), compresses them,
// and forms the products of its numerators and denominators.  It publishes
// those products at once, and the products of everything before it
// ("inclusive") as soon as it knows them: a decoupled look-back in which one
// warp reads the states of the 32 preceding tiles at a time and multiplies
// their products until it meets an inclusive one.  Every wait is bounded;
// one that gives up sets an error flag that the host turns into a status.
// With the prefix (N_pre, D_pre) known, the tile takes one inversion,
// inv = (D_pre D_tile)^-1, and writes Z_i = N_pre N_{<i} D_{>=i} inv, where
// N_{<i} and D_{>=i} run inside the tile (block scans with warp shuffles).
// X and Y are read once and Z written once.  Products inside the scan (the
// thread, block and look-back products) stay in [0, 2^64), congruent mod p;
// only the Z words written out are reduced to [0, p).  A second, small launch zeroes
// the column of an instance whose denominator product is zero (alpha equal
// to some compressed y).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/v3c_seteq.h"
#include "ctx.h"
#include "gl.cuh"
#include "internal.h"

namespace v3c {

using gl::u32;
using gl::u64;

constexpr u32 kSeqThreads = 256;
constexpr u32 kSeqPer = 8;
constexpr u32 kSeqMinBlocks = 3;  // resident CTAs per SM the scan is compiled for (80 registers)
constexpr u32 kSeqTile = kSeqThreads * kSeqPer;

struct SeqJob {
    const u64* x;
    const u64* y;
    u64* z;
    u64 L;
    u64 alpha, beta;
    u64 beta2, beta3;  // beta^2, beta^3 (width-4 tuples)
    u32* status;  // the instance's status word: 1 when its denominator product is zero
    u32 T;
    u32 tile0;    // first global tile
    u32 ntiles;
    u32 pad;
};

// Look-back state of one tile: its own products (flag 1) and the products
// of its instance up to and including it (flag 2).
struct SeqTile {
    u64 agg_n, agg_d, inc_n, inc_d;
};

__device__ __forceinline__ u32 seq_find(const SeqJob* __restrict__ jobs, u32 njobs, u32 tile)
{
    u32 lo = 0, hi = njobs;
    while (hi - lo > 1) {
        u32 mid = (lo + hi) >> 1;
        if (jobs[mid].tile0 <= tile) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ u64 compress(const u64* __restrict__ t, u32 T, u64 beta)
{
    // Horner from the last component: sum_k t_k beta^k, on values in
    // [0, 2^64) congruent mod p, canonical at the end.  A tuple of even
    // width at a 16-byte aligned address is read in 16-byte pairs.
    u64 s;
    if (!(T & 1) && !((uintptr_t)t & 15)) {
        const ulonglong2* t2 = reinterpret_cast<const ulonglong2*>(t);
        ulonglong2 q = __ldg(t2 + (T >> 1) - 1);
        s = gl::add_nc(gl::mul_nc(q.y, beta), q.x);
        for (int k = (int)(T >> 1) - 2; k >= 0; k--) {
            q = __ldg(t2 + k);
            s = gl::add_nc(gl::mul_nc(s, beta), q.y);
            s = gl::add_nc(gl::mul_nc(s, beta), q.x);
        }
    } else {
        s = __ldg(t + T - 1);
        for (int k = (int)T - 2; k >= 0; k--) s = gl::add_nc(gl::mul_nc(s, beta), __ldg(t + k));
    }
    return gl::canon(s);
}

// numerator and denominator of element e (1 and 1 past the end).
__device__ __forceinline__ void seq_terms(const SeqJob& J, u64 e, u64& num, u64& den)
{
    if (e < J.L) {
        num = gl::sub(J.alpha, compress(J.x + e * J.T, J.T, J.beta));
        den = gl::sub(J.alpha, compress(J.y + e * J.T, J.T, J.beta));
    } else {
        num = den = 1;
    }
}

// Block-wide exclusive product over threads in thread order (prefix) or in
// reverse order (suffix).  sh holds 32 words.  All threads must call it.
template <bool SUFFIX>
__device__ __forceinline__ u64 block_exclusive(u64 v, u64* sh)
{
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    u64 inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u64 t = SUFFIX ? __shfl_down_sync(0xffffffffu, inc, o) : __shfl_up_sync(0xffffffffu, inc, o);
        bool take = SUFFIX ? lane + o < 32 : lane >= (u32)o;
        if (take) inc = gl::mul_nc(inc, t);
    }
    u64 excl = SUFFIX ? __shfl_down_sync(0xffffffffu, inc, 1) : __shfl_up_sync(0xffffffffu, inc, 1);
    if (SUFFIX ? lane == 31 : lane == 0) excl = 1;
    if (SUFFIX ? lane == 0 : lane == 31) sh[wid] = inc;  // warp total
    __syncthreads();
    if (threadIdx.x == 0) {
        // exclusive product of warp totals, in the scan's direction
        u64 run = 1;
        for (u32 k = 0; k < nw; k++) {
            u32 w = SUFFIX ? nw - 1 - k : k;
            u64 t = sh[w];
            sh[w] = run;
            run = gl::mul_nc(run, t);
        }
    }
    __syncthreads();
    u64 r = gl::mul_nc(excl, sh[wid]);
    __syncthreads();
    return r;
}

// x^(p-2), the inverse of x (0 for 0).  p - 2 has bits 63..33 and 31..0
// set, so x^(p-2) = (x^(2^31 - 1))^(2^33) x^(2^32 - 1); x^(2^31 - 1) comes
// from the chain 2^k - 1 for k = 1, 2, 3, 6, 12, 15, 30, 31 (each step
// e_{a+b} = e_a^(2^b) e_b): 64 squarings and 9 products in all.
__device__ u64 seq_inverse(u64 x)
{
    auto sq = [](u64 v, int n) {
        for (int i = 0; i < n; i++) v = gl::mul(v, v);
        return v;
    };
    const u64 e1 = x;
    const u64 e2 = gl::mul(sq(e1, 1), e1);
    const u64 e3 = gl::mul(sq(e2, 1), e1);
    const u64 e6 = gl::mul(sq(e3, 3), e3);
    const u64 e12 = gl::mul(sq(e6, 6), e6);
    const u64 e15 = gl::mul(sq(e12, 3), e3);
    const u64 e30 = gl::mul(sq(e15, 15), e15);
    const u64 e31 = gl::mul(sq(e30, 1), e1);
    const u64 e32 = gl::mul(sq(e31, 1), e1);
    return gl::mul(sq(e31, 33), e32);
}

// The terms alpha - Compress(X_i), alpha - Compress(Y_i) of the tile at
// tbase into bn, bd (padded layout; 1 past the end), computed by the threads
// [first, first + nthr) of the CTA, thread j taking elements j + nthr k.
// Width-4 tuples at 16-byte aligned addresses (the query circuit's (list,
// slot, distance, item)) are requested two elements at a time, eight
// 16-byte loads in flight per thread, before any is compressed; their
// Compress is t_0 + t_1 beta + t_2 beta^2 + t_3 beta^3 as three independent
// 64x64 products summed unreduced in 192 bits and reduced once.
__device__ __forceinline__ u32 seq_pad(u32 i);
__device__ __forceinline__ void seq_load(const SeqJob& J, u64 tbase, u64* bn, u64* bd, u32 first, u32 nthr)
{
    const u32 j = threadIdx.x - first;
    if (J.T == 4 && !(((uintptr_t)J.x | (uintptr_t)J.y) & 15)) {
        const ulonglong2* x2 = reinterpret_cast<const ulonglong2*>(J.x);
        const ulonglong2* y2 = reinterpret_cast<const ulonglong2*>(J.y);
        for (u32 i0 = j; i0 < kSeqTile; i0 += 2 * nthr) {
            ulonglong2 xa[2], xb[2], ya[2], yb[2];
#pragma unroll
            for (u32 k = 0; k < 2; k++) {
                const u64 e = tbase + i0 + k * nthr;
                if (i0 + k * nthr < kSeqTile && e < J.L) {
                    xa[k] = __ldcs(x2 + 2 * e);
                    xb[k] = __ldcs(x2 + 2 * e + 1);
                    ya[k] = __ldcs(y2 + 2 * e);
                    yb[k] = __ldcs(y2 + 2 * e + 1);
                }
            }
#pragma unroll
            for (u32 k = 0; k < 2; k++) {
                const u32 i = i0 + k * nthr;
                if (i >= kSeqTile) break;
                u64 n = 1, d = 1;
                if (tbase + i < J.L) {
                    u64 lo = xa[k].x, mid = 0;
                    u32 hi = 0;
                    gl::mac192(lo, mid, hi, xa[k].y, J.beta);
                    gl::mac192(lo, mid, hi, xb[k].x, J.beta2);
                    gl::mac192(lo, mid, hi, xb[k].y, J.beta3);
                    n = gl::sub(J.alpha, gl::fold192(lo, mid, hi));
                    lo = ya[k].x;
                    mid = 0;
                    hi = 0;
                    gl::mac192(lo, mid, hi, ya[k].y, J.beta);
                    gl::mac192(lo, mid, hi, yb[k].x, J.beta2);
                    gl::mac192(lo, mid, hi, yb[k].y, J.beta3);
                    d = gl::sub(J.alpha, gl::fold192(lo, mid, hi));
                }
                bn[seq_pad(i)] = n;
                bd[seq_pad(i)] = d;
            }
        }
    } else {
        for (u32 i = j; i < kSeqTile; i += nthr) {
            u64 n, d;
            seq_terms(J, tbase + i, n, d);
            bn[seq_pad(i)] = n;
            bd[seq_pad(i)] = d;
        }
    }
}

// Polls of one look-back window before the wait gives up (with a short
// sleep between polls, on the order of a second in all).
constexpr u32 kSeqSpinLimit = 1u << 22;

// Shared words are padded by one per 8 (index i + i/8): the 8-word stride of
// a thread's contiguous elements becomes 9, an odd number of 8-byte words,
// so a warp's accesses fall in distinct bank pairs.
__device__ __forceinline__ u32 seq_pad(u32 i) { return i + (i >> 3); }

__device__ __forceinline__ u64 warp_product(u64 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = gl::mul_nc(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Warp 0's part of a tile: publish the tile's products, find the products of
// the instance before the tile (decoupled look-back), publish the inclusive
// products, and return (N_pre, D_pre) in lane 0.
__device__ __forceinline__ void seq_lookback(const SeqJob& J, u32 tile, u64 Nt, u64 Dt, SeqTile* st, u32* flags,
                                             u32* err, u64& Np, u64& Dp)
{
    const u32 lane = threadIdx.x & 31;
    const u32 lt = tile - J.tile0;
    Np = 1;
    Dp = 1;
    if (lane == 0) {
        SeqTile& me = st[tile];
        if (lt == 0) {
            me.inc_n = Nt;
            me.inc_d = Dt;
        } else {
            me.agg_n = Nt;
            me.agg_d = Dt;
        }
        __threadfence();
        atomicExch(&flags[tile], lt == 0 ? 2u : 1u);
    }
    if (lt == 0) return;
    int p = (int)tile - 1;  // nearest predecessor not folded in yet
    u32 spins = 0;
    for (;;) {
        const int q = p - (int)lane;
        const bool in = q >= (int)J.tile0;
        const u32 f = in ? *(volatile const u32*)(flags + q) : 2u;  // before the instance: identity
        const u32 inc = __ballot_sync(0xffffffffu, f == 2u);
        const u32 upto = inc ? (u32)__ffs(inc) - 1 : 31u;             // lanes 0..upto take part
        const u32 relevant = upto == 31 ? 0xffffffffu : ((2u << upto) - 1);
        if (__ballot_sync(0xffffffffu, f == 0u) & relevant) {
            if (++spins > kSeqSpinLimit) {  // a predecessor never published: give up
                if (lane == 0) atomicOr(err, 1u);
                return;
            }
            __nanosleep(64);
            continue;
        }
        __threadfence();
        u64 vn = 1, vd = 1;
        if (in && lane <= upto) {
            const SeqTile& o = st[q];
            if (lane == upto && inc) {
                vn = __ldcv(&o.inc_n);
                vd = __ldcv(&o.inc_d);
            } else {
                vn = __ldcv(&o.agg_n);
                vd = __ldcv(&o.agg_d);
            }
        }
        vn = warp_product(vn);
        vd = warp_product(vd);
        Np = gl::mul_nc(Np, vn);
        Dp = gl::mul_nc(Dp, vd);
        if (inc) break;
        p -= 32;
        spins = 0;
    }
    if (lane == 0) {
        SeqTile& me = st[tile];
        me.inc_n = gl::mul_nc(Np, Nt);
        me.inc_d = gl::mul_nc(Dp, Dt);
        __threadfence();
        atomicExch(&flags[tile], 2u);
    }
}

// The scan.  A CTA takes tiles from the global counter until none is left,
// one tile ahead: while warp 0 runs the look-back and the inversion of the
// current tile (a chain of dependent products), warps 1..7 already compute
// the next tile's terms into the other half of the double buffer.  Per tile:
// the terms (coalesced loads, thread j taking elements j + 224 k or
// j + 256 k) land in shared memory; thread t then owns the contiguous
// elements 8t .. 8t+7 and forms their products; block scans give the
// numerators of the earlier threads and the denominators of the later ones;
// Z goes out through shared memory for coalesced stores.
__global__ void __launch_bounds__(kSeqThreads, kSeqMinBlocks) k_seteq_scan(const SeqJob* __restrict__ jobs, u32 njobs,
                                                                          u32 ntiles, SeqTile* st, u32* flags,
                                                                          u32* counter, u32* err)
{
    __shared__ u64 sh[32];
    __shared__ u64 s_num[2][kSeqTile + kSeqTile / 8];
    __shared__ u64 s_den[2][kSeqTile + kSeqTile / 8];
    __shared__ u64 s_tot[2];  // the tile's numerator and denominator products
    __shared__ u64 s_k;       // N_pre (D_pre D_tile)^-1
    __shared__ u32 s_tile[2];
    const u32 t = threadIdx.x;
    if (t == 0) s_tile[0] = atomicAdd(counter, 1u);
    __syncthreads();
    u32 tile = s_tile[0];
    u32 b = 0;
    if (tile < ntiles) {
        const SeqJob& J = jobs[seq_find(jobs, njobs, tile)];
        seq_load(J, (u64)(tile - J.tile0) * kSeqTile, s_num[0], s_den[0], 0, blockDim.x);
    }
    __syncthreads();
    while (tile < ntiles) {
        const SeqJob& J = jobs[seq_find(jobs, njobs, tile)];
        const u64 tbase = (u64)(tile - J.tile0) * kSeqTile;
        if (t == 0) s_tile[b ^ 1] = atomicAdd(counter, 1u);  // the next tile, seen after the scans' barriers
        u64 pn = 1, pd = 1;
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            pn = gl::mul_nc(pn, s_num[b][seq_pad(kSeqPer * t + k)]);
            pd = gl::mul_nc(pd, s_den[b][seq_pad(kSeqPer * t + k)]);
        }
        const u64 en = block_exclusive<false>(pn, sh);  // numerators of the earlier threads
        const u64 sd = block_exclusive<true>(pd, sh);   // denominators of the later threads
        if (t == blockDim.x - 1) s_tot[0] = gl::mul_nc(en, pn);
        if (t == 0) s_tot[1] = gl::mul_nc(sd, pd);
        __syncthreads();
        const u32 next = s_tile[b ^ 1];
        if (t < 32) {
            u64 Np, Dp;
            seq_lookback(J, tile, s_tot[0], s_tot[1], st, flags, err, Np, Dp);
            if (t == 0) {
                const u64 inv = seq_inverse(gl::mul(Dp, s_tot[1]));
                if (inv == 0) atomicOr(J.status, 1u);
                s_k = gl::mul_nc(Np, inv);
            }
        } else if (next < ntiles) {
            const SeqJob& Jn = jobs[seq_find(jobs, njobs, next)];
            seq_load(Jn, (u64)(next - Jn.tile0) * kSeqTile, s_num[b ^ 1], s_den[b ^ 1], 32, blockDim.x - 32);
        }
        __syncthreads();
        // Z_i = N_pre N_{<i} D_{>=i} (D_pre D_tile)^-1, D_{>=i} within the tile.
        u64 num[kSeqPer], den[kSeqPer];
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            num[k] = s_num[b][seq_pad(kSeqPer * t + k)];
            den[k] = s_den[b][seq_pad(kSeqPer * t + k)];
        }
        u64 N = gl::mul_nc(s_k, en);
        u64 S = sd;
        u64 suf[kSeqPer];
#pragma unroll
        for (int k = kSeqPer - 1; k >= 0; k--) {
            S = gl::mul_nc(S, den[k]);
            suf[k] = S;
        }
        const u64 ebase = tbase + (u64)kSeqPer * t;
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            s_num[b][seq_pad(kSeqPer * t + k)] = gl::mul(N, suf[k]);  // each thread rewrites only its own words
            N = gl::mul_nc(N, num[k]);
            if (ebase + k + 1 == J.L) J.z[J.L] = gl::canon(N);
        }
        __syncthreads();
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            const u32 i = t + k * kSeqThreads;
            if (tbase + i < J.L) __stcs(J.z + tbase + i, s_num[b][seq_pad(i)]);
        }
        __syncthreads();
        tile = next;
        b ^= 1;
    }
}

// Columns of instances whose denominator product is zero are all zero.
__global__ void k_seteq_zero(const SeqJob* __restrict__ jobs, u32 njobs)
{
    for (u32 j = blockIdx.x; j < njobs; j += gridDim.x) {
        const SeqJob& J = jobs[j];
        if (!*(volatile const u32*)J.status) continue;
        for (u64 i = threadIdx.x; i <= J.L; i += blockDim.x) J.z[i] = 0;
    }
}
}  // namespace v3c

using namespace v3c::detail;

extern "C" v3c_status v3c_seteq(v3c_ctx* ctx, const v3c_seteq_desc* descs, uint32_t n, uint32_t* h_status,
                                void* stream)
{
    NvtxScope range("v3c_seteq");
    if (!ctx) return V3C_EINVAL;
    if (!descs || !n) return fail(ctx, V3C_EINVAL, "v3c_seteq: no instances");
    u64 tiles = 0;
    for (u32 i = 0; i < n; i++) {
        const v3c_seteq_desc& d = descs[i];
        if (!d.x || !d.y || !d.z || d.T < 1 || d.T > 32 || d.L == 0 || d.L >= ((u64)1 << 40) || d.alpha >= gl::P ||
            d.beta >= gl::P)
            return fail(ctx, V3C_EINVAL, "v3c_seteq: bad instance %u", i);
        tiles += (d.L + kSeqTile - 1) / kSeqTile;
    }
    if (tiles >= ((u64)1 << 31)) return fail(ctx, V3C_EINVAL, "v3c_seteq: too many elements");
    v3c_status r = use_device(ctx);
    if (r) return r;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> g(ctx->mu);
    // Scratch: jobs, tile states, then (zeroed) tile flags, the tile counter,
    // the error flag and the per-instance statuses.
    const size_t job_words = (sizeof(SeqJob) * n + 15) / 16 * 2;  // an even word count
    const size_t tile_words = 4 * tiles;
    const size_t flag_words = (tiles + 2 + n + 1) / 2 + 1;        // u32 words, rounded up
    const size_t words = job_words + tile_words + flag_words;
    u64* mem = nullptr;
    CK(cudaMallocAsync((void**)&mem, words * 8, s));
    SeqTile* dst = reinterpret_cast<SeqTile*>(mem + job_words);
    u32* flags = reinterpret_cast<u32*>(mem + job_words + tile_words);
    u32* counter = flags + tiles;
    u32* err = counter + 1;
    u32* status = err + 1;
    std::vector<SeqJob> jobs(n);
    u32 t0 = 0;
    for (u32 i = 0; i < n; i++) {
        const v3c_seteq_desc& d = descs[i];
        SeqJob& J = jobs[i];
        memset(&J, 0, sizeof J);
        J.x = d.x;
        J.y = d.y;
        J.z = d.z;
        J.L = d.L;
        J.T = d.T;
        J.alpha = d.alpha;
        J.beta = d.beta;
        J.beta2 = gl::h_mul(d.beta, d.beta);
        J.beta3 = gl::h_mul(J.beta2, d.beta);
        J.tile0 = t0;
        J.ntiles = (u32)((d.L + kSeqTile - 1) / kSeqTile);
        J.status = status + i;
        t0 += J.ntiles;
    }
    cudaError_t e = cudaMemcpyAsync(mem, jobs.data(), sizeof(SeqJob) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, flag_words * 8, s);
    const SeqJob* dj = reinterpret_cast<const SeqJob*>(mem);
    // Persistent grid: the resident CTAs of all SMs (tiles are handed out in
    // order, so every tile a CTA waits for is held by a running CTA).
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_seteq_scan, kSeqThreads, 0);
    const int grid = (int)std::min<u64>(tiles, (u64)num_sms() * std::max(per_sm, 1));
    if (e == cudaSuccess) {
        StageTimer tm(ctx, 8, s);
        k_seteq_scan<<<grid, kSeqThreads, 0, s>>>(dj, n, (u32)tiles, dst, flags, counter, err);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            k_seteq_zero<<<(int)std::min<u32>(n, (u32)num_sms() * 2), 256, 0, s>>>(dj, n);
            e = cudaGetLastError();
        }
        tm.done();
        ctx->launches += 2;
    }
    // The statuses and the error flag come back when the caller waits.
    std::vector<u32> st;
    if (e == cudaSuccess && h_status) {
        st.resize(1 + (size_t)n);
        e = cudaMemcpyAsync(st.data(), err, 4 * (1 + (size_t)n), cudaMemcpyDeviceToHost, s);
    }
    cudaFreeAsync(mem, s);
    if (e == cudaSuccess && h_status) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "v3c_seteq: %s", cudaGetErrorString(e));
    if (h_status) {
        if (st[0]) return fail(ctx, V3C_ETIMEDOUT, "v3c_seteq: a tile's look-back wait gave up");
        for (u32 i = 0; i < n; i++) h_status[i] = st[1 + (size_t)i];
    }
    return V3C_OK;
}
