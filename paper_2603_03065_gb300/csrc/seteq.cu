// Multiset-equality gadget (Sec. 4.5, Gadgets and Cost Model): the SetEq
// grand-product column Z_{i+1} = Z_i (alpha - x_i) / (alpha - y_i) over
// tuples compressed by Compress(t; beta) = sum_k t_k beta^k.
//
// GB300 mapping: a multiplicative scan over F_p in three persistent launches
// over all instances.  (1) Every CTA takes a tile of 2048 elements, 8 per
// thread, and writes the tile's products of numerators and denominators.
// (2) One CTA per instance scans the tile products: the prefix of
// numerators before each tile, the suffix of denominators after it, and the
// inverse of the full denominator product (the instance's only inversion).
// (3) Every tile reads its numerators and denominators back, scans them with
// warp shuffles and one shared-memory step per CTA, and writes
// Z_i = N_{<i} * D_{>=i} * D_all^-1.  Loads and stores are coalesced: the
// order-free product of phase 1 takes strided elements, and phase 3
// transposes through shared memory.
// X and Y are read once (phase 1); the compressed terms cost 16 bytes per
// tuple to write and read back instead of a second pass over X, Y and the
// Horner evaluations.
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
constexpr u32 kSeqTile = kSeqThreads * kSeqPer;

struct SeqJob {
    const u64* x;
    const u64* y;
    u64* z;
    u64 L;
    u64 alpha, beta;
    ulonglong2* nd;  // [L]: (alpha - x_i, alpha - y_i), written by phase 1, read by phase 3
    u64* agg;     // [ntiles][2]: tile products of numerators, denominators
    u64* carry;   // [ntiles][2]: numerator product before, denominator product after the tile
    u64* inv;     // [2]: inverse of the denominator product (0 if it is 0), status
    u32 T;
    u32 tile0;    // first global tile
    u32 ntiles;
    u32 pad;
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
        if (take) inc = gl::mul(inc, t);
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
            run = gl::mul(run, t);
        }
    }
    __syncthreads();
    u64 r = gl::mul(excl, sh[wid]);
    __syncthreads();
    return r;
}

// Phase 1: tile products of the numerators and denominators.  A product
// does not depend on order, so thread t takes elements t + 256 k: the warp's
// loads of one tuple component are then one contiguous run.
__global__ void __launch_bounds__(kSeqThreads) k_seteq_reduce(const SeqJob* __restrict__ jobs, u32 njobs, u32 ntiles)
{
    __shared__ u64 sh[32];
    for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const SeqJob& J = jobs[seq_find(jobs, njobs, tile)];
        const u32 lt = tile - J.tile0;
        const u64 base = (u64)lt * kSeqTile + threadIdx.x;
        u64 pn = 1, pd = 1;
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            const u64 e = base + (u64)k * kSeqThreads;
            u64 n, d;
            seq_terms(J, e, n, d);
            if (e < J.L) J.nd[e] = make_ulonglong2(n, d);
            pn = gl::mul(pn, n);
            pd = gl::mul(pd, d);
        }
        // Tile totals: exclusive prefix of the last thread times its own value.
        u64 en = block_exclusive<false>(pn, sh);
        u64 ed = block_exclusive<false>(pd, sh);
        if (threadIdx.x == blockDim.x - 1) {
            J.agg[2 * lt] = gl::mul(en, pn);
            J.agg[2 * lt + 1] = gl::mul(ed, pd);
        }
    }
}

// Phase 2: per instance, carries across tiles and the one inversion.
__global__ void __launch_bounds__(1024) k_seteq_carries(const SeqJob* __restrict__ jobs, u32 njobs)
{
    __shared__ u64 sh[32];
    __shared__ u64 tot[2];
    for (u32 j = blockIdx.x; j < njobs; j += gridDim.x) {
        const SeqJob& J = jobs[j];
        const u32 nt = J.ntiles;
        // Thread t takes the contiguous tiles [t c, (t+1) c).
        const u32 c = (nt + blockDim.x - 1) / blockDim.x;
        const u32 t0 = min(nt, threadIdx.x * c), t1 = min(nt, t0 + c);
        u64 pn = 1, pd = 1;
        for (u32 t = t0; t < t1; t++) {
            pn = gl::mul(pn, J.agg[2 * t]);
            pd = gl::mul(pd, J.agg[2 * t + 1]);
        }
        u64 before = block_exclusive<false>(pn, sh);  // numerators of tiles before t0
        u64 after = block_exclusive<true>(pd, sh);    // denominators of tiles from t1 on
        if (threadIdx.x == blockDim.x - 1) tot[0] = gl::mul(before, pn);
        if (threadIdx.x == 0) tot[1] = gl::mul(after, pd);
        // running carries inside the thread's range
        u64 run = before;
        for (u32 t = t0; t < t1; t++) {
            J.carry[2 * t] = run;
            run = gl::mul(run, J.agg[2 * t]);
        }
        run = after;
        for (u32 t = t1; t > t0; t--) {
            J.carry[2 * (t - 1) + 1] = run;
            run = gl::mul(run, J.agg[2 * (t - 1) + 1]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const u64 D = tot[1];
            J.inv[0] = gl::pow(D, gl::P - 2);  // 0 when D = 0
            J.inv[1] = D == 0;
        }
        __syncthreads();
    }
}

// Phase 3: Z_i = N_{<i} D_{>=i} D^-1 for every element of every tile, and
// Z_L = N_{<L} D^-1 from the thread that holds element L - 1.  Terms are
// computed with coalesced loads (thread t, elements t + 256 k), transposed
// through shared memory so that thread t scans the contiguous elements
// 8t .. 8t+7, and Z goes back through shared memory for coalesced stores.
// Shared words are padded by one per 8 (index i + i/8): the 8-word stride of
// the contiguous reads becomes 9, an odd number of 8-byte words, so a warp's
// accesses fall in distinct bank pairs.
__device__ __forceinline__ u32 seq_pad(u32 i) { return i + (i >> 3); }

__global__ void __launch_bounds__(kSeqThreads) k_seteq_apply(const SeqJob* __restrict__ jobs, u32 njobs, u32 ntiles)
{
    __shared__ u64 sh[32];
    __shared__ u64 s_num[kSeqTile + kSeqTile / 8];
    __shared__ u64 s_den[kSeqTile + kSeqTile / 8];
    const u32 t = threadIdx.x;
    for (u32 tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const SeqJob& J = jobs[seq_find(jobs, njobs, tile)];
        const u32 lt = tile - J.tile0;
        const u64 tbase = (u64)lt * kSeqTile;
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            const u32 i = t + k * kSeqThreads;
            ulonglong2 v = tbase + i < J.L ? __ldcs(J.nd + tbase + i) : make_ulonglong2(1, 1);
            s_num[seq_pad(i)] = v.x;
            s_den[seq_pad(i)] = v.y;
        }
        __syncthreads();
        u64 num[kSeqPer], den[kSeqPer];
        u64 pn = 1, pd = 1;
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            num[k] = s_num[seq_pad(kSeqPer * t + k)];
            den[k] = s_den[seq_pad(kSeqPer * t + k)];
            pn = gl::mul(pn, num[k]);
            pd = gl::mul(pd, den[k]);
        }
        // N carries the factor D^-1 from the start: Z_i = (N_{<i} D^-1) D_{>=i}.
        const u64 inv = __ldg(J.inv);
        u64 N = gl::mul(gl::mul(__ldg(J.carry + 2 * lt), inv), block_exclusive<false>(pn, sh));
        u64 S = gl::mul(__ldg(J.carry + 2 * lt + 1), block_exclusive<true>(pd, sh));
        // S: denominators after this thread's elements; walk them backwards.
        u64 suf[kSeqPer];
#pragma unroll
        for (int k = kSeqPer - 1; k >= 0; k--) {
            S = gl::mul(S, den[k]);
            suf[k] = S;
        }
        const u64 ebase = tbase + (u64)kSeqPer * t;
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            s_num[seq_pad(kSeqPer * t + k)] = gl::mul(N, suf[k]);  // every read above is done
            N = gl::mul(N, num[k]);
            if (ebase + k + 1 == J.L) J.z[J.L] = N;
        }
        __syncthreads();
#pragma unroll
        for (u32 k = 0; k < kSeqPer; k++) {
            const u32 i = t + k * kSeqThreads;
            if (tbase + i < J.L) J.z[tbase + i] = s_num[seq_pad(i)];
        }
        __syncthreads();
    }
}

}  // namespace v3c

using namespace v3c::detail;

extern "C" v3c_status v3c_seteq(v3c_ctx* ctx, const v3c_seteq_desc* descs, uint32_t n, uint32_t* h_status,
                                void* stream)
{
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
    // Scratch: jobs, per-tile products and carries, per-instance inverse/status.
    u64 elems = 0;
    for (u32 i = 0; i < n; i++) elems += descs[i].L;
    const size_t job_words = (sizeof(SeqJob) * n + 15) / 16 * 2;  // an even word count
    const size_t words = job_words + 4 * tiles + 2 * (size_t)n + 2 * elems;
    u64* mem = nullptr;
    CK(cudaMallocAsync((void**)&mem, words * 8, s));
    std::vector<SeqJob> jobs(n);
    u64* agg = mem + job_words;
    u64* carry = agg + 2 * tiles;
    u64* inv = carry + 2 * tiles;
    u64* nd = inv + 2 * (size_t)n;  // 16-byte aligned: every earlier part has an even word count
    u64 e0 = 0;
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
        J.tile0 = t0;
        J.ntiles = (u32)((d.L + kSeqTile - 1) / kSeqTile);
        J.agg = agg + 2 * (size_t)t0;
        J.carry = carry + 2 * (size_t)t0;
        J.inv = inv + 2 * (size_t)i;
        J.nd = reinterpret_cast<ulonglong2*>(nd + 2 * e0);
        e0 += d.L;
        t0 += J.ntiles;
    }
    cudaError_t e = cudaMemcpyAsync(mem, jobs.data(), sizeof(SeqJob) * n, cudaMemcpyHostToDevice, s);
    const SeqJob* dj = reinterpret_cast<const SeqJob*>(mem);
    const int grid = (int)std::min<u64>(tiles, (u64)num_sms() * 8);
    if (e == cudaSuccess) {
        StageTimer tm(ctx, 8, s);
        k_seteq_reduce<<<grid, kSeqThreads, 0, s>>>(dj, n, (u32)tiles);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            k_seteq_carries<<<(int)std::min<u32>(n, (u32)num_sms() * 2), 1024, 0, s>>>(dj, n);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) {
            k_seteq_apply<<<grid, kSeqThreads, 0, s>>>(dj, n, (u32)tiles);
            e = cudaGetLastError();
        }
        tm.done();
        ctx->launches += 3;
    }
    std::vector<u64> st;
    if (e == cudaSuccess && h_status) {
        st.resize(2 * (size_t)n);
        e = cudaMemcpyAsync(st.data(), inv, 16 * (size_t)n, cudaMemcpyDeviceToHost, s);
    }
    cudaFreeAsync(mem, s);
    if (e == cudaSuccess && h_status) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(ctx, V3C_ECUDA, "v3c_seteq: %s", cudaGetErrorString(e));
    if (h_status)
        for (u32 i = 0; i < n; i++) h_status[i] = (uint32_t)st[2 * (size_t)i + 1];
    return V3C_OK;
}
