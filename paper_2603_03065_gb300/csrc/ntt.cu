// Coset low-degree extension kernels (stages A, B and C of internal.h).
//
// The prover's cost sits in FFT-based polynomial arithmetic over a padded
// power-of-two domain (Sec. 2.1, binning effect; Sec. 5.2, Metrics).  For
// each column the LDE is the evaluation of the interpolant on the coset
// 7 * <w_N>:
//     a = iNTT_n(col),  b_i = a_i 7^i (i < n),  E_j = sum_i b_i w_N^{ij},
// and committed row t holds E_{bitrev_{log N}(t)}.
//
// GB300 mapping: one CTA owns one small DFT (or a few side by side) held in
// shared memory.  The data moves through HBM three times: x -> Y -> Z -> rows.
// Every global read and write is a contiguous run of at least 32 bytes.
// The last stage writes the row-major, bit-reversed LDE directly.  Each
// stage is one persistent launch over all jobs of a batch.
#include <cuda_runtime.h>
#include <algorithm>

#include "gl.cuh"
#include "internal.h"

namespace v3c {

using gl::u32;
using gl::u64;

// ---------------------------------------------------------------- plan tables

void plan_split(u32 log_n, u32 r, u32& log_n1, u32& log_n2)
{
    // Stage B holds M = n2 * 2^r values (<= 2^13, 64 KiB) per CTA, stage A
    // and C hold n1-point DFTs (n1 <= 2^11).
    u32 cap = r >= 13 ? 0 : 13 - r;
    log_n2 = std::min(log_n, cap);
    log_n1 = log_n - log_n2;
}

static inline size_t half_or_one(u32 log_l) { return log_l ? (size_t)1 << (log_l - 1) : 1; }

size_t plan_table_words(u32 log_n, u32 r)
{
    u32 l1, l2;
    plan_split(log_n, r, l1, l2);
    size_t n = (size_t)1 << log_n, N = n << r;
    size_t w = n;                          // scale
    if (l1) w += n + N;                    // twa, twb
    w += half_or_one(l1) * 2 + half_or_one(l2) + half_or_one(l2 + r);
    return w;
}

static u64 hmul(u64 a, u64 b) { return (u64)((unsigned __int128)a * b % gl::P); }
static u64 hpow(u64 a, u64 e)
{
    u64 r = 1;
    while (e) {
        if (e & 1) r = hmul(r, a);
        a = hmul(a, a);
        e >>= 1;
    }
    return r;
}
static u64 hroot(u32 log_m) { return hpow(7, (gl::P - 1) >> log_m); }
static u64 hinv(u64 a) { return hpow(a, gl::P - 2); }

struct TableArgs {
    u64* twa;
    u64* scale;
    u64* twb;
    u64* rinv_n1;
    u64* rinv_n2;
    u64* rfwd_M;
    u64* rfwd_n1;
    u64 w_n_inv, w_N, w_n1_inv, w_n2_inv, w_M, w_n1, n_inv;
    u32 log_n, log_n1, log_n2, log_M, log_N;
    u64 seg[8];  // cumulative segment ends
};

__global__ void k_plan_tables(TableArgs a)
{
    u64 total = a.seg[6];
    u32 n1 = 1u << a.log_n1, n2 = 1u << a.log_n2;
    u64 n_mask = ((u64)1 << a.log_n) - 1, N_mask = ((u64)1 << a.log_N) - 1;
    for (u64 e = blockIdx.x * (u64)blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        if (e < a.seg[0]) {  // twa[k1][i2]
            u64 k1 = e >> a.log_n2, i2 = e & (n2 - 1);
            a.twa[e] = gl::pow(a.w_n_inv, (k1 * i2) & n_mask);
        } else if (e < a.seg[1]) {  // scale[k1][t]
            u64 i = e - a.seg[0];
            u64 k1 = i >> a.log_n2, t = i & (n2 - 1);
            u64 j = k1 + (u64)n1 * gl::bitrev((u32)t, a.log_n2);
            a.scale[i] = gl::mul(gl::pow(7, j), a.n_inv);
        } else if (e < a.seg[2]) {  // twb[k1][q]
            u64 i = e - a.seg[1];
            u64 k1 = i >> a.log_M, q = i & (((u64)1 << a.log_M) - 1);
            a.twb[i] = gl::pow(a.w_N, (k1 * q) & N_mask);
        } else if (e < a.seg[3]) {
            u64 i = e - a.seg[2];
            a.rinv_n1[i] = gl::pow(a.w_n1_inv, i);
        } else if (e < a.seg[4]) {
            u64 i = e - a.seg[3];
            a.rinv_n2[i] = gl::pow(a.w_n2_inv, i);
        } else if (e < a.seg[5]) {
            u64 i = e - a.seg[4];
            a.rfwd_M[i] = gl::pow(a.w_M, i);
        } else {
            u64 i = e - a.seg[5];
            a.rfwd_n1[i] = gl::pow(a.w_n1, i);
        }
    }
}

cudaError_t build_plan_tables(Plan& p, u64* base, cudaStream_t s)
{
    u32 l1, l2;
    plan_split(p.log_n, p.r, l1, l2);
    p.log_n1 = l1;
    p.log_n2 = l2;
    p.log_M = l2 + p.r;
    p.log_N = p.log_n + p.r;
    size_t n = (size_t)1 << p.log_n, N = n << p.r;
    TableArgs a;
    u64* cur = base;
    a.twa = l1 ? cur : nullptr;
    cur += l1 ? n : 0;
    a.scale = cur;
    cur += n;
    a.twb = l1 ? cur : nullptr;
    cur += l1 ? N : 0;
    a.rinv_n1 = cur;
    cur += half_or_one(l1);
    a.rinv_n2 = cur;
    cur += half_or_one(l2);
    a.rfwd_M = cur;
    cur += half_or_one(p.log_M);
    a.rfwd_n1 = cur;
    cur += half_or_one(l1);
    a.seg[0] = l1 ? n : 0;
    a.seg[1] = a.seg[0] + n;
    a.seg[2] = a.seg[1] + (l1 ? N : 0);
    a.seg[3] = a.seg[2] + half_or_one(l1);
    a.seg[4] = a.seg[3] + half_or_one(l2);
    a.seg[5] = a.seg[4] + half_or_one(p.log_M);
    a.seg[6] = a.seg[5] + half_or_one(l1);
    a.w_n_inv = hinv(hroot(p.log_n));
    a.w_N = hroot(p.log_N);
    a.w_n1_inv = hinv(hroot(l1));
    a.w_n2_inv = hinv(hroot(l2));
    a.w_M = hroot(p.log_M);
    a.w_n1 = hroot(l1);
    a.n_inv = hinv(n % gl::P);
    a.log_n = p.log_n;
    a.log_n1 = l1;
    a.log_n2 = l2;
    a.log_M = p.log_M;
    a.log_N = p.log_N;
    p.twa = a.twa;
    p.scale = a.scale;
    p.twb = a.twb;
    p.rinv_n1 = a.rinv_n1;
    p.rinv_n2 = a.rinv_n2;
    p.rfwd_M = a.rfwd_M;
    p.rfwd_n1 = a.rfwd_n1;
    u64 total = a.seg[6];
    int grid = (int)std::min<u64>((total + 255) / 256, (u64)num_sms() * 8);
    k_plan_tables<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- in-CTA DFTs

// B transforms of size L = 2^logL stored back to back in shared memory.
// Decimation in frequency: natural order in, bit-reversed order out.
// tw[j] = w_L^j (or w_L^-j) for j < L/2.  Butterfly (i, i+h) of the stage
// with half-span h uses w_{2h}^pos = tw[pos << s].
__device__ __forceinline__ void dft_dif(u64* a, u32 B, u32 logL, const u64* tw)
{
    if (logL == 0) return;
    u32 half = 1u << (logL - 1);
    u32 total = B << (logL - 1);
    for (u32 s = 0; s < logL; s++) {
        u32 h = half >> s;
        for (u32 b = threadIdx.x; b < total; b += blockDim.x) {
            u32 tr = b >> (logL - 1);
            u32 bb = b & (half - 1);
            u32 pos = bb & (h - 1);
            u32 i = ((bb - pos) << 1) + pos;
            u64* x = a + ((size_t)tr << logL);
            u64 u = x[i], v = x[i + h];
            x[i] = gl::add(u, v);
            x[i + h] = gl::mul(gl::sub(u, v), tw[pos << s]);
        }
        __syncthreads();
    }
}

// Decimation in time: bit-reversed order in, natural order out.  Stages
// s < first are skipped (the caller has already applied them).
__device__ __forceinline__ void dft_dit(u64* a, u32 B, u32 logL, const u64* tw, u32 first)
{
    if (logL == 0) return;
    u32 half = 1u << (logL - 1);
    u32 total = B << (logL - 1);
    for (u32 s = first; s < logL; s++) {
        u32 h = 1u << s;
        for (u32 b = threadIdx.x; b < total; b += blockDim.x) {
            u32 tr = b >> (logL - 1);
            u32 bb = b & (half - 1);
            u32 pos = bb & (h - 1);
            u32 i = ((bb - pos) << 1) + pos;
            u64* x = a + ((size_t)tr << logL);
            u64 u = x[i];
            u64 t = gl::mul(x[i + h], tw[pos << (logL - 1 - s)]);
            x[i] = gl::add(u, t);
            x[i + h] = gl::sub(u, t);
        }
        __syncthreads();
    }
}

__device__ __forceinline__ u32 find_job(const u32* first, u32 njobs, u32 item)
{
    u32 lo = 0, hi = njobs;
    while (hi - lo > 1) {
        u32 mid = (lo + hi) >> 1;
        if (first[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- stage A

u32 stage_a_items(const LdeJob& j, const Tiles&)
{
    if (!j.plan.log_n1) return 0;
    return j.c * ((1u << j.plan.log_n2) / j.a_cols);
}

size_t stage_a_smem(const LdeJob& j, const Tiles&)
{
    if (!j.plan.log_n1) return 0;
    size_t n1 = (size_t)1 << j.plan.log_n1;
    return (j.a_cols * n1 + n1 / 2) * sizeof(u64);
}

__global__ void __launch_bounds__(256) k_stage_a(const LdeJob* __restrict__ jobs, StageList L)
{
    extern __shared__ u64 sm[];
    for (u32 item = blockIdx.x; item < L.total; item += gridDim.x) {
        u32 jid = find_job(L.first, L.njobs, item);
        const LdeJob& J = jobs[jid];
        u32 local = item - L.first[jid];
        const u32 l1 = J.plan.log_n1, l2 = J.plan.log_n2;
        const u32 n1 = 1u << l1, n2 = 1u << l2;
        const u32 T2 = J.a_cols, lT2 = __ffs(T2) - 1;
        const u32 tiles = n2 >> lT2;
        const u32 col = local / tiles, i20 = (local % tiles) << lT2;
        const u64* x = J.x + ((size_t)col << J.plan.log_n);
        u64* data = sm;
        u64* tw = sm + ((size_t)T2 << l1);
        for (u32 e = threadIdx.x; e < n1 / 2; e += blockDim.x) tw[e] = J.plan.rinv_n1[e];
        for (u32 e = threadIdx.x; e < (T2 << l1); e += blockDim.x) {
            u32 u = e & (T2 - 1), i1 = e >> lT2;
            data[((size_t)u << l1) + i1] = x[i20 + u + ((size_t)i1 << l2)];
        }
        __syncthreads();
        dft_dif(data, T2, l1, tw);
        u64* Y = J.Y + ((size_t)col << J.plan.log_n);
        for (u32 e = threadIdx.x; e < (T2 << l1); e += blockDim.x) {
            u32 u = e & (T2 - 1), t = e >> lT2;
            u32 k1 = gl::bitrev(t, l1);
            size_t o = ((size_t)k1 << l2) + i20 + u;
            Y[o] = gl::mul(data[((size_t)u << l1) + t], J.plan.twa[o]);
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- stage B

u32 stage_b_items(const LdeJob& j) { return j.c << j.plan.log_n1; }

size_t stage_b_smem(const LdeJob& j)
{
    size_t n2 = (size_t)1 << j.plan.log_n2, M = (size_t)1 << j.plan.log_M;
    return (M + n2 + std::max<size_t>(n2 / 2, 1) + std::max<size_t>(M / 2, 1)) * sizeof(u64);
}

__global__ void __launch_bounds__(512) k_stage_b(const LdeJob* __restrict__ jobs, StageList L)
{
    extern __shared__ u64 sm[];
    for (u32 item = blockIdx.x; item < L.total; item += gridDim.x) {
        u32 jid = find_job(L.first, L.njobs, item);
        const LdeJob& J = jobs[jid];
        u32 local = item - L.first[jid];
        const u32 l1 = J.plan.log_n1, l2 = J.plan.log_n2, lM = J.plan.log_M, r = J.plan.r;
        const u32 n1 = 1u << l1, n2 = 1u << l2, M = 1u << lM;
        const u32 col = local >> l1, k1 = local & (n1 - 1);
        u64* data = sm;              // [M]
        u64* stage = sm + M;         // [n2]
        u64* twi = stage + n2;       // [n2/2]
        u64* twf = twi + std::max(n2 / 2, 1u);  // [M/2]
        for (u32 e = threadIdx.x; e < n2 / 2; e += blockDim.x) twi[e] = J.plan.rinv_n2[e];
        for (u32 e = threadIdx.x; e < M / 2; e += blockDim.x) twf[e] = J.plan.rfwd_M[e];
        const u64* src = l1 ? J.Y + ((size_t)col << J.plan.log_n) + ((size_t)k1 << l2)
                            : J.x + ((size_t)col << J.plan.log_n);
        for (u32 e = threadIdx.x; e < n2; e += blockDim.x) stage[e] = src[e];
        __syncthreads();
        dft_dif(stage, 1, l2, twi);  // position t: n * a_{k1 + n1*bitrev(t)}
        const u64* sc = J.plan.scale + ((size_t)k1 << l2);
        // Scale by 7^j / n and spread for the zero-padded size-M transform.
        // In bit-reversed order over log M bits, coefficient k2 sits at
        // bitrev_n2(k2) << r; the first r DIT stages only copy each value
        // into the 2^r slots after it, so they are applied here directly.
        for (u32 e = threadIdx.x; e < M; e += blockDim.x) {
            u32 t = e >> r;
            data[e] = gl::mul(stage[t], sc[t]);
        }
        __syncthreads();
        dft_dit(data, 1, lM, twf, r);
        if (l1) {
            u64* Z = J.Z + ((size_t)col << J.plan.log_N) + ((size_t)k1 << lM);
            const u64* tb = J.plan.twb + ((size_t)k1 << lM);
            for (u32 e = threadIdx.x; e < M; e += blockDim.x) Z[e] = gl::mul(data[e], tb[e]);
        } else {
            // n1 = 1: this CTA holds the whole column; write committed rows.
            const bool pad = (col + 1 == J.c) && (J.c & 1) && J.c < J.ld;
            for (u32 e = threadIdx.x; e < M; e += blockDim.x) {
                size_t row = gl::bitrev(e, lM);
                J.lde[row * J.ld + col] = data[e];
                if (pad) J.lde[row * J.ld + col + 1] = 0;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- stage C

u32 stage_c_items(const LdeJob& j, const Tiles&)
{
    if (!j.plan.log_n1) return 0;
    u32 pairs = (j.c + 1) / 2;
    return pairs * ((1u << j.plan.log_M) / j.c_q);
}

size_t stage_c_smem(const LdeJob& j, const Tiles&)
{
    if (!j.plan.log_n1) return 0;
    size_t n1 = (size_t)1 << j.plan.log_n1;
    return (2 * j.c_q * n1 + n1 / 2) * sizeof(u64);
}

__global__ void __launch_bounds__(256) k_stage_c(const LdeJob* __restrict__ jobs, StageList L)
{
    extern __shared__ u64 sm[];
    for (u32 item = blockIdx.x; item < L.total; item += gridDim.x) {
        u32 jid = find_job(L.first, L.njobs, item);
        const LdeJob& J = jobs[jid];
        u32 local = item - L.first[jid];
        const u32 l1 = J.plan.log_n1, lM = J.plan.log_M;
        const u32 n1 = 1u << l1;
        const u32 Q = J.c_q, lQ = __ffs(Q) - 1;
        const u32 pairs = (J.c + 1) / 2;
        const u32 cp = local % pairs, q0 = (local / pairs) << lQ;  // pairs fastest: shared rows
        u64* data = sm;                          // [2][Q][n1]
        u64* tw = sm + ((size_t)2 * Q << l1);    // [n1/2]
        for (u32 e = threadIdx.x; e < n1 / 2; e += blockDim.x) tw[e] = J.plan.rfwd_n1[e];
        const u32 per = Q << l1;
        for (u32 e = threadIdx.x; e < 2 * per; e += blockDim.x) {
            u32 w = e / per, rem = e - w * per;
            u32 v = rem & (Q - 1), k1 = rem >> lQ;
            u32 col = 2 * cp + w;
            u64 val = 0;
            if (col < J.c)
                val = J.Z[((size_t)col << J.plan.log_N) + ((size_t)k1 << lM) + q0 + v];
            data[((size_t)(w * Q + v) << l1) + k1] = val;
        }
        __syncthreads();
        dft_dif(data, 2 * Q, l1, tw);
        const u32 c0 = 2 * cp;
        const bool two = c0 + 1 < J.ld;
        for (u32 e = threadIdx.x; e < per; e += blockDim.x) {
            u32 u = e & (n1 - 1), v = e >> l1;
            size_t row = ((size_t)gl::bitrev(q0 + v, lM) << l1) + u;
            u64 a = data[((size_t)v << l1) + u];
            u64 b = data[((size_t)(Q + v) << l1) + u];
            u64* dst = J.lde + row * J.ld + c0;
            if (J.vec_ok) {
                *reinterpret_cast<ulonglong2*>(dst) = make_ulonglong2(a, b);
            } else {
                dst[0] = a;
                if (two) dst[1] = b;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- launchers

// grid <= 0 picks a persistent grid: resident CTAs per SM (from the
// occupancy calculator) times the SM count, capped at the item count.
template <typename K>
static cudaError_t launch_persistent(K kernel, int threads, size_t smem, int grid, cudaStream_t s,
                                     const LdeJob* jobs, StageList l)
{
    if (l.total == 0) return cudaSuccess;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (grid <= 0) {
        int nb = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem);
        if (e != cudaSuccess) return e;
        grid = std::max(nb, 1) * num_sms();
    }
    grid = (int)std::min<u32>((u32)grid, l.total);
    kernel<<<grid, threads, smem, s>>>(jobs, l);
    return cudaGetLastError();
}

cudaError_t launch_stage_a(const LdeJob* d_jobs, StageList l, size_t smem, const Tiles& t, int grid,
                           cudaStream_t s)
{
    return launch_persistent(k_stage_a, t.a_threads, smem, grid, s, d_jobs, l);
}

cudaError_t launch_stage_b(const LdeJob* d_jobs, StageList l, size_t smem, const Tiles& t, int grid,
                           cudaStream_t s)
{
    return launch_persistent(k_stage_b, t.b_threads, smem, grid, s, d_jobs, l);
}

cudaError_t launch_stage_c(const LdeJob* d_jobs, StageList l, size_t smem, const Tiles& t, int grid,
                           cudaStream_t s)
{
    return launch_persistent(k_stage_c, t.c_threads, smem, grid, s, d_jobs, l);
}

// ---------------------------------------------------------------- misc kernels

__global__ void k_validate(const u64* __restrict__ x, u64 count, u32* flag)
{
    for (u64 i = blockIdx.x * (u64)blockDim.x + threadIdx.x; i < count; i += (u64)gridDim.x * blockDim.x)
        if (x[i] >= gl::P) {
            atomicOr(flag, 1u);
            return;
        }
}

cudaError_t launch_validate(const u64* x, u64 count, u32* d_flag, cudaStream_t s)
{
    if (!count) return cudaSuccess;
    int grid = (int)std::min<u64>((count + 255) / 256, (u64)num_sms() * 8);
    k_validate<<<grid, 256, 0, s>>>(x, count, d_flag);
    return cudaGetLastError();
}

// Integer-pipe microbenchmark: each thread runs 8 independent chains of
// 32x32->64 multiply-adds (mad.wide.u32), `iters` steps each.
__global__ void k_int_peak(u64* out, u32 iters)
{
    u32 a = threadIdx.x * 2654435761u + blockIdx.x;
    u64 acc[8];
#pragma unroll
    for (int k = 0; k < 8; k++) acc[k] = (u64)(a + k) * 0x9E3779B9u;
    for (u32 i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
#pragma unroll
            for (int rep = 0; rep < 4; rep++) acc[k] = (u64)(u32)acc[k] * (a | 1u) + acc[k];
        }
    }
    u64 x = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) x ^= acc[k];
    if (x == 0x123456789ull) out[blockIdx.x] = x;
}

cudaError_t launch_int_peak(u64* out, int grid, int threads, u32 iters, cudaStream_t s)
{
    k_int_peak<<<grid, threads, 0, s>>>(out, iters);
    return cudaGetLastError();
}

}  // namespace v3c
