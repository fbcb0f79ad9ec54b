// Poseidon-w12 permutation shared by one warp, for latency-bound chains
// (the codebook sponge of a snapshot, the small top levels of Merkle trees).
//
// Lane l < 12 holds state word s_l, non-canonical in [0, 2^64); lanes 12-31
// take part in the shuffles only.  A round applies the S-box (every lane in
// a full round, lane 0 in a partial one) and forms its MDS row plus the next
// round's constant,
//   s'_l = sum_j m[(j - l) mod 12] s_j + rc_(r+1)[l],
// on 21/21/22-bit limbs: every lane splits its word once, each term is three
// 32-bit shuffles and three 32-bit multiply-adds in two accumulators per
// limb (no carries: sum m < 2^9 and the constant limbs are below 2^22, so
// every sum stays below 2^32), and the limb sums are folded once per round.
// In partial rounds the 11 terms of the pre-S-box words accumulate while
// lane 0 runs its S-box.  The round constants' limbs sit in shared memory,
// one 16-byte row per lane and round.  The rounds are those of
// poseidon.cuh (4 full, 22 partial, 4 full, Sec. 4.3).
#pragma once
#include "gl.cuh"
#include "poseidon.cuh"

namespace v3c {
namespace pos {

__constant__ u32 c_mds_row_w[12] = V3C_MDS_ROW_INIT;

// Limbs (a, b, c) of rc_r[l] for r < 30; row 30 is zero.
struct WarpRc {
    uint4 v[31][12];
};

// Fills t; every thread of the block calls it, then the block synchronises.
__device__ __forceinline__ void warp_rc_init(WarpRc& t, u32 tid, u32 nthreads)
{
    for (u32 e = tid; e < 31 * 12; e += nthreads) {
        const u32 r = e / 12, i = e % 12;
        const u64 v = r < 30 ? c_rc[r][i] : 0;
        t.v[r][i] = make_uint4((u32)v & 0x1FFFFFu, (u32)(v >> 21) & 0x1FFFFFu, (u32)(v >> 42), 0);
    }
}

// This lane's MDS row: m[j] = row[(j - l) mod 12].
__device__ __forceinline__ void warp_mds_row(u32 (&m)[12], u32 lane)
{
    const u32 li = lane < 12 ? lane : 0;
#pragma unroll
    for (int j = 0; j < 12; j++) m[j] = c_mds_row_w[(j + 12 - li) % 12];
}

// Products for a latency-bound chain: the reduction written with compares
// (gl::reduce128) has a shorter dependency chain than the carry-chain form.
__device__ __forceinline__ u64 mul_lat(u64 a, u64 b) { return gl::reduce128(a * b, __umul64hi(a, b)); }

// x^7 on non-canonical values (inputs and output in [0, 2^64)).
__device__ __forceinline__ u64 sbox7_lat(u64 x)
{
    u64 x2 = mul_lat(x, x);
    u64 x3 = mul_lat(x2, x);
    u64 x4 = mul_lat(x2, x2);
    return mul_lat(x3, x4);
}

__device__ __forceinline__ void limbs21(u64 v, u32& a, u32& b, u32& c)
{
    a = (u32)v & 0x1FFFFFu;
    b = (u32)(v >> 21) & 0x1FFFFFu;
    c = (u32)(v >> 42);
}

// Accumulates the MDS terms j in [J0, 12) of this lane's row from the
// senders' limbs into two accumulators per limb (shorter chains).
template <int J0>
__device__ __forceinline__ void warp_mds_terms(u32 a, u32 b, u32 c, const u32 (&m)[12], u32 (&A)[2], u32 (&B)[2],
                                               u32 (&C)[2])
{
#pragma unroll
    for (int j = J0; j < 12; j++) {
        A[j & 1] += __shfl_sync(0xffffffffu, a, j) * m[j];
        B[j & 1] += __shfl_sync(0xffffffffu, b, j) * m[j];
        C[j & 1] += __shfl_sync(0xffffffffu, c, j) * m[j];
    }
}

// One round on this lane's word; the accumulators start from the next
// round's constant limbs.
__device__ __forceinline__ u64 warp_round(u64 x, int r, bool full, const WarpRc& t, const u32 (&m)[12], u32 lane)
{
    const bool own = lane < 12;
    const uint4 k = t.v[r + 1][own ? lane : 0];
    u32 A[2] = {own ? k.x : 0, 0}, B[2] = {own ? k.y : 0, 0}, C[2] = {own ? k.z : 0, 0};
    u32 a, b, c;
    if (full) {
        limbs21(sbox7_lat(x), a, b, c);
        warp_mds_terms<0>(a, b, c, m, A, B, C);
    } else {
        // Terms j >= 1 use the pre-S-box words and overlap lane 0's S-box.
        limbs21(x, a, b, c);
        warp_mds_terms<1>(a, b, c, m, A, B, C);
        u32 ya, yb, yc;
        limbs21(sbox7_lat(x), ya, yb, yc);
        A[0] += __shfl_sync(0xffffffffu, ya, 0) * m[0];
        B[0] += __shfl_sync(0xffffffffu, yb, 0) * m[0];
        C[0] += __shfl_sync(0xffffffffu, yc, 0) * m[0];
    }
    return limb_fold21(A[0] + A[1], B[0] + B[1], C[0] + C[1]);
}

// The permutation of the state held one word per lane; every lane of the
// warp calls it (the shuffles use the full mask).
__device__ __forceinline__ u64 permute_warp(u64 x, const WarpRc& t, const u32 (&m)[12], u32 lane)
{
    x = gl::add_nc_small(x, lane < 12 ? c_rc[0][lane] : 0);  // round 0's constant; later ones ride the MDS
#pragma unroll 1
    for (int r = 0; r < 4; r++) x = warp_round(x, r, true, t, m, lane);
#pragma unroll 1
    for (int r = 4; r < 26; r++) x = warp_round(x, r, false, t, m, lane);
#pragma unroll 1
    for (int r = 26; r < 30; r++) x = warp_round(x, r, true, t, m, lane);
    return x;
}

}  // namespace pos
}  // namespace v3c
