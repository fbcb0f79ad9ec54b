// Poseidon-w12 permutation on the device (one thread per state).
//
// The hash is Poseidon (Sec. 4.3): width 12, S-box x^7, rounds 4 full,
// 22 partial and 4 full, each round ARC -> S-box -> MDS.  The constants are
// generated at build time (gen_params.cpp).
//
// Evaluation orders (all exact; selected by the Cfg template):
//   plain  the round loop as defined, one loop body for all 30 rounds so the
//          code stays small enough for the instruction cache;
//   fast   the partial rounds in the equivalent sparse form of the Poseidon
//          paper (Grassi et al., "efficient partial rounds").  Each partial
//          round adds one scalar to lane 0, applies the S-box to lane 0 and
//          multiplies by [[m_0, v_k^T], [w_k, I]].  A dense 11x11 block D_0 is
//          applied after the MDS of round 3.  gen_params.cpp derives the
//          constants and checks on the host that both orders agree.
// MDS products (the MDS row has entries below 64):
//   wide   each 32-bit half of a lane times the entry, a 32x32->64
//          multiply-add into a 42-bit accumulator;
//   limb   each lane in 22-bit limbs, so that every product and its
//          12-term sum fit one 32-bit multiply-add (full-rate IMAD);
//   split  limbs of 21, 21 and 22 bits through the block form of the
//          circulant ([[A, B], [B, A]], two 6x6 products per limb), the two
//          21-bit limbs through a second 3x3 block split (54 products per
//          limb instead of 72): 180 32-bit multiply-adds per MDS.
// Values inside the permutation are non-canonical in [0, 2^64).
#pragma once
#include "gl.cuh"
#include "poseidon_params.h"

namespace v3c {
namespace pos {

using gl::u32;
using gl::u64;

__constant__ u64 c_rc[30][12] = V3C_RC_INIT;
__constant__ u64 c_fast_a[22] = V3C_FAST_A_INIT;
__constant__ u64 c_fast_v[22 * 11] = V3C_FAST_V_INIT;
__constant__ u64 c_fast_w[22 * 11] = V3C_FAST_W_INIT;
__constant__ u64 c_fast_d0[11 * 11] = V3C_FAST_D0_INIT;
// Full rounds 0-3, then 26-29 with the constants carried out of the fast
// partial rounds folded into round 26.
__constant__ u64 c_rc_full[8 * 12] = V3C_FAST_RC_FULL_INIT;
// Round constants as 22-bit limbs [round 0..30][lane][3]; row 30 is zero.
__constant__ u32 c_rc_limbs[31 * 12 * 3] = V3C_RC_LIMBS_INIT;
// Round constants for the split MDS [round 0..30][36] (see gen_params.cpp).
__constant__ u32 c_rc_split[31 * 36] = V3C_RC_SPLIT_INIT;
// Zero accumulator starts, for an MDS that adds no constant.
__constant__ u32 c_zero36[36] = {0};

__host__ __device__ constexpr u32 mds_coef(int k)
{
    constexpr u32 row[12] = V3C_MDS_ROW_INIT;
    return row[k];
}

enum MulKind { MUL_INTRINSIC = 0, MUL_PTX = 1, MUL_WIDE = 2 };
// MDS_SPLIT: 21-bit limbs (the top one 22 bits); every limb vector uses the
// block form of the circulant, two 6x6 products instead of one 12x12 (see
// mds_split).
enum MdsKind { MDS_WIDE = 0, MDS_LIMB = 1, MDS_SPLIT = 2 };

// FOLD2: the limb sums are recombined with 32x32->64 multiply-adds and one
// carry chain instead of shifts and compares.  ARCM: the round constants of
// round r+1 start the limb accumulators of round r's MDS, so the constant
// addition costs nothing after round 0.
// FOLD3 / RED: the limb fold and the 128-bit reduction written as PTX
// carry chains (no compares or selects).
template <int MUL_, int MDS_, bool SQR_, bool FAST_, bool FOLD2_ = false, bool ARCM_ = false,
          bool FOLD3_ = false, bool RED_ = false, int SHIFT_ = 0>
struct Cfg {
    static constexpr int MUL = MUL_;
    static constexpr int MDS = MDS_;
    static constexpr bool SQR = SQR_;
    static constexpr bool FAST = FAST_;
    static constexpr bool FOLD2 = FOLD2_;
    static constexpr bool ARCM = ARCM_;
    static constexpr bool FOLD3 = FOLD3_;
    static constexpr bool RED = RED_;
    static constexpr int SHIFT = SHIFT_;
};

// A + B 2^22 + C 2^44 (A, B, C < 2^32) to [0, 2^64) with carry chains:
// w0 = A + (B << 22) carries c0; w1 = (B >> 10) + (C << 12 mod 2^32) + c0
// carries c1; the multiple of 2^64 is h = (C >> 20) + c1 < 2^13, folded as
// h EPS = h 2^32 - h.  (w1:w0) + h EPS carries at most once, and after a
// carry the sum is below 2^45, so adding EPS cannot carry again.
__device__ __forceinline__ u64 limb_fold3(u32 A, u32 B, u32 Cc)
{
    u64 r;
    asm("{\n\t"
        ".reg .u32 t, u, v, w0, w1, hh, h, u0, u1, r0, r1, c;\n\t"
        "shl.b32 t, %2, 22;\n\t"
        "add.cc.u32 w0, %1, t;\n\t"
        "shr.b32 u, %2, 10;\n\t"
        "shl.b32 v, %3, 12;\n\t"
        "addc.cc.u32 w1, u, v;\n\t"
        "shr.b32 hh, %3, 20;\n\t"
        "addc.u32 h, hh, 0;\n\t"
        "sub.cc.u32 u0, 0, h;\n\t"
        "subc.u32 u1, h, 0;\n\t"
        "add.cc.u32 r0, w0, u0;\n\t"
        "addc.cc.u32 r1, w1, u1;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "sub.cc.u32 r0, r0, c;\n\t"       // + c EPS = + c 2^32 - c
        "subc.u32 r1, r1, 0;\n\t"
        "add.u32 r1, r1, c;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "r"(A), "r"(B), "r"(Cc));
    return r;
}
// The configuration the library's kernels use (fastest measured on GB300:
// split MDS, round constants merged into the MDS accumulators, PTX
// carry-chain reduction, compiler 64x64 products, plain round order).  The
// permutation is bound by the IMAD (FMA-heavy) pipe.
typedef Cfg<MUL_INTRINSIC, MDS_SPLIT, false, false, false, true, false, true> Default;

struct U128 {
    u64 lo, hi;
};

__device__ __forceinline__ U128 mul128_ptx(u64 a, u64 b)
{
    u32 r0, r1, r2, r3;
    asm("{\n\t"
        ".reg .u32 a0, a1, b0, b1;\n\t"
        "mov.b64 {a0, a1}, %4;\n\t"
        "mov.b64 {b0, b1}, %5;\n\t"
        "mul.lo.u32 %0, a0, b0;\n\t"
        "mul.hi.u32 %1, a0, b0;\n\t"
        "mad.lo.cc.u32 %1, a0, b1, %1;\n\t"
        "madc.hi.u32 %2, a0, b1, 0;\n\t"
        "mad.lo.cc.u32 %1, a1, b0, %1;\n\t"
        "madc.hi.cc.u32 %2, a1, b0, %2;\n\t"
        "madc.hi.u32 %3, a1, b1, 0;\n\t"
        "mad.lo.cc.u32 %2, a1, b1, %2;\n\t"
        "addc.u32 %3, %3, 0;\n\t"
        "}"
        : "=&r"(r0), "=&r"(r1), "=&r"(r2), "=&r"(r3)
        : "l"(a), "l"(b));
    U128 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.lo) : "r"(r0), "r"(r1));
    asm("mov.b64 %0, {%1, %2};" : "=l"(r.hi) : "r"(r2), "r"(r3));
    return r;
}

// Four 32x32->64 products assembled with 64-bit adds.
__device__ __forceinline__ U128 mul128_wide(u64 a, u64 b)
{
    u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    u64 p00 = (u64)a0 * b0, p01 = (u64)a0 * b1, p10 = (u64)a1 * b0, p11 = (u64)a1 * b1;
    u64 mid = p01 + p10;
    u64 cm = mid < p01;
    u64 lo = p00 + (mid << 32);
    u64 c = lo < p00;
    u64 hi = p11 + (mid >> 32) + (cm << 32) + c;
    return {lo, hi};
}

// x^2 from three 32x32->64 products (the cross term doubled).
__device__ __forceinline__ U128 sqr128_wide(u64 x)
{
    u32 a0 = (u32)x, a1 = (u32)(x >> 32);
    u64 p00 = (u64)a0 * a0, p11 = (u64)a1 * a1, p01 = (u64)a0 * a1;
    u64 cm = p01 >> 63;
    u64 mid = p01 << 1;
    u64 lo = p00 + (mid << 32);
    u64 c = lo < p00;
    u64 hi = p11 + (mid >> 32) + (cm << 32) + c;
    return {lo, hi};
}

template <class C>
__device__ __forceinline__ U128 mul128(u64 a, u64 b)
{
    if (C::MUL == MUL_PTX) return mul128_ptx(a, b);
    if (C::MUL == MUL_WIDE) return mul128_wide(a, b);
    return {a * b, __umul64hi(a, b)};
}

template <class C>
__device__ __forceinline__ u64 reduce(U128 p)
{
    return C::RED ? gl::reduce128_ptx(p.lo, p.hi) : gl::reduce128(p.lo, p.hi);
}

template <class C>
__device__ __forceinline__ u64 mulmod(u64 a, u64 b)
{
    return reduce<C>(mul128<C>(a, b));
}

template <class C>
__device__ __forceinline__ u64 sqrmod(u64 a)
{
    if (C::SQR) return reduce<C>(sqr128_wide(a));
    return mulmod<C>(a, a);
}

template <class C>
__device__ __forceinline__ u64 sbox(u64 x)
{
    u64 x2 = sqrmod<C>(x);
    u64 x3 = mulmod<C>(x2, x);
    u64 x4 = sqrmod<C>(x2);
    return mulmod<C>(x3, x4);
}

// L + H * 2^32 for L, H < 2^42, folded to [0, 2^64).
__device__ __forceinline__ u64 mds_fold(u64 L, u64 H)
{
    u32 hl = (u32)H, hh = (u32)(H >> 32);
    u64 v = L + ((u64)hl << 32);
    u32 c = v < L;
    u32 x = hh + c;
    u64 t = ((u64)x << 32) - x;
    u64 r = v + t;
    if (r < t) r += gl::EPS;
    return r;
}

// A + B 2^22 + C 2^44 for A, B, C < 2^32, folded to [0, 2^64).
__device__ __forceinline__ u64 limb_fold(u32 A, u32 B, u32 Cc)
{
    u64 x = (u64)A + ((u64)B << 22);              // < 2^55
    u64 y = x + ((u64)(Cc & 0xFFFFFu) << 44);     // may carry once
    u32 c = y < x;
    u32 h = (Cc >> 20) + c;                        // multiple of 2^64, < 2^13
    u64 t = ((u64)h << 32) - h;                    // h * (2^64 mod p)
    u64 r = y + t;
    if (r < t) r += gl::EPS;
    return r;
}

// A + B 2^22 + C 2^44 for A, B, C < 2^32, folded to [0, 2^64) with wide
// multiply-adds: x = A + B 2^22 (< 2^55); t = hi32(x) + C 2^12 (< 2^45) is the
// word above bit 32, so V = lo32(x) + lo32(t) 2^32 + h 2^64 with h = t >> 32
// (< 2^13), and 2^64 = EPS (mod p).  v + h EPS carries at most once, and
// after a carry the sum is below 2^45, so adding EPS cannot carry again.
__device__ __forceinline__ u64 limb_fold2(u32 A, u32 B, u32 Cc)
{
    u64 x = (u64)B * (1u << 22) + A;
    u64 t = (u64)Cc * (1u << 12) + (u32)(x >> 32);
    u32 h = (u32)(t >> 32);
    u64 v = ((u64)(u32)t << 32) | (u32)x;
    u64 u = (u64)h * 0xFFFFFFFFu;
    u64 r;
    u32 c;
    asm("{\n\t"
        ".reg .u32 v0, v1, u0, u1, r0, r1;\n\t"
        "mov.b64 {v0, v1}, %2;\n\t"
        "mov.b64 {u0, u1}, %3;\n\t"
        "add.cc.u32 r0, v0, u0;\n\t"
        "addc.cc.u32 r1, v1, u1;\n\t"
        "addc.u32 %1, 0, 0;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r), "=r"(c)
        : "l"(v), "l"(u));
    return (u64)c * 0xFFFFFFFFu + r;
}

// A + B 2^21 + C 2^42 (A, B, C < 2^32) to [0, 2^64): w0 = A + (B << 21)
// carries c0; w1 = (B >> 11) + (C << 10 mod 2^32) + c0 carries c1; the
// multiple of 2^64 is h = (C >> 22) + c1 < 2^11, folded as h EPS.  The last
// step carries at most once, and after a carry the sum is below 2^43.
__device__ __forceinline__ u64 limb_fold21(u32 A, u32 B, u32 Cc)
{
    u64 r;
    asm("{\n\t"
        ".reg .u32 t, u, v, w0, w1, hh, h, u0, u1, r0, r1, c;\n\t"
        "shl.b32 t, %2, 21;\n\t"
        "add.cc.u32 w0, %1, t;\n\t"
        "shr.b32 u, %2, 11;\n\t"
        "shl.b32 v, %3, 10;\n\t"
        "addc.cc.u32 w1, u, v;\n\t"
        "shr.b32 hh, %3, 22;\n\t"
        "addc.u32 h, hh, 0;\n\t"
        "sub.cc.u32 u0, 0, h;\n\t"
        "subc.u32 u1, h, 0;\n\t"
        "add.cc.u32 r0, w0, u0;\n\t"
        "addc.cc.u32 r1, w1, u1;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "sub.cc.u32 r0, r0, c;\n\t"
        "subc.u32 r1, r1, 0;\n\t"
        "add.u32 r1, r1, c;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "r"(A), "r"(B), "r"(Cc));
    return r;
}


// acc + x K for a constant K (mod 2^32; K is a compile-time constant once the
// MDS loops are unrolled).  With shift set, constants with at most two set
// bits, or of the form 2^a - 2^b, are built from shifts and adds (integer ALU
// pipe) instead of one multiply-add (the IMAD pipe, which the permutation
// otherwise saturates).  Negative K subtracts.
// Bit counts of 0 <= a < 256 with fixed-bound loops, so that they fold to
// constants after the MDS loops are unrolled.
__host__ __device__ __forceinline__ constexpr int cpop(int a)
{
    int n = 0;
    for (int b = 0; b < 8; b++) n += (a >> b) & 1;
    return n;
}
__host__ __device__ __forceinline__ constexpr int chi(int a)
{
    int h = 0;
    for (int b = 0; b < 8; b++)
        if ((a >> b) & 1) h = b;
    return h;
}
__host__ __device__ __forceinline__ constexpr int clo(int a)
{
    int l = 0;
    for (int b = 7; b >= 0; b--)
        if ((a >> b) & 1) l = b;
    return l;
}

// shift: 0 never; 1 for constants with one bit set (one shift-add, LEA, in
// place of one multiply-add); 2 for up to two bits set; 3 also for
// 2^(hi+1) - 2^lo.
__device__ __forceinline__ u32 mac_const(u32 acc, u32 x, int K, int shift)
{
    const int A = K < 0 ? -K : K;
    const int pc = cpop(A), hi = chi(A), lo = clo(A);
    const bool sub_form = pc > 2 && ((1 << (hi + 1)) - (1 << lo)) == A;
    const bool use = shift >= 3 ? (pc <= 2 || sub_form) : shift >= pc;
    if (!use || A == 0) return acc + x * (u32)K;
    u32 t;
    if (pc == 1)
        t = x << lo;
    else if (pc == 2)
        t = (x << hi) + (x << lo);
    else
        t = (x << (hi + 1)) - (x << lo);
    return K < 0 ? acc - t : acc + t;
}

// Block form of the circulant: with x = (x_top, x_bot) in halves of 6,
// M = [[A, B], [B, A]], so y_top + y_bot = (A + B)(x_top + x_bot) and
// y_top - y_bot = (A - B)(x_top - x_bot).  A + B is the 6x6 circulant of
// s_k = m_k + m_(k+6); A - B has entries m[(j-i) mod 12] - m[(j-i+6) mod 12].
__host__ __device__ constexpr u32 split_s(int k) { return mds_coef(k) + mds_coef(k + 6); }
__host__ __device__ constexpr u32 split_d(int i, int j)
{
    return mds_coef(((j - i) % 12 + 12) % 12) - mds_coef(((j - i + 6) % 12 + 12) % 12);  // mod 2^32
}

// Sums over the MDS row and over one row of |A - B|, for the bounds below.
__host__ __device__ constexpr u32 mds_row_sum()
{
    u32 t = 0;
    for (int k = 0; k < 12; k++) t += mds_coef(k);
    return t;
}
__host__ __device__ constexpr u32 split_d_abs_sum()
{
    u32 t = 0;
    for (int j = 0; j < 6; j++) {
        int d = (int)mds_coef(j) - (int)mds_coef(j + 6);
        t += (u32)(d < 0 ? -d : d);
    }
    return t;
}
// Limbs below 2^22 (the top limb of a 64-bit lane; the low limbs are
// narrower), constants' limbs below 2^22 as well.  P sums S = sum(m) < 2^10
// products of u = x_j + x_(j+6) < 2^23; Q sums products of |v| < 2^22 with
// |A - B| entries; y = sum_j m x_j + rc < S 2^22 + 2^22, and P + Q, P - Q are
// 2 y, so none of them leaves [0, 2^32) (|Q| stays below 2^31).
static_assert((unsigned long long)mds_row_sum() * ((1u << 23) - 2) + (1u << 23) < (1ull << 32), "P bound");
static_assert((unsigned long long)(split_d_abs_sum() + 1) * (1u << 22) < (1ull << 31), "Q bound");
static_assert(2ull * ((unsigned long long)mds_row_sum() * ((1u << 22) - 1) + (1u << 22)) < (1ull << 32),
              "output bound");

// y = M x + rc for one vector of limbs below 2^22.  The 32-bit sums are exact
// (bounds above): P and Q as signed values mod 2^32, P + Q and P - Q as the
// even values 2 y, so the halving is a logical shift.  init = [P inits (6),
// Q inits (6)]: rc_i + rc_(i+6) and rc_i - rc_(i+6).
template <class C>
__device__ __forceinline__ void split6(const u32 (&x)[12], const u32* init, u32 (&y)[12])
{
    u32 u[6], v[6];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        u[j] = x[j] + x[j + 6];
        v[j] = x[j] - x[j + 6];
    }
#pragma unroll
    for (int i = 0; i < 6; i++) {
        u32 P = init[i], Q = init[6 + i];
#pragma unroll
        for (int j = 0; j < 6; j++) {
            P = mac_const(P, u[j], (int)split_s((j - i + 6) % 6), C::SHIFT);
            Q = mac_const(Q, v[j], (int)split_d(i, j), C::SHIFT);
        }
        y[i] = (P + Q) >> 1;
        y[i + 6] = (P - Q) >> 1;
    }
}

// The circulant part A + B (entries s_k) is itself [[S0, S1], [S1, S0]] in
// 3 x 3 blocks: S0 + S1 is the 3-circulant of s_k + s_(k+3), S0 - S1 has
// entries s_((j-i) mod 6) - s_((j-i+3) mod 6).  For limbs below 2^21 this
// second split keeps every sum in 32 bits, and both halvings are merged:
// with P' = P_i + P_(i+3), Q' = P_i - P_(i+3) (i < 3) and Q2 = 2 Q,
//   y_i = (P' + Q' + Q2_i) / 4,        y_(i+6) = (P' + Q' - Q2_i) / 4,
//   y_(i+3) = (P' - Q' + Q2_(i+3)) / 4, y_(i+9) = (P' - Q' - Q2_(i+3)) / 4.
// 54 multiply-adds per limb vector instead of 72.
__host__ __device__ constexpr u32 split_sp(int k) { return split_s(k) + split_s(k + 3); }
__host__ __device__ constexpr u32 split_dd(int i, int j)
{
    return split_s(((j - i) % 6 + 6) % 6) - split_s(((j - i + 3) % 6 + 6) % 6);  // mod 2^32
}
__host__ __device__ constexpr u32 split_dd_abs_sum()
{
    u32 t = 0;
    for (int j = 0; j < 3; j++) {
        int d = (int)split_dd(0, j);
        t += (u32)(d < 0 ? -d : d);
    }
    return t;
}
// Limbs and constant limbs below 2^21: P' < S (2^23 - 4) + 2^23, |Q'| and
// |Q2| below 2^31, and 4 y < 4 (S (2^21 - 1) + 2^21) < 2^32.
static_assert((unsigned long long)mds_row_sum() * ((1u << 23) - 4) + (1u << 23) < (1ull << 32), "P' bound");
static_assert((unsigned long long)(split_dd_abs_sum() + 1) * (1u << 23) < (1ull << 31), "Q' bound");
static_assert(2ull * (split_d_abs_sum() + 1) * (1u << 21) < (1ull << 31), "Q2 bound");
static_assert(4ull * ((unsigned long long)mds_row_sum() * ((1u << 21) - 1) + (1u << 21)) < (1ull << 32),
              "4y bound");

// y = M x + rc for one vector of limbs below 2^21.  init = [P' inits (3),
// Q' inits (3), Q2 inits (6)], from the constants' limbs as for the values.
template <class C>
__device__ __forceinline__ void split6_2(const u32 (&x)[12], const u32* init, u32 (&y)[12])
{
    u32 u[6], v[6], up[3], vp[3];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        u[j] = x[j] + x[j + 6];
        v[j] = x[j] - x[j + 6];
    }
#pragma unroll
    for (int j = 0; j < 3; j++) {
        up[j] = u[j] + u[j + 3];
        vp[j] = u[j] - u[j + 3];
    }
    u32 A[3], B[3], Q2[6];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        u32 Pp = init[i], Qp = init[3 + i];
#pragma unroll
        for (int j = 0; j < 3; j++) {
            Pp = mac_const(Pp, up[j], (int)split_sp((j - i + 3) % 3), C::SHIFT);
            Qp = mac_const(Qp, vp[j], (int)split_dd(i, j), C::SHIFT);
        }
        A[i] = Pp + Qp;
        B[i] = Pp - Qp;
    }
#pragma unroll
    for (int i = 0; i < 6; i++) {
        u32 q = init[6 + i];
#pragma unroll
        for (int j = 0; j < 6; j++) q = mac_const(q, v[j], (int)(2u * split_d(i, j)), C::SHIFT);
        Q2[i] = q;
    }
#pragma unroll
    for (int i = 0; i < 3; i++) {
        y[i] = (A[i] + Q2[i]) >> 2;
        y[i + 6] = (A[i] - Q2[i]) >> 2;
        y[i + 3] = (B[i] + Q2[i + 3]) >> 2;
        y[i + 9] = (B[i] - Q2[i + 3]) >> 2;
    }
}

// s <- M s (+ the next round's constants, from init) with limbs of 21, 21
// and 22 bits, each through the block form; the two 21-bit limbs through the
// second split as well.
template <class C>
__device__ __forceinline__ void mds_split(u64 (&s)[12], const u32* init)
{
    u32 a[12], b[12], c[12];
#pragma unroll
    for (int j = 0; j < 12; j++) {
        a[j] = (u32)s[j] & 0x1FFFFFu;
        b[j] = (u32)(s[j] >> 21) & 0x1FFFFFu;
        c[j] = (u32)(s[j] >> 42);
    }
    u32 ya[12], yb[12], yc[12];
    split6_2<C>(a, init, ya);
    split6_2<C>(b, init + 12, yb);
    split6<C>(c, init + 24, yc);
#pragma unroll
    for (int i = 0; i < 12; i++) s[i] = limb_fold21(ya[i], yb[i], yc[i]);
}

// s <- M s, M[i][j] = m[(j - i) mod 12].  With C::ARCM the accumulators start
// from the limbs `init` (the next round's constants), so the output is
// M s + RC.
template <class C>
__device__ __forceinline__ void mds(u64 (&s)[12], const u32* init = nullptr)
{
    if constexpr (C::MDS == MDS_SPLIT) {
        mds_split<C>(s, init ? init : c_zero36);
        return;
    }
    u64 out[12];
    if (C::MDS == MDS_LIMB) {
        u32 a[12], b[12], c[12];
#pragma unroll
        for (int j = 0; j < 12; j++) {
            a[j] = (u32)s[j] & 0x3FFFFFu;
            b[j] = (u32)(s[j] >> 22) & 0x3FFFFFu;
            c[j] = (u32)(s[j] >> 44);
        }
#pragma unroll
        for (int i = 0; i < 12; i++) {
            // Bounds: 12 * 63 * (2^22 - 1) + 2^22 < 2^32, so no limb sum wraps.
            u32 A = 0, B = 0, Cc = 0;
            if (C::ARCM) {
                A = init[3 * i];
                B = init[3 * i + 1];
                Cc = init[3 * i + 2];
            }
#pragma unroll
            for (int j = 0; j < 12; j++) {
                const u32 m = mds_coef((j - i + 12) % 12);
                A += a[j] * m;
                B += b[j] * m;
                Cc += c[j] * m;
            }
            out[i] = C::FOLD3 ? limb_fold3(A, B, Cc) : C::FOLD2 ? limb_fold2(A, B, Cc) : limb_fold(A, B, Cc);
        }
    } else {
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
            out[i] = mds_fold(L, H);
        }
    }
#pragma unroll
    for (int i = 0; i < 12; i++) s[i] = out[i];
}

// ---------------------------------------------------------------- plain form

// Rounds 0-3 and 26-29 full, 4-25 partial, in one loop body.
template <class C>
__device__ __forceinline__ void permute_plain(u64 (&s)[12])
{
    if constexpr (C::ARCM) {
        // Round 0's constants are added here; every MDS adds the next round's.
#pragma unroll
        for (int i = 0; i < 12; i++) s[i] = gl::add_nc_small(s[i], c_rc[0][i]);
#pragma unroll 1
        for (int r = 0; r < 30; r++) {
            if (r < 4 || r >= 26) {
#pragma unroll
                for (int i = 0; i < 12; i++) s[i] = sbox<C>(s[i]);
            } else {
                s[0] = sbox<C>(s[0]);
            }
            mds<C>(s, (C::MDS == MDS_SPLIT ? c_rc_split : c_rc_limbs) + (r + 1) * 36);
        }
    } else {
#pragma unroll 1
        for (int r = 0; r < 30; r++) {
            if (r < 4 || r >= 26) {
#pragma unroll
                for (int i = 0; i < 12; i++) s[i] = sbox<C>(gl::add_nc_small(s[i], c_rc[r][i]));
            } else {
#pragma unroll
                for (int i = 0; i < 12; i++) s[i] = gl::add_nc_small(s[i], c_rc[r][i]);
                s[0] = sbox<C>(s[0]);
            }
            mds<C>(s);
        }
    }
}

// ---------------------------------------------------------------- fast form

// Accumulates 64x64 products into a 3-word (lo, hi, top) integer.
struct Acc {
    u64 lo, hi;
    u32 top;
};

template <class C>
__device__ __forceinline__ void acc_add(Acc& a, u64 x, u64 k)
{
    U128 p = mul128<C>(x, k);
    if (C::RED) {
        // (lo, hi, top) += p as one carry chain.
        asm("add.cc.u64 %0, %0, %3;\n\t"
            "addc.cc.u64 %1, %1, %4;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+l"(a.lo), "+l"(a.hi), "+r"(a.top)
            : "l"(p.lo), "l"(p.hi));
        return;
    }
    u64 lo = a.lo + p.lo;
    u64 c1 = lo < p.lo;
    u64 hi = a.hi + p.hi;
    u32 c2 = hi < p.hi;
    u64 hi2 = hi + c1;
    c2 += hi2 < hi;
    a.lo = lo;
    a.hi = hi2;
    a.top += c2;
}

// lo + 2^64 hi + 2^128 top (top < 2^32) to [0, 2^64); 2^128 = -2^32 (mod p).
__device__ __forceinline__ u64 acc_reduce(const Acc& a)
{
    u64 r = gl::reduce128_ptx(a.lo, a.hi);
    u64 t = (u64)a.top << 32;
    u64 d = r - t;
    // On borrow d = r - t + 2^64 = r - t + EPS (mod p), and d >= 2^64 - 2^36 > EPS.
    if (r < t) d -= gl::EPS;
    return d;
}

template <class C>
__device__ __forceinline__ void apply_d0(u64 (&s)[12])
{
    u64 t[11];
#pragma unroll
    for (int i = 0; i < 11; i++) {
        Acc a{0, 0, 0};
#pragma unroll
        for (int j = 0; j < 11; j++) acc_add<C>(a, s[1 + j], c_fast_d0[i * 11 + j]);
        t[i] = acc_reduce(a);
    }
#pragma unroll
    for (int i = 0; i < 11; i++) s[1 + i] = t[i];
}

template <class C>
__device__ __forceinline__ void partial_fast(u64 (&s)[12], int k)
{
    u64 x0 = sbox<C>(gl::add_nc_small(s[0], c_fast_a[k]));
    Acc a{0, 0, 0};
    acc_add<C>(a, x0, (u64)mds_coef(0));
#pragma unroll
    for (int j = 0; j < 11; j++) acc_add<C>(a, s[1 + j], c_fast_v[k * 11 + j]);
#pragma unroll
    for (int j = 0; j < 11; j++) s[1 + j] = gl::add_nc(s[1 + j], mulmod<C>(x0, c_fast_w[k * 11 + j]));
    s[0] = acc_reduce(a);
}

template <class C>
__device__ __forceinline__ void full_round_idx(u64 (&s)[12], int f)
{
#pragma unroll
    for (int i = 0; i < 12; i++) s[i] = sbox<C>(gl::add_nc_small(s[i], c_rc_full[f * 12 + i]));
    mds<C>(s);
}

template <class C>
__device__ __forceinline__ void permute_fast(u64 (&s)[12])
{
#pragma unroll 1
    for (int h = 0; h < 2; h++) {
#pragma unroll 1
        for (int r = 0; r < 4; r++) full_round_idx<C>(s, 4 * h + r);
        if (h == 0) {
            apply_d0<C>(s);
#pragma unroll 1
            for (int k = 0; k < 22; k++) partial_fast<C>(s, k);
        }
    }
}

template <class C>
__device__ __forceinline__ void permute(u64 (&s)[12])
{
    if (C::FAST) permute_fast<C>(s);
    else permute_plain<C>(s);
}

}  // namespace pos
}  // namespace v3c
