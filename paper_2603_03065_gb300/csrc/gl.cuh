// Goldilocks field arithmetic on the device: p = 2^64 - 2^32 + 1.
//
// The reduction uses the special form of p instead of Montgomery or Barrett:
// 2^64 = 2^32 - 1 (mod p) and 2^96 = -1 (mod p).  A 128-bit value
// x = lo + 2^64 * (h0 + 2^32 * h1) is therefore congruent to
// lo - h1 + h0 * (2^32 - 1).  This needs one subtraction, one shifted
// subtraction and one addition, each with a single carry fix-up.
//
// Two value conventions are used:
//   canonical      values in [0, p), at every API boundary and in the NTT;
//   non-canonical  values in [0, 2^64), congruent mod p, inside the Poseidon
//                  permutation, to skip the conditional subtractions.
#pragma once
#include <stdint.h>

namespace gl {

typedef uint64_t u64;
typedef uint32_t u32;

constexpr u64 P = 0xFFFFFFFF00000001ull;
constexpr u64 EPS = 0xFFFFFFFFull;  // 2^64 mod p

__host__ __device__ __forceinline__ u64 canon(u64 x) { return x >= P ? x - P : x; }

// 128-bit (hi:lo) -> a value in [0, 2^64) congruent mod p.
__host__ __device__ __forceinline__ u64 reduce128(u64 lo, u64 hi)
{
    u32 h0 = (u32)hi;
    u32 h1 = (u32)(hi >> 32);
    u64 t0 = lo - h1;
    // Borrow: the wrapped value is lo - h1 + 2^64 = (lo - h1) + EPS (mod p),
    // and it is at least 2^64 - 2^32 + 1 > EPS, so subtracting EPS cannot wrap.
    if (lo < (u64)h1) t0 -= EPS;
    u64 t1 = ((u64)h0 << 32) - h0;  // h0 * (2^32 - 1) < 2^64
    u64 r = t0 + t1;
    // Carry: r + 2^64 = r + EPS; r < 2^64 - 2^33 here, so one fix-up suffices.
    if (r < t1) r += EPS;
    return r;
}

// The same reduction as PTX carry chains (no compares or selects).
// r = lo + h0 EPS carries c, then r - h1 borrows b; the true value is
// r + (c - b) 2^64 = r + (c - b) EPS (mod p).  With c = 1, b = 0:
// r < h0 EPS < 2^64 - 2^33, so r + EPS fits.  With c = 0, b = 1:
// r >= 2^64 - 2^32, so r - EPS >= 0.  With c = b there is no correction.
// The correction k EPS is added as a 64-bit two's-complement value: low word
// -k, high word the sign of k.
__device__ __forceinline__ u64 reduce128_ptx(u64 lo, u64 hi)
{
    u64 r;
    asm("{\n\t"
        ".reg .u32 l0, l1, h0, h1, u0, u1, r0, r1, c, b, k, nk, sk;\n\t"
        "mov.b64 {l0, l1}, %1;\n\t"
        "mov.b64 {h0, h1}, %2;\n\t"
        "sub.cc.u32 u0, 0, h0;\n\t"
        "subc.u32 u1, h0, 0;\n\t"
        "add.cc.u32 r0, l0, u0;\n\t"
        "addc.cc.u32 r1, l1, u1;\n\t"
        "addc.u32 c, 0, 0;\n\t"
        "sub.cc.u32 r0, r0, h1;\n\t"
        "subc.cc.u32 r1, r1, 0;\n\t"
        "subc.u32 b, 0, 0;\n\t"
        "add.u32 k, c, b;\n\t"
        "sub.u32 nk, 0, k;\n\t"
        "shr.s32 sk, k, 31;\n\t"
        "add.cc.u32 r0, r0, nk;\n\t"
        "addc.u32 r1, r1, sk;\n\t"
        "mov.b64 %0, {r0, r1};\n\t"
        "}"
        : "=l"(r)
        : "l"(lo), "l"(hi));
    return r;
}

// Non-canonical product: inputs in [0, 2^64), output in [0, 2^64).
__device__ __forceinline__ u64 mul_nc(u64 a, u64 b) { return reduce128_ptx(a * b, __umul64hi(a, b)); }

// Canonical product: inputs in [0, 2^64), output in [0, p).
__device__ __forceinline__ u64 mul(u64 a, u64 b) { return canon(mul_nc(a, b)); }

// Canonical sub: a in [0, 2^64), b canonical; the result is canonical when
// a is.  On a borrow the wrapped d = a - b + 2^64 stands for d - EPS, and
// d >= 2^64 - (p - 1) > EPS, so d - EPS neither wraps nor reaches p.  On the
// device this is one borrow chain: the borrow, as a 0 / 0xFFFFFFFF mask, is
// EPS itself, subtracted from the low word.
__host__ __device__ __forceinline__ u64 sub(u64 a, u64 b)
{
#ifdef __CUDA_ARCH__
    u64 r;
    asm("{\n\t"
        ".reg .u32 a0, a1, b0, b1, d0, d1, m;\n\t"
        "mov.b64 {a0, a1}, %1;\n\t"
        "mov.b64 {b0, b1}, %2;\n\t"
        "sub.cc.u32 d0, a0, b0;\n\t"
        "subc.cc.u32 d1, a1, b1;\n\t"
        "subc.u32 m, 0, 0;\n\t"
        "sub.cc.u32 d0, d0, m;\n\t"
        "subc.u32 d1, d1, 0;\n\t"
        "mov.b64 %0, {d0, d1};\n\t"
        "}"
        : "=l"(r)
        : "l"(a), "l"(b));
    return r;
#else
    u64 d = a - b;
    if (a < b) d += P;  // wrapped a - b + 2^64, plus p (mod 2^64) = a - b + p
    return d;
#endif
}

// Canonical add: a + b = a - (p - b) for canonical b (with b = 0 the
// subtrahend is p: a - p borrows, and the borrow's correction brings it back
// to a), so the device form is two more instructions in front of the borrow
// chain of sub.
__host__ __device__ __forceinline__ u64 add(u64 a, u64 b)
{
#ifdef __CUDA_ARCH__
    return sub(a, P - b);
#else
    u64 s = a + b;
    // On carry the true sum is s + 2^64 < 2p, and s - p (mod 2^64) = s + EPS.
    if (s < a || s >= P) s -= P;
    return s;
#endif
}

// The 128-bit reduction for code that also runs on the host: the carry-chain
// form on the device (it moves part of the work off the integer ALU pipe),
// the compare form on the host.  Both return a value below 2^64 congruent
// to lo + 2^64 hi.
__host__ __device__ __forceinline__ u64 reduce_any(u64 lo, u64 hi)
{
#ifdef __CUDA_ARCH__
    return reduce128_ptx(lo, hi);
#else
    return reduce128(lo, hi);
#endif
}

// x 2^e mod p for canonical x and 0 <= e < 96, canonical result; e is a
// constant wherever this is inlined into unrolled code, so only one branch
// remains.  With 2^64 = 2^32 - 1 and 2^128 = -2^32 (mod p):
// Multiplying by 2^(e+96) is the negation of this (2^96 = -1 mod p).
//   e < 32:       x 2^e = lo + 2^64 h (h < 2^32) = lo + h (2^32 - 1);
//   32 <= e < 64: lo + 2^64 hi, the 128-bit reduction;
//   64 <= e < 96: x 2^e = -x 2^-k with k = 96 - e in (0, 32].  Since
//                 2^32 - 2^64 = 1 (mod p), 2^-k = 2^(32-k) - 2^(64-k); with
//                 x = q 2^k + r (r < 2^k) this gives x 2^e = A - B, where
//                 A = r 2^(64-k) = (r 2^(32-k)) 2^32 <= 2^64 - 2^32 < p and
//                 B = q + r 2^(32-k) < 2^63 + 2^32 < p, so one conditional
//                 addition of p makes it canonical.
__host__ __device__ __forceinline__ u64 mul_pow2(u64 x, u32 e)
{
    if (e == 0) return x;
    if (e < 32) {
#ifdef __CUDA_ARCH__
        // lo = x 2^e mod 2^64 and h = x >> (64 - e) < 2^32; x 2^e = lo + h 2^64
        // = lo - h + h 2^32 (mod p).  That sum is V = r + c 2^64 with
        // c in {-1, 0, 1}; V = r + c EPS (mod p) stays within [0, p) for
        // c != 0, and a final compare-subtract handles c = 0.
        u64 r;
        asm("{\n\t"
            ".reg .u32 x0, x1, l0, l1, h, r0, r1, b, c, nc, sc;\n\t"
            ".reg .pred q;\n\t"
            "mov.b64 {x0, x1}, %1;\n\t"
            "shl.b32 l0, x0, %2;\n\t"
            "shf.l.wrap.b32 l1, x0, x1, %2;\n\t"
            "shr.b32 h, x1, %3;\n\t"
            "sub.cc.u32 r0, l0, h;\n\t"
            "subc.cc.u32 r1, l1, 0;\n\t"
            "subc.u32 b, 0, 0;\n\t"
            "add.cc.u32 r1, r1, h;\n\t"
            "addc.u32 c, b, 0;\n\t"
            "neg.s32 nc, c;\n\t"
            "shr.s32 sc, c, 31;\n\t"
            "add.cc.u32 r0, r0, nc;\n\t"
            "addc.u32 r1, r1, sc;\n\t"
            "setp.eq.u32 q, r1, 0xFFFFFFFF;\n\t"
            "setp.ne.and.u32 q, r0, 0, q;\n\t"
            "@q add.u32 r0, r0, 0xFFFFFFFF;\n\t"
            "@q mov.u32 r1, 0;\n\t"
            "mov.b64 %0, {r0, r1};\n\t"
            "}"
            : "=l"(r)
            : "l"(x), "r"(e), "r"(32 - e));
        return r;
#else
        u64 lo = x << e;
        u64 h = x >> (64 - e);
        u64 t = (h << 32) - h;  // < 2^64 - 2^32
        u64 r = lo + t;
        if (r < t) r += EPS;    // carry: r + 2^64 = r + EPS, and r < t here
        return canon(r);
#endif
    }
    if (e < 64) return canon(reduce_any(x << e, x >> (64 - e)));
    const u32 k = 96 - e;
    const u64 q = x >> k;
    const u64 ah = (k == 32 ? (x & 0xFFFFFFFFull) : ((x & ((1ull << k) - 1)) << (32 - k)));
    const u64 A = ah << 32, B = q + ah;
    return A >= B ? A - B : A - B + P;
}

// a in [0, 2^64), k canonical: a + k mod p as a value in [0, 2^64).
// On carry, s + 2^64 = s + EPS with s < p, so s + EPS < 2^64.
__device__ __forceinline__ u64 add_nc_small(u64 a, u64 k)
{
    u64 s = a + k;
    if (s < k) s += EPS;
    return s;
}

// a, b in [0, 2^64): a + b mod p as a value in [0, 2^64).  After a carry,
// s + EPS can carry again only when s > 2^64 - 2^32, and then the wrapped
// value is below EPS, so a second EPS cannot carry.
__device__ __forceinline__ u64 add_nc(u64 a, u64 b)
{
    u64 s = a + b;
    if (s < b) {
        s += EPS;
        if (s < EPS) s += EPS;
    }
    return s;
}

__device__ __forceinline__ u64 pow(u64 a, u64 e)
{
    u64 r = 1, x = a;
    while (e) {
        if (e & 1) r = mul(r, x);
        x = mul(x, x);
        e >>= 1;
    }
    return r;
}

// Host-side arithmetic for the planners (per-round constants, tables).
inline u64 h_mul(u64 a, u64 b) { return (u64)((unsigned __int128)a * b % P); }
inline u64 h_pow(u64 a, u64 e)
{
    u64 r = 1;
    while (e) {
        if (e & 1) r = h_mul(r, a);
        a = h_mul(a, a);
        e >>= 1;
    }
    return r;
}
inline u64 h_inv(u64 a) { return h_pow(a, P - 2); }
// w_m = 7^((p-1)/m) for m = 2^log_m (7 generates the multiplicative group).
inline u64 h_root(u32 log_m) { return h_pow(7, (P - 1) >> log_m); }

__host__ __device__ __forceinline__ u32 bitrev(u32 x, u32 bits)
{
#ifdef __CUDA_ARCH__
    return bits ? (__brev(x) >> (32 - bits)) : 0;
#else
    u32 r = 0;
    for (u32 i = 0; i < bits; i++) r |= ((x >> i) & 1u) << (bits - 1 - i);
    return r;
#endif
}

// (lo, mid, hi) += a * b: a 64x64 -> 128-bit product added into a 192-bit
// accumulator whose top word counts the carries (at most one per product).
// The product is four 32x32 + 64 -> 64 wide multiply-adds, each taking the
// carry word of the one before: t = a0 b1 + hi(a0 b0), u = a1 b0 + lo(t),
// high half a1 b1 + hi(t) + hi(u); no sum leaves 64 bits.  On the IMAD pipe
// this is a third cheaper than a 64-bit multiply's low and high halves.
__device__ __forceinline__ void mac192(u64& lo, u64& mid, u32& hi, u64 a, u64 b)
{
    asm("{\n\t"
        ".reg .u32 a0, a1, b0, b1, p0, p1, t0, t1, u0, u1;\n\t"
        ".reg .u64 p, t, u, h, c, pl;\n\t"
        "mov.b64 {a0, a1}, %3;\n\t"
        "mov.b64 {b0, b1}, %4;\n\t"
        "mul.wide.u32 p, a0, b0;\n\t"
        "mov.b64 {p0, p1}, p;\n\t"
        "cvt.u64.u32 c, p1;\n\t"
        "mad.wide.u32 t, a0, b1, c;\n\t"
        "mov.b64 {t0, t1}, t;\n\t"
        "cvt.u64.u32 c, t0;\n\t"
        "mad.wide.u32 u, a1, b0, c;\n\t"
        "mov.b64 {u0, u1}, u;\n\t"
        "cvt.u64.u32 c, t1;\n\t"
        "mad.wide.u32 h, a1, b1, c;\n\t"
        "cvt.u64.u32 c, u1;\n\t"
        "add.u64 h, h, c;\n\t"
        "mov.b64 pl, {p0, u0};\n\t"
        "add.cc.u64 %0, %0, pl;\n\t"
        "addc.cc.u64 %1, %1, h;\n\t"
        "addc.u32 %2, %2, 0;\n\t"
        "}"
        : "+l"(lo), "+l"(mid), "+r"(hi)
        : "l"(a), "l"(b));
}

// The accumulator's value lo + mid 2^64 + hi 2^128 mod p.  With 2^64 = 2^32 - 1
// and 2^128 = (2^32 - 1)^2 = 2^64 - 2^33 + 1 = -2^32 (mod p), it is
// reduce(lo + mid 2^64) - hi 2^32, and hi 2^32 < 2^63 < p for hi < 2^31.
__device__ __forceinline__ u64 fold192(u64 lo, u64 mid, u32 hi)
{
    return sub(canon(reduce128_ptx(lo, mid)), (u64)hi << 32);
}

}  // namespace gl
