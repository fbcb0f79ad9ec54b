"""The pass structure of the CUDA NTT, restated in Python integers and
checked against the DFT definition (no GPU, no oracle).

A radix-2^K pass is a 2^K-point DFT of the values a thread holds plus one
twiddle per value (the Cooley-Tukey split); the in-register DFTs multiply only
by 32nd roots of unity, which are powers of 2 mod p (w_32 = 7^((p-1)/32) =
2^78), with 2^(e+96) = -2^e folded into the butterflies' signs.  Element j of a
pass sits at shared-memory word sw(i0) ^ sw(j 2^st) because the swizzle is
linear over XOR and i0 has no bit in the stride field.  This model uses the
kernels' index arithmetic (lo, hi, i0, bitrev_K, root exponents) and the half
or full twiddle tables."""
import random

import pytest

P = 2**64 - 2**32 + 1


def root(logm, inv=False):
    w = pow(7, (P - 1) >> logm, P)
    return pow(w, P - 2, P) if inv else w


G32 = 78


def root_exp(K, inv, m):
    e = (G32 * (32 >> K) * m) % 192
    return (192 - e) % 192 if inv else e


def bitrev(j, K):
    return int(format(j, f"0{K}b")[::-1], 2) if K else 0


def mul_pow2(x, e):
    assert e < 96
    return x * pow(2, e, P) % P


def small_dif(v, K, inv):
    R = 1 << K
    for t in range(K):
        h = R >> (t + 1)
        for j in range(R):
            if j & h:
                continue
            e = root_exp(K, inv, (j & (h - 1)) << t)
            x, y = v[j], v[j + h]
            v[j] = (x + y) % P
            v[j + h] = mul_pow2((x - y) % P, e) if e < 96 else mul_pow2((y - x) % P, e - 96)


def small_dit(v, K, inv):
    for t in range(K):
        h = 1 << t
        for j in range(1 << K):
            if j & h:
                continue
            e = root_exp(K, inv, (j & (h - 1)) << (K - 1 - t))
            x, y = v[j], mul_pow2(v[j + h], e if e < 96 else e - 96)
            v[j], v[j + h] = ((x + y) % P, (x - y) % P) if e < 96 else ((x - y) % P, (x + y) % P)


def mul_tw(v, tw, e, logL, full):
    if full:
        return v * tw[e] % P
    half = (1 << logL) >> 1
    t = tw[e & (half - 1)] if half else tw[0]
    if half and (e & half):
        t = P - t
    return v * t % P


def table(logL, inv, full):
    w = root(logL, inv)
    return [pow(w, i, P) for i in range(max(((1 << logL) if full else (1 << logL) >> 1), 1))]


def dft_dif(a, B, logL, inv, kmax, full):
    tw, s = table(logL, inv, full), 0
    while s < logL:
        K = min(kmax, logL - s)
        lst = logL - s - K
        for g in range(B << (logL - K)):
            tr, gg = g >> (logL - K), g & ((1 << (logL - K)) - 1)
            lo, hi = gg & ((1 << lst) - 1), gg >> lst
            i0 = (tr << logL) + (hi << (lst + K)) + lo
            v = [a[i0 + (j << lst)] for j in range(1 << K)]
            small_dif(v, K, inv)
            if lst:
                for j in range(1, 1 << K):
                    v[j] = mul_tw(v[j], tw, (lo * bitrev(j, K)) << s, logL, full)
            for j in range(1 << K):
                a[i0 + (j << lst)] = v[j]
        s += K


def dft_dit(a, logL, inv, first, kmax):
    tw, s = table(logL, inv, False), first
    while s < logL:
        K = min(kmax, logL - s)
        for g in range(1 << (logL - K)):
            lo, hi = g & ((1 << s) - 1), g >> s
            i0 = (hi << (s + K)) + lo
            v = [a[i0 + (j << s)] for j in range(1 << K)]
            if s:
                for j in range(1, 1 << K):
                    v[j] = mul_tw(v[j], tw, (lo * bitrev(j, K)) << (logL - s - K), logL, False)
            small_dit(v, K, inv)
            for j in range(1 << K):
                a[i0 + (j << s)] = v[j]
        s += K


def radix2_dit(a, logL, inv, first):
    """The radix-2 DIT stages s >= first, stage by stage (the definition the passes replace)."""
    tw, L = table(logL, inv, False), 1 << logL
    for s in range(first, logL):
        h = 1 << s
        for e in range(L):
            if e & h:
                continue
            t = a[e + h] * tw[(e % h) << (logL - 1 - s)] % P if s else a[e + h]
            a[e], a[e + h] = (a[e] + t) % P, (a[e] - t) % P


def test_roots_are_powers_of_two():
    assert pow(2, G32, P) == root(5)
    for K in range(1, 6):
        for m in range(1 << K):
            assert pow(2, root_exp(K, False, m), P) == pow(root(K), m, P)
            assert pow(2, root_exp(K, True, m), P) == pow(root(K, True), m, P)


@pytest.mark.parametrize("logL", [1, 2, 3, 5, 6, 8])
@pytest.mark.parametrize("inv", [False, True])
def test_dif_passes_equal_the_dft(logL, inv):
    rng = random.Random(logL * 2 + inv)
    L = 1 << logL
    w = root(logL, inv)
    for kmax in (1, 2, 3, 4, 5):
        for full in (False, True):
            B = 2
            x = [rng.randrange(P) for _ in range(B * L)]
            a = list(x)
            dft_dif(a, B, logL, inv, kmax, full)
            for b in range(B):
                X = [sum(x[b * L + n] * pow(w, n * k, P) for n in range(L)) % P for k in range(L)]
                assert all(a[b * L + t] == X[bitrev(t, logL)] for t in range(L))


@pytest.mark.parametrize("logL,first", [(5, 0), (8, 3), (10, 3), (10, 0)])
def test_dit_passes_equal_radix2_stages(logL, first):
    rng = random.Random(logL + first)
    for kmax in (2, 4, 5):
        y = [rng.randrange(P) for _ in range(1 << logL)]
        a1, a2 = list(y), list(y)
        dft_dit(a1, logL, False, first, kmax)
        radix2_dit(a2, logL, False, first)
        assert a1 == a2


def test_pass_words_are_xor_offsets():
    def sw(i):
        return i ^ ((i >> 4) & 15)

    for K in range(1, 6):
        for st in range(0, 12):
            for i0 in range(0, 1 << 13, 7):
                if (i0 >> st) & ((1 << K) - 1):
                    continue
                for j in range(1 << K):
                    word = sw(i0) + (j << st) if st >= 8 else sw(i0) ^ sw(j << st)
                    assert word == sw(i0 + (j << st))
