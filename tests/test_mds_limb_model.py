"""The limb arithmetic of the CUDA Poseidon MDS, restated in Python integers
and checked against M s + rc mod p (no GPU, no oracle).

Lanes in [0, 2^64) split into limbs of 21, 21 and 22 bits.  The circulant
M = [[A, B], [B, A]] (6 x 6 blocks) gives P = (A + B)(x + x'), Q =
(A - B)(x - x'), y = (P + Q) / 2 and (P - Q) / 2 per limb vector; for the two
21-bit limbs A + B is split again into 3 x 3 blocks and both halvings merge
into one shift by 2.  The warp-shared permutation uses the direct 12-term
form.  Every sum must stay in 32 bits (signed where it is a difference),
which these checks assert on random and extreme states."""
import os
import random
import re

import pytest

P = 2**64 - 2**32 + 1
M32 = 2**32 - 1
ROW = [59, 23, 38, 43, 50, 3, 41, 22, 2, 55, 6, 30]


def m(k):
    return ROW[k % 12]


S = [m(k) + m(k + 6) for k in range(6)]


def d(i, j):
    return m(j - i) - m(j - i + 6)


SP = [S[k] + S[k + 3] for k in range(3)]


def dd(i, j):
    return S[(j - i) % 6] - S[(j - i + 3) % 6]


def split6(x, init):
    """One-level block form; init = [P (6), Q (6)] mod 2^32."""
    u = [(x[j] + x[j + 6]) & M32 for j in range(6)]
    v = [(x[j] - x[j + 6]) & M32 for j in range(6)]
    y = [0] * 12
    for i in range(6):
        p, q, p_true = init[i], init[6 + i], init[i]
        for j in range(6):
            p = (p + u[j] * S[(j - i + 6) % 6]) & M32
            p_true += u[j] * S[(j - i + 6) % 6]
            q = (q + v[j] * (d(i, j) & M32)) & M32
        assert p_true < 2**32
        y[i], y[i + 6] = ((p + q) & M32) >> 1, ((p - q) & M32) >> 1
    return y


def split6_2(x, init):
    """Two-level form for 21-bit limbs; init = [P' (3), Q' (3), Q2 (6)]."""
    u = [(x[j] + x[j + 6]) & M32 for j in range(6)]
    v = [(x[j] - x[j + 6]) & M32 for j in range(6)]
    up = [(u[j] + u[j + 3]) & M32 for j in range(3)]
    vp = [(u[j] - u[j + 3]) & M32 for j in range(3)]
    A, B, Q2 = [0] * 3, [0] * 3, [0] * 6
    for i in range(3):
        pp, qq, pp_true = init[i], init[3 + i], init[i]
        for j in range(3):
            pp = (pp + up[j] * SP[(j - i + 3) % 3]) & M32
            pp_true += up[j] * SP[(j - i + 3) % 3]
            qq = (qq + vp[j] * (dd(i, j) & M32)) & M32
        assert pp_true < 2**32
        A[i], B[i] = (pp + qq) & M32, (pp - qq) & M32
    for i in range(6):
        q = init[6 + i]
        for j in range(6):
            q = (q + v[j] * ((2 * d(i, j)) & M32)) & M32
        Q2[i] = q
    y = [0] * 12
    for i in range(3):
        y[i], y[i + 6] = ((A[i] + Q2[i]) & M32) >> 2, ((A[i] - Q2[i]) & M32) >> 2
        y[i + 3], y[i + 9] = ((B[i] + Q2[i + 3]) & M32) >> 2, ((B[i] - Q2[i + 3]) & M32) >> 2
    return y


def limbs(v):
    return v & 0x1FFFFF, (v >> 21) & 0x1FFFFF, v >> 42


def init1(l):
    return [(l[i] + l[i + 6]) & M32 for i in range(6)] + [(l[i] - l[i + 6]) & M32 for i in range(6)]


def init2(l):
    p = [l[i] + l[i + 6] for i in range(6)]
    return ([(p[i] + p[i + 3]) & M32 for i in range(3)] + [(p[i] - p[i + 3]) & M32 for i in range(3)]
            + [(2 * (l[i] - l[i + 6])) & M32 for i in range(6)])


def states(n):
    rng = random.Random(11)
    fixed = [([0] * 12, [0] * 12), ([2**64 - 1] * 12, [P - 1] * 12), ([P - 1] * 12, [P - 1] * 12),
             ([2**63] * 12, [12345] * 12), ([2**64 - 1 if j % 2 else 0 for j in range(12)], [P - 1] * 12)]
    return fixed + [([rng.getrandbits(64) for _ in range(12)], [rng.randrange(P) for _ in range(12)])
                    for _ in range(n)]


def test_row_matches_the_generated_constants():
    hdr = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2603_03065_gb300",
                       "_build", "poseidon_params.h")
    if not os.path.exists(hdr):
        pytest.skip("library not built")
    mrow = re.search(r"V3C_MDS_ROW_INIT\s*\{([^}]*)\}", open(hdr).read())
    assert [int(v.strip().rstrip("uU")) for v in mrow.group(1).split(",") if v.strip()] == ROW


def test_block_forms_equal_the_circulant():
    for s, rc in states(3000):
        la, lb, lc = zip(*[limbs(v) for v in rc])
        a, b, c = zip(*[limbs(v) for v in s])
        ya, yb, yc = split6_2(a, init2(la)), split6_2(b, init2(lb)), split6(c, init1(lc))
        assert ya == split6(a, init1(la)) and yb == split6(b, init1(lb))
        for i in range(12):
            assert yc[i] < 2**32
            got = (ya[i] + yb[i] * 2**21 + yc[i] * 2**42) % P
            assert got == (sum(m(j - i) * s[j] for j in range(12)) + rc[i]) % P


def test_direct_limb_form_of_the_warp_permutation():
    for s, rc in states(500):
        for i in range(12):
            acc = [limbs(rc[i])[k] for k in range(3)]
            for j in range(12):
                for k in range(3):
                    acc[k] += limbs(s[j])[k] * m(j - i)
            assert max(acc) < 2**32
            assert (acc[0] + acc[1] * 2**21 + acc[2] * 2**42) % P == (sum(m(j - i) * s[j] for j in range(12)) + rc[i]) % P
