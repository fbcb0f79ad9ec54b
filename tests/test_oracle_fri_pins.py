"""Pins of the oracle's FRI commit phase against facts outside oracle.c.

The fold is checked against the coefficient-split definition
    f(X) = sum_{i < 2^a} X^i f_i(X^(2^a)),  fold_beta(f) = sum_i beta^i f_i,
evaluated here with plain Python integers (Horner on the split coefficient
lists); the oracle instead interpolates each coset (inverse DFT with x^-i).
The combine is brute-forced, the interpolation is re-evaluated, and the
whole commit phase must end on a polynomial whose degree is the input degree
divided by the total folding factor (the FRI completeness property).
"""
import numpy as np
import pytest

import oracle

P = oracle.P


def horner(coefs, x):
    acc = 0
    for c in reversed(coefs):
        acc = (acc * x + c) % P
    return acc


def root(log_m):
    # 7 generates F_p^*, so 7^((p-1)/m) has order exactly m.
    return pow(7, (P - 1) >> log_m, P)


def brev(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def coset_codeword(coefs, log_m, shift):
    """Values of the polynomial at shift * w_m^bitrev(t), t = 0..m-1."""
    w = root(log_m)
    return [horner(coefs, shift * pow(w, brev(t, log_m), P) % P) for t in range(1 << log_m)]


@pytest.mark.parametrize("a", [1, 2, 3, 4])
def test_fold_matches_coefficient_split(a):
    rng = np.random.default_rng(10 + a)
    log_m, deg = 7, 40
    coefs = [int(v) for v in rng.integers(0, P, size=deg, dtype=np.uint64)]
    shift = 7
    f = coset_codeword(coefs, log_m, shift)
    beta = int(rng.integers(1, P, dtype=np.uint64))
    got = oracle.fri_fold(np.array(f, dtype=np.uint64), shift, a, beta)
    A = 1 << a
    padded = coefs + [0] * (-len(coefs) % A)
    parts = [padded[i::A] for i in range(A)]  # f_i: coefficients i, i+A, i+2A, ...
    folded = [sum(pow(beta, i, P) * parts[i][j] for i in range(A)) % P for j in range(len(parts[0]))]
    want = coset_codeword(folded, log_m - a, pow(shift, A, P))
    assert [int(v) for v in got] == want


def test_fold_with_zero_challenge_is_the_even_part():
    # beta = 0, arity 2: (f(x) + f(-x)) / 2, where the two points of a coset
    # are adjacent positions 2u, 2u+1 of the bit-reversed order.
    rng = np.random.default_rng(3)
    f = rng.integers(0, P, size=1 << 6, dtype=np.uint64)
    got = oracle.fri_fold(f, 7, 1, 0)
    inv2 = pow(2, P - 2, P)
    want = [(int(f[2 * u]) + int(f[2 * u + 1])) * inv2 % P for u in range(32)]
    assert [int(v) for v in got] == want


def test_adjacent_positions_are_negatives():
    # The reading that makes the fold local: x_{2u+1} = -x_{2u}.
    log_m = 9
    w = root(log_m)
    for u in range(1 << (log_m - 1)):
        x0 = 7 * pow(w, brev(2 * u, log_m), P) % P
        x1 = 7 * pow(w, brev(2 * u + 1, log_m), P) % P
        assert (x0 + x1) % P == 0


def test_combine_brute_force():
    rng = np.random.default_rng(4)
    m1 = rng.integers(0, P, size=(16, 6), dtype=np.uint64)  # width 5, ld 6
    m2 = rng.integers(0, P, size=(16, 4), dtype=np.uint64)  # width 3, ld 4
    alpha = int(rng.integers(1, P, dtype=np.uint64))
    got = oracle.fri_combine([m1, m2], [5, 3], alpha)
    for t in range(16):
        vals = [int(v) for v in m1[t, :5]] + [int(v) for v in m2[t, :3]]
        want = sum(pow(alpha, e, P) * v for e, v in enumerate(vals)) % P
        assert int(got[t]) == want


def test_interpolate_reevaluates():
    rng = np.random.default_rng(5)
    log_m, shift = 5, pow(7, 1 << 4, P)
    f = rng.integers(0, P, size=1 << log_m, dtype=np.uint64)
    c = [int(v) for v in oracle.fri_interpolate(f, shift)]
    assert coset_codeword(c, log_m, shift) == [int(v) for v in f]


@pytest.mark.parametrize("arity_bits,final_log", [(1, 3), (2, 2), (3, 4), (4, 5)])
def test_commit_phase_ends_low_degree(arity_bits, final_log):
    # Columns of n = 2^6 rows extended at rate 2^3: every column, and so the
    # combination, has degree < 2^6.  After folding by 2^F in total the final
    # polynomial has degree < 2^6 / 2^F; the coefficients above are zero.
    rng = np.random.default_rng(6)
    cols = rng.integers(0, P, size=(5, 64), dtype=np.uint64)
    e = oracle.lde(cols, 3)
    betas = [int(v) for v in rng.integers(1, P, size=10, dtype=np.uint64)]
    st = oracle.fri_commit([e], [5], 987654321, betas, arity_bits, final_log, 2)
    F = 9 - final_log
    assert sum(st["arities"]) == F
    bound = max(1, 64 >> F)
    assert all(int(v) == 0 for v in st["final"][bound:])
    assert any(int(v) != 0 for v in st["final"][:bound])


def test_verifier_accepts_honest_and_rejects_tampered_openings():
    rng = np.random.default_rng(7)
    cols = rng.integers(0, P, size=(4, 32), dtype=np.uint64)
    e = oracle.lde(cols, 2)
    alpha = 31337
    betas = [int(v) for v in rng.integers(1, P, size=4, dtype=np.uint64)]
    st = oracle.fri_commit([e], [4], alpha, betas, 2, 2, 1)
    f0 = st["layers"][0]
    for t0 in [0, 1, 77, 127]:
        op = oracle.fri_query(st, t0)
        assert oracle.fri_verify_query(st["caps"], st["heights"], st["arities"], st["betas"], st["final"],
                                       7, t0, int(f0[t0]), op)
        bad = [(v.copy(), p.copy()) for v, p in op]
        bad[1][0][0] = (int(bad[1][0][0]) + 1) % P  # a planted error in the second layer's coset
        assert not oracle.fri_verify_query(st["caps"], st["heights"], st["arities"], st["betas"],
                                           st["final"], 7, t0, int(f0[t0]), bad)


# --- quadratic extension F_p[u] / (u^2 - 7) ----------------------------------

def emul(a, b):
    return ((a[0] * b[0] + 7 * a[1] * b[1]) % P, (a[0] * b[1] + a[1] * b[0]) % P)


def test_extension_is_a_field_and_arithmetic_matches():
    # 7 generates F_p^*, so it is a non-residue (Euler's criterion) and
    # u^2 - 7 is irreducible.
    assert pow(7, (P - 1) // 2, P) == P - 1
    rng = np.random.default_rng(20)
    for _ in range(20):
        a = tuple(int(v) for v in rng.integers(0, P, size=2, dtype=np.uint64))
        b = tuple(int(v) for v in rng.integers(0, P, size=2, dtype=np.uint64))
        assert oracle.ext_mul(a, b) == emul(a, b)
        ai = oracle.ext_inv(a)
        assert emul(a, ai) == (1, 0)


@pytest.mark.parametrize("a", [1, 2, 4])
def test_extension_fold_matches_coefficient_split(a):
    rng = np.random.default_rng(30 + a)
    log_m, deg, shift = 6, 24, 7
    coefs = [tuple(int(v) for v in rng.integers(0, P, size=2, dtype=np.uint64)) for _ in range(deg)]
    w = root(log_m)
    xs = [shift * pow(w, brev(t, log_m), P) % P for t in range(1 << log_m)]
    f = np.array([[horner([c[0] for c in coefs], x), horner([c[1] for c in coefs], x)] for x in xs], np.uint64)
    beta = tuple(int(v) for v in rng.integers(1, P, size=2, dtype=np.uint64))
    got = oracle.fri_fold(f, shift, a, beta, ext=2)
    A = 1 << a
    padded = coefs + [(0, 0)] * (-len(coefs) % A)
    parts = [padded[i::A] for i in range(A)]
    bp = [(1, 0)]
    for _ in range(A - 1):
        bp.append(emul(bp[-1], beta))
    folded = []
    for j in range(len(parts[0])):
        acc = (0, 0)
        for i in range(A):
            t = emul(bp[i], parts[i][j])
            acc = ((acc[0] + t[0]) % P, (acc[1] + t[1]) % P)
        folded.append(acc)
    ys = [pow(shift, A, P) * pow(root(log_m - a), brev(t, log_m - a), P) % P for t in range(1 << (log_m - a))]
    want = [[horner([c[0] for c in folded], y), horner([c[1] for c in folded], y)] for y in ys]
    assert [[int(v) for v in row] for row in got] == want


def test_extension_path_reduces_to_the_base_path():
    rng = np.random.default_rng(40)
    cols = rng.integers(0, P, size=(3, 32), dtype=np.uint64)
    e = oracle.lde(cols, 2)
    base = oracle.fri_commit([e], [3], 12345, [11, 22, 33], 2, 1, 1)
    ext = oracle.fri_commit([e], [3], (12345, 0), [(11, 0), (22, 0), (33, 0)], 2, 1, 1, ext=2)
    assert np.array_equal(ext["final"][:, 0], base["final"]) and not ext["final"][:, 1].any()
    for k in range(len(base["layers"])):
        assert np.array_equal(ext["layers"][k][:, 0], base["layers"][k])


def test_extension_commit_phase_ends_low_degree_and_verifies():
    rng = np.random.default_rng(50)
    cols = rng.integers(0, P, size=(5, 64), dtype=np.uint64)
    e = oracle.lde(cols, 3)
    alpha = (987654321, 123456789)
    betas = [tuple(int(v) for v in rng.integers(1, P, size=2, dtype=np.uint64)) for _ in range(4)]
    st = oracle.fri_commit([e], [5], alpha, betas, 2, 3, 2, ext=2)
    bound = 64 >> 6
    assert not st["final"][bound:].any() and st["final"][:bound].any()
    f0 = st["layers"][0]
    for t0 in [0, 5, 511]:
        op = oracle.fri_query(st, t0)
        assert oracle.fri_verify_query(st["caps"], st["heights"], st["arities"], st["betas"], st["final"], 9, t0,
                                       f0[t0], op, ext=2)
        bad = [(v.copy(), p.copy()) for v, p in op]
        bad[0][0][1] = (int(bad[0][0][1]) + 1) % P  # the imaginary part of one opened value
        assert not oracle.fri_verify_query(st["caps"], st["heights"], st["arities"], st["betas"], st["final"], 9,
                                           t0, f0[t0], bad, ext=2)
