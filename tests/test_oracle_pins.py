"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test checks the oracle against something the mathematics or a
published value fixes: brute-force DFT sums, Horner evaluation, inverse
permutations, exact-integer determinants, published SplitMix64 outputs and
the paper's printed G -> G_B pairs.  Python restatements here are written
from the definitions, not from oracle.c.
"""
import itertools
import os
import random

import numpy as np
import pytest

import oracle
import synth

P = oracle.P
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EDGE = [0, 1, 2, P - 1, P - 2, 1 << 32, (1 << 32) - 1, (1 << 64) - (1 << 32), (1 << 63) % P, 7]


def rnd_elems(rng, k):
    return [rng.randrange(P) for _ in range(k)]


# ---------------------------------------------------------------- field
def test_field_ops_against_python_ints():
    rng = random.Random(11)
    vals = EDGE + rnd_elems(rng, 200)
    for a in vals:
        for b in vals[:40]:
            assert oracle.mul(a, b) == (a * b) % P
            assert oracle.add(a, b) == (a + b) % P
            assert oracle.sub(a, b) == (a - b) % P


def test_field_special_form_identities():
    # 2^64 = 2^32 - 1 and 2^96 = -1 (mod p): the identities a special-form
    # reduction relies on.
    two32 = 1 << 32
    assert oracle.mul(two32, two32) == two32 - 1
    assert oracle.mul(oracle.mul(two32, two32), two32) == P - 1
    rng = random.Random(3)
    for a in EDGE[1:] + rnd_elems(rng, 50):
        if a % P:
            assert oracle.mul(a, oracle.inv(a)) == 1


def test_seven_generates_the_multiplicative_group():
    assert P - 1 == (1 << 32) * 3 * 5 * 17 * 257 * 65537
    for q in (2, 3, 5, 17, 257, 65537):
        assert pow(7, (P - 1) // q, P) != 1
    # x -> x^7 is a permutation of F_p (gcd(7, p-1) = 1).
    assert (P - 1) % 7 != 0


@pytest.mark.parametrize("log_m", list(range(0, 33)))
def test_roots_of_unity(log_m):
    w = oracle.root_of_unity(log_m)
    assert pow(w, 1 << log_m, P) == 1
    if log_m:
        assert pow(w, 1 << (log_m - 1), P) == P - 1


# ---------------------------------------------------------------- NTT
def dft_bruteforce(x, inverse=False):
    m = len(x)
    log_m = m.bit_length() - 1
    w = pow(7, (P - 1) >> log_m, P)
    if inverse:
        w = pow(w, P - 2, P)
    out = [sum(xi * pow(w, i * j, P) for i, xi in enumerate(x)) % P for j in range(m)]
    if inverse:
        minv = pow(m, P - 2, P)
        out = [(v * minv) % P for v in out]
    return out


@pytest.mark.parametrize("log_m", [0, 1, 2, 3, 5, 7])
def test_ntt_matches_bruteforce_dft(log_m):
    rng = random.Random(100 + log_m)
    x = rnd_elems(rng, 1 << log_m)
    assert oracle.ntt(x).tolist() == dft_bruteforce(x)
    assert oracle.intt(x).tolist() == dft_bruteforce(x, inverse=True)


def test_ntt_roundtrip_impulse_constant():
    rng = np.random.default_rng(5)
    n = 1 << 12
    x = rng.integers(0, P, size=n, dtype=np.uint64)
    assert np.array_equal(oracle.intt(oracle.ntt(x)), x)
    d = np.zeros(n, np.uint64)
    d[0] = 1
    assert np.all(oracle.ntt(d) == 1)                  # delta_0 -> all ones
    cst = np.full(n, 12345, np.uint64)
    f = oracle.ntt(cst)
    assert int(f[0]) == (12345 * n) % P and np.all(f[1:] == 0)  # constant -> n delta_0


# ---------------------------------------------------------------- LDE
def lde_by_definition(col, r):
    """Committed rows of one column by the definition: coefficients by
    brute-force inverse DFT, then P(7 w_N^j) by Horner at j = bitrev(t)."""
    n = len(col)
    log_N = n.bit_length() - 1 + r
    a = dft_bruteforce(list(col), inverse=True)
    wN = pow(7, (P - 1) >> log_N, P)
    out = []
    for t in range(1 << log_N):
        j = int(format(t, f"0{log_N}b")[::-1], 2) if log_N else 0
        x = 7 * pow(wN, j, P) % P
        acc = 0
        for ai in reversed(a):
            acc = (acc * x + ai) % P
        out.append(acc)
    return out


@pytest.mark.parametrize("log_n,r", [(0, 2), (1, 1), (3, 0), (4, 2), (5, 3)])
def test_lde_matches_horner_at_coset_points(log_n, r):
    rng = random.Random(7 * log_n + r)
    c = 3
    cols = [rnd_elems(rng, 1 << log_n) for _ in range(c)]
    e = oracle.lde(cols, r)
    assert e.shape == ((1 << (log_n + r)), 4)          # ld rounds 3 up to 4
    assert np.all(e[:, 3] == 0)
    for j in range(c):
        assert e[:, j].tolist() == lde_by_definition(cols[j], r)


def test_lde_reinterpolates_to_degree_below_n():
    rng = random.Random(21)
    log_n, r = 5, 2
    n, N = 1 << log_n, 1 << (log_n + r)
    col = rnd_elems(rng, n)
    e = oracle.lde([col], r)[:, 0].tolist()
    natural = [0] * N
    for t in range(N):
        natural[int(format(t, f"0{log_n + r}b")[::-1], 2)] = e[t]
    coef = dft_bruteforce(natural, inverse=True)        # coefficients of f(7x)
    ginv = pow(7, P - 2, P)
    a = [(coef[i] * pow(ginv, i, P)) % P for i in range(N)]
    assert a[:n] == dft_bruteforce(col, inverse=True)
    assert all(v == 0 for v in a[n:])


def test_lde_constant_linear_and_r0():
    rng = np.random.default_rng(9)
    n, r = 1 << 6, 3
    cst = np.full((1, n), 99, np.uint64)
    assert np.all(oracle.lde(cst, r)[:, 0] == 99)
    x = rng.integers(0, P, size=(2, n), dtype=np.uint64)
    al, be = 123456789, P - 5
    comb = np.array([[(al * int(u) + be * int(v)) % P for u, v in zip(x[0], x[1])]], np.uint64)
    ex = oracle.lde(x, r)
    ec = oracle.lde(comb, r)[:, 0]
    want = [(al * int(u) + be * int(v)) % P for u, v in zip(ex[:, 0], ex[:, 1])]
    assert ec.tolist() == want
    # r = 0: evaluations on the coset 7 H_n, rows bit-reversed.
    col = x[0].tolist()
    assert oracle.lde([col], 0)[:, 0].tolist() == lde_by_definition(col, 0)


def test_lde_rows_route_agrees_with_ntt_route():
    x = synth.columns(seed=1, c=5, log_n=9, mix="trace")
    e = oracle.lde(x, 2)
    co = oracle.coeffs(x)
    rows = np.array([0, 1, 2, 77, 511, 1024, 2047], np.uint64)
    assert np.array_equal(oracle.lde_rows(co, 2, rows), e[rows.astype(np.int64), :5])


# ---------------------------------------------------------------- SplitMix64
def test_splitmix64_published_outputs():
    import ctypes

    for line in open(os.path.join(GOLDEN, "splitmix64.txt")):
        if line.startswith("#") or not line.strip():
            continue
        st0, idx, out = (int(v) for v in line.split())
        st = ctypes.c_uint64(st0)
        for _ in range(idx + 1):
            v = oracle.lib().orc_splitmix64_next(ctypes.byref(st))
        assert v == out
        # the input generator's counter form gives the same stream
        assert int(synth.draws(st0, idx, 1)[0]) == out


# ---------------------------------------------------------------- Poseidon
def derive_constants_python():
    """Constant derivation restated from the spec: RC draws kept iff < p,
    then candidate MDS rows of (draw & 63) with zeros redrawn."""
    st = 0x56334442504F5331                           # "V3DBPOS1"
    assert st == int.from_bytes(b"V3DBPOS1", "big")
    rc = []
    while len(rc) < 360:
        st, d = synth.splitmix64(st)
        if d < P:
            rc.append(d)
    row = []
    while len(row) < 12:
        st, d = synth.splitmix64(st)
        if d & 63:
            row.append(d & 63)
    return rc, row


def det_exact(A):
    """Exact integer determinant by fraction-free (Bareiss) elimination."""
    A = [r[:] for r in A]
    n, sign, prev = len(A), 1, 1
    for k in range(n - 1):
        if A[k][k] == 0:
            for i in range(k + 1, n):
                if A[i][k]:
                    A[k], A[i] = A[i], A[k]
                    sign = -sign
                    break
            else:
                return 0
        for i in range(k + 1, n):
            for j in range(k + 1, n):
                A[i][j] = (A[i][j] * A[k][k] - A[i][k] * A[k][j]) // prev
        prev = A[k][k]
    return sign * A[n - 1][n - 1]


def test_poseidon_constants_follow_the_generator():
    rc, mds, tries = oracle.poseidon_params()
    rc_py, row_py = derive_constants_python()
    assert rc.reshape(-1).tolist() == rc_py
    assert tries == 1                                  # first candidate row is MDS
    circ = [[row_py[(j - i) % 12] for j in range(12)] for i in range(12)]
    assert mds.tolist() == circ


def test_mds_minors_nonzero_by_exact_determinants():
    _, mds, _ = oracle.poseidon_params()
    M = mds.tolist()
    for k in (1, 2, 3):
        for R in itertools.combinations(range(12), k):
            for C in itertools.combinations(range(12), k):
                assert det_exact([[M[r][c] for c in C] for r in R]) % P != 0
    rng = random.Random(4)
    for _ in range(400):
        k = rng.randint(4, 12)
        R = sorted(rng.sample(range(12), k))
        C = sorted(rng.sample(range(12), k))
        assert det_exact([[M[r][c] for c in C] for r in R]) % P != 0


def test_mds_check_rejects_singular_minors_and_accepts_cauchy():
    _, mds, _ = oracle.poseidon_params()
    assert oracle.mds_check(mds) == 1
    bad = mds.copy()
    bad[3, 5] = 0                                      # a zero 1x1 minor
    assert oracle.mds_check(bad) == 0
    row = [5, 10, 3, 6, 1, 2, 7, 9, 11, 4, 8, 12]      # small entries with product coincidences
    M = [[row[(j - i) % 12] for j in range(12)] for i in range(12)]
    zero_2x2 = any(
        det_exact([[M[r][c] for c in C] for r in R]) % P == 0
        for R in itertools.combinations(range(12), 2)
        for C in itertools.combinations(range(12), 2)
    )
    assert oracle.mds_check(np.array(M, np.uint64)) == (0 if zero_2x2 else 1)
    assert zero_2x2
    # Cauchy matrices 1/(x_i - y_j) with distinct x, y are MDS by construction.
    xs = list(range(1, 13))
    ys = list(range(100, 112))
    cauchy = [[pow(x - y, P - 2, P) for y in ys] for x in xs]
    assert oracle.mds_check(np.array(cauchy, np.uint64)) == 1


def inverse_permutation(state, rc, mds):
    """Perm^-1 from the spec: undo MDS (Gauss-Jordan inverse mod p), undo the
    S-box with exponent 7^-1 mod (p-1), subtract the round constants; rounds
    29 down to 0, rounds 0-3 and 26-29 full."""
    n = 12
    A = [list(map(int, r)) + [1 if i == j else 0 for j in range(n)] for i, r in enumerate(mds)]
    for col in range(n):
        piv = next(i for i in range(col, n) if A[i][col] % P)
        A[col], A[piv] = A[piv], A[col]
        iv = pow(A[col][col], P - 2, P)
        A[col] = [(v * iv) % P for v in A[col]]
        for i in range(n):
            if i != col and A[i][col]:
                f = A[i][col]
                A[i] = [(a - f * b) % P for a, b in zip(A[i], A[col])]
    minv = [r[n:] for r in A]
    d = pow(7, -1, P - 1)
    s = [int(v) for v in state]
    for rho in range(29, -1, -1):
        s = [sum(minv[i][j] * s[j] for j in range(n)) % P for i in range(n)]
        full = rho < 4 or rho >= 26
        for i in range(n if full else 1):
            s[i] = pow(s[i], d, P)
        s = [(s[i] - int(rc[rho][i])) % P for i in range(n)]
    return s


def test_permutation_inverts():
    rc, mds, _ = oracle.poseidon_params()
    rng = random.Random(17)
    states = [[0] * 12, [P - 1] * 12, list(range(12))] + [rnd_elems(rng, 12) for _ in range(4)]
    for s in states:
        out = oracle.permute(s)
        assert all(int(v) < P for v in out)
        assert inverse_permutation(out, rc, mds) == s


def test_sponge_and_compression_rules():
    rng = random.Random(23)
    x = rnd_elems(rng, 20)
    for k in range(0, 5):                              # hash-or-noop
        assert oracle.hash_(x[:k]).tolist() == x[:k] + [0] * (4 - k)
    s = oracle.permute(x[:8] + [0] * 4)
    assert oracle.hash_(x[:8]).tolist() == s[:4].tolist()
    s9 = s.copy()
    s9[0] = x[8]                                       # overwrite lane 0, keep 1..11
    assert oracle.hash_(x[:9]).tolist() == oracle.permute(s9)[:4].tolist()
    s16 = s.copy()
    s16[:8] = x[8:16]
    assert oracle.hash_(x[:16]).tolist() == oracle.permute(s16)[:4].tolist()
    s15 = s.copy()
    s15[:7] = x[8:15]                                  # ragged chunk of 7 keeps lane 7
    assert oracle.hash_(x[:15]).tolist() == oracle.permute(s15)[:4].tolist()
    L, R = x[:4], x[4:8]
    assert oracle.compress(L, R).tolist() == oracle.permute(L + R + [0] * 4)[:4].tolist()
    assert oracle.compress(L, R).tolist() != oracle.compress(R, L).tolist()


# ---------------------------------------------------------------- Merkle
def merkle_root_recursive(digests):
    if len(digests) == 1:
        return digests[0]
    h = len(digests) // 2
    return oracle.compress(merkle_root_recursive(digests[:h]), merkle_root_recursive(digests[h:])).tolist()


@pytest.mark.parametrize("log_rows", [1, 2, 3, 4])
def test_merkle_against_recursive_definition_and_paths(log_rows):
    rng = np.random.default_rng(log_rows)
    width = 9
    rows = rng.integers(0, P, size=(1 << log_rows, 10), dtype=np.uint64)
    leaves = [oracle.hash_(r[:width]).tolist() for r in rows]
    for h in range(0, log_rows + 1):
        tree, cap = oracle.merkle(rows, width, h)
        assert tree.size == oracle.tree_len(log_rows, h)
        k = log_rows - h
        want_cap = [merkle_root_recursive(leaves[i << k:(i + 1) << k]) for i in range(1 << h)]
        assert cap.tolist() == want_cap
        if k:
            assert tree[: 4 << log_rows].reshape(-1, 4).tolist() == leaves
        for t in range(1 << log_rows):
            path = oracle.merkle_path(tree, log_rows, h, t)
            assert oracle.merkle_verify(rows[t, :width], width, log_rows, h, t, path, cap)
            if k:
                bad = path.copy()
                bad[rng.integers(0, k), rng.integers(0, 4)] ^= np.uint64(1)
                assert not oracle.merkle_verify(rows[t, :width], width, log_rows, h, t, bad, cap)
                assert not oracle.merkle_verify(rows[t, :width], width, log_rows, h, t ^ 1, path, cap)
            row = rows[t, :width].copy()
            row[rng.integers(0, width)] ^= np.uint64(2)
            assert not oracle.merkle_verify(row, width, log_rows, h, t, path, cap)


# ---------------------------------------------------------------- paper goldens
def test_padded_domain_matches_paper_table():
    for line in open(os.path.join(GOLDEN, "binning.txt")):
        if line.startswith("#") or not line.strip():
            continue
        G, k = (int(v) for v in line.split())
        assert oracle.domain_log2(G) == k


# ---------------------------------------------------------------- whole commit
def test_small_commit_is_self_consistent():
    s = synth.Shape(c=13, log_n=6, rate_bits=2, cap_height=2, seed=4)
    x = s.inputs()
    e, tree, cap = oracle.commit(x, s.rate_bits, s.cap_height)
    assert e.shape == (1 << s.log_N, 14)
    assert np.all(e[:, 13] == 0)
    leaves = oracle.leaf_hashes(e, 13)
    assert np.array_equal(tree[: leaves.size].reshape(-1, 4), leaves)
    assert cap.tolist() == [merkle_root_recursive(leaves[i << 6:(i + 1) << 6].tolist()) for i in range(4)]
