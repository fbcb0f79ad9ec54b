"""Pins of the oracle's multiset-equality gadget (Sec. 4.5, Gadgets and Cost
Model): Compress(x; beta) = sum_k x_k beta^k and the grand-product column
Z_{i+1} = Z_i (alpha - x_i) / (alpha - y_i) of SetEq.

Pinned by brute force in Python integers, by the identity the gadget exists
for (Z_L = 1 exactly when the multisets agree, for a random alpha), and by
the tuple compression making tuple multisets comparable.
"""
import numpy as np

import oracle

P = oracle.P


def brute(X, Y, alpha, beta):
    def comp(t):
        return sum(int(v) * pow(beta, k, P) for k, v in enumerate(t)) % P

    z = [1]
    for x, y in zip(X, Y):
        den = (alpha - comp(y)) % P
        z.append(z[-1] * (alpha - comp(x)) * pow(den, P - 2, P) % P)
    return z


def test_compress_is_horner_in_beta():
    rng = np.random.default_rng(1)
    x = rng.integers(0, P, size=7, dtype=np.uint64)
    beta = 0x1234567890ABCDEF
    want = 0
    for v in reversed([int(t) for t in x]):
        want = (want * beta + v) % P
    assert oracle.compress_tuple(x, beta) == want
    assert oracle.compress_tuple(x, 0) == int(x[0])
    assert oracle.compress_tuple(x, 1) == sum(int(t) for t in x) % P


def test_partial_products_brute_force():
    rng = np.random.default_rng(2)
    X = rng.integers(0, P, size=(40, 3), dtype=np.uint64)
    Y = rng.integers(0, P, size=(40, 3), dtype=np.uint64)
    alpha, beta = 987654321987654321, 123456789
    z = oracle.seteq_partial_products(X, Y, alpha, beta)
    assert [int(v) for v in z] == brute(X, Y, alpha, beta)


def test_permuted_multiset_closes_to_one():
    rng = np.random.default_rng(3)
    X = rng.integers(0, 1 << 20, size=(500, 4), dtype=np.uint64)
    X[::7] = X[3]  # repeated tuples: multiplicities count
    Y = X[rng.permutation(500)]
    z = oracle.seteq_partial_products(X, Y, 0xDEADBEEF12345, 77777)
    assert int(z[-1]) == 1
    assert int(z[0]) == 1 and len({int(v) for v in z}) > 400


def test_different_multisets_do_not_close():
    rng = np.random.default_rng(4)
    X = rng.integers(0, 1 << 20, size=(300, 2), dtype=np.uint64)
    Y = X[rng.permutation(300)].copy()
    Y[17, 1] ^= np.uint64(1)  # one component of one tuple
    assert int(oracle.seteq_partial_products(X, Y, 0xABCDEF987, 31)[-1]) != 1
    # a multiplicity change: same set, different multiset
    Y = X.copy()
    Y[5] = X[6]
    assert int(oracle.seteq_partial_products(X, Y, 0xABCDEF987, 31)[-1]) != 1


def test_tuple_order_inside_a_row_matters_only_through_beta():
    # Swapping two components of one x tuple keeps the multiset of rows
    # equal only if beta cannot tell them apart: with beta = 1 it closes,
    # with a random beta it does not.
    X = np.array([[1, 2], [3, 4], [5, 6]], np.uint64)
    Y = np.array([[4, 3], [1, 2], [5, 6]], np.uint64)
    assert int(oracle.seteq_partial_products(X, Y, 1 << 40, 1)[-1]) == 1
    assert int(oracle.seteq_partial_products(X, Y, 1 << 40, 99)[-1]) != 1


def test_alpha_hitting_a_denominator_is_reported():
    X = np.array([[5], [6]], np.uint64)
    Y = np.array([[6], [7]], np.uint64)
    assert oracle.seteq_partial_products(X, Y, 7, 3) is None
