"""Pins of the oracle's snapshot commitment (Sec. 4.3, Snapshot Commitments).

The C routine is compared with the paper's equations composed here in
Python from the separately pinned sponge (oracle.hash_) and Merkle tree
(oracle.merkle, whose width-4 leaves are the digests themselves):
    hash_{i,j} = Hash(i, j, f, item, v^(0..M-1)),  root_i = MerkleTree(hash_{i,.}),
    hash_i = Hash(i, mu_i, root_i),  root_mk = MerkleTree(hash_.),
    root_cb = Hash(C_{0,0}, ..., C_{M-1,K-1}).
Binding properties close the loop: a change to any committed value moves
exactly the roots that cover it.
"""
import numpy as np

import oracle
import synth

P = oracle.P


def u64(*xs):
    return np.array(xs, dtype=np.uint64)


def compose(rec, mu, cb, log_nlist, log_n):
    nlist, n = 1 << log_nlist, 1 << log_n
    leaves = np.stack([oracle.hash_(np.concatenate([u64(t // n, t % n), rec[t]])) for t in range(nlist * n)])
    roots = np.stack([oracle.merkle(leaves[i * n:(i + 1) * n], 4, 0)[1][0] for i in range(nlist)])
    cent = np.stack([oracle.hash_(np.concatenate([u64(i), mu[i], roots[i]])) for i in range(nlist)])
    mk = oracle.merkle(cent, 4, 0)[1][0]
    cbr = oracle.hash_(cb.reshape(-1))
    return leaves, roots, cent, mk, cbr


def test_snapshot_matches_the_composed_equations():
    rec, mu, cb = synth.snapshot(11, 3, 4, 16, 4, 16, valid=0.6)
    leaves, roots, cent, mk, cbr = compose(rec, mu, cb, 3, 4)
    assert np.array_equal(oracle.snapshot_slot_leaves(rec, 3, 4), leaves)
    st = oracle.snapshot_commit(rec, mu, cb, 3, 4)
    assert np.array_equal(st["list_roots"], roots)
    assert np.array_equal(st["centroid_digests"], cent)
    assert np.array_equal(st["root_mk"], mk)
    assert np.array_equal(st["root_cb"], cbr)


def test_per_list_helpers_agree_with_the_whole_commit():
    rec, mu, cb = synth.snapshot(16, 3, 3, 8, 2, 4)
    st = oracle.snapshot_commit(rec, mu, cb, 3, 3)
    for i in range(8):
        root = oracle.snapshot_list_root(rec[i * 8:(i + 1) * 8], i, 3)
        assert np.array_equal(root, st["list_roots"][i])
        assert np.array_equal(oracle.snapshot_centroid_digest(i, mu[i], root), st["centroid_digests"][i])


def test_single_list_and_single_slot_edges():
    # nlist = 1: root_mk is hash_0 itself; n = 1: root_i is the slot digest.
    rec, mu, cb = synth.snapshot(12, 0, 3, 8, 2, 4)
    _, roots, cent, mk, _ = compose(rec, mu, cb, 0, 3)
    st = oracle.snapshot_commit(rec, mu, cb, 0, 3)
    assert np.array_equal(st["root_mk"], cent[0]) and np.array_equal(mk, cent[0])
    rec, mu, cb = synth.snapshot(13, 2, 0, 8, 2, 4)
    leaves, roots, _, _, _ = compose(rec, mu, cb, 2, 0)
    st = oracle.snapshot_commit(rec, mu, cb, 2, 0)
    assert np.array_equal(st["list_roots"], leaves)


def test_binding_moves_exactly_the_covering_roots():
    rec, mu, cb = synth.snapshot(14, 2, 3, 8, 4, 8)
    base = oracle.snapshot_commit(rec, mu, cb, 2, 3)
    # one PQ code component of slot (2, 5)
    r2 = rec.copy()
    r2[2 * 8 + 5, 2 + 3] = (int(r2[2 * 8 + 5, 2 + 3]) + 1) % 8
    st = oracle.snapshot_commit(r2, mu, cb, 2, 3)
    changed = [not np.array_equal(st["list_roots"][i], base["list_roots"][i]) for i in range(4)]
    assert changed == [False, False, True, False]
    assert not np.array_equal(st["root_mk"], base["root_mk"])
    assert np.array_equal(st["root_cb"], base["root_cb"])
    # one centroid coordinate
    m2 = mu.copy()
    m2[1, 0] = (int(m2[1, 0]) + 1) % P
    st = oracle.snapshot_commit(rec, m2, cb, 2, 3)
    assert np.array_equal(st["list_roots"], base["list_roots"])
    assert not np.array_equal(st["root_mk"], base["root_mk"])
    # one codebook coordinate
    c2 = cb.copy()
    c2[3, 7, 1] = (int(c2[3, 7, 1]) + 1) % P
    st = oracle.snapshot_commit(rec, mu, c2, 2, 3)
    assert np.array_equal(st["root_mk"], base["root_mk"])
    assert not np.array_equal(st["root_cb"], base["root_cb"])


def test_field_order_is_canonical():
    # Hash(i, j, f, item, v^(0), v^(1), ...): swapping two code components, or
    # the two indices, changes the digest.
    r = np.array([1, 77, 3, 5, 0, 2], np.uint64)
    a = oracle.hash_(np.concatenate([u64(1, 2), r]))
    b = oracle.hash_(np.concatenate([u64(2, 1), r]))
    r2 = r.copy()
    r2[2], r2[3] = r[3], r[2]
    c = oracle.hash_(np.concatenate([u64(1, 2), r2]))
    assert not np.array_equal(a, b) and not np.array_equal(a, c)


def test_fixed_point_inputs_are_canonical_and_signed():
    rec, mu, cb = synth.snapshot(15, 4, 2, 32, 8, 16)
    for a in (rec, mu, cb):
        assert (a < np.uint64(P)).all()
    signed = np.where(mu > np.uint64(P // 2), -(P - mu.astype(object)), mu.astype(object))
    assert signed.min() >= -65535 and signed.max() <= 65535 and signed.min() < 0 < signed.max()
    assert set(np.unique(rec[:, 0]).tolist()) <= {0, 1}
    assert (rec[rec[:, 0] == 0, 1:] == 0).all()
