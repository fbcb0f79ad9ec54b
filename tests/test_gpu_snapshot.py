"""Snapshot commitment (Sec. 4.3) on the GPU against the CPU oracle.

Bit-exact: root_mk, root_cb, every list root and the top-level paths of
probed lists.  Small shapes cover one list, one slot per list, host and
device inputs and record widths that are not a multiple of the sponge rate;
the SIFT1M high-accuracy layout (8192 lists x 256 slots, D = 128, M = 8,
K = 256) is compared in full.  The MS MARCO high-accuracy layout (8192 x
2048, D = 384) is checked on sampled lists: the oracle recomputes each
sampled list root from its records alone, binds it to its centroid, and
verifies the GPU's top-level path against the GPU's root_mk; root_cb is
compared in full.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v3c():
    from paper_2603_03065_gb300 import build

    build.build()
    import paper_2603_03065_gb300 as m

    return m


@pytest.fixture(scope="module")
def ctx(v3c):
    c = v3c.Context(0)
    yield c
    c.close()


def check_full(v3c, ctx, seed, log_nlist, log_n, D, M, K, device):
    rec, mu, cb = synth.snapshot(seed, log_nlist, log_n, D, M, K)
    if device:
        sid = ctx.snapshot_commit(v3c.to_device_u64(rec), v3c.to_device_u64(mu), v3c.to_device_u64(cb),
                                  log_nlist, log_n)
    else:
        sid = ctx.snapshot_commit(rec, mu, cb, log_nlist, log_n)
    mk, cbr = ctx.snapshot_roots(sid)
    st = oracle.snapshot_commit(rec, mu, cb, log_nlist, log_n)
    assert np.array_equal(ctx.snapshot_list_roots(sid, log_nlist), st["list_roots"])
    assert np.array_equal(mk, st["root_mk"])
    assert np.array_equal(cbr, st["root_cb"])
    if log_nlist:
        tree, cap = oracle.merkle(st["centroid_digests"], 4, 0)
        lists = np.array([0, (1 << log_nlist) - 1, (1 << log_nlist) // 3], np.uint32)
        paths = ctx.snapshot_open_lists(sid, lists, log_nlist)
        for q, i in enumerate(lists):
            assert np.array_equal(paths[q], oracle.merkle_path(tree, log_nlist, 0, int(i)))
            assert oracle.merkle_verify(st["centroid_digests"][i], 4, log_nlist, 0, int(i), paths[q], mk.reshape(1, 4))
    ctx.snapshot_release(sid)


SNAP_CASES = [
    # seed, log_nlist, log_n, D, M, K, device input
    (1, 3, 4, 16, 4, 16, True),
    (2, 3, 4, 16, 4, 16, False),
    (3, 0, 3, 8, 2, 4, True),     # one list: root_mk = hash_0
    (4, 2, 0, 8, 2, 4, True),     # one slot per list: root_i = hash_{i,0}
    (5, 5, 6, 40, 5, 8, True),    # record width 7: one permutation per slot, ragged
    (6, 4, 5, 24, 12, 4, False),  # record width 14: two permutations per slot
    (7, 6, 3, 3, 1, 1, True),     # D = 3, M = K = 1: a 3-word codebook is its own padded digest
]


@pytest.mark.parametrize("seed,log_nlist,log_n,D,M,K,device", SNAP_CASES)
def test_snapshot_matches_oracle(v3c, ctx, seed, log_nlist, log_n, D, M, K, device):
    check_full(v3c, ctx, seed, log_nlist, log_n, D, M, K, device)


def test_snapshot_sift1m_high_acc_full(v3c, ctx):
    p = synth.SNAP_SIFT1M
    check_full(v3c, ctx, 21, p["log_nlist"], p["log_n"], p["D"], p["M"], p["K"], True)


def test_snapshot_msmarco_high_acc_sampled(v3c, ctx):
    p = synth.SNAP_MSMARCO
    ln, lnn = p["log_nlist"], p["log_n"]
    n = 1 << lnn
    rec, mu, cb = synth.snapshot(24, ln, lnn, p["D"], p["M"], p["K"], valid=p["valid"])
    sid = ctx.snapshot_commit(v3c.to_device_u64(rec), v3c.to_device_u64(mu), v3c.to_device_u64(cb), ln, lnn)
    mk, cbr = ctx.snapshot_roots(sid)
    assert np.array_equal(cbr, oracle.hash_(cb.reshape(-1)))
    roots = ctx.snapshot_list_roots(sid, ln)
    rng = np.random.default_rng(24)
    lists = np.unique(np.concatenate([[0, (1 << ln) - 1], rng.integers(0, 1 << ln, size=6)])).astype(np.uint32)
    paths = ctx.snapshot_open_lists(sid, lists, ln)
    for q, i in enumerate(lists):
        root = oracle.snapshot_list_root(rec[int(i) * n:(int(i) + 1) * n], int(i), lnn)
        assert np.array_equal(roots[i], root)
        leaf = oracle.snapshot_centroid_digest(int(i), mu[i], root)
        assert oracle.merkle_verify(leaf, 4, ln, 0, int(i), paths[q], mk.reshape(1, 4))
    ctx.snapshot_release(sid)


def test_snapshot_codebook_digest_cache(v3c):
    # The context reuses root_cb only for codebooks equal word for word: a
    # stale digest would show up as a mismatch against the oracle here.
    with v3c.Context(0) as c:
        rec, mu, cb = synth.snapshot(40, 3, 3, 16, 4, 8)
        rec2, mu2, _ = synth.snapshot(41, 3, 3, 16, 4, 8)
        cb_changed = cb.copy()
        cb_changed[3, 5, 2] = (int(cb_changed[3, 5, 2]) + 1) % oracle.P
        _, _, cb_other = synth.snapshot(42, 3, 3, 16, 4, 4)  # another shape: K = 4
        seq = [(rec, mu, cb), (rec2, mu2, cb), (rec, mu, cb_changed), (rec2, mu2, cb_other), (rec, mu, cb)]
        for r, m, k in seq:
            sid = c.snapshot_commit(v3c.to_device_u64(r), v3c.to_device_u64(m), v3c.to_device_u64(k), 3, 3)
            mk, cbr = c.snapshot_roots(sid)
            assert np.array_equal(cbr, oracle.hash_(k.reshape(-1)))
            assert np.array_equal(mk, oracle.snapshot_commit(r, m, k, 3, 3)["root_mk"])
            c.snapshot_release(sid)


def test_snapshot_errors(v3c, ctx):
    rec, mu, cb = synth.snapshot(8, 2, 2, 8, 2, 4)
    with pytest.raises(v3c.V3CError):
        ctx.snapshot_commit(rec, mu, cb, 21, 2)  # too many lists
    sid = ctx.snapshot_commit(rec, mu, cb, 2, 2)
    with pytest.raises(v3c.V3CError):
        ctx.snapshot_open_lists(sid, [4], 2)  # list out of range
    ctx.snapshot_release(sid)
    with pytest.raises(v3c.V3CError):
        ctx.snapshot_roots(sid)
