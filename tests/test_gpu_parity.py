"""Bit-exact parity of the CUDA path (through the C ABI) with the CPU oracle.

All values are field elements; the tolerance is zero.  Small shapes are
compared element by element over the whole LDE, tree and cap.  They span
several tiles, ragged column counts (odd, not a multiple of 8) and every
stage split (n1 = 1 and n1 > 1).  The 135 x 2^16 workload is compared in
full; the 135 x 2^20 workload on sampled rows, leaves and nodes and by
whole-column properties, in the launch configuration the benchmark times.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

P = oracle.P


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


def gpu_lde(v3c, ctx, x, r, ld=None):
    import torch

    d = v3c.to_device_u64(x)
    out = ctx.lde(d, r, ld=ld)
    torch.cuda.synchronize()
    return v3c.to_host_u64(out)


def gpu_merkle(v3c, ctx, rows, width, h):
    import torch

    d = v3c.to_device_u64(rows)
    tree, cap = ctx.merkle(d, width, h)
    torch.cuda.synchronize()
    t = v3c.to_host_u64(tree) if tree is not None else np.zeros(0, np.uint64)
    return t, v3c.to_host_u64(cap)


LDE_SHAPES = [
    (1, 0, 0), (1, 0, 3), (2, 1, 1), (3, 3, 0), (8, 10, 3), (13, 5, 2), (5, 11, 2), (4, 13, 0),
    (13, 12, 3), (9, 14, 1), (6, 15, 3), (3, 16, 2), (2, 17, 3),
]


@pytest.mark.parametrize("c,log_n,r", LDE_SHAPES)
def test_lde_bit_exact(v3c, ctx, c, log_n, r):
    x = synth.columns(seed=c * 100 + log_n * 10 + r, c=c, log_n=log_n, mix="trace" if c >= 4 else "uniform")
    want = oracle.lde(x, r)
    got = gpu_lde(v3c, ctx, x, r)
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("ld", [13, 20])
def test_lde_odd_and_padded_row_stride(v3c, ctx, ld):
    x = synth.columns(seed=77, c=13, log_n=12, mix="trace")
    want = oracle.lde(x, 3, ld=ld)
    got = gpu_lde(v3c, ctx, x, 3, ld=ld)
    assert np.array_equal(got, want)


def test_lde_extremes_of_the_field(v3c, ctx):
    n = 1 << 12
    x = np.stack([np.full(n, P - 1, np.uint64), np.zeros(n, np.uint64),
                  np.array([(P - 1) if i % 2 else 1 for i in range(n)], np.uint64)])
    assert np.array_equal(gpu_lde(v3c, ctx, x, 2), oracle.lde(x, 2))


@pytest.mark.parametrize("width,log_rows,h", [
    (1, 3, 0), (4, 5, 2), (5, 6, 1), (8, 7, 0), (9, 9, 3), (16, 8, 8), (17, 10, 4), (135, 9, 4), (24, 12, 0),
])
def test_merkle_bit_exact(v3c, ctx, width, log_rows, h):
    rng = np.random.default_rng(width * 1000 + log_rows)
    ld = width + (width & 1)
    rows = rng.integers(0, P, size=(1 << log_rows, ld), dtype=np.uint64)
    want_tree, want_cap = oracle.merkle(rows, width, h)
    got_tree, got_cap = gpu_merkle(v3c, ctx, rows, width, h)
    assert np.array_equal(got_cap.reshape(-1, 4), want_cap)
    assert np.array_equal(got_tree, want_tree)


def test_merkle_unaligned_row_stride(v3c, ctx):
    rng = np.random.default_rng(5)
    rows = rng.integers(0, P, size=(1 << 8, 11), dtype=np.uint64)   # odd ld: scalar loads
    want_tree, want_cap = oracle.merkle(rows, 11, 2)
    got_tree, got_cap = gpu_merkle(v3c, ctx, rows, 11, 2)
    assert np.array_equal(got_tree, want_tree) and np.array_equal(got_cap.reshape(-1, 4), want_cap)


def check_object(ctx, cid, x, r, h):
    e, tree, cap = oracle.commit(x, r, h)
    got = ctx.commit_views(cid, x.shape[0])
    assert np.array_equal(got["lde"], e)
    assert np.array_equal(got["tree"], tree)
    assert np.array_equal(got["cap"], cap)
    assert np.array_equal(ctx.cap(cid), cap)


def test_plain_commit_8x2_10(v3c, ctx):
    s = synth.PLAIN_8x2_10
    x = s.inputs()
    cid = ctx.commit([(v3c.to_device_u64(x), s.rate_bits, s.cap_height)])[0]
    check_object(ctx, cid, x, s.rate_bits, s.cap_height)
    ctx.release(cid)


def test_batched_uneven_commit_matches_each_alone(v3c, ctx):
    shapes = [synth.Shape(c=c, log_n=ln, rate_bits=r, cap_height=h, seed=9, batch=b)
              for b, (c, ln, r, h) in enumerate([(20, 12, 1, 4), (33, 13, 2, 4), (7, 9, 3, 0), (135, 10, 3, 4),
                                                 (21, 14, 2, 4), (5, 3, 1, 4)])]
    xs = [s.inputs() for s in shapes]
    # half host inputs, half device inputs
    items = [(x if i % 2 else v3c.to_device_u64(x), s.rate_bits, s.cap_height)
             for i, (x, s) in enumerate(zip(xs, shapes))]
    ids = ctx.commit(items)
    for cid, x, s in zip(ids, xs, shapes):
        check_object(ctx, cid, x, s.rate_bits, s.cap_height)
    for cid in ids:
        ctx.release(cid)


def test_open_paths_verify_against_oracle(v3c, ctx):
    s = synth.Shape(c=19, log_n=9, rate_bits=2, cap_height=3, seed=12)
    x = s.inputs()
    cid = ctx.commit([(x, s.rate_bits, s.cap_height)])[0]
    cap = ctx.cap(cid)
    e = oracle.lde(x, s.rate_bits)
    rng = np.random.default_rng(1)
    for leaf in list(rng.integers(0, 1 << s.log_N, size=12)) + [0, (1 << s.log_N) - 1]:
        o = ctx.open(cid, int(leaf), s.c)
        assert np.array_equal(o.row, e[leaf, : s.c])
        assert o.path.shape == (s.log_N - s.cap_height, 4)
        assert oracle.merkle_verify(o.row, s.c, s.log_N, s.cap_height, int(leaf), o.path, cap)
        bad = o.path.copy()
        bad[0, 0] ^= np.uint64(1)
        assert not oracle.merkle_verify(o.row, s.c, s.log_N, s.cap_height, int(leaf), bad, cap)
    ctx.release(cid)


def test_errors_are_reported(v3c):
    import torch

    with v3c.Context(0, flags=v3c.FLAG_VALIDATE) as c:
        x = np.full((3, 16), P, np.uint64)                  # not canonical
        with pytest.raises(v3c.V3CError) as ei:
            c.commit([(x, 1, 0)])
        assert ei.value.status == v3c.V3C_EINVAL
        with pytest.raises(v3c.V3CError) as ei:
            c.release(12345)
        assert ei.value.status == v3c.V3C_ENOTFOUND
        with pytest.raises(v3c.V3CError) as ei:
            c.commit([(np.zeros((2, 8), np.uint64), 1, 9)])  # cap height > log N
        assert ei.value.status == v3c.V3C_EINVAL
    with v3c.Context(0, hbm_budget_bytes=1 << 20) as c:
        with pytest.raises(v3c.V3CError) as ei:
            c.commit([(np.zeros((8, 1 << 12), np.uint64), 3, 0)])
        assert ei.value.status == v3c.V3C_ENOMEM
        cid = c.commit([(np.zeros((2, 8), np.uint64), 1, 0)])[0]  # small one fits
        c.release(cid)
    torch.cuda.synchronize()


# ---------------------------------------------------------------- full-size workloads

def test_trace_commit_135x2_16_full(v3c, ctx):
    s = synth.TRACE_135x2_16
    x = s.inputs()
    cid = ctx.commit([(v3c.to_device_u64(x), s.rate_bits, s.cap_height)])[0]
    got = ctx.commit_views(cid, s.c)
    want_lde = oracle.lde(x, s.rate_bits)
    assert np.array_equal(got["lde"], want_lde)
    # every leaf, and every tree node from its children
    N = 1 << s.log_N
    leaves = oracle.leaf_hashes(want_lde, s.c)
    tree = got["tree"]
    assert np.array_equal(tree[: 4 * N].reshape(-1, 4), leaves)
    off, cnt = 0, N
    for k in range(s.log_N - s.cap_height):
        below = tree[off: off + 4 * cnt]
        above = oracle.merkle_level(below)
        off += 4 * cnt
        cnt //= 2
        nxt = tree[off: off + 4 * cnt].reshape(-1, 4) if k + 1 < s.log_N - s.cap_height else got["cap"]
        assert np.array_equal(above, nxt)
    ctx.release(cid)


def test_large_commit_135x2_20_sampled(v3c, ctx):
    import torch

    s = synth.LARGE_135x2_20
    x = s.inputs()
    d = v3c.to_device_u64(x)
    cid = ctx.commit([(d, s.rate_bits, s.cap_height)])[0]
    torch.cuda.synchronize()
    b = ctx.buffers(cid)
    N = 1 << s.log_N
    lde_t = _wrap(b["lde"], N * b["ld"]).view(N, b["ld"])
    tree_t = _wrap(b["tree"], v3c.tree_words(s.log_N, s.cap_height))
    cap = ctx.cap(cid)
    rng = np.random.default_rng(2024)
    rows = np.unique(np.concatenate([[0, 1, N - 1, N // 2], rng.integers(0, N, size=12)])).astype(np.uint64)
    co = oracle.coeffs(x)
    want_rows = oracle.lde_rows(co, s.rate_bits, rows)
    got_rows = lde_t[torch.as_tensor(rows.astype(np.int64), device="cuda")].cpu().numpy().view(np.uint64)
    assert np.array_equal(got_rows[:, : s.c], want_rows)
    assert np.all(got_rows[:, s.c:] == 0)
    # sampled leaves
    tree_h = tree_t.cpu().numpy().view(np.uint64)
    leaves = oracle.leaf_hashes(np.ascontiguousarray(want_rows), s.c)
    assert np.array_equal(tree_h[: 4 * N].reshape(-1, 4)[rows.astype(np.int64)], leaves)
    # sampled nodes at every level, and the cap from the level below it
    off, cnt = 0, N
    top = s.log_N - s.cap_height
    for k in range(top):
        lvl = tree_h[off: off + 4 * cnt].reshape(-1, 4)
        nxt_off = off + 4 * cnt
        above_cnt = cnt // 2
        above = tree_h[nxt_off: nxt_off + 4 * above_cnt].reshape(-1, 4) if k + 1 < top else cap
        idx = np.unique(rng.integers(0, above_cnt, size=min(above_cnt, 64)))
        pairs = np.concatenate([lvl[2 * idx], lvl[2 * idx + 1]], axis=1).reshape(-1, 4)
        assert np.array_equal(oracle.merkle_level(pairs), above[idx])
        off, cnt = nxt_off, above_cnt
    # whole-column property: the committed column re-interpolates to the
    # oracle coefficients times 7^i, with nothing at degree >= n
    for j in (0, s.c - 1):
        col = lde_t[:, j].cpu().numpy().view(np.uint64)
        natural = np.empty_like(col)
        natural[_bitrev_indices(s.log_N)] = col          # row t holds E_bitrev(t)
        a = oracle.intt(natural)                          # coefficients of P(7x)
        n = 1 << s.log_n
        assert np.all(a[n:] == 0)
        sample = rng.integers(0, n, size=32)
        for i in sample:
            assert int(a[i]) == (int(co[j, i]) * pow(7, int(i), P)) % P
    ctx.release(cid)


def _bitrev_indices(bits):
    idx = np.arange(1 << bits, dtype=np.uint64)
    out = np.zeros_like(idx)
    for b in range(bits):
        out |= ((idx >> np.uint64(b)) & np.uint64(1)) << np.uint64(bits - 1 - b)
    return out.astype(np.int64)


def _wrap(ptr, words):
    import torch

    class _A:
        __cuda_array_interface__ = {"shape": (words,), "typestr": "<i8", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_A(), device="cuda")


def test_graph_replay_matches_direct_launches(v3c):
    # Five calls with one batch signature: more than the ring of three captured
    # instances, so job tables of reused instances are rewritten between replays.
    shapes = [(20, 12, 1, 4), (33, 11, 2, 3), (135, 10, 3, 4)]
    with v3c.Context(0) as g, v3c.Context(0, flags=v3c.FLAG_NO_GRAPH) as d:
        for rep in range(5):
            xs = [synth.columns(seed=60 + rep, c=c, log_n=ln, batch=i) for i, (c, ln, r, h) in enumerate(shapes)]
            items = [(v3c.to_device_u64(x), r, h) for x, (c, ln, r, h) in zip(xs, shapes)]
            ids_g = g.commit(items)
            ids_d = d.commit(items)
            for ig, idd, x, (c, ln, r, h) in zip(ids_g, ids_d, xs, shapes):
                vg, vd = g.commit_views(ig, c), d.commit_views(idd, c)
                for key in ("lde", "tree", "cap"):
                    assert np.array_equal(vg[key], vd[key])
                if rep == 0:
                    check_object(g, ig, x, r, h)
            for i in ids_g:
                g.release(i)
            for i in ids_d:
                d.release(i)


def test_autotuned_commit_matches_oracle(v3c):
    with v3c.Context(0, autotune=True) as ctx:
        for (c, ln, r, h) in [(13, 12, 3, 4), (40, 14, 1, 2)]:
            x = synth.columns(seed=70 + ln, c=c, log_n=ln)
            cid = ctx.commit([(x, r, h)])[0]
            check_object(ctx, cid, x, r, h)
            ctx.release(cid)


# Large host inputs are copied in column chunks on a copy stream, and the
# LDE's first stages run per chunk as the copies land.
@pytest.mark.parametrize("c,log_n,r,h", [(135, 16, 3, 4), (65, 16, 2, 2), (4099, 10, 2, 3)])
def test_chunked_host_input_commit(v3c, ctx, c, log_n, r, h):
    x = synth.columns(seed=c + log_n, c=c, log_n=log_n, mix="trace")
    cid = ctx.commit([(x, r, h)])[0]
    got = ctx.commit_views(cid, c)
    lde, tree, cap = oracle.commit(x, r, h)
    assert np.array_equal(got["lde"].reshape(lde.shape), lde)
    assert np.array_equal(got["cap"].reshape(cap.shape), cap)
    assert np.array_equal(got["tree"], tree)
    ctx.release(cid)


def test_chunked_and_plain_inputs_in_one_batch(v3c, ctx):
    a = synth.columns(seed=1, c=9, log_n=12, mix="trace")     # device input
    b = synth.columns(seed=2, c=40, log_n=17, mix="trace")    # host, chunked
    c_ = synth.columns(seed=3, c=7, log_n=11, mix="trace")    # host, small
    ids = ctx.commit([(v3c.to_device_u64(a), 3, 2), (b, 2, 4), (c_, 1, 0)])
    for cid, (x, r, h) in zip(ids, [(a, 3, 2), (b, 2, 4), (c_, 1, 0)]):
        got = ctx.commit_views(cid, x.shape[0])
        lde, tree, cap = oracle.commit(x, r, h)
        assert np.array_equal(got["lde"].reshape(lde.shape), lde)
        assert np.array_equal(got["cap"].reshape(cap.shape), cap)
        ctx.release(cid)


def test_maximum_size_commit_sampled(v3c):
    # The largest shape the library accepts: 2^22 input rows at rate 3, i.e.
    # 2^25 LDE rows (the V3C_MAX_LOG_LDE limit).  Three columns (rows of
    # width <= 4 are their own zero-padded leaf digests).  Sampled rows are
    # checked against the oracle's Horner evaluation, and their Merkle paths,
    # read back with the batched opening, must verify against the GPU's cap.
    import torch

    c, log_n, r, h = 3, 22, 3, 4
    x = synth.columns(seed=2222, c=c, log_n=log_n, mix="trace")
    with v3c.Context(0) as big:
        cid = big.commit([(v3c.to_device_u64(x), r, h)])[0]
        torch.cuda.synchronize()
        N = 1 << (log_n + r)
        rng = np.random.default_rng(22)
        rows = np.unique(np.concatenate([[0, 1, N - 1, N // 2], rng.integers(0, N, size=8)])).astype(np.uint64)
        got_rows, paths = big.open_batch(cid, rows, c)
        want_rows = oracle.lde_rows(oracle.coeffs(x), r, rows)
        assert np.array_equal(got_rows, want_rows)
        cap = big.cap(cid)
        for q, t in enumerate(rows):
            assert oracle.merkle_verify(want_rows[q], c, log_n + r, h, int(t), paths[q], cap)
        big.release(cid)
    with v3c.Context(0) as small:
        with pytest.raises(v3c.V3CError):
            small.commit([(v3c.to_device_u64(synth.columns(seed=1, c=1, log_n=log_n, mix="uniform")), 4, 0)])


def test_pipelined_host_input_commits(v3c):
    """Commits of large host inputs enqueued back to back, each cap read only
    after the next commit is enqueued (the input copies of commit k+1 run on
    the copy stream while commit k computes): every object equals the
    oracle's commit of its own input."""
    import torch

    # 64 x 2^16 words: at the 2^22-word threshold of the chunked copy path
    shapes = [synth.Shape(c=64, log_n=16, rate_bits=2, cap_height=3, seed=71, batch=b) for b in range(3)]
    xs = [s.inputs() for s in shapes]
    pinned = [torch.from_numpy(x.view(np.int64)).pin_memory().numpy().view(np.uint64) for x in xs]
    with v3c.Context(0) as c:
        stream = torch.cuda.current_stream()
        ids = []
        for p, s in zip(pinned, shapes):
            ids.append(c.commit([(p, s.rate_bits, s.cap_height)], stream=stream)[0])
        for cid, x, s in zip(ids, xs, shapes):
            lde, tree, cap = oracle.commit(x, s.rate_bits, s.cap_height)
            assert np.array_equal(c.cap(cid), cap)
            got = c.commit_views(cid, s.c)
            assert np.array_equal(got["lde"], lde)
            c.release(cid)
