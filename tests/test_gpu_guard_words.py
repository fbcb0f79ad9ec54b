"""Guard words around caller-owned output buffers.

The entry points that write into buffers the caller passes (v3c_lde,
v3c_merkle, v3c_coeffs, v3c_seteq, v3c_lde_noalloc) get each output as a
view inside a larger device buffer whose words before and after it hold a
fixed pattern.  After the call the pattern must be intact (no write outside
the output) and the output must equal the oracle's, on shapes that span
several tiles with ragged edges, odd and even row strides, and a view that
starts 8 bytes past a 16-byte boundary (the scalar-store path; v3c_merkle,
whose digests are 16-byte pairs, must refuse such a view and leave it as it
was).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

PATTERN = 0x5A5A5A5A5A5A5A5A
GUARD = 4096  # words on each side


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


def guarded(words: int, offset: int = 0):
    """A device buffer of `words` words between two guard regions; `offset`
    extra words shift the view's start (1 = 8 bytes past 16-byte alignment)."""
    import torch

    buf = torch.full((words + 2 * GUARD + offset,), PATTERN, dtype=torch.int64, device="cuda")
    return buf, buf[GUARD + offset:GUARD + offset + words]


def intact(v3c, buf, words: int, offset: int = 0) -> bool:
    import torch

    torch.cuda.synchronize()
    h = v3c.to_host_u64(buf)
    lo, hi = h[:GUARD + offset], h[GUARD + offset + words:]
    return bool((lo == np.uint64(PATTERN)).all() and (hi == np.uint64(PATTERN)).all())


@pytest.mark.parametrize("c,log_n,r,ld,offset", [(5, 11, 2, 7, 0), (5, 11, 2, 6, 0), (5, 11, 2, 6, 1),
                                                  (9, 13, 3, 10, 0), (3, 4, 1, 3, 1)])
def test_lde_writes_only_its_output(v3c, ctx, c, log_n, r, ld, offset):
    x = synth.columns(seed=40 + c, c=c, log_n=log_n, mix="trace")
    N = 1 << (log_n + r)
    buf, view = guarded(N * ld, offset)
    out = view.view(N, ld)
    ctx.lde(v3c.to_device_u64(x), r, ld=ld, out=out)
    assert intact(v3c, buf, N * ld, offset)
    got = v3c.to_host_u64(out)
    want = oracle.lde(x, r)
    assert np.array_equal(got[:, :c], want[:, :c])
    assert not got[:, c:].any()


@pytest.mark.parametrize("log_rows,width,ld,h", [(13, 5, 6, 3), (10, 16, 17, 0), (9, 8, 8, 9)])
def test_merkle_writes_only_its_tree_and_cap(v3c, ctx, log_rows, width, ld, h):
    import torch

    N = 1 << log_rows
    rows = synth.columns(seed=60 + width, c=ld, log_n=log_rows, mix="uniform").T.copy()  # [N][ld]
    d_rows = v3c.to_device_u64(rows)
    tw = oracle.tree_len(log_rows, h)
    tbuf, tree = guarded(max(tw, 1))
    cbuf, cap = guarded(4 << h)
    ctx.merkle(d_rows, width, h, tree=tree if tw else None, cap=cap.view(1 << h, 4))
    torch.cuda.synchronize()
    assert intact(v3c, tbuf, max(tw, 1))
    assert intact(v3c, cbuf, 4 << h)
    # Digests are stored as 16-byte pairs: a cap 8 bytes off alignment is refused, untouched.
    mbuf, mcap = guarded(4 << h, 1)
    with pytest.raises(v3c.V3CError) as e:
        ctx.merkle(d_rows, width, h, tree=tree if tw else None, cap=mcap.view(1 << h, 4))
    assert e.value.status == v3c.V3C_EINVAL
    assert intact(v3c, mbuf, 4 << h, 1)
    assert (v3c.to_host_u64(mcap) == np.uint64(PATTERN)).all()
    want_tree, want_cap = oracle.merkle(rows, width, h)
    assert np.array_equal(v3c.to_host_u64(cap).reshape(-1), np.asarray(want_cap, np.uint64).reshape(-1))
    if tw:
        assert np.array_equal(v3c.to_host_u64(tree)[:tw], np.asarray(want_tree, np.uint64).reshape(-1)[:tw])


@pytest.mark.parametrize("c,log_n,offset", [(6, 12, 0), (3, 10, 1)])
def test_coeffs_writes_only_its_output(v3c, ctx, c, log_n, offset):
    x = synth.columns(seed=80 + c, c=c, log_n=log_n, mix="trace")
    n = 1 << log_n
    buf, view = guarded(c * n, offset)
    ctx.coeffs(v3c.to_device_u64(x), out=view.view(c, n))
    assert intact(v3c, buf, c * n, offset)
    assert np.array_equal(v3c.to_host_u64(view).reshape(c, n), oracle.coeffs(x))


@pytest.mark.parametrize("L,T", [(3001, 4), (2049, 3), (1, 4)])
def test_seteq_writes_only_its_column(v3c, ctx, L, T):
    import torch

    X, Y = synth.seteq_instance(90 + T, L, T, equal=True)
    ch = synth.challenges(90 + L, 2)
    buf, z = guarded(L + 1, 1)
    st = ctx.seteq([(v3c.to_device_u64(X), v3c.to_device_u64(Y), z, ch[0], ch[1])])
    torch.cuda.synchronize()
    assert st == [0]
    assert intact(v3c, buf, L + 1, 1)
    assert np.array_equal(v3c.to_host_u64(z), oracle.seteq_partial_products(X, Y, ch[0], ch[1]))


def test_lde_noalloc_writes_only_its_output(v3c, ctx):
    c, log_n, r, ld = 7, 12, 3, 9
    x = synth.columns(seed=99, c=c, log_n=log_n, mix="trace")
    N = 1 << (log_n + r)
    buf, view = guarded(N * ld)
    out = view.view(N, ld)
    assert v3c.lde_noalloc(v3c.to_device_u64(x), r, out, ld=ld) == 0
    assert intact(v3c, buf, N * ld)
    got = v3c.to_host_u64(out)
    assert np.array_equal(got[:, :c], oracle.lde(x, r)[:, :c])
    assert not got[:, c:].any()
