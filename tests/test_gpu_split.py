"""The kernels of the multi-GPU row split, on one GPU (tolerance zero).

v3c_coeffs gives each column's interpolant coefficients (compared with the
oracle's inverse NTT), computed here shard by shard as the ranks would.
v3c_commit_part then commits each part q of G from the whole coefficient
table; its rows must equal the rows [q N/G, (q+1) N/G) of the oracle's LDE,
its tree the oracle's subtree over that block and its cap the matching slice
of the oracle's cap.  The parts are run one after another on the same GPU
(no collective is exercised here; the exchange is covered by the gloo test).
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


def _coeffs_by_shards(v3c, ctx, x, world):
    import torch

    from paper_2603_03065_gb300 import split

    c, n = x.shape
    parts = []
    for rank in range(world):
        c0, c1 = split.column_shard(c, world, rank)
        if c1 > c0:
            parts.append(ctx.coeffs(v3c.to_device_u64(x[c0:c1])))
    torch.cuda.synchronize()
    return torch.cat(parts, dim=0).contiguous()


@pytest.mark.parametrize("c,log_n,r,h,log_parts", [
    (8, 10, 3, 4, 1), (13, 12, 3, 4, 2), (9, 9, 2, 2, 2), (5, 13, 3, 3, 3), (20, 14, 1, 1, 1), (3, 6, 3, 4, 3),
    (17, 16, 2, 4, 2),
])
def test_parts_equal_blocks_of_the_single_commit(v3c, c, log_n, r, h, log_parts):
    import torch

    from paper_2603_03065_gb300 import split

    s = synth.Shape(c=c, log_n=log_n, rate_bits=r, cap_height=h, seed=31)
    x = s.inputs()
    lde, _, cap = oracle.commit(x, r, h)
    with v3c.Context(0) as ctx:
        co = _coeffs_by_shards(v3c, ctx, x, 1 << log_parts)
        assert np.array_equal(co.cpu().numpy().view(np.uint64), oracle.coeffs(x))
        for q in range(1 << log_parts):
            cid = ctx.commit_part(co, r, h, log_parts, q)
            got = ctx.commit_views(cid, c)
            r0, r1 = split.part_rows(s.log_N, log_parts, q)
            assert np.array_equal(got["lde"], lde[r0:r1])
            tree, sub_cap = oracle.merkle(lde[r0:r1], c, h - log_parts)
            assert np.array_equal(got["tree"], tree)
            e0, e1 = split.cap_slice(h, log_parts, q)
            assert np.array_equal(got["cap"], cap[e0:e1])
            assert np.array_equal(sub_cap, cap[e0:e1])
            ctx.release(cid)
        torch.cuda.synchronize()


def test_trace_135x2_16_in_eight_parts(v3c):
    """The 135 x 2^16 workload at rate 3 split into its eight cosets: the
    concatenated caps equal the single commit's cap, every part's rows its
    block of the LDE."""
    import torch

    from paper_2603_03065_gb300 import split

    s = synth.TRACE_135x2_16
    x = s.inputs()
    lde, _, cap = oracle.commit(x, s.rate_bits, s.cap_height)
    with v3c.Context(0) as ctx:
        co = _coeffs_by_shards(v3c, ctx, x, 8)
        caps = []
        for q in range(8):
            cid = ctx.commit_part(co, s.rate_bits, s.cap_height, 3, q)
            got = ctx.commit_views(cid, s.c)
            r0, r1 = split.part_rows(s.log_N, 3, q)
            assert np.array_equal(got["lde"], lde[r0:r1])
            caps.append(got["cap"])
            ctx.release(cid)
        torch.cuda.synchronize()
    assert np.array_equal(np.concatenate(caps), cap)


def test_part_arguments_are_checked(v3c):
    import torch

    co = torch.zeros((4, 1 << 8), dtype=torch.int64, device="cuda")
    with v3c.Context(0) as ctx:
        for r, h, lp, q in [(2, 4, 3, 0), (3, 1, 2, 0), (3, 4, 2, 4)]:   # parts > 2^r, > 2^h, part >= G
            with pytest.raises(v3c.V3CError) as ei:
                ctx.commit_part(co, r, h, lp, q)
            assert ei.value.status == v3c.V3C_EINVAL
