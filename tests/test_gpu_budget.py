"""HBM budget: over-budget commits are refused with V3C_ENOMEM and leak nothing.

A context with a 64 MB budget is asked, again and again, for a commit whose
resident LDE alone is 268 MB, and for a batch in which one of two requests is
that large (the whole batch is refused), between commits that fit and are
released.  Every refusal must leave the context's resident bytes, the bytes
in use in the device's stream-ordered pool and the scratch arena where they
were, and the commits that fit must still equal the oracle.
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


def test_budget_refusals_and_releases_leak_nothing(v3c):
    import torch

    small = synth.columns(seed=5, c=8, log_n=8, mix="trace")
    big = np.zeros((64, 1 << 16), np.uint64)
    _, _, want = oracle.commit(small, 2, 1)
    with v3c.Context(0, hbm_budget_bytes=64 << 20) as c:
        cid = c.commit([(small, 2, 1)])[0]  # warm: plan tables and scratch arena
        c.release(cid)
        torch.cuda.synchronize()
        base = c.mem_stats()
        assert base["resident"] == 0
        for _ in range(10):
            with pytest.raises(v3c.V3CError) as e:
                c.commit([(big, 3, 4)])
            assert e.value.status == v3c.V3C_ENOMEM
            with pytest.raises(v3c.V3CError) as e:
                c.commit([(small, 2, 1), (big, 3, 4)])
            assert e.value.status == v3c.V3C_ENOMEM
            assert c.mem_stats()["resident"] == 0
            ids = c.commit([(small, 2, 1), (small, 2, 1)])
            assert c.mem_stats()["resident"] > 0
            for cid in ids:
                assert np.array_equal(np.asarray(c.cap(cid)).reshape(-1), np.asarray(want).reshape(-1))
                c.release(cid)
        torch.cuda.synchronize()
        end = c.mem_stats()
        assert end["resident"] == 0
        assert end["pool_used"] == base["pool_used"]
        assert end["arena"] == base["arena"]
