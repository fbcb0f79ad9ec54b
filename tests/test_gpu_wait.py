"""Bounded device waits give up and report, and the context stays usable.

The library's waiting kernels (the SetEq look-back, the FRI copy pipeline)
limit every wait and turn an expired one into V3C_ETIMEDOUT.  Their waits are
always satisfied in normal operation, so v3c_wait_selftest runs a kernel
whose wait nothing satisfies: an mbarrier phase that never completes (the
FRI pipeline's wait) and a device word that nothing sets.  Each must give up
after its limit, report the time-out, and leave the context able to commit
bit-exactly against the oracle.
"""
import time

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


def commit_matches_oracle(v3c, ctx):
    x = synth.columns(seed=77, c=8, log_n=8, mix="uniform")
    cid = ctx.commit([(v3c.to_device_u64(x), 2, 1)])[0]
    cap = ctx.cap(cid)
    ctx.release(cid)
    _, _, want = oracle.commit(x, 2, 1)
    return np.array_equal(np.asarray(cap, np.uint64).reshape(-1), np.asarray(want, np.uint64).reshape(-1))


@pytest.mark.parametrize("kind", [0, 1])
def test_wait_gives_up_and_context_stays_usable(v3c, ctx, kind):
    limit_us = 50_000
    t0 = time.perf_counter()
    with pytest.raises(v3c.V3CError) as e:
        ctx.wait_selftest(kind, limit_us)
    dt = time.perf_counter() - t0
    assert e.value.status == v3c.V3C_ETIMEDOUT
    assert dt >= limit_us * 1e-6
    assert dt < 10.0
    assert commit_matches_oracle(v3c, ctx)
    # A second expired wait on the same context behaves the same.
    with pytest.raises(v3c.V3CError) as e:
        ctx.wait_selftest(kind, 1000)
    assert e.value.status == v3c.V3C_ETIMEDOUT
    assert commit_matches_oracle(v3c, ctx)


def test_wait_selftest_rejects_bad_arguments(v3c, ctx):
    for kind, limit in [(2, 1000), (0, 0), (1, 2_000_001)]:
        with pytest.raises(v3c.V3CError) as e:
            ctx.wait_selftest(kind, limit)
        assert e.value.status == v3c.V3C_EINVAL
