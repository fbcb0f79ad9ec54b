"""Serving loop (continuous batching) on the GPU.

Requests of different shapes arrive while others run.  Each request's cap
must equal the oracle's and the cap of the same commit made alone (tolerance
zero).  Objects stay resident after DONE until released.  Admission respects
the HBM budget, and stop() resolves queued requests with ECANCELED, as does
a failure of the scheduler thread (injected on the host).
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


def wait_done(ctx, v3c, tickets, caps, timeout=120.0):
    pending = set(tickets)
    out = {}
    t0 = time.time()
    while pending and time.time() - t0 < timeout:
        for t in list(pending):
            st, state, cap, times = ctx.serve_poll(t, caps[t])
            if st == v3c.V3C_OK:
                out[t] = (cap, times)
                pending.discard(t)
            elif st != v3c.V3C_EAGAIN:
                raise AssertionError(f"ticket {t} failed with status {st}")
        time.sleep(0.002)
    assert not pending, f"{len(pending)} requests not done"
    return out


def test_mixed_requests_equal_alone_and_oracle(v3c):
    shapes = [synth.Shape(c=c, log_n=ln, rate_bits=r, cap_height=h, seed=21, batch=b)
              for b, (c, ln, r, h) in enumerate([(80, 10, 3, 4), (135, 11, 3, 4), (20, 12, 1, 4), (7, 8, 2, 0),
                                                 (33, 9, 2, 3), (80, 10, 3, 4), (135, 9, 3, 4), (9, 13, 1, 4),
                                                 (64, 8, 3, 2), (21, 12, 2, 4)])]
    xs = [s.inputs() for s in shapes]
    with v3c.Context(0, max_inflight=3) as ctx:
        ctx.serve_start(max_batch=4)
        tickets, caps = [], {}
        for i, (s, x) in enumerate(zip(shapes, xs)):
            t = ctx.serve_submit(x, s.rate_bits, s.cap_height)
            assert t > 0
            tickets.append(t)
            caps[t] = s.cap_height
            if i % 3 == 2:
                time.sleep(0.01)        # later arrivals join while earlier ones run
        done = wait_done(ctx, v3c, tickets, caps)
        for t, s, x in zip(tickets, shapes, xs):
            cap, times = done[t]
            _, _, want_cap = oracle.commit(x, s.rate_bits, s.cap_height)
            assert np.array_equal(cap, want_cap)
            ts, ta, tst, td = times
            assert ts <= ta <= tst <= td
            alone = ctx.commit([(x, s.rate_bits, s.cap_height)])[0]
            assert np.array_equal(ctx.cap(alone), cap)
            ctx.release(alone)
            # resident after DONE: open a leaf and verify it against the cap
            o = ctx.open(t, 3, s.c)
            assert oracle.merkle_verify(o.row, s.c, s.log_N, s.cap_height, 3, o.path, cap)
        for t in tickets:
            ctx.release(t)
        ctx.serve_stop()


def test_admission_waits_for_budget_and_stop_cancels(v3c):
    s = synth.Shape(c=16, log_n=12, rate_bits=2, cap_height=4, seed=3)
    fp = v3c.footprint(s.c, s.log_n, s.rate_bits, s.cap_height)
    x = s.inputs()
    # budget for two resident objects: the third request waits until a release
    with v3c.Context(0, hbm_budget_bytes=2 * fp + fp // 2, max_inflight=2) as ctx:
        ctx.serve_start(max_batch=8)
        t1 = ctx.serve_submit(x, s.rate_bits, s.cap_height)
        t2 = ctx.serve_submit(x, s.rate_bits, s.cap_height)
        t3 = ctx.serve_submit(x, s.rate_bits, s.cap_height)
        done = wait_done(ctx, v3c, [t1, t2], {t1: s.cap_height, t2: s.cap_height})
        time.sleep(0.05)
        st, state, _, _ = ctx.serve_poll(t3, s.cap_height)
        assert st == v3c.V3C_EAGAIN and state == v3c.REQ_QUEUED
        ctx.release(t1)                  # frees budget: t3 is admitted
        done3 = wait_done(ctx, v3c, [t3], {t3: s.cap_height})
        assert np.array_equal(done3[t3][0], done[t1][0])
        ctx.release(t2)
        ctx.release(t3)
        # a request that can never fit is refused at submit
        big = synth.Shape(c=64, log_n=16, rate_bits=3, cap_height=4)
        with pytest.raises(v3c.V3CError):
            ctx.serve_submit(np.zeros((big.c, 1 << big.log_n), np.uint64), big.rate_bits, big.cap_height)
        # queued work is cancelled by stop
        t4 = ctx.serve_submit(x, s.rate_bits, s.cap_height)
        t5 = ctx.serve_submit(x, s.rate_bits, s.cap_height)
        t6 = ctx.serve_submit(x, s.rate_bits, s.cap_height)
        ctx.serve_stop()
        assert ctx.lib.v3c_serve_poll(ctx.h, t6, None, None, None) == v3c.V3C_ECANCELED
        for t in (t4, t5):
            try:
                ctx.release(t)
            except v3c.V3CError:
                pass


def test_scheduler_failure_fails_queued_requests_and_keeps_the_context(v3c):
    # Host-side injection: the scheduler thread raises.  Requests already on
    # the device finish (DONE, caps equal to the oracle's); those waiting for
    # memory resolve to FAILED with ECANCELED; later submits are refused;
    # stop still works and the context still commits.
    s = synth.Shape(c=16, log_n=12, rate_bits=2, cap_height=4, seed=4)
    fp = v3c.footprint(s.c, s.log_n, s.rate_bits, s.cap_height)
    x = s.inputs()
    _, _, want = oracle.commit(x, s.rate_bits, s.cap_height)
    with v3c.Context(0, hbm_budget_bytes=2 * fp + fp // 2, max_inflight=2) as ctx:
        ctx.serve_start(max_batch=8)
        tickets = [ctx.serve_submit(x, s.rate_bits, s.cap_height) for _ in range(5)]
        done = wait_done(ctx, v3c, tickets[:2], {t: s.cap_height for t in tickets[:2]})
        for t in tickets[:2]:
            assert np.array_equal(np.asarray(done[t][0]).reshape(-1), np.asarray(want).reshape(-1))
        time.sleep(0.05)
        for t in tickets[2:]:  # nothing released: they wait for memory
            st, state, _, _ = ctx.serve_poll(t, s.cap_height)
            assert st == v3c.V3C_EAGAIN and state == v3c.REQ_QUEUED
        ctx.serve_inject_failure(0)
        t0 = time.time()
        states = {}
        while len(states) < 3 and time.time() - t0 < 10:
            for t in tickets[2:]:
                st, state, _, _ = ctx.serve_poll(t, s.cap_height)
                if st != v3c.V3C_EAGAIN:
                    states[t] = (st, state)
            time.sleep(0.005)
        assert all(v == (v3c.V3C_ECANCELED, v3c.REQ_FAILED) for v in states.values()) and len(states) == 3
        with pytest.raises(v3c.V3CError) as e:
            ctx.serve_submit(x, s.rate_bits, s.cap_height)
        assert e.value.status == v3c.V3C_ECANCELED
        ctx.serve_stop()
        for t in tickets[:2]:
            ctx.release(t)
        cid = ctx.commit([(x, s.rate_bits, s.cap_height)])[0]
        assert np.array_equal(np.asarray(ctx.cap(cid)).reshape(-1), np.asarray(want).reshape(-1))
        ctx.release(cid)


def test_borrowed_pinned_and_device_inputs(v3c):
    import torch

    shapes = [synth.Shape(c=24, log_n=12, rate_bits=2, cap_height=4, seed=8, batch=b) for b in range(4)]
    xs = [s.inputs() for s in shapes]
    pinned = [torch.from_numpy(x.view(np.int64)).pin_memory() for x in xs]
    with v3c.Context(0) as ctx:
        ctx.serve_start(max_batch=3, slot_scratch_bytes=1 << 20)   # tiny cap: one request per pass
        tickets, caps = [], {}
        for i, (s, x, p) in enumerate(zip(shapes, xs, pinned)):
            src = p.numpy().view(np.uint64) if i % 2 == 0 else v3c.to_device_u64(x)
            t = ctx.serve_submit(src, s.rate_bits, s.cap_height, borrow=True)
            tickets.append(t)
            caps[t] = s.cap_height
        done = wait_done(ctx, v3c, tickets, caps)
        for t, s, x in zip(tickets, shapes, xs):
            _, _, want_cap = oracle.commit(x, s.rate_bits, s.cap_height)
            assert np.array_equal(done[t][0], want_cap)
            ctx.release(t)
        ctx.serve_stop()


def test_small_requests_do_not_wait_for_a_large_one(v3c):
    """Requests are batched by size class: small requests that arrive just
    after a large one run as their own batch (on a higher-priority stream)
    and finish before the large one, instead of completing with it."""
    big = synth.Shape(c=135, log_n=18, rate_bits=3, cap_height=4, seed=13)
    small = [synth.Shape(c=8, log_n=10, rate_bits=3, cap_height=4, seed=13, batch=b) for b in range(1, 6)]
    xb = big.inputs()
    xs = [s.inputs() for s in small]
    with v3c.Context(0, max_inflight=4) as ctx:
        # warm the plans of both shapes
        ctx.release(ctx.commit([(xb, 3, 4)])[0])
        ctx.release(ctx.commit([(xs[0], 3, 4)])[0])
        ctx.serve_start(max_batch=8)
        tb = ctx.serve_submit(xb, 3, 4)
        ts = [ctx.serve_submit(x, 3, 4) for x in xs]
        caps = {t: 4 for t in [tb] + ts}
        done = wait_done(ctx, v3c, [tb] + ts, caps)
        t_big = done[tb][1][3]
        for t, s, x in zip(ts, small, xs):
            cap, times = done[t]
            assert times[3] < t_big, "a small request completed only with the large one"
            _, _, want = oracle.commit(x, 3, 4)
            assert np.array_equal(cap, want)
        _, _, want_big = oracle.commit(xb, 3, 4)
        assert np.array_equal(done[tb][0], want_big)
        for t in [tb] + ts:
            ctx.release(t)
        ctx.serve_stop()
