"""Bit-exact parity on the commit workloads at their own sizes.

The commitment is the Merkle roots over the committed trace (Sec. 4.3), an
exact function of the input, so the tolerance is zero.  Three workloads are
compared with the CPU oracle (all host cores) at the sizes the benchmark runs
them, through the C ABI and in the launch configuration the benchmark times:

* the large commit, 135 x 2^20 at rate 3, cap height 4 (about 9 GB of LDE):
  every LDE word, every tree level and the cap;
* the 64 uneven column batches of seed 3 (log2 rows 12..18, 20..135 columns,
  rate 1..3, cap height 4) committed by ONE batched v3c_commit, replayed from
  its captured CUDA graph with autotuned tiles: every batch's LDE, tree and cap;
* a slice of the serving trace (the mixture 2^14 x 80 / 2^16 x 135 /
  2^18 x 135, rate 3, cap height 4), all requests submitted at once so that
  they are admitted and run side by side: each cap equals the oracle's and the
  same request committed alone, and one large request's LDE and tree are
  compared in full.

Device results are compared on the device in chunks against the oracle's
arrays, so host memory holds only the oracle's copy.
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


def _wrap(ptr, words):
    import torch

    class _A:
        __cuda_array_interface__ = {"shape": (words,), "typestr": "<i8", "data": (ptr, False), "version": 3}

    return torch.as_tensor(_A(), device="cuda")


def device_equal(ptr: int, want: np.ndarray, chunk_words: int = 1 << 25) -> bool:
    """Device words at ``ptr`` equal the host array ``want`` (flattened)."""
    import torch

    flat = np.ascontiguousarray(want, dtype=np.uint64).reshape(-1)
    dev = _wrap(ptr, flat.size)
    for lo in range(0, flat.size, chunk_words):
        part = torch.from_numpy(flat[lo: lo + chunk_words].view(np.int64)).to("cuda")
        if not torch.equal(dev[lo: lo + chunk_words], part):
            return False
    return True


def first_mismatch(ptr: int, want: np.ndarray) -> int:
    import torch

    flat = np.ascontiguousarray(want, dtype=np.uint64).reshape(-1)
    got = _wrap(ptr, flat.size).cpu().numpy().view(np.uint64)
    bad = np.nonzero(got != flat)[0]
    return int(bad[0]) if bad.size else -1


def check_full(ctx, cid, x, r, h):
    """The resident object's LDE, tree and cap equal the oracle's commit."""
    import torch

    torch.cuda.synchronize()
    lde, tree, cap = oracle.commit(x, r, h)
    b = ctx.buffers(cid)
    assert b["ld"] == lde.shape[1] and b["log_rows"] == x.shape[1].bit_length() - 1 + r
    for key, want in (("lde", lde), ("tree", tree), ("cap", cap)):
        if want.size == 0:
            continue
        ok = device_equal(b[key], want)
        assert ok, f"{key} differs from the oracle at word {first_mismatch(b[key], want)}"
    return cap


def test_large_commit_135x2_20_full(v3c):
    """The benchmark's default workload, compared word for word."""
    import torch

    s = synth.LARGE_135x2_20
    x = s.inputs()
    with v3c.Context(0, flags=v3c.FLAG_TIMING) as ctx:        # the benchmark's context flags
        d = v3c.to_device_u64(x)
        warm = ctx.commit([(d, s.rate_bits, s.cap_height)], stream=torch.cuda.current_stream())[0]
        ctx.release(warm)
        cid = ctx.commit([(d, s.rate_bits, s.cap_height)], stream=torch.cuda.current_stream())[0]
        cap = check_full(ctx, cid, x, s.rate_bits, s.cap_height)
        assert np.array_equal(ctx.cap(cid), cap)
        ctx.release(cid)


def test_uneven_64_batches_seed3_one_batched_commit(v3c):
    """C4: all 64 batches in one v3c_commit (one persistent launch per stage),
    the second call replayed from the captured graph with autotuned tiles."""
    import torch

    shapes = synth.uneven_batches(3)
    assert len(shapes) == 64
    xs = [s.inputs() for s in shapes]
    with v3c.Context(0, hbm_budget_bytes=64 << 30, autotune=True) as ctx:
        ds = [v3c.to_device_u64(x) for x in xs]
        items = [(d, s.rate_bits, s.cap_height) for d, s in zip(ds, shapes)]
        stream = torch.cuda.current_stream()
        for cid in ctx.commit(items, stream=stream):       # first sighting: direct launches
            ctx.release(cid)
        replays0 = ctx.graph_replays()
        ids = ctx.commit(items, stream=stream)              # second sighting: captured and replayed
        assert ctx.graph_replays() == replays0 + 1
        for cid, x, s in zip(ids, xs, shapes):
            check_full(ctx, cid, x, s.rate_bits, s.cap_height)
            ctx.release(cid)


def _serve_slice(count: int = 48):
    """The first ``count`` requests of the serving trace (seed 5).  Inputs:
    every 2^14 x 80 request its own; the 2^16 x 135 requests share a pool of
    three inputs and the 2^18 x 135 requests a pool of two, so the oracle runs
    once per distinct input."""
    trace = synth.poisson_trace(rate=200.0, duration=5.0, seed=5)[:count]
    pools = {16: 3, 18: 2}
    reqs = []
    for i, r in enumerate(trace):
        s = r.shape
        batch = s.batch if s.log_n not in pools else 5000 + 10 * s.log_n + i % pools[s.log_n]
        reqs.append(synth.Shape(c=s.c, log_n=s.log_n, rate_bits=3, cap_height=4, batch=batch, seed=5))
    return reqs


def test_serving_slice_matches_oracle_and_alone(v3c):
    import torch

    reqs = _serve_slice()
    kinds = {(s.log_n, s.c) for s in reqs}
    assert kinds == {(14, 80), (16, 135), (18, 135)}       # the slice spans the whole mixture
    inputs = {}
    for s in reqs:
        if s not in inputs:
            inputs[s] = s.inputs()
    want = {}
    big = next(s for s in reqs if s.log_n == 18)
    big_full = None
    for s, x in inputs.items():
        lde, tree, cap = oracle.commit(x, s.rate_bits, s.cap_height)
        want[s] = cap
        if s == big:
            big_full = (lde, tree)
        del lde, tree
    with v3c.Context(0, hbm_budget_bytes=150 << 30) as ctx:
        # warm plans for the three shapes, then serve every request at once
        for s in {(r.log_n, r.c): r for r in reqs}.values():
            ctx.release(ctx.commit([(inputs[s], 3, 4)])[0])
        torch.cuda.synchronize()
        pinned = {s: torch.from_numpy(x.view(np.int64)).pin_memory() for s, x in inputs.items()}
        ctx.serve_start(max_batch=8)
        tickets = [ctx.serve_submit(pinned[s].numpy().view(np.uint64), 3, 4, borrow=True) for s in reqs]
        assert all(t > 0 for t in tickets)
        caps = {}
        overlapped = 0
        times = {}
        import time

        deadline = time.time() + 300
        while len(caps) < len(tickets):
            assert time.time() < deadline, "serving did not finish"
            for tk, s in zip(tickets, reqs):
                if tk in caps:
                    continue
                st, state, cap, t = ctx.serve_poll(tk, cap_height=4)
                if st == v3c.V3C_EAGAIN:
                    continue
                assert st == v3c.V3C_OK, v3c.strerror(st)
                caps[tk] = cap
                times[tk] = t
            time.sleep(0.001)
        # requests ran side by side: some request started before another finished
        spans = sorted((t[2], t[3]) for t in times.values())
        overlapped = sum(1 for a, b in zip(spans, spans[1:]) if b[0] < a[1])
        assert overlapped > 0
        for tk, s in zip(tickets, reqs):
            assert np.array_equal(caps[tk], want[s]), f"served cap of {s} differs from the oracle"
        # one large request in full: its LDE and tree stay resident until release
        tk_big = tickets[reqs.index(big)]
        b = ctx.buffers(tk_big)
        assert device_equal(b["lde"], big_full[0]) and device_equal(b["tree"], big_full[1])
        ctx.serve_stop()
        # the same requests committed alone, one at a time
        for s in inputs:
            cid = ctx.commit([(inputs[s], 3, 4)])[0]
            assert np.array_equal(ctx.cap(cid), want[s])
            ctx.release(cid)
        for tk in tickets:
            ctx.release(tk)
