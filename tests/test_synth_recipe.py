"""The seeded input generator follows its stated recipe (no GPU, no oracle):
the counter-based SplitMix64 streams, the column-kind blocks and value ranges,
the running-product recurrence, the uneven-batch ranges and the serving
trace's arrival rate and mixture."""
import numpy as np
import pytest

import synth

P = synth.P


def test_counter_form_equals_the_sequential_stream():
    state = synth.stream_state(7, 3, 11)
    st, seq = state, []
    for _ in range(50):
        st, d = synth.splitmix64(st)
        seq.append(d)
    assert [int(v) for v in synth.draws(state, 0, 50)] == seq
    assert [int(v) for v in synth.draws(state, 17, 10)] == seq[17:27]


def test_stream_keys_separate_seed_batch_and_column():
    keys = {synth.stream_state(s, b, c) for s in (0, 1) for b in (0, 1) for c in (0, 1)}
    assert len(keys) == 8
    _, k = synth.splitmix64((5 << 32) | 9)
    assert synth.stream_state(0, 5, 9) == k and synth.stream_state(123, 5, 9) == 123 ^ k


def test_column_kind_blocks():
    kinds = synth.column_kinds(135)
    counts = [kinds.count(k) for k in (synth.UNIFORM, synth.SMALL, synth.SELECTOR, synth.RUNNING_PRODUCT)]
    assert counts == [54, 40, 27, 14]
    assert kinds == sorted(kinds)  # contiguous blocks in that order
    assert synth.column_kinds(8, "uniform") == [synth.UNIFORM] * 8


def test_column_values_follow_their_kind():
    x = synth.columns(0, 135, 10)
    kinds = synth.column_kinds(135)
    assert x.dtype == np.uint64 and x.shape == (135, 1024)
    assert (x < np.uint64(P)).all()
    for j, k in enumerate(kinds):
        col = [int(v) for v in x[j]]
        if k == synth.SMALL:
            assert max(col) < 1 << 16 and len(set(col)) > 500
        elif k == synth.SELECTOR:
            assert set(col) == {0, 1}
        elif k == synth.RUNNING_PRODUCT:
            # r_0 = u_0 and r_i = r_(i-1) u_i with u the stream's nonzero draws below p
            st = synth.stream_state(0, 0, j)
            u = [int(v) for v in synth.draws(st, 0, 4000) if 0 < int(v) < P][:1024]
            r = u[0]
            assert col[0] == r
            for i in range(1, 1024):
                r = r * u[i] % P
                assert col[i] == r
        else:
            st = synth.stream_state(0, 0, j)
            want = [int(v) for v in synth.draws(st, 0, 2000) if int(v) < P][:1024]
            assert col == want
    # deterministic, and another batch is another stream
    assert np.array_equal(x, synth.columns(0, 135, 10))
    assert not np.array_equal(x, synth.columns(0, 135, 10, batch=1))


def test_uneven_batches_ranges():
    shapes = synth.uneven_batches(3)
    assert len(shapes) == 64
    assert all(12 <= s.log_n <= 18 and 20 <= s.c <= 135 and 1 <= s.rate_bits <= 3 and s.cap_height == 4
               for s in shapes)
    assert [s.batch for s in shapes] == list(range(64))
    assert len({(s.c, s.log_n, s.rate_bits) for s in shapes}) > 50
    assert shapes == synth.uneven_batches(3)


@pytest.mark.parametrize("rate", [60.0, 200.0])
def test_serving_trace_rate_and_mixture(rate):
    tr = synth.poisson_trace(rate=rate, duration=30.0, seed=5)
    n = len(tr)
    assert abs(n - rate * 30) < 5 * (rate * 30) ** 0.5  # Poisson count within 5 sigma
    assert all(a.t_arrive < b.t_arrive for a, b in zip(tr, tr[1:]))
    small = sum(1 for r in tr if r.shape.log_n == 14) / n
    large = sum(1 for r in tr if r.shape.log_n == 18) / n
    assert abs(small - 0.50) < 0.06 and abs(large - 0.15) < 0.05
    assert all(r.shape.rate_bits == 3 and r.shape.cap_height == 4 for r in tr)
