"""Library log callback and the autotune cache.

The log callback receives failures at level 0 (the same text as
v3c_last_error_detail) and resource messages at level 1, and nothing once
removed.  Autotuned tile choices exported from one context and imported into
another spare the second one the timing runs (far fewer kernel launches) and
give the same, oracle-exact commitment; text for another SM count or with
out-of-range values is refused and changes nothing.
"""
import json

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


def test_log_callback_levels_and_silence(v3c):
    import torch

    got = []
    with v3c.Context(0) as ctx:
        ctx.set_log(lambda level, text: got.append((level, text)), max_level=1)
        x = synth.columns(seed=3, c=4, log_n=9, mix="trace")
        cid = ctx.commit([(x, 2, 1)])[0]  # a new shape: plan tables and arena are built
        ctx.release(cid)
        assert any(level == 1 and "plan tables" in text for level, text in got)
        assert any(level == 1 and "scratch arena" in text for level, text in got)
        assert all(level <= 1 for level, _ in got)
        n = len(got)
        with pytest.raises(v3c.V3CError) as e:
            ctx.commit([(np.zeros((2, 8), np.uint64), 1, 9)])  # cap height above log N
        assert e.value.status == v3c.V3C_EINVAL
        assert [lv for lv, _ in got[n:]] == [0]
        assert got[n][1] == ctx.lib.v3c_last_error_detail(ctx.h).decode()
        ctx.set_log(None)
        n = len(got)
        with pytest.raises(v3c.V3CError):
            ctx.commit([(np.zeros((2, 8), np.uint64), 1, 9)])
        cid = ctx.commit([(synth.columns(seed=4, c=4, log_n=10, mix="trace"), 2, 1)])[0]
        ctx.release(cid)
        assert len(got) == n
    torch.cuda.synchronize()


def test_tune_cache_round_trip(v3c):
    shape = (12, 2)  # log_n, rate_bits
    x = synth.columns(seed=11, c=24, log_n=shape[0], mix="trace")
    _, _, want = oracle.commit(x, shape[1], 3)
    with v3c.Context(0, autotune=True) as a:
        l0 = a.kernel_launches()
        cid = a.commit([(x, shape[1], 3)])[0]
        tuning_launches = a.kernel_launches() - l0
        cap_a = np.asarray(a.cap(cid))
        a.release(cid)
        text = a.tune_export()
    doc = json.loads(text)
    assert doc["sm_count"] > 0
    entries = {(e["log_n"], e["rate_bits"]): e for e in doc["entries"]}
    assert shape in entries
    assert set(entries[shape]) == {"log_n", "rate_bits", "a_cols", "c_q", "c_qc", "kcap", "h_threads"}
    with v3c.Context(0, autotune=True) as b:
        b.tune_import(text)
        assert json.loads(b.tune_export()) == doc
        l0 = b.kernel_launches()
        cid = b.commit([(x, shape[1], 3)])[0]
        plain_launches = b.kernel_launches() - l0
        cap_b = np.asarray(b.cap(cid))
        b.release(cid)
        # refused texts leave the imported choices as they were
        bad = dict(doc, sm_count=doc["sm_count"] + 1)
        with pytest.raises(v3c.V3CError) as e:
            b.tune_import(json.dumps(bad))
        assert e.value.status == v3c.V3C_EINVAL
        worse = json.loads(text)
        worse["entries"][0]["kcap"] = 9
        with pytest.raises(v3c.V3CError) as e:
            b.tune_import(json.dumps(worse))
        assert e.value.status == v3c.V3C_EINVAL
        with pytest.raises(v3c.V3CError) as e:
            b.tune_import('{"sm_count": 1')
        assert e.value.status == v3c.V3C_EINVAL
        assert json.loads(b.tune_export()) == doc
    assert plain_launches * 3 < tuning_launches
    assert np.array_equal(cap_a.reshape(-1), np.asarray(want).reshape(-1))
    assert np.array_equal(cap_b.reshape(-1), np.asarray(want).reshape(-1))
