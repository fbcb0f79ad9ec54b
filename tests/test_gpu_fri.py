"""FRI commit phase and batched openings on the GPU against the CPU oracle.

Bit-exact (tolerance zero): every layer cap, the final polynomial and every
query record are compared with the oracle on the same seeded inputs and
challenges.  Shapes cover arities 2..16, a ragged last round, one and two
combined commitments, cap heights clamped by small layers, and the
135 x 2^16 trace workload in full.  At 135 x 2^20 the check is by
properties that hold at any size: the final polynomial has the degree FRI
completeness demands, and the oracle's verifier accepts sampled queries
whose initial rows match the oracle's Horner evaluation.
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


def oracle_records(st, idx):
    out = []
    for t0 in idx:
        rec = []
        for vals, path in oracle.fri_query(st, int(t0)):
            rec.append(np.asarray(vals, np.uint64).reshape(-1))
            rec.append(np.asarray(path, np.uint64).reshape(-1))
        out.append(np.concatenate(rec))
    return np.stack(out)


def run_case(v3c, ctx, shapes, r, h_lde, arity_bits, final_log, cap_height, seed, stepwise=False, ext=1):
    xs = [synth.columns(seed=seed + i, c=c, log_n=log_n, mix="trace" if c >= 4 else "uniform")
          for i, (c, log_n) in enumerate(shapes)]
    ids = ctx.commit([(v3c.to_device_u64(x), r, h_lde) for x in xs])
    ch = synth.challenges(seed, 80)
    if ext == 1:
        alpha, betas = ch[0], ch[1:30]
    else:
        alpha, betas = (ch[0], ch[1]), [(ch[2 + 2 * k], ch[3 + 2 * k]) for k in range(30)]
    log_N = shapes[0][1] + r
    R = len(oracle.fri_arities(log_N, arity_bits, final_log))
    if stepwise:
        fid = ctx.fri_begin(ids, alpha, arity_bits, final_log, cap_height, ext=ext)
        caps_early = [ctx.fri_cap(fid, 0)]
        for k in range(R):
            ctx.fri_fold(fid, [betas[k]])
            if k + 1 < R:
                caps_early.append(ctx.fri_cap(fid, k + 1))
    else:
        fid = ctx.fri_begin(ids, alpha, arity_bits, final_log, cap_height, betas=betas[:R], ext=ext)
    info = ctx.fri_info(fid)
    assert info["ext"] == ext
    ldes = [oracle.lde(x, r) for x in xs]
    st = oracle.fri_commit(ldes, [x.shape[0] for x in xs], alpha, betas, arity_bits, final_log, cap_height, ext=ext)
    assert info["rounds"] == R == len(st["arities"])
    assert info["arities"] == st["arities"]
    assert info["heights"] == st["heights"]
    for k in range(R):
        assert np.array_equal(ctx.fri_cap(fid, k), st["caps"][k]), f"layer {k} cap"
        if stepwise:
            assert np.array_equal(caps_early[k], st["caps"][k])
    assert np.array_equal(ctx.fri_final(fid), st["final"])
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, 1 << log_N, size=23, dtype=np.uint64)
    idx[:3] = [0, (1 << log_N) - 1, 1]
    if R:
        got = ctx.fri_query(fid, idx)
        assert got.shape == (idx.size, info["query_words"])
        assert np.array_equal(got, oracle_records(st, idx))
    ctx.fri_release(fid)
    for i in ids:
        ctx.release(i)
    return st


FRI_CASES = [
    # shapes [(c, log_n)], r, h_lde, arity_bits, final_log, cap_height
    ([(8, 10)], 3, 0, 4, 5, 4),
    ([(8, 10)], 3, 0, 3, 5, 2),     # rounds 3, 3, 2: ragged last round
    ([(5, 9)], 2, 1, 1, 3, 3),      # arity 2, leaves hashed as zero-padded pairs
    ([(3, 8)], 1, 0, 2, 0, 6),      # down to one value; caps clamped by small layers
    ([(135, 10)], 3, 4, 4, 5, 4),   # wide rows, several 64-column passes per warp
    ([(13, 11), (6, 11)], 3, 2, 4, 4, 3),  # two commitments combined
    ([(1, 4)], 1, 0, 4, 5, 0),      # no fold at all: log N = 5 = final_log
    # Copy-engine (tiled) combination: at least 16 columns and 256 rows.
    ([(17, 9), (33, 9)], 2, 1, 3, 4, 3),   # two tiled objects, the second at an odd power offset
    ([(21, 10), (5, 10)], 3, 2, 4, 5, 4),  # one tiled, one register-load, summed
    ([(16, 8)], 1, 0, 2, 3, 2),            # whole tiles only (no partial column chunk)
    ([(20, 7)], 1, 0, 4, 5, 4),            # exactly one tile of 256 rows
    ([(16, 15)], 2, 0, 4, 5, 4),           # 512 tiles: several tiles per CTA, one chunk each
]


@pytest.mark.parametrize("shapes,r,h_lde,a,final_log,h", FRI_CASES)
def test_fri_matches_oracle(v3c, ctx, shapes, r, h_lde, a, final_log, h):
    run_case(v3c, ctx, shapes, r, h_lde, a, final_log, h, seed=sum(c for c, _ in shapes) + a)


EXT_CASES = [
    ([(8, 10)], 3, 0, 4, 5, 4),
    ([(8, 10)], 3, 0, 3, 5, 2),     # ragged last round
    ([(5, 9)], 2, 1, 1, 3, 3),      # arity 2: leaves of 4 words, zero-padded, not hashed
    ([(13, 11), (6, 11)], 3, 2, 4, 4, 3),
    ([(1, 4)], 1, 0, 4, 5, 0),      # no fold
    ([(17, 9), (33, 9)], 2, 1, 3, 4, 3),   # tiled combination, two objects
    ([(21, 10), (5, 10)], 3, 2, 4, 5, 4),  # tiled + register-load
    ([(20, 7)], 1, 0, 4, 5, 4),            # one tile
    ([(40, 14)], 3, 2, 4, 5, 4),           # 512 tiles, three chunks per tile
]


@pytest.mark.parametrize("shapes,r,h_lde,a,final_log,h", EXT_CASES)
def test_fri_extension_matches_oracle(v3c, ctx, shapes, r, h_lde, a, final_log, h):
    run_case(v3c, ctx, shapes, r, h_lde, a, final_log, h, seed=100 + sum(c for c, _ in shapes) + a, ext=2)


def test_fri_extension_stepwise_and_trace_135x2_16(v3c, ctx):
    run_case(v3c, ctx, [(9, 10)], 3, 0, 2, 3, 4, seed=191, stepwise=True, ext=2)
    run_case(v3c, ctx, [(135, 16)], 3, 4, 4, 5, 4, seed=235, ext=2)


def test_fri_stepwise_equals_oracle(v3c, ctx):
    run_case(v3c, ctx, [(9, 10)], 3, 0, 2, 3, 4, seed=91, stepwise=True)


def test_fri_trace_135x2_16_full(v3c, ctx):
    run_case(v3c, ctx, [(135, 16)], 3, 4, 4, 5, 4, seed=135)


def test_open_batch_matches_oracle_and_single_open(v3c, ctx):
    x = synth.columns(4, 11, 9)
    cid = ctx.commit([(v3c.to_device_u64(x), 2, 3)])[0]
    e = oracle.lde(x, 2)
    tree, cap = oracle.merkle(e, 11, 3)
    idx = np.array([0, 5, 2047, 1024, 5, 77], np.uint64)
    rows, paths = ctx.open_batch(cid, idx, 11)
    for q, t in enumerate(idx):
        assert np.array_equal(rows[q], e[int(t), :11])
        assert np.array_equal(paths[q], oracle.merkle_path(tree, 11, 3, int(t)))
        one = ctx.open(cid, int(t), 11)
        assert np.array_equal(one.row, rows[q]) and np.array_equal(one.path, paths[q])
    r_only, none = ctx.open_batch(cid, idx, 11, paths=False)
    assert none is None and np.array_equal(r_only, rows)
    ctx.release(cid)


def test_fri_errors(v3c, ctx):
    x = synth.columns(5, 4, 8)
    y = synth.columns(6, 4, 9)
    a, b = ctx.commit([(v3c.to_device_u64(x), 1, 0), (v3c.to_device_u64(y), 1, 0)])
    with pytest.raises(v3c.V3CError):
        ctx.fri_begin([a, b], 3)  # different row counts
    with pytest.raises(v3c.V3CError):
        ctx.fri_begin([a], 3, arity_bits=5)
    with pytest.raises(v3c.V3CError):
        ctx.fri_begin([a], P)  # alpha not canonical
    with pytest.raises(v3c.V3CError):
        ctx.fri_begin([12345678], 3)  # unknown commitment
    fid = ctx.fri_begin([a], 3, arity_bits=2, final_log=3)
    R = ctx.fri_info(fid)["rounds"]
    with pytest.raises(v3c.V3CError):
        ctx.fri_query(fid, [0])  # rounds not done
    with pytest.raises(v3c.V3CError):
        ctx.fri_final(fid)
    with pytest.raises(v3c.V3CError):
        ctx.fri_cap(fid, 1)  # layer 1 not committed yet
    with pytest.raises(v3c.V3CError):
        ctx.fri_fold(fid, [1] * (R + 1))
    ctx.fri_fold(fid, [1] * R)
    with pytest.raises(v3c.V3CError):
        ctx.fri_query(fid, [1 << 9])  # out of range
    with pytest.raises(v3c.V3CError):
        ctx.fri_fold(fid, [1])
    ctx.fri_release(fid)
    with pytest.raises(v3c.V3CError):
        ctx.fri_release(fid)
    ctx.release(a)
    ctx.release(b)


def test_fri_respects_the_hbm_budget(v3c):
    # Room for the commitment and 100 KB more; the FRI state of arity 2 down
    # to one value needs f_0 (64 KB) plus layer 0's tree (260 KB) and more.
    with v3c.Context(0, hbm_budget_bytes=v3c.footprint(8, 10, 3, 4) + 100_000) as small:
        x = synth.columns(8, 8, 10)
        cid = small.commit([(v3c.to_device_u64(x), 3, 4)])[0]
        with pytest.raises(v3c.V3CError) as e:
            small.fri_begin([cid], 3, arity_bits=1, final_log=0)
        assert e.value.status == 2
        small.release(cid)


def test_fri_large_135x2_20_properties(v3c, ctx):
    # The benchmark's launch configuration: one commitment of the 135 x 2^20
    # trace workload, arity 16 down to 2^5 values, cap height 4.
    s = synth.LARGE_135x2_20
    x = s.inputs()
    cid = ctx.commit([(v3c.to_device_u64(x), s.rate_bits, s.cap_height)])[0]
    ch = synth.challenges(2020, 8)
    fid = ctx.fri_begin([cid], ch[0], 4, 5, 4, betas=ch[1:6])
    info = ctx.fri_info(fid)
    assert info["arities"] == [4, 4, 4, 4, 2] and info["log_sizes"] == [23, 19, 15, 11, 7, 5]
    # The committed columns have degree < 2^20; folded by 2^18 in total, the
    # final polynomial has degree < 4 of its 32 coefficients.
    fin = ctx.fri_final(fid)
    assert not fin[4:].any() and fin[:4].any()
    # Sampled queries: rows from the batched opening equal the oracle's
    # Horner evaluation and authenticate against the commitment cap; the
    # oracle's verifier accepts the FRI openings built on them.
    coef = oracle.coeffs(x)
    rng = np.random.default_rng(20)
    idx = rng.integers(0, 1 << 23, size=3, dtype=np.uint64)
    rows, paths = ctx.open_batch(cid, idx, s.c)
    want_rows = oracle.lde_rows(coef, s.rate_bits, idx)
    assert np.array_equal(rows, want_rows)
    cap = ctx.cap(cid)
    recs = ctx.fri_query(fid, idx)
    caps = [ctx.fri_cap(fid, k) for k in range(info["rounds"])]
    for q, t0 in enumerate(idx):
        assert oracle.merkle_verify(rows[q], s.c, 23, s.cap_height, int(t0), paths[q], cap)
        f0 = int(oracle.fri_combine([rows[q:q + 1]], [s.c], ch[0])[0])
        ops, off = [], 0
        for k, a in enumerate(info["arities"]):
            depth = info["log_sizes"][k] - a - info["heights"][k]
            vals = recs[q, off:off + (1 << a)]
            path = recs[q, off + (1 << a): off + (1 << a) + 4 * depth].reshape(-1, 4)
            ops.append((vals, path))
            off += (1 << a) + 4 * depth
        assert oracle.fri_verify_query(caps, info["heights"], info["arities"], ch[1:6], fin, 23, int(t0), f0, ops)
    ctx.fri_release(fid)
    ctx.release(cid)
