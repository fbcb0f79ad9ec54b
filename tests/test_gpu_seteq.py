"""SetEq grand-product columns (Sec. 4.5) on the GPU against the CPU oracle.

Bit-exact over whole columns: single instances whose lengths straddle the
2048-element tiles (1, 7, 2047, 2048, 2049, 6145, 2^16 + 3), tuple widths 1 to
32, a batch of uneven instances in one call, a batch of width-4 instances (the
16-byte pair loads and the three-product compression, across the field) and
one at an 8-byte offset (the one-word loads), the 64 x 2^17 batched workload (two
instances compared in full, every instance closing to 1), unequal multisets,
and the degenerate challenge (alpha equal to a compressed y).
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


def run(v3c, ctx, cases):
    import torch

    inst, host = [], []
    for X, Y, alpha, beta in cases:
        z = torch.empty(X.shape[0] + 1, dtype=torch.int64, device="cuda")
        inst.append((v3c.to_device_u64(X), v3c.to_device_u64(Y), z, alpha, beta))
        host.append((X, Y, alpha, beta))
    st = ctx.seteq(inst)
    torch.cuda.synchronize()
    return st, [v3c.to_host_u64(i[2]) for i in inst]


@pytest.mark.parametrize("L,T", [(1, 1), (7, 3), (2047, 4), (2048, 1), (2049, 2), (5000, 32), ((1 << 16) + 3, 4),
                                 (1, 4), (1024, 4), (1025, 4), (2048, 4), (2049, 4), (3073, 4), (6145, 4)])
def test_seteq_matches_oracle(v3c, ctx, L, T):
    X, Y = synth.seteq_instance(L + T, L, T, equal=(L % 2 == 1))
    ch = synth.challenges(L, 2)
    st, (z,) = run(v3c, ctx, [(X, Y, ch[0], ch[1])])
    want = oracle.seteq_partial_products(X, Y, ch[0], ch[1])
    assert st == [0]
    assert np.array_equal(z, want)
    if L % 2 == 1:
        assert int(z[-1]) == 1


def test_seteq_batch_of_uneven_instances(v3c, ctx):
    cases = []
    for b, (L, T) in enumerate([(3, 1), (4096, 4), (10000, 2), (1, 5), (2500, 4), (65, 7)]):
        X, Y = synth.seteq_instance(90, L, T, equal=b % 2 == 0, batch=b)
        ch = synth.challenges(90 + b, 2)
        cases.append((X, Y, ch[0], ch[1]))
    st, zs = run(v3c, ctx, cases)
    assert st == [0] * len(cases)
    for (X, Y, a, bta), z in zip(cases, zs):
        assert np.array_equal(z, oracle.seteq_partial_products(X, Y, a, bta))


def test_seteq_batch_of_width4_instances(v3c, ctx):
    # Every instance of width 4 and 16-byte aligned (16-byte pair loads and the
    # three-product compression), with ragged last tiles and a one-element tile.
    cases = []
    for b, L in enumerate([5000, 1, 2048, 77, 12289, 4095]):
        X, Y = synth.seteq_instance(300, L, 4, equal=b % 2 == 1, batch=b)
        ch = synth.challenges(300 + b, 2)
        cases.append((X, Y, ch[0], ch[1]))
    st, zs = run(v3c, ctx, cases)
    assert st == [0] * len(cases)
    for (X, Y, a, bta), z in zip(cases, zs):
        assert np.array_equal(z, oracle.seteq_partial_products(X, Y, a, bta))


def test_seteq_width4_full_range_words(v3c, ctx):
    # Words and challenges across the whole field (p - 1 included), so the
    # 192-bit sums of the width-4 compression carry into their top word.
    rng = np.random.default_rng(4242)
    L = 4099
    X = rng.integers(0, P, size=(L, 4), dtype=np.uint64)
    X[: L // 3] = np.uint64(P - 1) - X[: L // 3] % np.uint64(1 << 20)
    X[7] = np.uint64(P - 1)
    X[8] = 0
    Y = X[rng.permutation(L)].copy()
    alpha, beta = P - 3, P - 2
    st, (z,) = run(v3c, ctx, [(X, Y, alpha, beta)])
    assert st == [0]
    want = oracle.seteq_partial_products(X, Y, alpha, beta)
    assert np.array_equal(z, want)
    assert int(z[-1]) == 1


def test_seteq_width4_at_an_8_byte_offset(v3c, ctx):
    # Tuples that start 8 bytes past a 16-byte boundary take the one-word loads
    # and Horner's rule; the result is the same.
    import torch

    L = 3001
    X, Y = synth.seteq_instance(301, L, 4, equal=True)
    ch = synth.challenges(301, 2)
    fx = v3c.to_device_u64(np.concatenate([np.zeros(1, np.uint64), X.reshape(-1)]))
    fy = v3c.to_device_u64(np.concatenate([np.zeros(1, np.uint64), Y.reshape(-1)]))
    x, y = fx[1:].view(L, 4), fy[1:].view(L, 4)
    assert x.data_ptr() % 16 == 8
    z = torch.empty(L + 1, dtype=torch.int64, device="cuda")
    st = ctx.seteq([(x, y, z, ch[0], ch[1])])
    torch.cuda.synchronize()
    assert st == [0]
    assert np.array_equal(v3c.to_host_u64(z), oracle.seteq_partial_products(X, Y, ch[0], ch[1]))


def test_seteq_64_queries_x_2_17(v3c, ctx):
    p = synth.SETEQ_MSMARCO
    L = 1 << p["log_L"]
    cases = []
    for q in range(p["instances"]):
        X, Y = synth.seteq_instance(7, L, p["T"], batch=q)
        ch = synth.challenges(1000 + q, 2)
        cases.append((X, Y, ch[0], ch[1]))
    st, zs = run(v3c, ctx, cases)
    assert st == [0] * len(cases)
    assert all(int(z[-1]) == 1 and int(z[0]) == 1 for z in zs)
    for q in (0, len(cases) - 1):
        X, Y, a, b = cases[q]
        assert np.array_equal(zs[q], oracle.seteq_partial_products(X, Y, a, b))


def test_seteq_degenerate_alpha(v3c, ctx):
    X, Y = synth.seteq_instance(5, 3000, 2)
    beta = 12345
    alpha = oracle.compress_tuple(Y[1234], beta)  # alpha - y_1234 = 0
    ok_X, ok_Y = synth.seteq_instance(6, 100, 2)
    st, zs = run(v3c, ctx, [(X, Y, alpha, beta), (ok_X, ok_Y, 99, beta)])
    assert st == [1, 0]
    assert not zs[0].any()
    assert oracle.seteq_partial_products(X, Y, alpha, beta) is None
    assert np.array_equal(zs[1], oracle.seteq_partial_products(ok_X, ok_Y, 99, beta))


def test_seteq_degenerate_alpha_width4(v3c, ctx):
    X, Y = synth.seteq_instance(8, 5000, 4)
    beta = 777
    alpha = oracle.compress_tuple(Y[4321], beta)
    ok_X, ok_Y = synth.seteq_instance(9, 2500, 4)
    st, zs = run(v3c, ctx, [(X, Y, alpha, beta), (ok_X, ok_Y, 99, beta)])
    assert st == [1, 0]
    assert not zs[0].any()
    assert np.array_equal(zs[1], oracle.seteq_partial_products(ok_X, ok_Y, 99, beta))


def test_seteq_rejects_bad_arguments(v3c, ctx):
    import torch

    x = torch.zeros((4, 33), dtype=torch.int64, device="cuda")
    z = torch.zeros(5, dtype=torch.int64, device="cuda")
    with pytest.raises(v3c.V3CError):
        ctx.seteq([(x, x, z, 1, 1)])  # T = 33
    x = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(v3c.V3CError):
        ctx.seteq([(x, x, z, P, 1)])  # alpha not canonical
