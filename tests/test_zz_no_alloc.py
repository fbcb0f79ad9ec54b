"""The allocation-free LDE entry point (v3c_lde_noalloc).

Some callers cannot allocate device memory: a process that shares the GPU
with a server whose caching allocator already owns the HBM, or a latency
critical path that must not take the device-wide synchronisation a
cudaMalloc/cudaFree may imply.  v3c_lde_noalloc serves them from a fixed
device array.  This test calls it through the C ABI, twice in a row (the
array keeps the previous call's contents), and checks each result against
the allocating entry point v3c_lde, element for element (field elements:
tolerance zero).  It also checks that a shape larger than the array is
refused.  It lives in a file that pytest collects last.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def v3c():
    from paper_2603_03065_gb300 import build

    build.build()
    import paper_2603_03065_gb300 as m

    return m


def test_noalloc_lde_matches_v3c_lde_on_two_calls(v3c):
    import torch

    torch.cuda.set_device(0)
    with v3c.Context(0) as ctx:
        # Two calls in a row with different shapes, both of which use the
        # scratch (n > 2^(13 - rate_bits)); the second also runs over the
        # leftovers of the first.
        for seed, (c, log_n, r) in enumerate([(13, 12, 3), (7, 14, 2), (13, 12, 3)]):
            x = synth.columns(seed=40 + seed, c=c, log_n=log_n, mix="trace")
            d = v3c.to_device_u64(x)
            want = ctx.lde(d, r)
            out = torch.full_like(want, -1)                 # caller-owned output
            st = v3c.lde_noalloc(d, r, out)
            assert st == v3c.V3C_OK, v3c.strerror(st)
            torch.cuda.synchronize()
            assert torch.equal(out, want)


def test_noalloc_call_allocates_no_device_memory(v3c):
    """The property the entry point exists for: once its array is reserved
    (the first call on the device), a call changes the device's free memory
    by nothing."""
    import torch

    torch.cuda.set_device(0)
    x = synth.columns(seed=47, c=9, log_n=13, mix="trace")
    d = v3c.to_device_u64(x)
    out = torch.empty((1 << 16, 10), dtype=torch.int64, device="cuda")
    assert v3c.lde_noalloc(d, 3, out) == v3c.V3C_OK               # warm: module and array in place
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert v3c.lde_noalloc(d, 3, out) == v3c.V3C_OK
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_binding_checks_the_output_shape(v3c):
    import torch

    torch.cuda.set_device(0)
    d = v3c.to_device_u64(synth.columns(seed=48, c=4, log_n=10, mix="trace"))
    with pytest.raises(ValueError):
        v3c.lde_noalloc(d, 3, torch.empty((1 << 12, 4), dtype=torch.int64, device="cuda"))   # rows for rate 1
    with pytest.raises(ValueError):
        v3c.lde_noalloc(d, 3, torch.empty((1 << 13, 3), dtype=torch.int64, device="cuda"))   # fewer than c columns
    with pytest.raises(ValueError):
        v3c.lde_noalloc(d[:, :1000], 3, torch.empty((8000, 4), dtype=torch.int64, device="cuda"))  # n not 2^k


def test_noalloc_refuses_shapes_over_the_limit(v3c):
    import torch

    torch.cuda.set_device(0)
    d = torch.zeros(16, dtype=torch.int64, device="cuda")
    # 135 x 2^14 rows at rate 3 needs ~160 MB of work space: refused before
    # anything is enqueued (the pointers are never touched).
    st = v3c.load().v3c_lde_noalloc(d.data_ptr(), 135, 14, 3, d.data_ptr(), 136,
                                   torch.cuda.current_stream().cuda_stream)
    assert st == v3c.V3C_EINVAL
    assert np.isclose(v3c.NOALLOC_SCRATCH_BYTES, 32 << 20)
