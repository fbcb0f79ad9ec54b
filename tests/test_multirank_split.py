"""One commit split over ranks by LDE row blocks, on CPU gloo ranks.

Each rank computes the coefficients of its share of the columns, the ranks
all-gather the coefficient table, each rank commits its part (the row block
[q N/G, (q+1) N/G), a whole subtree) and rank 0 gathers the cap slices.  The
orchestration and the partition arithmetic are the library's
(paper_2603_03065_gb300.split); the oracle stands in for the device calls:
coefficients by its inverse NTT, and a part by Horner evaluation of the
part's rows at 7 w_N^bitrev(t) (its own definition of the committed rows),
then its sponge and Merkle tree over the block.  The gathered cap must equal
the single-process oracle commit's cap bit for bit, and each part's rows the
matching block of the single-process LDE.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SHAPE = dict(c=11, log_n=6, rate_bits=3, cap_height=3, seed=17)


def _worker(rank, world, port, out_path):
    import json

    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import synth
    from paper_2603_03065_gb300 import split

    s = synth.Shape(**SHAPE)
    x = s.inputs()
    c0, c1 = split.column_shard(s.c, world, rank)
    shard = torch.from_numpy(x[c0:c1].view(np.int64).copy())

    def coeffs_of(t):
        a = oracle.coeffs(t.numpy().view(np.uint64), threads=1)
        return torch.from_numpy(a.view(np.int64))

    def new_table(rows, cols):
        return torch.empty((rows, cols), dtype=torch.int64)

    def commit_part(coeffs, log_parts, part):
        a = coeffs.numpy().view(np.uint64)
        r0, r1 = split.part_rows(s.log_N, log_parts, part)
        rows = oracle.lde_rows(a, s.rate_bits, np.arange(r0, r1, dtype=np.uint64), threads=1)
        block = np.zeros((r1 - r0, s.ld), np.uint64)
        block[:, : s.c] = rows
        _, cap = oracle.merkle(block, s.c, s.cap_height - log_parts, threads=1)
        return (r0, block.tolist()), torch.from_numpy(cap.view(np.int64).copy())

    (r0, block), cap = split.commit_split(shard, s.c, s.log_n, s.rate_bits, s.cap_height, coeffs_of=coeffs_of,
                                          commit_part=commit_part, new_table=new_table)
    dist.barrier()
    dist.destroy_process_group()
    with open(f"{out_path}.{rank}", "w") as f:
        json.dump({"rank": rank, "r0": r0, "block": block,
                   "cap": cap.numpy().view(np.uint64).tolist() if cap is not None else None}, f)


@pytest.mark.timeout(300)
@pytest.mark.parametrize("world", [2, 4])
def test_split_commit_over_gloo_ranks_equals_single_process(tmp_path, world):
    import json

    import torch.multiprocessing as mp

    import oracle
    import synth

    oracle.build()
    port = _free_port()
    out = str(tmp_path / "rank")
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    res = [json.load(open(f"{out}.{r}")) for r in range(world)]
    s = synth.Shape(**SHAPE)
    lde, _, cap = oracle.commit(s.inputs(), s.rate_bits, s.cap_height)
    assert res[0]["cap"] is not None
    assert np.array_equal(np.array(res[0]["cap"], np.uint64).reshape(-1, 4), cap)
    size = lde.shape[0] // world
    for q in range(world):
        assert res[q]["r0"] == q * size
        assert np.array_equal(np.array(res[q]["block"], np.uint64), lde[q * size:(q + 1) * size])


def test_partition_arithmetic():
    from paper_2603_03065_gb300 import split

    assert split.log_parts_for(8, 3, 4) == 3
    for bad in (3, 16):
        with pytest.raises(ValueError):
            split.log_parts_for(bad, 3, 4)
    with pytest.raises(ValueError):
        split.log_parts_for(4, 3, 1)            # cap height below log2(parts)
    # parts tile the rows and the cap, in order
    assert [split.part_rows(10, 2, q) for q in range(4)] == [(0, 256), (256, 512), (512, 768), (768, 1024)]
    assert [split.cap_slice(4, 2, q) for q in range(4)] == [(0, 4), (4, 8), (8, 12), (12, 16)]
    assert [split.part_coset(2, q) for q in range(4)] == [0, 2, 1, 3]
    shards = [split.column_shard(135, 8, r) for r in range(8)]
    assert shards[0] == (0, 17) and shards[-1] == (119, 135)
    assert sum(b - a for a, b in shards) == 135
