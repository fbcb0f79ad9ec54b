"""Host logic of the multi-GPU bench path on CPU: two gloo ranks.

Under torchrun each rank commits its own independent batch of the same
shape (no data-path collective), and the reported time is the slowest
rank's.  This runs those two steps (bench.shard_workload and
bench.max_over_ranks) with world_size 2 on the gloo backend.  The oracle
stands in for each rank's GPU commit.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import json
    import time

    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    import synth

    s = bench.shard_workload(synth.Shape(c=9, log_n=6, rate_bits=2, cap_height=1, seed=11), rank)
    x = s.inputs()
    t0 = time.perf_counter()
    _, _, cap = oracle.commit(x, s.rate_bits, s.cap_height, threads=1)
    dt = time.perf_counter() - t0 + 0.05 * rank   # make the ranks' times differ
    slowest = bench.max_over_ranks(dt, device="cpu")
    caps = [None] * world
    dist.all_gather_object(caps, cap.tolist())
    times = [None] * world
    dist.all_gather_object(times, dt)
    dist.barrier()
    dist.destroy_process_group()
    with open(f"{out_path}.{rank}", "w") as f:
        json.dump({"rank": rank, "batch": s.batch, "slowest": slowest, "times": times, "caps": caps}, f)


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_and_take_the_slowest(tmp_path):
    import json

    import torch.multiprocessing as mp

    import oracle
    import synth

    oracle.build()
    port = _free_port()
    out = str(tmp_path / "rank")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    res = [json.load(open(f"{out}.{r}")) for r in range(2)]
    assert [r["batch"] for r in res] == [0, 1]                       # one batch per rank
    for r in res:
        assert r["slowest"] == pytest.approx(max(r["times"]))          # max over ranks
    assert res[0]["caps"][0] != res[0]["caps"][1]                      # independent problems
    for rank in range(2):                                              # each rank's commit is right
        s = synth.Shape(c=9, log_n=6, rate_bits=2, cap_height=1, seed=11, batch=rank)
        _, _, cap = oracle.commit(s.inputs(), s.rate_bits, s.cap_height)
        assert res[0]["caps"][rank] == cap.tolist()
