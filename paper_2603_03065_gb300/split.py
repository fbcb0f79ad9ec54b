"""One commit split over G = 2^k GPUs by LDE row blocks (host-side logic).

In the committed (bit-reversed) row order, the LDE rows [q N/G, (q+1) N/G)
are the evaluations of each column's interpolant on the coset
7 w_N^kappa <w_{N/G}> with kappa = bitrev_k(q), again in bit-reversed order
(v3c_commit_part).  That block is a whole subtree of the Merkle tree, so when
the cap height h is at least k its top level is the slice
[q 2^h / G, (q+1) 2^h / G) of the cap.  The only exchange is the
coefficient table: each rank computes the coefficients of its share of the
columns (v3c_coeffs), all ranks gather the whole [c][n] table, and each rank
commits its own part.  The cap is the parts' cap slices in order of q,
gathered to rank 0 (512 bytes at h = 4).

This module holds the partition arithmetic and the exchange.  The device
work is passed in as two callables, so the same orchestration runs with the
library on GPUs (NCCL) and with the CPU oracle standing in (gloo tests).
No field arithmetic happens here.
"""
from __future__ import annotations

from typing import Callable


def log_parts_for(world: int, rate_bits: int, cap_height: int) -> int:
    """log2 of the number of parts for ``world`` ranks: one part per rank.
    The split needs a power-of-two world of at most 2^min(rate_bits, h)."""
    if world < 1 or world & (world - 1):
        raise ValueError(f"the row split needs a power-of-two number of ranks, got {world}")
    k = world.bit_length() - 1
    if k > rate_bits or k > cap_height:
        raise ValueError(f"{world} parts exceed 2^min(rate_bits={rate_bits}, cap_height={cap_height})")
    return k


def bitrev(x: int, bits: int) -> int:
    out = 0
    for _ in range(bits):
        out = (out << 1) | (x & 1)
        x >>= 1
    return out


def part_rows(log_N: int, log_parts: int, part: int) -> tuple[int, int]:
    """Committed rows [r0, r1) of part ``part``."""
    size = 1 << (log_N - log_parts)
    return part * size, (part + 1) * size


def part_coset(log_parts: int, part: int) -> int:
    """kappa: part q's rows are the evaluations at 7 w_N^(kappa + G j)."""
    return bitrev(part, log_parts)


def cap_slice(cap_height: int, log_parts: int, part: int) -> tuple[int, int]:
    """Cap entries [e0, e1) that part ``part`` produces."""
    size = 1 << (cap_height - log_parts)
    return part * size, (part + 1) * size


def column_shard(c: int, world: int, rank: int) -> tuple[int, int]:
    """Columns [c0, c1) whose coefficients rank ``rank`` computes: contiguous
    blocks of ceil(c / world) columns (the last ones may be short or empty)."""
    per = -(-c // world)
    return min(c, rank * per), min(c, (rank + 1) * per)


def commit_split(x_shard, c: int, log_n: int, rate_bits: int, cap_height: int, *,
                 coeffs_of: Callable, commit_part: Callable, new_table: Callable, group=None):
    """Runs one rank's share of a split commit and returns (part result, cap).

    x_shard     this rank's columns [c1 - c0][n] (column_shard), a tensor on
                the collective's device
    coeffs_of   x_shard -> its coefficients [c1 - c0][n] (same device)
    new_table   (rows, n) -> an empty int64 tensor on the collective's device
    commit_part (coeffs [c][n], log_parts, part) -> (part result, cap slice
                tensor [2^(h - log_parts)][4] on the collective's device)
    Returns this rank's part result and, on rank 0, the whole cap
    [2^h][4] (None elsewhere).  Every rank passes equal shard shapes to the
    all-gather: shards are padded to ceil(c / world) columns."""
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    log_parts = log_parts_for(world, rate_bits, cap_height)
    per = -(-c // world)
    n = 1 << log_n
    c0, c1 = column_shard(c, world, rank)
    mine = new_table(per, n)
    if c1 > c0:
        mine[: c1 - c0] = coeffs_of(x_shard)
    if c1 - c0 < per:
        mine[c1 - c0:] = 0
    table = new_table(per * world, n)
    dist.all_gather_into_tensor(table, mine, group=group)
    coeffs = table[:c] if per * world != c else table
    result, cap_part = commit_part(coeffs.contiguous(), log_parts, rank)
    caps = [new_table(1 << (cap_height - log_parts), 4) for _ in range(world)] if rank == 0 else None
    dist.gather(cap_part, caps, dst=0, group=group)
    cap = None
    if rank == 0:
        import torch

        cap = torch.cat(caps, dim=0)
    return result, cap
