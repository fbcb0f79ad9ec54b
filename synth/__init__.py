"""Seeded synthetic inputs for the commitment workloads.

This module is the one piece shared by the oracle-side tests and the CUDA
path's tests and benchmark.  It only draws input data; it contains none of
the commitment's arithmetic (no NTT, hash or tree).  The running-product
column kind is part of the input recipe itself and uses plain Python
integers.

Recipe (stand-in for the paper's Plonky2 trace columns, whose witnesses and
datasets are not available; trace heights are powers of two as in the
padded domain G_B = 2^ceil(log2 G) of Sec. 2.1 and Table zkivfpq-bench):

* Every (seed, batch, column) owns one SplitMix64 stream (Steele, Lea and
  Flood, OOPSLA 2014).  Its starting state is ``seed XOR k`` where ``k`` is
  the first SplitMix64 output from state ``(batch << 32) | column``.  Values
  are drawn in row order.
* Column kinds, in contiguous blocks in this order: floor(0.4c) uniform
  field elements (draws kept iff < p), floor(0.3c) small integers
  (draw & 0xFFFF), floor(0.2c) selectors (draw & 1), and the rest running
  products r_0 = u_0, r_i = r_{i-1} * u_i mod p of uniform nonzero u.
* ``mix="uniform"`` makes every column uniform (the 8 x 2^10 workload).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

P = 0xFFFFFFFF00000001
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1

UNIFORM, SMALL, SELECTOR, RUNNING_PRODUCT = 0, 1, 2, 3


def splitmix64(state: int) -> tuple[int, int]:
    """One SplitMix64 step: returns (new_state, output)."""
    state = (state + GAMMA) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def _mix_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def draws(state: int, start: int, count: int) -> np.ndarray:
    """Outputs number start .. start+count-1 (0-based) of the stream that
    begins at ``state``.  SplitMix64 is counter based: output i is the mix
    of state + (i + 1) * gamma."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(state) + idx * np.uint64(GAMMA)
        return _mix_np(z)


def stream_state(seed: int, batch: int, column: int) -> int:
    _, k = splitmix64(((batch & 0xFFFFFFFF) << 32) | (column & 0xFFFFFFFF))
    return (seed ^ k) & M64


def _filtered(state: int, n: int, keep) -> np.ndarray:
    """First n draws of the stream that satisfy ``keep`` (rejection)."""
    out = np.empty(0, dtype=np.uint64)
    start = 0
    want = n
    while out.size < n:
        chunk = want + 64
        d = draws(state, start, chunk)
        start += chunk
        out = np.concatenate([out, d[keep(d)]])
        want = n - out.size
    return out[:n]


def column_kinds(c: int, mix: str = "trace") -> list[int]:
    if mix == "uniform":
        return [UNIFORM] * c
    nu, ns, nsel = (4 * c) // 10, (3 * c) // 10, (2 * c) // 10
    return [UNIFORM] * nu + [SMALL] * ns + [SELECTOR] * nsel + [RUNNING_PRODUCT] * (c - nu - ns - nsel)


def column(seed: int, batch: int, col: int, n: int, kind: int) -> np.ndarray:
    st = stream_state(seed, batch, col)
    if kind == UNIFORM:
        return _filtered(st, n, lambda d: d < np.uint64(P))
    if kind == SMALL:
        return draws(st, 0, n) & np.uint64(0xFFFF)
    if kind == SELECTOR:
        return draws(st, 0, n) & np.uint64(1)
    if kind == RUNNING_PRODUCT:
        u = _filtered(st, n, lambda d: (d < np.uint64(P)) & (d != np.uint64(0))).tolist()
        return np.array(list(itertools.accumulate(u, lambda r, ui: (r * ui) % P)), dtype=np.uint64)
    raise ValueError(f"unknown column kind {kind}")


def columns(seed: int, c: int, log_n: int, batch: int = 0, mix: str = "trace") -> np.ndarray:
    """Column-major [c][n] uint64 array of canonical field elements."""
    n = 1 << log_n
    kinds = column_kinds(c, mix)
    out = np.empty((c, n), dtype=np.uint64)
    for j, k in enumerate(kinds):
        out[j] = column(seed, batch, j, n, k)
    return out


def challenges(seed: int, count: int) -> list[int]:
    """Verifier challenges (FRI alpha, betas, query positions are drawn by the
    caller from these): the first ``count`` canonical nonzero draws of the
    stream of (seed, batch 0xFFFFFFFF, column 0)."""
    st = stream_state(seed, 0xFFFFFFFF, 0)
    return [int(v) for v in _filtered(st, count, lambda d: (d < np.uint64(P)) & (d != np.uint64(0)))]


def uniform_int(state: int, k: int) -> tuple[int, int]:
    """Unbiased integer in [0, k) by rejection from a SplitMix64 stream."""
    limit = ((1 << 64) // k) * k
    while True:
        state, d = splitmix64(state)
        if d < limit:
            return state, d % k


@dataclass(frozen=True)
class Shape:
    c: int
    log_n: int
    rate_bits: int
    cap_height: int
    batch: int = 0
    seed: int = 0
    mix: str = "trace"

    @property
    def ld(self) -> int:
        return self.c + (self.c & 1)

    @property
    def log_N(self) -> int:
        return self.log_n + self.rate_bits

    def lde_elems(self) -> int:
        return self.c << self.log_N

    def perms(self) -> int:
        """Poseidon permutations of the commit: leaves then tree nodes."""
        N = 1 << self.log_N
        leaf = 0 if self.c <= 4 else -(-self.c // 8)
        return N * leaf + (N - (1 << self.cap_height))

    def inputs(self) -> np.ndarray:
        return columns(self.seed, self.c, self.log_n, self.batch, self.mix)


# The five workloads: sizes, mixes and seeds.
PLAIN_8x2_10 = Shape(c=8, log_n=10, rate_bits=3, cap_height=0, seed=0, mix="uniform")
TRACE_135x2_16 = Shape(c=135, log_n=16, rate_bits=3, cap_height=4, seed=0)
LARGE_135x2_20 = Shape(c=135, log_n=20, rate_bits=3, cap_height=4, seed=0)
# Profiling case: the per-CTA shapes of the 135 x 2^20 commit (n1 = n2 = 2^10) on 8 columns.
PROFILE_8x2_20 = Shape(c=8, log_n=20, rate_bits=3, cap_height=4, seed=0)


def uneven_batches(seed: int = 3, count: int = 64) -> list[Shape]:
    """64 column-batches: log2 rows uniform in {12..18}, columns in {20..135},
    rate_bits in {1,2,3}, cap height 4.  Shapes come from the SplitMix64
    stream that starts at the seed itself; each batch's data from its own
    (seed, batch, column) streams."""
    st = seed & M64
    out = []
    for b in range(count):
        st, dn = uniform_int(st, 7)
        st, dc = uniform_int(st, 116)
        st, dr = uniform_int(st, 3)
        out.append(Shape(c=20 + dc, log_n=12 + dn, rate_bits=1 + dr, cap_height=4, batch=b, seed=seed))
    return out


SERVE_MIX = ((0.50, 14, 80), (0.35, 16, 135), (0.15, 18, 135))


@dataclass(frozen=True)
class Request:
    t_arrive: float
    shape: Shape


def poisson_trace(rate: float = 200.0, duration: float = 60.0, seed: int = 5) -> list[Request]:
    """Arrivals with Exp(rate) gaps over ``duration`` seconds; each request's
    shape from the mixture (rate_bits 3, cap height 4); request i's data uses
    batch index i of the same seed."""
    st = seed & M64
    t = 0.0
    out: list[Request] = []
    i = 0
    while True:
        st, d = splitmix64(st)
        u = (d >> 11) * (1.0 / (1 << 53))
        t += -math.log1p(-u) / rate
        if t >= duration:
            break
        st, d = splitmix64(st)
        v = (d >> 11) * (1.0 / (1 << 53))
        acc = 0.0
        for prob, log_n, c in SERVE_MIX:
            acc += prob
            if v < acc:
                break
        out.append(Request(t, Shape(c=c, log_n=log_n, rate_bits=3, cap_height=4, batch=i, seed=seed)))
        i += 1
    return out


# --- IVF-PQ snapshots --------------------------------------------------------
# A fixed-shape IVF-PQ snapshot: nlist lists of n slots, each slot a record
# [f, item, v^(0), ..., v^(M-1)]; centroids mu [nlist][D]; PQ codebooks
# [M][K][d], d = D / M.  Coordinates are 16-bit fixed point, the encoding
# round((2^16 - 1) v / v_max) of real coordinates in [-v_max, v_max],
# embedded in F_p (a negative x as p + x).  Padding slots (f = 0) hold zeros.
SNAP_SIFT1M = dict(log_nlist=13, log_n=8, D=128, M=8, K=256, valid=1e6 / (1 << 21))
SNAP_MSMARCO = dict(log_nlist=13, log_n=11, D=384, M=8, K=256, valid=8.8e6 / (1 << 24))


def _fixed_point(state: int, count: int) -> np.ndarray:
    span = np.uint64(2 * 65535 + 1)
    u = draws(state, 0, count) % span           # x + 65535, x in [-65535, 65535]
    neg = u < np.uint64(65535)
    return np.where(neg, np.uint64(P - 65535) + u, u - np.uint64(65535))


def snapshot(seed: int, log_nlist: int, log_n: int, D: int, M: int = 8, K: int = 256, valid: float = 0.5):
    """(records [nlist * n][2 + M], mu [nlist][D], codebooks [M][K][D / M])."""
    N = 1 << (log_nlist + log_n)
    base = 0xFFFF0000
    f = (draws(stream_state(seed, base, 0), 0, N) & np.uint64(0xFFFF)) < np.uint64(int(valid * 65536))
    item = draws(stream_state(seed, base, 1), 0, N) & np.uint64(0xFFFFFFFF)
    codes = (draws(stream_state(seed, base, 2), 0, N * M) & np.uint64(K - 1)).reshape(N, M)
    rec = np.zeros((N, 2 + M), np.uint64)
    rec[:, 0] = f.astype(np.uint64)
    rec[:, 1] = np.where(f, item, 0)
    rec[:, 2:] = np.where(f[:, None], codes, 0)
    mu = _fixed_point(stream_state(seed, base, 3), (1 << log_nlist) * D).reshape(1 << log_nlist, D)
    cb = _fixed_point(stream_state(seed, base, 4), M * K * (D // M)).reshape(M, K, D // M)
    return rec, mu, cb


# --- multiset-equality instances -------------------------------------------
# SetEq over the candidate tuples of the multiset-based query circuit: X holds
# L tuples (list, slot, distance, item) of the scan budget N_sel, Y the same
# tuples in another order (a valid permutation witness), or with one tuple
# altered when equal=False.  Distances are 32-bit fixed point.
SETEQ_MSMARCO = dict(instances=64, log_L=17, T=4)   # N_sel = 2^24 / 128 per query, 64 queries


def seteq_instance(seed: int, L: int, T: int = 4, equal: bool = True, batch: int = 0):
    base = 0xFFFE0000
    cols = []
    for k in range(T):
        d = draws(stream_state(seed, base + batch, k), 0, L)
        cols.append(d & np.uint64(0xFFFFFFFF if k >= 2 else 0x1FFF))
    X = np.stack(cols, axis=1).astype(np.uint64)
    order = np.argsort(draws(stream_state(seed, base + batch, T), 0, L), kind="stable")
    Y = X[order].copy()
    if not equal:
        Y[L // 2, T - 1] ^= np.uint64(1)
    return X, Y
