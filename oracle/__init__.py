"""CPU oracle for the coset LDE + Poseidon-w12 Merkle commitment.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library never loads it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, ``unsigned __int128`` and
``%``); this module only builds it with gcc and marshals numpy arrays.
Every function below follows one step of the commitment definition; the
paper passage each follows is cited in ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

P = 0xFFFFFFFF00000001
HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

_lock = threading.Lock()
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc, no CUDA)."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, SRC, "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(LIB)
            u64, u32, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
            sig = {
                "orc_add": (u64, [u64, u64]),
                "orc_sub": (u64, [u64, u64]),
                "orc_mul": (u64, [u64, u64]),
                "orc_pow": (u64, [u64, u64]),
                "orc_inv": (u64, [u64]),
                "orc_root_of_unity": (u64, [u32]),
                "orc_bitrev": (u32, [u64, u32]),
                "orc_ntt": (i32, [_u64p, u32, i32]),
                "orc_lde": (i32, [_u64p, u32, u32, u32, _u64p, u32, i32]),
                "orc_coeffs": (i32, [_u64p, u32, u32, _u64p, i32]),
                "orc_lde_rows": (i32, [_u64p, u32, u32, u32, _u64p, u32, _u64p, i32]),
                "orc_splitmix64_next": (u64, [_u64p]),
                "orc_mds_check": (i32, [_u64p]),
                "orc_poseidon_params": (u32, [_u64p, _u64p]),
                "orc_permute": (None, [_u64p]),
                "orc_hash": (None, [_u64p, u32, _u64p]),
                "orc_compress": (None, [_u64p, _u64p, _u64p]),
                "orc_leaf_hashes": (i32, [_u64p, u32, u32, u64, _u64p, i32]),
                "orc_merkle_level": (i32, [_u64p, u64, _u64p, i32]),
                "orc_merkle": (i32, [_u64p, u32, u32, u32, u32, _u64p, _u64p, i32]),
                "orc_merkle_path": (i32, [_u64p, u32, u32, u64, _u64p]),
                "orc_merkle_verify": (i32, [_u64p, u32, u32, u32, u64, _u64p, _u64p]),
                "orc_commit": (i32, [_u64p, u32, u32, u32, u32, _u64p, u32, _u64p, _u64p, i32]),
                "orc_domain_log2": (u32, [u64]),
                "orc_fri_combine": (i32, [_u64p, u32, u32, u64, u64, u64, i32, _u64p, i32]),
                "orc_fri_fold_coset": (u64, [_u64p, u32, u64, u32, u64, u64]),
                "orc_fri_fold": (i32, [_u64p, u32, u64, u32, u64, _u64p, i32]),
                "orc_fri_interpolate": (i32, [_u64p, u32, u64, _u64p]),
                "orc_ext_mul": (None, [_u64p, _u64p, _u64p]),
                "orc_ext_inv": (None, [_u64p, _u64p]),
                "orc_fri_combine_ext": (i32, [_u64p, u32, u32, u64, _u64p, u64, i32, _u64p, i32]),
                "orc_fri_fold_coset_ext": (None, [_u64p, u32, u64, u32, _u64p, u64, _u64p]),
                "orc_fri_fold_ext": (i32, [_u64p, u32, u64, u32, _u64p, _u64p, i32]),
                "orc_snapshot_slot_leaves": (i32, [_u64p, u32, u32, u32, _u64p, i32]),
                "orc_snapshot_list_root": (i32, [_u64p, u64, u32, u32, _u64p]),
                "orc_compress_tuple": (u64, [_u64p, u32, u64]),
                "orc_seteq_partial_products": (i32, [_u64p, _u64p, u64, u32, u64, u64, _u64p]),
                "orc_snapshot_centroid_digest": (None, [u64, _u64p, u32, _u64p, _u64p]),
                "orc_snapshot_commit": (i32, [_u64p, u32, u32, u32, _u64p, u32, _u64p, u32, u32, _u64p, _u64p,
                                              _u64p, _u64p, i32]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def _p(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags.c_contiguous
    return a.ctypes.data_as(_u64p)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


# --- field ------------------------------------------------------------
def add(a: int, b: int) -> int:
    return lib().orc_add(a, b)


def sub(a: int, b: int) -> int:
    return lib().orc_sub(a, b)


def mul(a: int, b: int) -> int:
    return lib().orc_mul(a, b)


def pow_(a: int, e: int) -> int:
    return lib().orc_pow(a, e)


def inv(a: int) -> int:
    return lib().orc_inv(a)


def root_of_unity(log_m: int) -> int:
    return lib().orc_root_of_unity(log_m)


def bitrev(x: int, bits: int) -> int:
    return lib().orc_bitrev(x, bits)


# --- NTT / LDE ---------------------------------------------------------
def ntt(x, inverse: bool = False) -> np.ndarray:
    a = _u64(x).copy()
    log_m = int(a.size).bit_length() - 1
    assert a.size == 1 << log_m
    assert lib().orc_ntt(_p(a), log_m, 1 if inverse else 0) == 0
    return a


def intt(x) -> np.ndarray:
    return ntt(x, inverse=True)


def ld_for(c: int) -> int:
    return c + (c & 1)


def lde(cols, rate_bits: int, ld: int | None = None, threads: int | None = None) -> np.ndarray:
    """cols [c][n] -> row-major LDE [N][ld] in bit-reversed row order."""
    a = _u64(cols)
    c, n = a.shape
    log_n = n.bit_length() - 1
    ld = ld_for(c) if ld is None else ld
    out = np.empty(((n << rate_bits), ld), dtype=np.uint64)
    rc = lib().orc_lde(_p(a), c, log_n, rate_bits, _p(out), ld, threads or default_threads())
    assert rc == 0
    return out


def coeffs(cols, threads: int | None = None) -> np.ndarray:
    a = _u64(cols)
    c, n = a.shape
    out = np.empty_like(a)
    lib().orc_coeffs(_p(a), c, n.bit_length() - 1, _p(out), threads or default_threads())
    return out


def lde_rows(coef, rate_bits: int, rows, threads: int | None = None) -> np.ndarray:
    """Committed LDE rows ``rows`` (bit-reversed indices) by Horner evaluation
    of the coefficient columns at 7 * w_N^bitrev(t)."""
    a = _u64(coef)
    c, n = a.shape
    r = _u64(rows)
    out = np.empty((r.size, c), dtype=np.uint64)
    lib().orc_lde_rows(_p(a), c, n.bit_length() - 1, rate_bits, _p(r), r.size, _p(out),
                       threads or default_threads())
    return out


# --- Poseidon ------------------------------------------------------------
def poseidon_params() -> tuple[np.ndarray, np.ndarray, int]:
    rc = np.zeros(360, np.uint64)
    mds = np.zeros(144, np.uint64)
    tries = lib().orc_poseidon_params(_p(rc), _p(mds))
    return rc.reshape(30, 12), mds.reshape(12, 12), tries


def mds_check(m) -> int:
    a = _u64(m).reshape(144).copy()
    return lib().orc_mds_check(_p(a))


def permute(state) -> np.ndarray:
    s = _u64(state).copy()
    assert s.size == 12
    lib().orc_permute(_p(s))
    return s


def hash_(x) -> np.ndarray:
    a = _u64(x)
    out = np.zeros(4, np.uint64)
    lib().orc_hash(_p(a) if a.size else None, a.size, _p(out))
    return out


def compress(left, right) -> np.ndarray:
    out = np.zeros(4, np.uint64)
    lib().orc_compress(_p(_u64(left)), _p(_u64(right)), _p(out))
    return out


def leaf_hashes(rows: np.ndarray, width: int, threads: int | None = None) -> np.ndarray:
    a = _u64(rows)
    nrows, ld = a.shape
    out = np.empty((nrows, 4), np.uint64)
    lib().orc_leaf_hashes(_p(a), ld, width, nrows, _p(out), threads or default_threads())
    return out


def merkle_level(below: np.ndarray, threads: int | None = None) -> np.ndarray:
    a = _u64(below).reshape(-1, 4)
    cnt = a.shape[0] // 2
    out = np.empty((cnt, 4), np.uint64)
    lib().orc_merkle_level(_p(a), cnt, _p(out), threads or default_threads())
    return out


def tree_len(log_rows: int, cap_height: int) -> int:
    """u64 words below the cap: levels 0 .. logN-h-1 of N >> k digests."""
    N = 1 << log_rows
    return (2 * N - (2 << cap_height)) * 4


def merkle(rows: np.ndarray, width: int, cap_height: int, threads: int | None = None):
    a = _u64(rows)
    nrows, ld = a.shape
    log_rows = nrows.bit_length() - 1
    tree = np.zeros(tree_len(log_rows, cap_height), np.uint64)
    cap = np.zeros((1 << cap_height) * 4, np.uint64)
    rc = lib().orc_merkle(_p(a), ld, width, log_rows, cap_height, _p(tree) if tree.size else None,
                          _p(cap), threads or default_threads())
    assert rc == 0
    return tree, cap.reshape(-1, 4)


def merkle_path(tree: np.ndarray, log_rows: int, cap_height: int, t: int) -> np.ndarray:
    path = np.zeros(max(1, log_rows - cap_height) * 4, np.uint64)
    assert lib().orc_merkle_path(_p(_u64(tree)) if tree.size else None, log_rows, cap_height, t,
                                 _p(path)) == 0
    return path[: (log_rows - cap_height) * 4].reshape(-1, 4)


def merkle_verify(row, width: int, log_rows: int, cap_height: int, t: int, path, cap) -> bool:
    r = _u64(row)
    pth = _u64(path).reshape(-1)
    if pth.size == 0:
        pth = np.zeros(4, np.uint64)
    return bool(lib().orc_merkle_verify(_p(r), width, log_rows, cap_height, t, _p(pth),
                                        _p(_u64(cap).reshape(-1))))


def commit(cols, rate_bits: int, cap_height: int, threads: int | None = None):
    """Full commitment: returns (lde [N][ld], tree, cap [2^h][4])."""
    a = _u64(cols)
    c, n = a.shape
    e = lde(a, rate_bits, threads=threads)
    tree, cap = merkle(e, c, cap_height, threads=threads)
    return e, tree, cap


def domain_log2(G: int) -> int:
    return lib().orc_domain_log2(G)


# --- FRI commit phase ------------------------------------------------------
# The combine / fold / interpolate arithmetic is in oracle.c; below is only the
# round schedule and the bookkeeping of layers, trees and openings.
GENERATOR = 7


def ext_mul(a, b) -> tuple[int, int]:
    """(a0 + a1 u)(b0 + b1 u) in F_p[u] / (u^2 - 7)."""
    x, y, out = _u64(a), _u64(b), np.zeros(2, np.uint64)
    lib().orc_ext_mul(_p(x), _p(y), _p(out))
    return int(out[0]), int(out[1])


def ext_inv(a) -> tuple[int, int]:
    x, out = _u64(a), np.zeros(2, np.uint64)
    lib().orc_ext_inv(_p(x), _p(out))
    return int(out[0]), int(out[1])


def _ext_pair(v, ext: int):
    return [int(v)] if ext == 1 else [int(v[0]), int(v[1])]


def fri_combine(ldes, widths, alpha, threads: int | None = None, ext: int = 1) -> np.ndarray:
    """f_0[t] = sum over the committed matrices, in order, of alpha^e row_t[i],
    with e running on from one matrix to the next.  ext = 2: alpha = (re, im)
    in F_p[u]/(u^2 - 7) and the result has shape [N][2]."""
    f = None
    e0 = 0
    for m, c in zip(ldes, widths):
        a = _u64(m)
        nrows, ld = a.shape
        if ext == 1:
            if f is None:
                f = np.zeros(nrows, np.uint64)
            assert lib().orc_fri_combine(_p(a), ld, c, nrows, int(alpha), e0, 1, _p(f),
                                         threads or default_threads()) == 0
        else:
            if f is None:
                f = np.zeros((nrows, 2), np.uint64)
            al = _u64(_ext_pair(alpha, 2))
            assert lib().orc_fri_combine_ext(_p(a), ld, c, nrows, _p(al), e0, 1, _p(f),
                                             threads or default_threads()) == 0
        e0 += c
    return f


def fri_fold(f, shift: int, arity_bits: int, beta, threads: int | None = None, ext: int = 1) -> np.ndarray:
    a = _u64(f)
    m = a.shape[0]
    logm = m.bit_length() - 1
    if ext == 1:
        out = np.empty(m >> arity_bits, np.uint64)
        assert lib().orc_fri_fold(_p(a), logm, shift, arity_bits, int(beta), _p(out),
                                  threads or default_threads()) == 0
    else:
        out = np.empty((m >> arity_bits, 2), np.uint64)
        b = _u64(_ext_pair(beta, 2))
        assert lib().orc_fri_fold_ext(_p(a), logm, shift, arity_bits, _p(b), _p(out),
                                      threads or default_threads()) == 0
    return out


def fri_fold_coset(vals, logm: int, shift: int, arity_bits: int, beta, w: int, ext: int = 1):
    if ext == 1:
        return int(lib().orc_fri_fold_coset(_p(_u64(vals)), logm, shift, arity_bits, int(beta), w))
    out = np.zeros(2, np.uint64)
    lib().orc_fri_fold_coset_ext(_p(_u64(vals).reshape(-1)), logm, shift, arity_bits,
                                 _p(_u64(_ext_pair(beta, 2))), w, _p(out))
    return int(out[0]), int(out[1])


def fri_interpolate(f, shift: int) -> np.ndarray:
    """Coefficients of the polynomial with values f on the coset (bit-reversed
    order).  Extension values ([m][2]) interpolate componentwise: the DFT is
    linear over F_p."""
    a = _u64(f)
    if a.ndim == 2:
        return np.stack([fri_interpolate(np.ascontiguousarray(a[:, k]), shift) for k in range(a.shape[1])], axis=1)
    out = np.empty_like(a)
    assert lib().orc_fri_interpolate(_p(a), a.size.bit_length() - 1, shift, _p(out)) == 0
    return out


def fri_arities(log_N: int, arity_bits: int, final_log: int) -> list[int]:
    """Arity exponent of each round: arity_bits while the layer stays at or
    above 2^final_log, then whatever remains."""
    out, m = [], log_N
    while m > final_log:
        a = min(arity_bits, m - final_log)
        out.append(a)
        m -= a
    return out


def fri_commit(ldes, widths, alpha, betas, arity_bits: int, final_log: int, cap_height: int,
               threads: int | None = None, ext: int = 1) -> dict:
    """Commit phase: layer k (k < R) is committed as a Merkle tree whose leaf w
    is the coset [w 2^a_k, (w+1) 2^a_k) of the layer (2^a_k ext-word values,
    flattened); the last layer is sent as polynomial coefficients."""
    f = fri_combine(ldes, widths, alpha, threads, ext)
    log_N = f.shape[0].bit_length() - 1
    ar = fri_arities(log_N, arity_bits, final_log)
    assert len(betas) >= len(ar)
    layers, trees, caps, shifts, heights = [f], [], [], [GENERATOR], []
    for k, a in enumerate(ar):
        cur = layers[-1]
        logL = (cur.shape[0].bit_length() - 1) - a
        h = min(cap_height, logL)
        width = (1 << a) * ext
        tree, cap = merkle(np.ascontiguousarray(cur).reshape(-1, width), width, h, threads)
        trees.append(tree)
        caps.append(cap)
        heights.append(h)
        layers.append(fri_fold(cur, shifts[-1], a, betas[k], threads, ext))
        shifts.append(pow_(shifts[-1], 1 << a))
    final = fri_interpolate(layers[-1], shifts[-1])
    return {"layers": layers, "trees": trees, "caps": caps, "shifts": shifts, "arities": ar, "ext": ext,
            "heights": heights, "final": final, "betas": list(betas[: len(ar)])}


def fri_query(st: dict, t0: int) -> list[tuple[np.ndarray, np.ndarray]]:
    """Openings of query position t0 (in layer 0): per round, the coset values
    holding the query's position (flattened) and their Merkle path."""
    out, t = [], t0
    for k, a in enumerate(st["arities"]):
        cur = st["layers"][k]
        logL = (cur.shape[0].bit_length() - 1) - a
        leaf = t >> a
        vals = np.ascontiguousarray(cur[leaf << a: (leaf + 1) << a]).reshape(-1).copy()
        path = merkle_path(st["trees"][k], logL, st["heights"][k], leaf)
        out.append((vals, path))
        t = leaf
    return out


def fri_verify_query(caps, heights, arities, betas, final, log_N: int, t0: int, f0_value, openings,
                     ext: int = 1) -> bool:
    """Verifier side of one query: the opened cosets authenticate against the
    layer caps, hold the running value at the query position, and fold into
    the next layer's value; the last value equals the final polynomial at the
    query's point.  ext = 2: values are (re, im) pairs."""
    t, shift, logm = t0, GENERATOR, log_N
    value = tuple(int(v) for v in (f0_value if ext == 2 else [f0_value]))
    for k, a in enumerate(arities):
        vals, path = openings[k]
        logL = logm - a
        leaf = t >> a
        pos = (t & ((1 << a) - 1)) * ext
        if tuple(int(v) for v in vals[pos: pos + ext]) != value:
            return False
        if not merkle_verify(vals, (1 << a) * ext, logL, heights[k], leaf, path, caps[k]):
            return False
        got = fri_fold_coset(vals, logm, shift, a, betas[k], leaf, ext)
        value = got if ext == 2 else (got,)
        t, logm, shift = leaf, logL, pow_(shift, 1 << a)
    x = mul(shift, pow_(root_of_unity(logm), bitrev(t, logm)))
    fin = _u64(final).reshape(-1, ext)
    acc = [0] * ext
    for row in reversed(fin):
        acc = [add(mul(acc[k], x), int(row[k])) for k in range(ext)]
    return tuple(acc) == value


# --- snapshot commitment (Sec. 4.3) ----------------------------------------
def snapshot_slot_leaves(records, log_nlist: int, log_n: int, threads: int | None = None) -> np.ndarray:
    r = _u64(records)
    N = 1 << (log_nlist + log_n)
    M = r.shape[1] - 2
    out = np.empty((N, 4), np.uint64)
    assert lib().orc_snapshot_slot_leaves(_p(r), 1 << log_nlist, 1 << log_n, M, _p(out),
                                          threads or default_threads()) == 0
    return out


def snapshot_commit(records, mu, codebooks, log_nlist: int, log_n: int, threads: int | None = None) -> dict:
    """Returns list roots [nlist][4], centroid digests [nlist][4], root_mk, root_cb."""
    r, m, cb = _u64(records), _u64(mu), _u64(codebooks)
    nlist = 1 << log_nlist
    M = r.shape[1] - 2
    D = m.shape[1]
    Mc, K, d = cb.shape
    roots = np.empty((nlist, 4), np.uint64)
    cent = np.empty((nlist, 4), np.uint64)
    mk = np.empty(4, np.uint64)
    cbr = np.empty(4, np.uint64)
    assert lib().orc_snapshot_commit(_p(r), log_nlist, log_n, M, _p(m), D, _p(cb), K, d, _p(roots), _p(cent),
                                     _p(mk), _p(cbr), threads or default_threads()) == 0
    return {"list_roots": roots, "centroid_digests": cent, "root_mk": mk, "root_cb": cbr}


def snapshot_list_root(list_records, i: int, log_n: int) -> np.ndarray:
    """root_i from the n records of list i alone."""
    r = _u64(list_records)
    out = np.empty(4, np.uint64)
    assert lib().orc_snapshot_list_root(_p(r), i, log_n, r.shape[1] - 2, _p(out)) == 0
    return out


def snapshot_centroid_digest(i: int, mu_i, root_i) -> np.ndarray:
    m, rt = _u64(mu_i), _u64(root_i)
    out = np.empty(4, np.uint64)
    lib().orc_snapshot_centroid_digest(i, _p(m), m.size, _p(rt), _p(out))
    return out


# --- multiset equality (Sec. 4.5) -------------------------------------------
def compress_tuple(x, beta: int) -> int:
    a = _u64(x)
    return int(lib().orc_compress_tuple(_p(a), a.size, beta))


def seteq_partial_products(X, Y, alpha: int, beta: int):
    """Z [L + 1] with Z_0 = 1, Z_{i+1} = Z_i (alpha - x_i) / (alpha - y_i) over
    compressed tuples; None if some alpha - y_i is zero."""
    a, b = _u64(X), _u64(Y)
    L, T = a.shape
    z = np.empty(L + 1, np.uint64)
    rc = lib().orc_seteq_partial_products(_p(a), _p(b), L, T, alpha, beta, _p(z))
    return None if rc else z
