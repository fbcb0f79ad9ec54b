"""Python binding of libv3c.so: the LDE + Poseidon-Merkle polynomial commitment.

Argument marshalling only.  Every step of the commitment runs in the CUDA
kernels of ``libv3c.so``, and importing this module fails loudly if the
library has not been built (``python -m paper_2603_03065_gb300.build``).  PyTorch
provides device memory and streams.  Field elements are carried in int64
tensors that hold the uint64 bit patterns.

Example (x: canonical uint64 numpy array [c][n], n a power of two)::

    import paper_2603_03065_gb300 as v3c
    with v3c.Context(0) as ctx:
        cid = ctx.commit([(v3c.to_device_u64(x), 3, 4)])[0]  # rate_bits 3, cap height 4
        cap = ctx.cap(cid)                                   # [16][4] digests
        rows, paths = ctx.open_batch(cid, [0, 7], x.shape[0])
        fid = ctx.fri_begin([cid], alpha, 4, 5, 4, betas=betas)
        ...
        ctx.release(cid)
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libv3c.so")
P = 0xFFFFFFFF00000001

V3C_OK, V3C_EINVAL, V3C_ENOMEM, V3C_ECUDA, V3C_EAGAIN, V3C_ETIMEDOUT, V3C_ENOTFOUND, V3C_ECANCELED = range(8)
REQ_QUEUED, REQ_ADMITTED, REQ_RUNNING, REQ_DONE, REQ_FAILED = range(5)
FLAG_VALIDATE = 1
MAX_LOG_N, MAX_LOG_LDE, MAX_RATE_BITS = 22, 25, 4

_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_vp = ctypes.c_void_p
_u64p = ctypes.POINTER(ctypes.c_uint64)


_LOG_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_int, ctypes.c_char_p)


class V3CError(RuntimeError):
    def __init__(self, status: int, detail: str = ""):
        self.status = status
        super().__init__(f"v3c status {status}: {detail}")


class Config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", _u64), ("max_inflight", _u32), ("flags", _u32),
                ("autotune", _u32), ("timeout_ms", _u32)]


class CommitDesc(ctypes.Structure):
    _fields_ = [("cols", _vp), ("on_device", ctypes.c_int32), ("c", _u32), ("log_n", _u32),
                ("rate_bits", _u32), ("cap_height", _u32)]


class PartDesc(ctypes.Structure):
    _fields_ = [("coeffs", _vp), ("c", _u32), ("log_n", _u32), ("rate_bits", _u32), ("cap_height", _u32),
                ("log_parts", _u32), ("part", _u32)]


class ServeCfg(ctypes.Structure):
    _fields_ = [("queue_capacity", _u32), ("max_batch", _u32), ("max_inflight", _u32), ("flags", _u32),
                ("slot_scratch_bytes", _u64), ("batch_elems", _u64)]


FLAG_NO_GRAPH = 4
INPUT_HOST_COPY, INPUT_DEVICE, INPUT_HOST_BORROW = 0, 1, 2


FLAG_TIMING = 2
STAGES = ("lde_a", "lde_b", "lde_c", "leaf_hash", "merkle", "fri_combine", "fri_fold", "open", "seteq",
          "snapshot_slots", "snapshot_codebook")


class StageStats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * len(STAGES)), ("launches", ctypes.c_uint64 * len(STAGES))]


FRI_MAX_ROUNDS = 25


class FriCfg(ctypes.Structure):
    _fields_ = [("arity_bits", _u32), ("final_log", _u32), ("cap_height", _u32), ("ext_degree", _u32)]


class FriInfo(ctypes.Structure):
    _fields_ = [("rounds", _u32), ("rounds_done", _u32), ("log_N", _u32), ("n_columns", _u32),
                ("arity_bits", _u32 * FRI_MAX_ROUNDS), ("log_size", _u32 * (FRI_MAX_ROUNDS + 1)),
                ("cap_height", _u32 * FRI_MAX_ROUNDS), ("query_words", _u64), ("bytes", _u64),
                ("ext_degree", _u32), ("pad", _u32)]


class SnapshotDesc(ctypes.Structure):
    _fields_ = [("records", _vp), ("centroids", _vp), ("codebooks", _vp), ("on_device", ctypes.c_int32),
                ("log_nlist", _u32), ("log_n", _u32), ("M", _u32), ("D", _u32), ("K", _u32), ("d", _u32)]


class SeteqDesc(ctypes.Structure):
    _fields_ = [("x", _vp), ("y", _vp), ("z", _vp), ("L", _u64), ("T", _u32), ("pad", _u32), ("alpha", _u64),
                ("beta", _u64)]


class ReqTimes(ctypes.Structure):
    _fields_ = [("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


# Every symbol include/v3c.h declares, with its ctypes signature.
SIGNATURES = {
    "v3c_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "v3c_last_error_detail": (ctypes.c_char_p, [_vp]),
    "v3c_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(Config), ctypes.POINTER(_vp)]),
    "v3c_destroy": (ctypes.c_int, [_vp]),
    "v3c_lde": (ctypes.c_int, [_vp, _vp, _u32, _u32, _u32, _vp, _u32, _vp]),
    "v3c_merkle": (ctypes.c_int, [_vp, _vp, _u32, _u32, _u32, _u32, _vp, _vp, _vp]),
    "v3c_commit": (ctypes.c_int, [_vp, ctypes.POINTER(CommitDesc), _u32, _u64p, _vp]),
    "v3c_coeffs": (ctypes.c_int, [_vp, _vp, _u32, _u32, _vp, _vp]),
    "v3c_commit_part": (ctypes.c_int, [_vp, ctypes.POINTER(PartDesc), _u64p, _vp]),
    "v3c_commit_buffers": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(_vp), ctypes.POINTER(_u32),
                                          ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_u32),
                                          ctypes.POINTER(_u32)]),
    "v3c_commit_cap": (ctypes.c_int, [_vp, _u64, _u64p]),
    "v3c_open": (ctypes.c_int, [_vp, _u64, _u64, _u64p, _u64p]),
    "v3c_release": (ctypes.c_int, [_vp, _u64]),
    "v3c_commit_footprint": (_u64, [_u32, _u32, _u32, _u32]),
    "v3c_serve_start": (ctypes.c_int, [_vp, ctypes.POINTER(ServeCfg)]),
    "v3c_serve_submit": (ctypes.c_int, [_vp, ctypes.POINTER(CommitDesc), _u64p]),
    "v3c_serve_poll": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(ctypes.c_int), _u64p, ctypes.POINTER(ReqTimes)]),
    "v3c_serve_stop": (ctypes.c_int, [_vp]),
    "v3c_kernel_launches": (_u64, [_vp]),
    "v3c_graph_replays": (_u64, [_vp]),
    "v3c_stage_stats": (ctypes.c_int, [_vp, ctypes.c_void_p, ctypes.c_int]),
    "v3c_lde_noalloc": (ctypes.c_int, [_vp, _u32, _u32, _u32, _vp, _u32, _vp]),
    "v3c_int_peak": (ctypes.c_int, [_vp, _u32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "v3c_int_pipe_rate": (ctypes.c_int, [_vp, _u32, _u32, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double)]),
    "v3c_wait_selftest": (ctypes.c_int, [_vp, _u32, _u32, _vp]),
    "v3c_mem_stats": (ctypes.c_int, [_vp, _u64p]),
    "v3c_serve_inject_failure": (ctypes.c_int, [_vp, _u32]),
    "v3c_set_log": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int]),
    "v3c_tune_export": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "v3c_tune_import": (ctypes.c_int, [_vp, ctypes.c_char_p]),
    # include/v3c_fri.h
    "v3c_fri_begin": (ctypes.c_int, [_vp, _u64p, _u32, _u64p, ctypes.POINTER(FriCfg), _u64p, _u32, _u64p, _vp]),
    "v3c_fri_fold": (ctypes.c_int, [_vp, _u64, _u64p, _u32, _vp]),
    "v3c_fri_info": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(FriInfo)]),
    "v3c_fri_cap": (ctypes.c_int, [_vp, _u64, _u32, _u64p]),
    "v3c_fri_final": (ctypes.c_int, [_vp, _u64, _u64p]),
    "v3c_fri_query": (ctypes.c_int, [_vp, _u64, _u64p, _u32, _u64p]),
    "v3c_fri_release": (ctypes.c_int, [_vp, _u64]),
    "v3c_open_batch": (ctypes.c_int, [_vp, _u64, _u64p, _u32, _u64p, _u64p]),
    # include/v3c_snapshot.h
    "v3c_snapshot_commit": (ctypes.c_int, [_vp, ctypes.POINTER(SnapshotDesc), _u64p, _vp]),
    "v3c_snapshot_roots": (ctypes.c_int, [_vp, _u64, _u64p, _u64p]),
    "v3c_snapshot_list_roots": (ctypes.c_int, [_vp, _u64, _u64p]),
    "v3c_snapshot_open_lists": (ctypes.c_int, [_vp, _u64, ctypes.POINTER(_u32), _u32, _u64p]),
    "v3c_snapshot_release": (ctypes.c_int, [_vp, _u64]),
    # include/v3c_seteq.h
    "v3c_seteq": (ctypes.c_int, [_vp, ctypes.POINTER(SeteqDesc), _u32, ctypes.POINTER(_u32), _vp]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libv3c.so and binds every exported entry point.  Raises if the
    library is missing: there is no fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2603_03065_gb300.build` "
                          "(the CUDA library is required; there is no CPU fallback)")
    L = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(status: int) -> str:
    return load().v3c_strerror(status).decode()


def footprint(c: int, log_n: int, rate_bits: int, cap_height: int) -> int:
    return load().v3c_commit_footprint(c, log_n, rate_bits, cap_height)


def tree_words(log_rows: int, cap_height: int) -> int:
    N = 1 << log_rows
    return (2 * N - (2 << cap_height)) * 4


def _torch():
    import torch

    return torch


def _ptr(t) -> int | None:
    return None if t is None else t.data_ptr()


def _stream(stream) -> int | None:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def to_device_u64(a: np.ndarray, device="cuda"):
    """uint64 numpy array -> int64 CUDA tensor with the same bits."""
    torch = _torch()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


def to_host_u64(t) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint64)


NOALLOC_SCRATCH_BYTES = 32 << 20


def lde_noalloc(cols, rate_bits: int, out, ld: int | None = None, stream=None) -> int:
    """v3c_lde_noalloc on the current device: the LDE of ``cols`` into the
    caller's preallocated ``out`` [N][ld].  The library allocates nothing;
    its work space is a fixed device array, for callers that cannot allocate.
    Returns the v3c status (0 = ok).  The shapes are checked here, since
    the kernels write into ``out`` without knowing its size."""
    import torch

    c, n = cols.shape
    if n < 1 or n & (n - 1):
        raise ValueError(f"lde_noalloc: row count {n} is not a power of two")
    ld = out.shape[1] if ld is None else ld
    for name, t in (("cols", cols), ("out", out)):
        if t.dtype != torch.int64 or not t.is_contiguous() or t.device.type != "cuda":
            raise ValueError(f"lde_noalloc: {name} must be a contiguous int64 CUDA tensor")
        if t.device.index != torch.cuda.current_device():
            raise ValueError(f"lde_noalloc: {name} is not on the current CUDA device")
    if out.dim() != 2 or out.shape[0] != n << rate_bits:
        raise ValueError(f"lde_noalloc: out must have {n << rate_bits} rows, has {tuple(out.shape)}")
    if not c <= ld <= out.shape[1]:
        raise ValueError(f"lde_noalloc: need c <= ld <= out.shape[1] (c={c}, ld={ld}, out={tuple(out.shape)})")
    return load().v3c_lde_noalloc(_ptr(cols), c, n.bit_length() - 1, rate_bits, _ptr(out), ld, _stream(stream))


@dataclass
class Opening:
    row: np.ndarray
    path: np.ndarray


class Context:
    """One v3c context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_inflight: int = 0, flags: int = 0,
                 autotune: bool = False):
        self.lib = load()
        cfg = Config(hbm_budget_bytes, max_inflight, flags, 1 if autotune else 0, 0)
        self._borrowed = {}
        h = _vp()
        self._check(self.lib.v3c_create(device, ctypes.byref(cfg), ctypes.byref(h)), None)
        self.h = h
        self.device = device

    def _check(self, st: int, h=...):
        if st != V3C_OK:
            hh = self.h if h is ... else h
            detail = self.lib.v3c_last_error_detail(hh).decode() if hh else ""
            raise V3CError(st, f"{strerror(st)}: {detail}")

    def close(self):
        if getattr(self, "h", None):
            self.lib.v3c_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --------------------------------------------------------------- stages
    def lde(self, cols, rate_bits: int, ld: int | None = None, out=None, stream=None):
        """cols: int64 CUDA tensor [c][n] -> LDE [N][ld] (row-major, bit-reversed rows)."""
        torch = _torch()
        c, n = cols.shape
        log_n = n.bit_length() - 1
        ld = c + (c & 1) if ld is None else ld
        N = n << rate_bits
        if out is None:
            out = torch.empty((N, ld), dtype=torch.int64, device=cols.device)
        self._check(self.lib.v3c_lde(self.h, _ptr(cols), c, log_n, rate_bits, _ptr(out), ld, _stream(stream)))
        return out

    def merkle(self, rows, width: int, cap_height: int, tree=None, cap=None, stream=None):
        torch = _torch()
        N, ld = rows.shape
        log_rows = N.bit_length() - 1
        tw = tree_words(log_rows, cap_height)
        if tree is None and tw:
            tree = torch.empty(tw, dtype=torch.int64, device=rows.device)
        if cap is None:
            cap = torch.empty((1 << cap_height, 4), dtype=torch.int64, device=rows.device)
        self._check(self.lib.v3c_merkle(self.h, _ptr(rows), ld, width, log_rows, cap_height,
                                        _ptr(tree) if tw else None, _ptr(cap), _stream(stream)))
        return tree, cap

    def commit(self, items, stream=None) -> list[int]:
        """items: list of (cols, rate_bits, cap_height); cols an int64 CUDA tensor
        [c][n] or a uint64 numpy array (host input)."""
        descs = (CommitDesc * len(items))()
        keep = []
        for i, (cols, r, h) in enumerate(items):
            if isinstance(cols, np.ndarray):
                a = np.ascontiguousarray(cols, dtype=np.uint64)
                keep.append(a)
                descs[i] = CommitDesc(a.ctypes.data, 0, a.shape[0], a.shape[1].bit_length() - 1, r, h)
            else:
                descs[i] = CommitDesc(cols.data_ptr(), 1, cols.shape[0], cols.shape[1].bit_length() - 1, r, h)
        ids = (_u64 * len(items))()
        self._check(self.lib.v3c_commit(self.h, descs, len(items), ids, _stream(stream)))
        return list(ids)

    def coeffs(self, cols, out=None, stream=None):
        """v3c_coeffs: int64 CUDA tensor [c][n] of columns -> [c][n] natural-order
        coefficients of each column's interpolant (n^-1 applied)."""
        torch = _torch()
        c, n = cols.shape
        if n < 1 or n & (n - 1):
            raise ValueError(f"coeffs: row count {n} is not a power of two")
        if out is None:
            out = torch.empty((c, n), dtype=torch.int64, device=cols.device)
        elif tuple(out.shape) != (c, n) or not out.is_contiguous():
            raise ValueError("coeffs: out must be a contiguous [c][n] int64 tensor")
        self._check(self.lib.v3c_coeffs(self.h, _ptr(cols), c, n.bit_length() - 1, _ptr(out), _stream(stream)))
        return out

    def commit_part(self, coeffs, rate_bits: int, cap_height: int, log_parts: int, part: int, stream=None) -> int:
        """v3c_commit_part: part ``part`` of 2^log_parts of the commit whose
        coefficients are ``coeffs`` (int64 CUDA tensor [c][n]); returns the
        resident object's id (its rows are the commit's row block of the part)."""
        c, n = coeffs.shape
        d = PartDesc(coeffs.data_ptr(), c, n.bit_length() - 1, rate_bits, cap_height, log_parts, part)
        cid = _u64()
        self._check(self.lib.v3c_commit_part(self.h, ctypes.byref(d), ctypes.byref(cid), _stream(stream)))
        self._borrowed[cid.value] = coeffs
        return cid.value

    def buffers(self, cid: int):
        lde, tree, cap = _vp(), _vp(), _vp()
        ld, logr, h = _u32(), _u32(), _u32()
        self._check(self.lib.v3c_commit_buffers(self.h, cid, ctypes.byref(lde), ctypes.byref(ld),
                                                ctypes.byref(tree), ctypes.byref(cap), ctypes.byref(logr),
                                                ctypes.byref(h)))
        return dict(lde=lde.value, ld=ld.value, tree=tree.value, cap=cap.value, log_rows=logr.value,
                    cap_height=h.value)

    def commit_views(self, cid: int, c: int):
        """Copies of a resident object's LDE, tree and cap as numpy arrays."""
        torch = _torch()
        b = self.buffers(cid)
        N = 1 << b["log_rows"]
        out = {}
        for key, words in (("lde", N * b["ld"]), ("tree", tree_words(b["log_rows"], b["cap_height"])),
                           ("cap", 4 << b["cap_height"])):
            arr = np.empty(words, np.uint64)
            if words:
                torch.cuda.synchronize()
                cudart_memcpy_d2h(arr, b[key])
            out[key] = arr
        out["lde"] = out["lde"].reshape(N, b["ld"])
        out["cap"] = out["cap"].reshape(-1, 4)
        return out

    def cap(self, cid: int) -> np.ndarray:
        b = self.buffers(cid)
        out = np.empty((1 << b["cap_height"]) * 4, np.uint64)
        self._check(self.lib.v3c_commit_cap(self.h, cid, out.ctypes.data_as(_u64p)))
        return out.reshape(-1, 4)

    def open(self, cid: int, leaf: int, c: int) -> Opening:
        b = self.buffers(cid)
        k = b["log_rows"] - b["cap_height"]
        row = np.zeros(c, np.uint64)
        path = np.zeros(max(k, 1) * 4, np.uint64)
        self._check(self.lib.v3c_open(self.h, cid, leaf, row.ctypes.data_as(_u64p), path.ctypes.data_as(_u64p)))
        return Opening(row, path[: 4 * k].reshape(-1, 4))

    def release(self, cid: int):
        self._check(self.lib.v3c_release(self.h, cid))
        self._borrowed.pop(cid, None)

    # --------------------------------------------------------------- serving
    def serve_start(self, queue_capacity=0, max_batch=0, max_inflight=0, flags=0, slot_scratch_bytes=0,
                    batch_elems=0):
        cfg = ServeCfg(queue_capacity, max_batch, max_inflight, flags, slot_scratch_bytes, batch_elems)
        self._check(self.lib.v3c_serve_start(self.h, ctypes.byref(cfg)))

    def serve_submit(self, cols, rate_bits: int, cap_height: int, borrow: bool = False) -> int:
        """Submit one commit request.  ``cols``: uint64 numpy [c][n] (copied at
        submit, or borrowed when ``borrow``: then it must be pinned and kept
        alive until DONE), or an int64 CUDA tensor (borrowed)."""
        if isinstance(cols, np.ndarray):
            a = np.ascontiguousarray(cols, dtype=np.uint64)
            kind = INPUT_HOST_BORROW if borrow else INPUT_HOST_COPY
            ptr, c, n = a.ctypes.data, a.shape[0], a.shape[1]
        else:
            a = cols
            kind = INPUT_DEVICE
            ptr, c, n = cols.data_ptr(), cols.shape[0], cols.shape[1]
        d = CommitDesc(ptr, kind, c, n.bit_length() - 1, rate_bits, cap_height)
        t = _u64()
        st = self.lib.v3c_serve_submit(self.h, ctypes.byref(d), ctypes.byref(t))
        if st == V3C_EAGAIN:
            return -1
        self._check(st)
        if kind != INPUT_HOST_COPY:
            self._borrowed[t.value] = a   # keep the borrowed buffer alive until release
        return t.value

    def serve_poll(self, ticket: int, cap_height: int | None = None):
        """Returns (status, state, cap or None, times)."""
        state = ctypes.c_int()
        times = ReqTimes()
        cap = None
        capp = None
        if cap_height is not None:
            cap = np.zeros(4 << cap_height, np.uint64)
            capp = cap.ctypes.data_as(_u64p)
        st = self.lib.v3c_serve_poll(self.h, ticket, ctypes.byref(state), capp, ctypes.byref(times))
        t = (times.t_submit, times.t_admit, times.t_start, times.t_done)
        return st, state.value, (cap.reshape(-1, 4) if (cap is not None and st == V3C_OK) else None), t

    def serve_stop(self):
        self._check(self.lib.v3c_serve_stop(self.h))

    def serve_inject_failure(self, after_passes: int = 0):
        """v3c_serve_inject_failure: the scheduler thread raises at its pass
        `after_passes` from now (host-side failure injection for tests)."""
        self._check(self.lib.v3c_serve_inject_failure(self.h, after_passes))

    # --------------------------------------------------------------- openings
    def open_batch(self, cid: int, leaves, c: int, rows: bool = True, paths: bool = True):
        """Rows [nq][c] and paths [nq][log_N - h][4] of many leaves in one call."""
        b = self.buffers(cid)
        k = b["log_rows"] - b["cap_height"]
        idx = np.ascontiguousarray(leaves, dtype=np.uint64)
        nq = idx.size
        r = np.zeros((nq, c), np.uint64) if rows else None
        pth = np.zeros((nq, k, 4), np.uint64) if paths else None
        self._check(self.lib.v3c_open_batch(self.h, cid, idx.ctypes.data_as(_u64p), nq,
                                            r.ctypes.data_as(_u64p) if rows else None,
                                            pth.ctypes.data_as(_u64p) if paths and k else None))
        return r, pth

    # --------------------------------------------------------------- FRI
    def fri_begin(self, cids, alpha, arity_bits: int = 4, final_log: int = 5, cap_height: int = 4,
                  betas=(), ext: int = 1, stream=None) -> int:
        """alpha: an int (ext 1) or an (re, im) pair (ext 2); betas: a list of
        those."""
        ids = np.ascontiguousarray(cids, dtype=np.uint64)
        al = np.ascontiguousarray(np.array(alpha, dtype=object).reshape(-1).astype(np.uint64))
        bs = np.ascontiguousarray(np.array(list(betas), dtype=object).reshape(-1).astype(np.uint64))
        cfg = FriCfg(arity_bits, final_log, cap_height, ext)
        out = _u64()
        self._check(self.lib.v3c_fri_begin(self.h, ids.ctypes.data_as(_u64p), ids.size, al.ctypes.data_as(_u64p),
                                           ctypes.byref(cfg), bs.ctypes.data_as(_u64p) if bs.size else None,
                                           bs.size // ext, ctypes.byref(out), _stream(stream)))
        return out.value

    def fri_fold(self, fid: int, betas, stream=None):
        ext = self.fri_info(fid)["ext"]
        bs = np.ascontiguousarray(np.array(list(betas), dtype=object).reshape(-1).astype(np.uint64))
        self._check(self.lib.v3c_fri_fold(self.h, fid, bs.ctypes.data_as(_u64p), bs.size // ext, _stream(stream)))

    def fri_info(self, fid: int) -> dict:
        i = FriInfo()
        self._check(self.lib.v3c_fri_info(self.h, fid, ctypes.byref(i)))
        R = i.rounds
        return {"rounds": R, "rounds_done": i.rounds_done, "log_N": i.log_N, "n_columns": i.n_columns,
                "arities": list(i.arity_bits[:R]), "log_sizes": list(i.log_size[: R + 1]),
                "heights": list(i.cap_height[:R]), "query_words": i.query_words, "bytes": i.bytes,
                "ext": i.ext_degree}

    def fri_cap(self, fid: int, layer: int) -> np.ndarray:
        info = self.fri_info(fid)
        out = np.zeros((1 << info["heights"][layer]) * 4, np.uint64)
        self._check(self.lib.v3c_fri_cap(self.h, fid, layer, out.ctypes.data_as(_u64p)))
        return out.reshape(-1, 4)

    def fri_final(self, fid: int) -> np.ndarray:
        """Final coefficients: shape [m] (ext 1) or [m][2] (ext 2)."""
        info = self.fri_info(fid)
        m, ext = 1 << info["log_sizes"][-1], info["ext"]
        out = np.zeros(m * ext, np.uint64)
        self._check(self.lib.v3c_fri_final(self.h, fid, out.ctypes.data_as(_u64p)))
        return out if ext == 1 else out.reshape(m, ext)

    def fri_query(self, fid: int, indices) -> np.ndarray:
        """Raw opening records [nq][query_words]: per layer, the coset values
        then the Merkle path."""
        info = self.fri_info(fid)
        idx = np.ascontiguousarray(indices, dtype=np.uint64)
        out = np.zeros((idx.size, info["query_words"]), np.uint64)
        self._check(self.lib.v3c_fri_query(self.h, fid, idx.ctypes.data_as(_u64p), idx.size,
                                           out.ctypes.data_as(_u64p)))
        return out

    def fri_release(self, fid: int):
        self._check(self.lib.v3c_fri_release(self.h, fid))

    # --------------------------------------------------------------- snapshots
    def snapshot_commit(self, records, centroids, codebooks, log_nlist: int, log_n: int, stream=None) -> int:
        """records [nlist*n][2+M], centroids [nlist][D], codebooks [M][K][d]: all
        uint64 numpy arrays (host, copied) or all int64 CUDA tensors (device)."""
        on_dev = not isinstance(records, np.ndarray)
        if on_dev:
            ptrs = [records.data_ptr(), centroids.data_ptr(), codebooks.data_ptr()]
            M, D = records.shape[1] - 2, centroids.shape[1]
            _, K, d = codebooks.shape
        else:
            keep = [np.ascontiguousarray(a, dtype=np.uint64) for a in (records, centroids, codebooks)]
            ptrs = [a.ctypes.data for a in keep]
            M, D = keep[0].shape[1] - 2, keep[1].shape[1]
            _, K, d = keep[2].shape
        desc = SnapshotDesc(ptrs[0], ptrs[1], ptrs[2], INPUT_DEVICE if on_dev else INPUT_HOST_COPY, log_nlist, log_n,
                            M, D, K, d)
        out = _u64()
        self._check(self.lib.v3c_snapshot_commit(self.h, ctypes.byref(desc), ctypes.byref(out), _stream(stream)))
        return out.value

    def snapshot_roots(self, sid: int) -> tuple[np.ndarray, np.ndarray]:
        mk, cb = np.zeros(4, np.uint64), np.zeros(4, np.uint64)
        self._check(self.lib.v3c_snapshot_roots(self.h, sid, mk.ctypes.data_as(_u64p), cb.ctypes.data_as(_u64p)))
        return mk, cb

    def snapshot_list_roots(self, sid: int, log_nlist: int) -> np.ndarray:
        out = np.zeros((1 << log_nlist, 4), np.uint64)
        self._check(self.lib.v3c_snapshot_list_roots(self.h, sid, out.ctypes.data_as(_u64p)))
        return out

    def snapshot_open_lists(self, sid: int, lists, log_nlist: int) -> np.ndarray:
        idx = np.ascontiguousarray(lists, dtype=np.uint32)
        out = np.zeros((idx.size, log_nlist, 4), np.uint64)
        self._check(self.lib.v3c_snapshot_open_lists(self.h, sid, idx.ctypes.data_as(ctypes.POINTER(_u32)), idx.size,
                                                     out.ctypes.data_as(_u64p)))
        return out

    def snapshot_release(self, sid: int):
        self._check(self.lib.v3c_snapshot_release(self.h, sid))

    # --------------------------------------------------------------- SetEq
    def seteq(self, instances, wait: bool = True, stream=None):
        """instances: list of (x [L][T], y [L][T], z [L+1], alpha, beta), int64
        CUDA tensors.  Returns per-instance statuses (0 ok, 1 alpha equals a
        compressed y) when wait, else None."""
        descs = (SeteqDesc * len(instances))()
        for i, (x, y, z, alpha, beta) in enumerate(instances):
            L, T = x.shape
            descs[i] = SeteqDesc(x.data_ptr(), y.data_ptr(), z.data_ptr(), L, T, 0, alpha, beta)
        st = (_u32 * len(instances))() if wait else None
        self._check(self.lib.v3c_seteq(self.h, descs, len(instances), st, _stream(stream)))
        return list(st) if wait else None

    # --------------------------------------------------------------- misc
    def kernel_launches(self) -> int:
        return self.lib.v3c_kernel_launches(self.h)

    def graph_replays(self) -> int:
        """v3c_commit calls served by replaying a captured CUDA graph."""
        return self.lib.v3c_graph_replays(self.h)

    def stage_stats(self, reset: bool = False) -> dict:
        """Device time (ms) and launches per stage, from CUDA events the library
        records around each stage launch on its stream (needs FLAG_TIMING)."""
        st = StageStats()
        self._check(self.lib.v3c_stage_stats(self.h, ctypes.byref(st), 1 if reset else 0))
        return {name: (st.ms[i], st.launches[i]) for i, name in enumerate(STAGES)}

    def int_peak(self, reps: int = 10) -> tuple[float, float]:
        """Measured 32x32->64 wide multiply-adds per second and the SM MHz of that run."""
        return self.int_pipe_rate(0, reps)

    def set_log(self, fn=None, max_level: int = 1):
        """v3c_set_log: fn(level, text) receives the library's messages up to
        max_level (0 failures, 1 resources and choices, 2 detail); None
        silences it.  fn runs on library threads and must not call back."""
        if fn is None:
            self._log_cb = None
            self._check(self.lib.v3c_set_log(self.h, None, None, -1))
            return
        cb = _LOG_FN(lambda user, level, text: fn(level, text.decode(errors="replace")))
        self._log_cb = cb  # kept alive while the library may call it
        self._check(self.lib.v3c_set_log(self.h, ctypes.cast(cb, _vp), None, max_level))

    def tune_export(self) -> str:
        """v3c_tune_export: the autotuner's choices as JSON text."""
        n = ctypes.c_size_t(0)
        self.lib.v3c_tune_export(self.h, None, 0, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value + 1)
        self._check(self.lib.v3c_tune_export(self.h, buf, n.value + 1, ctypes.byref(n)))
        return buf.value.decode()

    def tune_import(self, text: str):
        """v3c_tune_import: adopt tile choices exported by tune_export."""
        self._check(self.lib.v3c_tune_import(self.h, text.encode()))

    def mem_stats(self) -> dict:
        """v3c_mem_stats: resident bytes counted against the budget, bytes in use
        in the device's default stream-ordered pool, and the scratch arena size."""
        out = (_u64 * 3)()
        self._check(self.lib.v3c_mem_stats(self.h, out))
        return {"resident": out[0], "pool_used": out[1], "arena": out[2]}

    def wait_selftest(self, kind: int, limit_us: int, stream=None) -> None:
        """v3c_wait_selftest: a device wait that nothing satisfies gives up after
        limit_us; raises V3CError with status V3C_ETIMEDOUT (the expected
        outcome)."""
        self._check(self.lib.v3c_wait_selftest(self.h, kind, limit_us, _stream(stream)))

    def int_pipe_rate(self, kind: int, reps: int = 10) -> tuple[float, float]:
        """v3c_int_pipe_rate: kind 0 = wide multiply-adds, 1 = 32-bit multiply-adds."""
        rate, mhz = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.v3c_int_pipe_rate(self.h, kind, reps, ctypes.byref(rate), ctypes.byref(mhz)))
        return rate.value, mhz.value


def cudart_memcpy_d2h(dst: np.ndarray, src_ptr: int):
    """Device -> host copy of raw device memory via torch (no compute)."""
    torch = _torch()
    n = dst.size
    # Wrap the raw pointer in a tensor view through the CUDA array interface.
    class _Arr:
        __cuda_array_interface__ = {"shape": (n,), "typestr": "<i8", "data": (src_ptr, False), "version": 3}

    t = torch.as_tensor(_Arr(), device="cuda")
    dst.view(np.int64)[:] = t.cpu().numpy()
