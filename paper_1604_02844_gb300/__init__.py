"""GB300-native level-synchronous top-down BFS (Paredes, Riley, Lujan,
"Breadth First Search Vectorization on the Intel Xeon Phi").

A thin ctypes binding over the C ABI in ``include/gbbfs.h`` (``libgbbfs.so``,
built in-tree by ``build.py``).  Every step of the search runs in the
library's CUDA kernels; this module only marshals arguments.  PyTorch is used
for device buffers and streams.  There is no CPU fallback: if the library is
missing the import-time load raises.

Functions keep the C names (``bfs_graph_create``, ``bfs_run``,
``bfs_run_batch``, ``bfs_server_create``, ``bfs_submit``, ``bfs_poll`` ...);
``Graph`` and ``Server`` wrap them for convenience.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

# The serving loop gives every resident graph its own CUDA stream.  With the
# default of 8 hardware work queues, those streams (and the caller's) share
# queues, so a small graph's result extraction waits behind a large graph's
# multi-millisecond round that happens to sit on the same queue.  32 queues
# (the most CUDA allows) keep the graphs apart.  The variable only counts
# before the process's first CUDA call, and an explicit setting is kept.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbbfs.so")

# bfs_status
BFS_OK = 0
BFS_NOT_READY = 1
BFS_ERR_INVALID_ARG = -1
BFS_ERR_INVALID_GRAPH = -2
BFS_ERR_OOM = -3
BFS_ERR_CUDA = -4
BFS_ERR_DEPTH = -5
BFS_ERR_TIMEOUT = -6
BFS_ERR_BUSY = -7

# bfs_option
BFS_OPT_BLOCK = 1
BFS_OPT_CTAS_PER_SM = 2
BFS_OPT_WARP_DEGREE = 3
BFS_OPT_CTA_DEGREE = 4
BFS_OPT_SEGMENT = 5
BFS_OPT_TIMEOUT_NS = 6
BFS_OPT_LAYER_STATS = 7
BFS_OPT_MAX_CTAS = 8
BFS_OPT_BATCH_WIDTH = 9
BFS_OPT_BATCH_BLOCK = 10
BFS_OPT_MODE = 11
BFS_OPT_ALPHA = 12
BFS_OPT_BETA = 13
BFS_OPT_BATCH_STREAMS = 14
MODE_WARP, MODE_BINNED, MODE_RESTORE, MODE_HYBRID = 0, 1, 2, 3

OPTION_NAMES = {
    "block": BFS_OPT_BLOCK, "ctas_per_sm": BFS_OPT_CTAS_PER_SM,
    "warp_degree": BFS_OPT_WARP_DEGREE, "cta_degree": BFS_OPT_CTA_DEGREE,
    "segment": BFS_OPT_SEGMENT, "timeout_ns": BFS_OPT_TIMEOUT_NS,
    "layer_stats": BFS_OPT_LAYER_STATS, "max_ctas": BFS_OPT_MAX_CTAS,
    "batch_width": BFS_OPT_BATCH_WIDTH, "batch_block": BFS_OPT_BATCH_BLOCK,
    "mode": BFS_OPT_MODE,
    "alpha": BFS_OPT_ALPHA,
    "beta": BFS_OPT_BETA,
    "batch_streams": BFS_OPT_BATCH_STREAMS,
}

# every symbol include/gbbfs.h declares, with (restype, argtypes)
_P = ctypes.c_void_p
_I32, _I64, _U64, _INT = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "bfs_abi_version": (_INT, []),
    "bfs_last_error": (ctypes.c_char_p, []),
    "bfs_last_status": (_INT, []),
    "bfs_graph_create": (_P, [_P, _P, _I64, _I64]),
    "bfs_graph_destroy": (_INT, [_P]),
    "bfs_graph_num_vertices": (_I64, [_P]),
    "bfs_graph_num_edges": (_I64, [_P]),
    "bfs_graph_set_option": (_INT, [_P, _INT, _I64]),
    "bfs_graph_get_option": (_I64, [_P, _INT]),
    "bfs_run": (_INT, [_P, _I32, _P, _P, _P]),
    "bfs_run_noalloc": (_INT, [_P, _P, _I64, _I64, _I32, _P, _P, _P]),
    "bfs_graph_status": (_INT, [_P]),
    "bfs_graph_layer_stats": (_INT, [_P, _P, _P, _P, _I32]),
    "bfs_graph_layer_times": (_INT, [_P, _P, _I32]),
    "bfs_graph_visited_bitmap": (_INT, [_P, _P, _I64]),
    "bfs_graph_autotune": (_INT, [_P, _INT, ctypes.c_int32]),
    "bfs_run_batch": (_INT, [_P, _P, _I32, _P]),
    "bfs_server_create": (_P, [_I64]),
    "bfs_server_destroy": (_INT, [_P]),
    "bfs_server_add_graph": (_INT, [_P, _P]),
    "bfs_submit": (_INT, [_P, _INT, _I32, _P, ctypes.POINTER(_U64)]),
    "bfs_poll": (_INT, [_P, _U64]),
    "bfs_server_drain": (_INT, [_P]),
    "bfs_ticket_times": (_INT, [_P, _U64, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "bfs_server_graph_stats": (_INT, [_P, _INT, ctypes.POINTER(_I64)]),
    "bfs_ticket_info": (_INT, [_P, _U64, _P]),
}


class TicketInfo(ctypes.Structure):
    """Layout of bfs_ticket_record (include/gbbfs.h)."""
    _fields_ = [("t_submit_ns", _I64), ("t_admit_ns", _I64), ("t_done_ns", _I64),
                ("join_iter", _I64), ("done_iter", _I64),
                ("graph_id", _I32), ("lane", _I32), ("lanes_busy_at_join", _I32), ("reserved", _I32)]


class BfsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"[{status}] {message}")
        self.status = status


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libgbbfs.so (or the library GBBFS_LIB names, e.g. the
    bounds-checking build libgbbfs_check.so); raises if it has not been built
    (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("GBBFS_LIB") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -c 'import __graft_entry__ as g; "
                           "g.build()'); this package has no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return load().bfs_last_error().decode(errors="replace")


def _check(status: int) -> int:
    if status < 0:
        raise BfsError(status, last_error())
    return status


def _ptr(a) -> int:
    """Address of a torch tensor or numpy array (contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    return int(a)


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


# ---- C-named functions ----------------------------------------------------

def bfs_abi_version() -> int:
    return load().bfs_abi_version()


def bfs_graph_create(row_offsets, col_idx, n: int | None = None, m: int | None = None) -> int:
    """Upload a CSR; arrays may be numpy, host or CUDA tensors (int32)."""
    n = (len(row_offsets) - 1) if n is None else n
    m = len(col_idx) if m is None else m
    h = load().bfs_graph_create(_ptr(row_offsets), _ptr(col_idx) if m > 0 else None, n, m)
    if not h:
        raise BfsError(load().bfs_last_status(), last_error())
    return h


def bfs_graph_destroy(g) -> None:
    _check(load().bfs_graph_destroy(g))


def bfs_run(g, root: int, level_out, parent_out=None, stream=None) -> None:
    _check(load().bfs_run(g, int(root), _ptr(level_out), _ptr(parent_out), _stream_handle(stream)))


NOALLOC_MAX_VERTICES = 131072
NOALLOC_MAX_EDGES = 4194304


def bfs_run_noalloc(row_offsets, col_idx, root: int, level_out, parent_out=None, stream=None,
                    n: int | None = None, m: int | None = None) -> None:
    """Search without any allocation (device CSR and outputs; blocks until done)."""
    n = (len(row_offsets) - 1) if n is None else n
    m = len(col_idx) if m is None else m
    _check(load().bfs_run_noalloc(_ptr(row_offsets), _ptr(col_idx) if m > 0 else None, n, m, int(root),
                                  _ptr(level_out), _ptr(parent_out), _stream_handle(stream)))


def bfs_graph_status(g) -> int:
    return _check(load().bfs_graph_status(g))


def bfs_run_batch(g, roots, level_out) -> None:
    r = np.ascontiguousarray(roots, dtype=np.int32)
    _check(load().bfs_run_batch(g, r.ctypes.data, int(r.shape[0]), _ptr(level_out)))


def bfs_graph_set_option(g, option, value: int) -> None:
    opt = OPTION_NAMES[option] if isinstance(option, str) else int(option)
    _check(load().bfs_graph_set_option(g, opt, int(value)))


def bfs_graph_get_option(g, option) -> int:
    opt = OPTION_NAMES[option] if isinstance(option, str) else int(option)
    v = load().bfs_graph_get_option(g, opt)
    return _check(v) if v < 0 else v


def bfs_graph_layer_stats(g, max_layers: int = 256):
    v = np.zeros(max_layers, np.int64)
    e = np.zeros(max_layers, np.int64)
    t = np.zeros(max_layers, np.int64)
    L = _check(load().bfs_graph_layer_stats(g, v.ctypes.data, e.ctypes.data, t.ctypes.data, max_layers))
    return v[:L], e[:L], t[:L]


def bfs_graph_layer_times(g, max_layers: int = 256) -> np.ndarray:
    t = np.zeros(max_layers, np.int64)
    L = _check(load().bfs_graph_layer_times(g, t.ctypes.data, max_layers))
    return t[:L]


BFS_TUNE_SINGLE, BFS_TUNE_BATCH, BFS_TUNE_MODE = 1, 2, 4


def bfs_graph_autotune(g, what: int, samples: int = 0) -> None:
    """Time candidate option values on sample searches and keep the fastest."""
    _check(load().bfs_graph_autotune(g, what, samples))


def bfs_graph_visited_bitmap(g, n: int) -> np.ndarray:
    words = np.zeros((n + 31) // 32, np.uint32)
    _check(load().bfs_graph_visited_bitmap(g, words.ctypes.data, words.shape[0]))
    return words


def bfs_server_create(hbm_budget_bytes: int = 0) -> int:
    h = load().bfs_server_create(int(hbm_budget_bytes))
    if not h:
        raise BfsError(load().bfs_last_status(), last_error())
    return h


def bfs_server_destroy(s) -> None:
    _check(load().bfs_server_destroy(s))


def bfs_server_add_graph(s, g) -> int:
    return _check(load().bfs_server_add_graph(s, g))


def bfs_submit(s, graph_id: int, root: int, level_out) -> int:
    t = ctypes.c_uint64(0)
    _check(load().bfs_submit(s, int(graph_id), int(root), _ptr(level_out), ctypes.byref(t)))
    return t.value


def bfs_poll(s, ticket: int) -> int:
    return _check(load().bfs_poll(s, int(ticket)))


def bfs_server_drain(s) -> None:
    _check(load().bfs_server_drain(s))


SERVER_PHASES = ("waiting for work", "admitting queries", "putting sources on the device",
                 "launching iterations", "reading the control block", "delivering results",
                 "waiting for workspace room", "stopped")


def bfs_server_graph_stats(s, graph_id: int) -> dict:
    out = (_I64 * 7)()
    _check(load().bfs_server_graph_stats(s, int(graph_id), out))
    return {"waiting": out[0], "running": out[1], "rounds": out[2], "iter": out[3], "has_workspace": bool(out[4]),
            "ns_since_round": out[5], "phase": SERVER_PHASES[out[6]] if 0 <= out[6] < len(SERVER_PHASES) else out[6]}


def bfs_ticket_times(s, ticket: int):
    a, b = ctypes.c_int64(0), ctypes.c_int64(0)
    _check(load().bfs_ticket_times(s, int(ticket), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def bfs_ticket_info(s, ticket: int) -> dict:
    """The path of one query: submission, admission, completion times and
    the search iterations at which its lane joined and finished."""
    info = TicketInfo()
    _check(load().bfs_ticket_info(s, int(ticket), ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in TicketInfo._fields_ if k != "reserved"}


# ---- convenience wrappers -------------------------------------------------

class Graph:
    """A resident CSR graph.  ``run`` returns CUDA tensors (level, parent)."""

    def __init__(self, row_offsets, col_idx, **options):
        self.n = len(row_offsets) - 1
        self.m = len(col_idx)
        self.handle = bfs_graph_create(row_offsets, col_idx, self.n, self.m)
        for k, v in options.items():
            self.set_option(k, v)

    def set_option(self, name, value):
        bfs_graph_set_option(self.handle, name, value)

    def get_option(self, name):
        return bfs_graph_get_option(self.handle, name)

    def run(self, root: int, level_out=None, parent_out=None, want_parent: bool = True, stream=None):
        import torch
        if level_out is None:
            level_out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        if parent_out is None and want_parent:
            parent_out = torch.empty(self.n, dtype=torch.int32, device="cuda")
        bfs_run(self.handle, root, level_out, parent_out, stream)
        return level_out, parent_out

    def status(self) -> int:
        return bfs_graph_status(self.handle)

    def run_batch(self, roots, level_out=None):
        import torch
        roots = np.ascontiguousarray(roots, dtype=np.int32)
        if level_out is None:
            level_out = torch.empty((roots.shape[0], self.n), dtype=torch.uint8, device="cuda")
        bfs_run_batch(self.handle, roots, level_out)
        return level_out

    def layer_stats(self, max_layers: int = 256):
        return bfs_graph_layer_stats(self.handle, max_layers)

    def layer_times(self, max_layers: int = 256):
        return bfs_graph_layer_times(self.handle, max_layers)

    def visited_bitmap(self):
        return bfs_graph_visited_bitmap(self.handle, self.n)

    def autotune(self, what: int = BFS_TUNE_SINGLE, samples: int = 0) -> dict:
        """Run the autotuner; returns the options it left set."""
        bfs_graph_autotune(self.handle, what, samples)
        return {k: self.get_option(k) for k in OPTION_NAMES}

    def close(self):
        if self.handle:
            bfs_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Server:
    """Continuous-batching request loop over resident graphs (C ABI
    bfs_server_*).  ``submit`` returns a ticket; ``poll``/``wait`` report
    completion; results land in the host uint8 buffer given at submit."""

    def __init__(self, hbm_budget_bytes: int = 0):
        self.handle = bfs_server_create(hbm_budget_bytes)
        self._keep = {}
        self._graphs = []  # registered graphs outlive the server (it frees their batch workspaces)

    def add_graph(self, graph: "Graph") -> int:
        gid = bfs_server_add_graph(self.handle, graph.handle)
        self._graphs.append(graph)
        return gid

    def submit(self, graph_id: int, root: int, level_out: np.ndarray) -> int:
        if not (isinstance(level_out, np.ndarray) and level_out.dtype == np.uint8 and level_out.flags["C_CONTIGUOUS"]):
            raise ValueError("level_out must be a C-contiguous numpy uint8 array")
        t = bfs_submit(self.handle, graph_id, root, level_out)
        self._keep[t] = level_out
        return t

    def poll(self, ticket: int) -> bool:
        return bfs_poll(self.handle, ticket) == BFS_OK

    def wait(self, ticket: int, sleep_s: float = 0.0, timeout_s: float | None = None) -> None:
        """Poll until the query completes (raises BfsError if it failed, and
        TimeoutError if timeout_s passes first)."""
        import time
        deadline = None if timeout_s is None else time.monotonic() + timeout_s
        while not self.poll(ticket):
            if deadline is not None and time.monotonic() > deadline:
                raise TimeoutError(f"query {ticket} still running after {timeout_s} s")
            if sleep_s:
                time.sleep(sleep_s)

    def drain(self) -> None:
        bfs_server_drain(self.handle)

    def times(self, ticket: int):
        return bfs_ticket_times(self.handle, ticket)

    def info(self, ticket: int) -> dict:
        return bfs_ticket_info(self.handle, ticket)

    def graph_stats(self, graph_id: int) -> dict:
        """Monitoring snapshot of one graph's queue and worker."""
        return bfs_server_graph_stats(self.handle, graph_id)

    def close(self):
        if self.handle:
            bfs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
