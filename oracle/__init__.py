"""CPU oracle for the BFS library -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The library itself never calls it and shares no
code with it.  The arithmetic lives in ``oracle.c`` (plain single-threaded C);
this module only compiles it with gcc and marshals numpy arrays.

Functions (paper: Paredes, Riley, Lujan, "Breadth First Search Vectorization
on the Intel Xeon Phi"):
  bfs             -- queue-based serial BFS (Sec. 3), init of Alg. 1
  bfs_batch       -- the same per source, uint8 source-major levels
  layer_profile   -- the per-layer columns of Table 1
  validate        -- the soft result check of Sec. 5.3, rules 1-5
Parity is pinned in tests/test_oracle.py against closed forms, brute-force
relaxation, scipy.sparse.csgraph and hand-checked fixtures in tests/golden/.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

VALIDATE_RULES = {
    0: "ok",
    1: "root is not its own parent at level 0",
    2: "parent edge missing or parent/level reach disagree",
    3: "parent not exactly one layer up",
    4: "an edge out of a reached vertex skips a layer or leaves the tree",
    5: "reached set differs from the oracle's",
}


def compile_source(src: str, out: str) -> str:
    """gcc -O2 of one oracle source file into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-Wall", src, "-o", tmp],
                   check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc -O2, single-threaded code)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB)
    return _LIB


def _bind(path: str) -> ctypes.CDLL:
    lib = ctypes.CDLL(path)
    p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32
    lib.oracle_bfs.argtypes = [p, p, i64, i32, p, p]
    lib.oracle_bfs.restype = i64
    lib.oracle_bfs_batch.argtypes = [p, p, i64, p, i32, p]
    lib.oracle_bfs_batch.restype = ctypes.c_int
    lib.oracle_layer_profile.argtypes = [p, i64, p, i64, p, p, p]
    lib.oracle_layer_profile.restype = i64
    lib.oracle_validate.argtypes = [p, p, i64, i32, p, p, p, p]
    lib.oracle_validate.restype = ctypes.c_int
    return lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _cols(col_idx):
    return _c(col_idx if len(col_idx) else np.zeros(1, np.int32), np.int32)


class Oracle:
    """The oracle functions bound to one compiled copy of oracle.c."""

    def __init__(self, path: str):
        self.path = path
        self.lib = _bind(path)

    def bfs(self, row_offsets, col_idx, root: int, want_parent: bool = True):
        """(level int32[n], parent int32[n] or None); -1 marks unreached."""
        ro, pro = _c(row_offsets, np.int32)
        ci, pci = _cols(col_idx)
        n = ro.shape[0] - 1
        level = np.empty(n, np.int32)
        parent = np.empty(n, np.int32) if want_parent else None
        r = self.lib.oracle_bfs(pro, pci, n, int(root), level.ctypes.data,
                                parent.ctypes.data if want_parent else None)
        if r < 0:
            raise ValueError(f"oracle_bfs: bad argument (root={root}, n={n})")
        return level, parent

    def bfs_batch(self, row_offsets, col_idx, roots):
        """uint8[k][n] levels (0xFF = unreached); raises on depth > 254."""
        ro, pro = _c(row_offsets, np.int32)
        ci, pci = _cols(col_idx)
        rt, prt = _c(roots, np.int32)
        n = ro.shape[0] - 1
        out = np.empty((rt.shape[0], n), np.uint8)
        rc = self.lib.oracle_bfs_batch(pro, pci, n, prt, rt.shape[0], out.ctypes.data)
        if rc == -5:
            raise OverflowError("a level exceeds 254")
        if rc != 0:
            raise ValueError("oracle_bfs_batch: bad argument")
        return out

    def layer_profile(self, row_offsets, level, max_layers: int = 4096):
        """Table 1 columns: (vertices[d], edges[d], traversed[d]) per layer d."""
        ro, pro = _c(row_offsets, np.int32)
        lv, plv = _c(level, np.int32)
        n = ro.shape[0] - 1
        v = np.zeros(max_layers, np.int64)
        e = np.zeros(max_layers, np.int64)
        t = np.zeros(max_layers, np.int64)
        L = self.lib.oracle_layer_profile(pro, n, plv, max_layers, v.ctypes.data,
                                          e.ctypes.data, t.ctypes.data)
        if L < 0:
            raise ValueError("more layers than max_layers")
        return v[:L], e[:L], t[:L]

    def validate(self, row_offsets, col_idx, root: int, level, parent, ref_level=None):
        """(rule, bad_vertex): rule 0 means every check passed."""
        ro, pro = _c(row_offsets, np.int32)
        ci, pci = _cols(col_idx)
        lv, plv = _c(level, np.int32)
        pa, ppa = _c(parent, np.int32)
        rl, prl = (None, None) if ref_level is None else _c(ref_level, np.int32)
        bad = ctypes.c_int64(-1)
        rule = self.lib.oracle_validate(pro, pci, ro.shape[0] - 1, int(root), plv, ppa, prl,
                                        ctypes.byref(bad))
        return int(rule), int(bad.value)

    def time_bfs(self, row_offsets, col_idx, roots):
        """Seconds of oracle_bfs per root (steady clock around the call only)."""
        ro, pro = _c(row_offsets, np.int32)
        ci, pci = _cols(col_idx)
        n = ro.shape[0] - 1
        level = np.empty(n, np.int32)
        parent = np.empty(n, np.int32)
        out = []
        for r in roots:
            t0 = time.perf_counter()
            self.lib.oracle_bfs(pro, pci, n, int(r), level.ctypes.data, parent.ctypes.data)
            out.append(time.perf_counter() - t0)
        return out


def default() -> Oracle:
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = Oracle(_LIB)
    return _lib


def bfs(row_offsets, col_idx, root: int, want_parent: bool = True):
    return default().bfs(row_offsets, col_idx, root, want_parent)


def bfs_batch(row_offsets, col_idx, roots):
    return default().bfs_batch(row_offsets, col_idx, roots)


def layer_profile(row_offsets, level, max_layers: int = 4096):
    return default().layer_profile(row_offsets, level, max_layers)


def validate(row_offsets, col_idx, root: int, level, parent, ref_level=None):
    return default().validate(row_offsets, col_idx, root, level, parent, ref_level)


def time_bfs(row_offsets, col_idx, roots):
    return default().time_bfs(row_offsets, col_idx, roots)
