"""Seeded synthetic graph inputs shared by the oracle tests, the GPU tests and
the benchmark.

This package only builds inputs (R-MAT/Kronecker and uniform tuples, the
vertex permutation, CSR assembly, seeded root choice).  It contains no BFS
arithmetic, and neither the oracle nor the CUDA library imports it.

Workload recipe (paper Sec. 4.1, Sec. 5.2): 2^scale vertices,
2^scale * edgefactor generated tuples with A/B/C/D = 0.57/0.19/0.19/0.05;
vertex ids permuted from the seed; symmetrised; self-loops and repeated
edges removed; int32 CSR with every row sorted.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

RMAT_A, RMAT_B, RMAT_C = 0.57, 0.19, 0.19


def build(force: bool = False) -> str:
    """Compile libgraphgen.so next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall",
               _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            i64, u64, i32p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p
            lib.gg_rmat_tuples.argtypes = [ctypes.c_int, i64, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, u64, i32p, i32p]
            lib.gg_rmat_tuples.restype = None
            lib.gg_uniform_tuples.argtypes = [i64, i64, u64, i32p, i32p]
            lib.gg_uniform_tuples.restype = None
            lib.gg_permutation.argtypes = [i64, u64, i32p]
            lib.gg_permutation.restype = None
            lib.gg_apply_permutation.argtypes = [i64, i32p, i32p, i32p]
            lib.gg_apply_permutation.restype = None
            lib.gg_build_csr.argtypes = [i64, i64, i32p, i32p, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, i32p, i32p]
            lib.gg_build_csr.restype = i64
            lib.gg_pick_roots.argtypes = [i64, i32p, i64, u64, ctypes.c_int, i32p]
            lib.gg_pick_roots.restype = i64
            lib.gg_num_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def rmat_tuples(scale: int, edgefactor: int, seed: int,
                A: float = RMAT_A, B: float = RMAT_B, C: float = RMAT_C):
    """Raw R-MAT tuples (src, dst), int32, before permutation and cleaning."""
    lib = _load()
    ne = (1 << scale) * edgefactor
    src = np.empty(ne, np.int32)
    dst = np.empty(ne, np.int32)
    lib.gg_rmat_tuples(scale, ne, A, B, C, seed, _ptr(src), _ptr(dst))
    return src, dst


def uniform_tuples(n: int, nedges: int, seed: int):
    lib = _load()
    src = np.empty(nedges, np.int32)
    dst = np.empty(nedges, np.int32)
    lib.gg_uniform_tuples(n, nedges, seed, _ptr(src), _ptr(dst))
    return src, dst


def permutation(n: int, seed: int) -> np.ndarray:
    lib = _load()
    perm = np.empty(n, np.int32)
    lib.gg_permutation(n, seed, _ptr(perm))
    return perm


def csr_from_tuples(n: int, src: np.ndarray, dst: np.ndarray, symmetrize: bool = True,
                    drop_loops: bool = True, dedup: bool = True):
    """(row_offsets int32[n+1], col_idx int32[m]) from tuples; rows sorted."""
    lib = _load()
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    ne = src.shape[0]
    ro = np.empty(n + 1, np.int32)
    col = np.empty(max(1, (2 if symmetrize else 1) * ne), np.int32)
    m = lib.gg_build_csr(n, ne, _ptr(src), _ptr(dst), int(symmetrize), int(drop_loops),
                         int(dedup), _ptr(ro), _ptr(col))
    if m < 0:
        raise ValueError(f"gg_build_csr failed with code {m}")
    return ro, col[:m].copy()


def kronecker(scale: int, edgefactor: int = 16, seed: int = 1):
    """Cleaned, permuted, symmetric Kronecker (R-MAT) graph as int32 CSR."""
    n = 1 << scale
    src, dst = rmat_tuples(scale, edgefactor, seed)
    lib = _load()
    perm = permutation(n, seed)
    lib.gg_apply_permutation(src.shape[0], _ptr(perm), _ptr(src), _ptr(dst))
    return csr_from_tuples(n, src, dst)


def erdos_renyi(scale: int, edgefactor: int = 16, seed: int = 1):
    """Uniform-endpoint graph with the Kronecker graph's n and tuple count."""
    n = 1 << scale
    src, dst = uniform_tuples(n, n * edgefactor, seed)
    return csr_from_tuples(n, src, dst)


def pick_roots(row_offsets: np.ndarray, k: int, seed: int, distinct: bool = True) -> np.ndarray:
    """k seeded vertices with out-degree >= 1 (distinct unless asked otherwise)."""
    lib = _load()
    ro = np.ascontiguousarray(row_offsets, np.int32)
    n = ro.shape[0] - 1
    out = np.empty(max(k, 1), np.int32)
    got = lib.gg_pick_roots(n, _ptr(ro), k, seed, int(distinct), _ptr(out))
    if got < 0:
        raise MemoryError("gg_pick_roots")
    return out[:got].copy()


def num_threads() -> int:
    return int(_load().gg_num_threads())
