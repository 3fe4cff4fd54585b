"""Every-root parity at full size: GPU searches checked against the oracle on
the host cores in parallel.

The oracle (plain single-threaded C) is called from host threads; ctypes
releases the GIL for the length of each call, so up to `workers` oracle
searches and validations run at once while the GPU computes the next roots.
Nothing here computes a BFS: the GPU results come from the caller's `run`,
the expected levels and the validation from `oracle`.
"""
import concurrent.futures as cf
import functools
import os

import numpy as np

import graphgen
import oracle


@functools.lru_cache(maxsize=4)
def big_graph(kind, scale, edgefactor=16, seed=1):
    """A seeded full-size input graph, generated once per test session."""
    ro, col = getattr(graphgen, kind)(scale, edgefactor, seed)
    ro.setflags(write=False)
    col.setflags(write=False)
    return ro, col


def host_workers():
    return max(1, min(16, os.cpu_count() or 1))


def check_roots(run, ro, col, roots, workers=None):
    """run(root) -> (level, parent) as host int32 arrays from the GPU.  Every
    root's levels must equal the oracle's bit for bit and its parents must
    pass the oracle's validation (rules 1-5 of the Sec. 5.3 soft check, the
    reached set against the oracle's).  Returns the failures (empty: all
    roots exact)."""
    workers = workers or host_workers()

    def check(r, lv, pa):
        ref = oracle.bfs(ro, col, r, want_parent=False)[0]
        if not np.array_equal(lv, ref):
            bad = np.flatnonzero(lv != ref)
            return f"root {r}: {len(bad)} levels differ, first at vertex {bad[0]}"
        rule, v = oracle.validate(ro, col, r, lv, pa, ref)
        if rule:
            return f"root {r}: {oracle.VALIDATE_RULES[rule]} at vertex {v}"
        return None

    fails, pending = [], []
    with cf.ThreadPoolExecutor(workers) as ex:
        for r in roots:
            lv, pa = run(int(r))
            pending.append(ex.submit(check, int(r), lv, pa))
            if len(pending) >= 2 * workers:  # bound the host arrays held at once
                fails += [f for f in (p.result() for p in pending[:workers]) if f]
                pending = pending[workers:]
        fails += [f for f in (p.result() for p in pending) if f]
    return fails
