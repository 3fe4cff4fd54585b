"""Small graph builders for the tests (plain Python/numpy, no BFS arithmetic)."""
import glob
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def csr_from_edges(n, edges, directed):
    """CSR that stores every listed edge exactly as listed (no cleaning);
    undirected edges are stored in both directions.  Row order follows the list."""
    rows = [[] for _ in range(n)]
    for u, v in edges:
        rows[u].append(v)
        if not directed:
            rows[v].append(u)
    ro = np.zeros(n + 1, np.int32)
    for u in range(n):
        ro[u + 1] = ro[u] + len(rows[u])
    col = np.array([v for r in rows for v in r], np.int32)
    return ro, col


def load_golden(path):
    spec = {"edges": [], "levels": None, "bitmap": None, "profile": None}
    section = None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] in ("n", "directed", "root"):
                spec[tok[0]] = int(tok[1])
                section = None
            elif tok[0] in ("edges", "levels", "bitmap", "profile"):
                section = tok[0]
            elif section == "edges":
                spec["edges"].append((int(tok[0]), int(tok[1])))
            elif section == "levels":
                spec["levels"] = (spec["levels"] or []) + [int(t) for t in tok]
            elif section == "bitmap":
                spec["bitmap"] = (spec["bitmap"] or []) + [int(t, 16) for t in tok]
            elif section == "profile":
                assert len(tok) == 3, path
                spec["profile"] = (spec["profile"] or []) + [[int(t) for t in tok]]
    assert len(spec["levels"]) == spec["n"], path
    ro, col = csr_from_edges(spec["n"], spec["edges"], spec["directed"])
    spec["row_offsets"], spec["col_idx"] = ro, col
    spec["levels"] = np.array(spec["levels"], np.int32)
    if spec["profile"] is not None:
        spec["profile"] = np.array(spec["profile"], np.int64)
    spec["name"] = os.path.basename(path)
    return spec


def golden_files():
    return sorted(glob.glob(os.path.join(GOLDEN, "*.txt")))


def golden_cases():
    return [load_golden(p) for p in golden_files() if not p.endswith("README.txt")]


# ---- closed-form families: (row_offsets, col_idx, expected levels) -------

def path_graph(n, root):
    ro, col = csr_from_edges(n, [(i, i + 1) for i in range(n - 1)], False)
    return ro, col, np.abs(np.arange(n) - root).astype(np.int32)


def cycle_graph(n, root):
    ro, col = csr_from_edges(n, [(i, (i + 1) % n) for i in range(n)], False)
    d = np.abs(np.arange(n) - root)
    return ro, col, np.minimum(d, n - d).astype(np.int32)


def grid_graph(w, h, root):
    e = []
    for r in range(h):
        for c in range(w):
            v = r * w + c
            if c + 1 < w:
                e.append((v, v + 1))
            if r + 1 < h:
                e.append((v, v + w))
    ro, col = csr_from_edges(w * h, e, False)
    rr, rc = divmod(root, w)
    lv = np.array([abs(v // w - rr) + abs(v % w - rc) for v in range(w * h)], np.int32)
    return ro, col, lv


def hypercube_graph(d, root):
    n = 1 << d
    e = [(v, v ^ (1 << b)) for v in range(n) for b in range(d) if v < v ^ (1 << b)]
    ro, col = csr_from_edges(n, e, False)
    lv = np.array([bin(v ^ root).count("1") for v in range(n)], np.int32)
    return ro, col, lv


def star_graph(leaves, root):
    n = leaves + 1
    ro, col = csr_from_edges(n, [(0, i) for i in range(1, n)], False)
    if root == 0:
        lv = np.ones(n, np.int32)
        lv[0] = 0
    else:
        lv = np.full(n, 2, np.int32)
        lv[0] = 1
        lv[root] = 0
    return ro, col, lv


def binary_tree(n, root=0):
    e = [((i - 1) // 2, i) for i in range(1, n)]
    ro, col = csr_from_edges(n, e, False)
    assert root == 0
    lv = np.array([int(np.floor(np.log2(i + 1))) for i in range(n)], np.int32)
    return ro, col, lv


def directed_path(n, root):
    """0->1->...->n-1: forward vertices reached at i-root, earlier ones not."""
    ro, col = csr_from_edges(n, [(i, i + 1) for i in range(n - 1)], True)
    lv = np.array([i - root if i >= root else -1 for i in range(n)], np.int32)
    return ro, col, lv


def brute_force_levels(ro, col, root):
    """Unit-weight Bellman-Ford: relax every edge until nothing changes."""
    n = len(ro) - 1
    INF = n + 1
    d = [INF] * n
    d[root] = 0
    changed = True
    while changed:
        changed = False
        for u in range(n):
            if d[u] == INF:
                continue
            for e in range(ro[u], ro[u + 1]):
                v = col[e]
                if d[u] + 1 < d[v]:
                    d[v] = d[u] + 1
                    changed = True
    return np.array([x if x < INF else -1 for x in d], np.int32)


def random_small_graph(rng, n, p, directed):
    e = [(u, v) for u in range(n) for v in range(n) if rng.random() < p]
    if not directed:
        e = [(u, v) for (u, v) in e if u <= v]
    return csr_from_edges(n, e, directed)
