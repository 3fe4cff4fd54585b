"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself:
  * hand-derived fixtures in tests/golden/ (paper Sec. 3 layer definition);
  * closed forms: path, cycle, grid (Manhattan), hypercube (Hamming), star,
    binary tree, directed path;
  * brute-force unit-weight relaxation of every edge on random graphs with
    at most 64 vertices;
  * scipy.sparse.csgraph (breadth-first distances, connected components) on
    seeded Kronecker and Erdos-Renyi graphs;
  * the validator (Sec. 5.3 soft check) accepts independent correct trees and
    rejects each kind of planted mistake;
  * hand-worked per-layer profiles (Table 1 columns: vertices, edges
    scanned, traversed) of five fixtures;
  * mutants of oracle.c (dropped term, wrong index, stack instead of queue,
    wrong root level, wrong parent, lenient validator, edges counted in the
    wrong layer) each fail some pin.
"""
import os
import random

import numpy as np
import pytest

import graphgen
import oracle
from fixtures import (binary_tree, brute_force_levels, cycle_graph, directed_path,
                      golden_cases, grid_graph, hypercube_graph, path_graph,
                      random_small_graph, star_graph)

scipy_sparse = pytest.importorskip("scipy.sparse")
csgraph = pytest.importorskip("scipy.sparse.csgraph")


# ---------------------------------------------------------------------------
# independent helpers (plain Python, no oracle code)

def independent_parent_check(ro, col, root, level, parent):
    """Parent edge exists and parent is one layer up; root is its own parent."""
    n = len(ro) - 1
    if parent[root] != root or level[root] != 0:
        return False
    for v in range(n):
        p = parent[v]
        if v == root:
            continue
        if (p >= 0) != (level[v] >= 0):
            return False
        if p < 0:
            continue
        if v not in set(col[ro[p]:ro[p + 1]].tolist()):
            return False
        if level[p] != level[v] - 1:
            return False
    return True


def tree_from_levels(ro, col, level, root):
    """A correct BFS tree built from exact levels: each vertex takes the first
    in-neighbour one layer up (independent of the oracle's FIFO choice)."""
    n = len(ro) - 1
    parent = np.full(n, -1, np.int32)
    parent[root] = root
    for u in range(n):
        if level[u] < 0:
            continue
        for v in col[ro[u]:ro[u + 1]]:
            if v != root and parent[v] == -1 and level[v] == level[u] + 1:
                parent[v] = u
    return parent


def closed_form_cases():
    cases = []
    for n in (1, 2, 7, 33):
        for r in {0, n // 2, n - 1}:
            cases.append(("path", *path_graph(n, r), r))
    for n in (3, 8, 31):
        for r in (0, n // 3):
            cases.append(("cycle", *cycle_graph(n, r), r))
    cases.append(("grid", *grid_graph(7, 5, 0), 0))
    cases.append(("grid", *grid_graph(7, 5, 17), 17))
    cases.append(("hypercube", *hypercube_graph(6, 0), 0))
    cases.append(("hypercube", *hypercube_graph(6, 45), 45))
    cases.append(("star", *star_graph(40, 0), 0))
    cases.append(("star", *star_graph(40, 7), 7))
    cases.append(("tree", *binary_tree(100), 0))
    cases.append(("dpath", *directed_path(12, 4), 4))
    return cases


def pin_failures(orc):
    """Every pin run against one compiled oracle; returns the failing pins."""
    bad = []
    for c in golden_cases():
        lv, pa = orc.bfs(c["row_offsets"], c["col_idx"], c["root"])
        if not np.array_equal(lv, c["levels"]):
            bad.append("golden:" + c["name"])
        elif not independent_parent_check(c["row_offsets"], c["col_idx"], c["root"], lv, pa):
            bad.append("golden-parent:" + c["name"])
        if c["profile"] is not None:  # hand-worked Table 1 columns, from the fixture's own levels
            v, e, t = orc.layer_profile(c["row_offsets"], c["levels"])
            if not np.array_equal(np.stack([v, e, t], axis=1), c["profile"]):
                bad.append("golden-profile:" + c["name"])
    for name, ro, col, expect, r in closed_form_cases():
        lv, pa = orc.bfs(ro, col, r)
        if not np.array_equal(lv, expect):
            bad.append(f"closed:{name}:{len(ro) - 1}:{r}")
        elif not independent_parent_check(ro, col, r, lv, pa):
            bad.append(f"closed-parent:{name}:{len(ro) - 1}:{r}")
    rng = random.Random(7)
    for i in range(60):
        n = rng.randint(1, 64)
        directed = bool(i % 2)
        ro, col = random_small_graph(rng, n, rng.choice([0.02, 0.05, 0.1, 0.3]), directed)
        r = rng.randrange(n)
        lv, pa = orc.bfs(ro, col, r)
        if not np.array_equal(lv, brute_force_levels(ro, col, r)):
            bad.append(f"brute:{i}")
        elif not independent_parent_check(ro, col, r, lv, pa):
            bad.append(f"brute-parent:{i}")
    # the validator accepts an independent correct tree, rejects planted mistakes
    ro, col, lv, r = *grid_graph(6, 6, 14)[:3], 14
    good = tree_from_levels(ro, col, lv, r)
    if orc.validate(ro, col, r, lv, good, lv)[0] != 0:
        bad.append("validate-accepts")
    for rule, mutate, use_ref in planted_mistakes(ro, col, lv, good, r):
        lv2, pa2 = mutate()
        if orc.validate(ro, col, r, lv2, pa2, lv if use_ref else None)[0] == 0:
            bad.append(f"validate-rejects:{rule}")
    ref = lv.copy()
    ref[int(np.argmax(lv))] = -1
    if orc.validate(ro, col, r, lv, good, ref)[0] != 5:
        bad.append("validate-reached-set")
    return bad


def planted_mistakes(ro, col, lv, pa, root):
    """(rule, thunk) pairs; each thunk returns a (level, parent) with one mistake."""
    n = len(ro) - 1
    far = int(np.argmax(lv))

    def root_parent():
        p = pa.copy()
        p[root] = col[ro[root]]
        return lv.copy(), p

    def missing_edge():
        # give `far` a parent one layer up that is not its neighbour
        p = pa.copy()
        nbrs = set(col[ro[far]:ro[far + 1]].tolist())
        cand = [u for u in range(n) if lv[u] == lv[far] - 1 and u not in nbrs]
        p[far] = cand[0]
        return lv.copy(), p

    def level_skip():
        l2 = lv.copy()
        l2[far] += 1
        return l2, pa.copy()

    def unreached_but_reachable():
        l2, p = lv.copy(), pa.copy()
        l2[far], p[far] = -1, -1
        return l2, p

    def cycle():
        # far's parent now points back at far: a two-cycle in the tree
        l2, p = lv.copy(), pa.copy()
        p[p[far]] = far
        return l2, p

    def all_levels_shifted():
        l2 = lv.copy()
        l2[l2 > 0] += 1
        return l2, pa.copy()

    # (rule, thunk, compare the reached set with the reference?)  The
    # unreached-but-reachable case runs without the reference so that only
    # rule 4 can see it.
    return [(1, root_parent, True), (2, missing_edge, True), (3, level_skip, True),
            (4, unreached_but_reachable, False), (3, cycle, True),
            (3, all_levels_shifted, True)]


# ---------------------------------------------------------------------------
# tests

@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_golden_fixture(case):
    lv, pa = oracle.bfs(case["row_offsets"], case["col_idx"], case["root"])
    np.testing.assert_array_equal(lv, case["levels"])
    assert oracle.validate(case["row_offsets"], case["col_idx"], case["root"], lv, pa,
                           case["levels"]) == (0, -1)


@pytest.mark.parametrize("idx", range(len(closed_form_cases())))
def test_closed_forms(idx):
    name, ro, col, expect, r = closed_form_cases()[idx]
    lv, pa = oracle.bfs(ro, col, r)
    np.testing.assert_array_equal(lv, expect)
    assert independent_parent_check(ro, col, r, lv, pa)
    assert oracle.validate(ro, col, r, lv, pa, expect)[0] == 0


def test_brute_force_relaxation_small_random():
    rng = random.Random(2024)
    for i in range(300):
        n = rng.randint(1, 64)
        directed = bool(i % 2)
        ro, col = random_small_graph(rng, n, rng.choice([0.01, 0.03, 0.06, 0.15, 0.5]), directed)
        r = rng.randrange(n)
        lv, pa = oracle.bfs(ro, col, r)
        np.testing.assert_array_equal(lv, brute_force_levels(ro, col, r))
        assert independent_parent_check(ro, col, r, lv, pa)
        assert oracle.validate(ro, col, r, lv, pa, lv)[0] == 0


def _scipy_levels(ro, col, root, directed):
    n = len(ro) - 1
    a = scipy_sparse.csr_matrix((np.ones(len(col)), col, ro), shape=(n, n))
    d = csgraph.shortest_path(a, method="D", directed=directed, unweighted=True, indices=root)
    return np.where(np.isinf(d), -1, d).astype(np.int32)


@pytest.mark.parametrize("kind,scale", [("kron", 10), ("kron", 12), ("kron", 14), ("er", 12)])
def test_scipy_cross_check(kind, scale):
    ro, col = (graphgen.kronecker if kind == "kron" else graphgen.erdos_renyi)(scale, 16, 3)
    roots = graphgen.pick_roots(ro, 6, 11)
    n = len(ro) - 1
    a = scipy_sparse.csr_matrix((np.ones(len(col)), col, ro), shape=(n, n))
    ncomp, label = csgraph.connected_components(a, directed=False)
    for r in roots:
        lv, pa = oracle.bfs(ro, col, r)
        np.testing.assert_array_equal(lv, _scipy_levels(ro, col, r, False))
        np.testing.assert_array_equal(lv >= 0, label == label[r])  # union-find reach
        assert oracle.validate(ro, col, r, lv, pa, lv)[0] == 0


def test_scipy_directed_random():
    rng = np.random.default_rng(5)
    n, ne = 3000, 9000
    src = rng.integers(0, n, ne).astype(np.int32)
    dst = rng.integers(0, n, ne).astype(np.int32)
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=False)
    for r in (0, 17, 2999):
        lv, pa = oracle.bfs(ro, col, r)
        np.testing.assert_array_equal(lv, _scipy_levels(ro, col, r, True))
        assert oracle.validate(ro, col, r, lv, pa, lv)[0] == 0


def test_validator_rejects_planted_mistakes():
    ro, col, lv = grid_graph(6, 6, 14)
    r = 14
    good = tree_from_levels(ro, col, lv, r)
    assert oracle.validate(ro, col, r, lv, good, lv) == (0, -1)
    for rule, mutate, use_ref in planted_mistakes(ro, col, lv, good, r):
        lv2, pa2 = mutate()
        got, _ = oracle.validate(ro, col, r, lv2, pa2, lv if use_ref else None)
        assert got == rule, (rule, got)


def test_validator_reached_set_rule():
    # a result that is internally consistent but misses a whole component
    # reachable only through... nothing: rule 5 compares with the reference
    ro, col, lv = path_graph(6, 0)
    pa = tree_from_levels(ro, col, lv, 0)
    ref = lv.copy()
    ref[5] = -1  # the reference claims 5 is unreachable
    assert oracle.validate(ro, col, 0, lv, pa, ref)[0] == 5


def test_batch_levels_and_sentinel():
    ro, col, _ = cycle_graph(20, 0)
    roots = np.array([0, 5, 19], np.int32)
    out = oracle.bfs_batch(ro, col, roots)
    assert out.shape == (3, 20) and out.dtype == np.uint8
    for i, r in enumerate(roots):
        np.testing.assert_array_equal(out[i], cycle_graph(20, int(r))[2].astype(np.uint8))
    ro2, col2 = graphgen.csr_from_tuples(6, np.array([0, 3], np.int32), np.array([1, 4], np.int32))
    out = oracle.bfs_batch(ro2, col2, np.array([0, 3], np.int32))
    np.testing.assert_array_equal(out[0], [0, 1, 255, 255, 255, 255])
    np.testing.assert_array_equal(out[1], [255, 255, 255, 0, 1, 255])


def test_batch_depth_overflow():
    ro, col, _ = path_graph(300, 0)
    with pytest.raises(OverflowError):
        oracle.bfs_batch(ro, col, np.array([0], np.int32))
    out = oracle.bfs_batch(ro, col, np.array([150], np.int32))  # depth 150 fits
    assert out[0].max() == 150


def test_golden_layer_profiles():
    """Hand-worked Table 1 columns (tests/golden, 'profile' sections)."""
    cases = [c for c in golden_cases() if c["profile"] is not None]
    assert len(cases) >= 5
    for c in cases:
        v, e, t = oracle.layer_profile(c["row_offsets"], c["levels"])
        np.testing.assert_array_equal(np.stack([v, e, t], axis=1), c["profile"], err_msg=c["name"])


def test_layer_profile_table1_invariants():
    ro, col = graphgen.kronecker(16, 16, 1)
    for r in graphgen.pick_roots(ro, 4, 2):
        lv, _ = oracle.bfs(ro, col, r, want_parent=False)
        v, e, t = oracle.layer_profile(ro, lv)
        deg = np.diff(ro)
        assert v[0] == 1 and v.sum() == (lv >= 0).sum()
        np.testing.assert_array_equal(t[:-1], v[1:])          # Table 1: next layer = traversed
        assert t[-1] == 0
        assert e.sum() == deg[lv >= 0].sum()
        # shape of Table 1: a few layers, the bulk of edges in the middle ones
        assert 3 <= len(v) <= 16
        assert e[np.argsort(e)[-2:]].sum() > 0.8 * e.sum()


def test_bad_root_rejected():
    ro, col, _ = path_graph(4, 0)
    with pytest.raises(ValueError):
        oracle.bfs(ro, col, 4)
    with pytest.raises(ValueError):
        oracle.bfs(ro, col, -1)


def test_pins_hold_for_the_oracle():
    assert pin_failures(oracle.default()) == []


MUTANTS = [
    ("dropped +1", "level[v] = level[u] + 1;", "level[v] = level[u];"),
    ("last neighbour skipped", "e < row_offsets[u + 1]; ++e) {\n            int32_t v = col_idx[e];\n            if (level[v] == -1)",
     "e < row_offsets[u + 1] - 1; ++e) {\n            int32_t v = col_idx[e];\n            if (level[v] == -1)"),
    ("row start off by one", "for (int64_t e = row_offsets[u]; e < row_offsets[u + 1]; ++e) {\n            int32_t v = col_idx[e];\n            if (level[v] == -1)",
     "for (int64_t e = row_offsets[u] + 1; e < row_offsets[u + 1]; ++e) {\n            int32_t v = col_idx[e];\n            if (level[v] == -1)"),
    ("stack instead of queue", "int32_t u = queue[head++];", "int32_t u = queue[--tail];"),
    ("root level 1", "level[root] = 0;\n    if (parent) parent[root] = root;\n    queue",
     "level[root] = 1;\n    if (parent) parent[root] = root;\n    queue"),
    ("parent is self", "if (parent) parent[v] = u;", "if (parent) parent[v] = v;"),
    ("validator drops rule 4", "if (level[v] < 0 || level[v] > level[u] + 1)", "if (0)"),
    ("validator rule 3 sign", "level[parent[v]] != level[v] - 1", "level[parent[v]] != level[v] + 1"),
    ("validator skips edge check", "if (parent[v] == u) found[v] = 1;", "found[v] = 1;"),
    ("validator drops rule 5", "if ((level[v] >= 0) != (ref_level[v] >= 0))", "if (0)"),
    ("validator drops root check", "if (parent[root] != root || level[root] != 0)", "if (0)"),
    ("profile edges counted at d+1", "edges[d] += row_offsets[v + 1] - row_offsets[v];",
     "if (d + 1 < max_layers) edges[d + 1] += row_offsets[v + 1] - row_offsets[v];"),
    ("profile edges only for d > 0", "edges[d] += row_offsets[v + 1] - row_offsets[v];",
     "if (d > 0) edges[d] += row_offsets[v + 1] - row_offsets[v];"),
    ("profile edges of unreached vertices", "if (d < 0) continue;\n        if (d >= max_layers)",
     "if (d < 0) { edges[0] += row_offsets[v + 1] - row_offsets[v]; continue; }\n        if (d >= max_layers)"),
    ("profile edges counted once per vertex", "edges[d] += row_offsets[v + 1] - row_offsets[v];",
     "edges[d] += 1;"),
    ("profile traversed at d", "if (d > 0) traversed[d - 1] += 1;", "traversed[d] += 1;"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutants_are_caught(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    assert src.count(old) == 1, name
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(mpath), str(tmp_path / "libmutant.so"))
    assert pin_failures(oracle.Oracle(lib)) != [], name
