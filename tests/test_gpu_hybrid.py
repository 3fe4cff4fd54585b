"""GPU parity of the direction-optimising search (mode 3).

Layers run top-down or bottom-up (every unvisited vertex looks for a parent
in the frontier bitmap); the results must not depend on the choice.  Levels
equal the oracle's bit for bit and parents pass its validation, whatever the
switching parameters.  The parameters below pin four regimes: the default
(alpha 14, beta 24); bottom-up from the first layer whose frontier has any
edge, never back (alpha, beta huge); a switch at every layer, which runs
both conversions (queue -> bitmap, bitmap -> queue) again and again (alpha
huge, beta 1); and top-down only (alpha 0).
"""
import numpy as np
import pytest

import graphgen
import oracle
from parity_pool import big_graph, check_roots
from fixtures import (binary_tree, csr_from_edges, cycle_graph, golden_cases, grid_graph,
                      hypercube_graph, path_graph, star_graph)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1604_02844_gb300 as gb  # noqa: E402
from paper_1604_02844_gb300 import build as lib_build  # noqa: E402

HYB = gb.MODE_HYBRID
BIG = 1 << 30
REGIMES = {
    "default": dict(alpha=14, beta=24),
    "bottom_up": dict(alpha=BIG, beta=BIG),
    "alternate": dict(alpha=BIG, beta=1),
    "top_down": dict(alpha=0, beta=24),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib_build.build()
    gb.load()


def check_root(g, ro, col, root, expect=None):
    level, parent = g.run(int(root))
    torch.cuda.synchronize()
    assert g.status() == gb.BFS_OK, gb.last_error()
    lv, pa = level.cpu().numpy(), parent.cpu().numpy()
    ref = oracle.bfs(ro, col, int(root), want_parent=False)[0] if expect is None else expect
    np.testing.assert_array_equal(lv, ref, err_msg=f"levels differ, root {root}")
    rule, bad = oracle.validate(ro, col, int(root), lv, pa, ref)
    assert rule == 0, f"root {root}: {oracle.VALIDATE_RULES[rule]} at vertex {bad}"
    return lv, pa


@pytest.mark.parametrize("regime", REGIMES)
@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_golden_fixtures(case, regime):
    with gb.Graph(case["row_offsets"], case["col_idx"], mode=HYB, **REGIMES[regime]) as g:
        check_root(g, case["row_offsets"], case["col_idx"], case["root"], case["levels"])
        if case["bitmap"] is not None:
            np.testing.assert_array_equal(g.visited_bitmap(), np.array(case["bitmap"], np.uint32))


CLOSED = [
    ("path", lambda: path_graph(1000, 613), 613),
    ("cycle", lambda: cycle_graph(4097, 5), 5),
    ("grid", lambda: grid_graph(300, 200, 30123), 30123),
    ("hypercube", lambda: hypercube_graph(14, 12345), 12345),
    ("star-hub", lambda: star_graph(300000, 0), 0),
    ("star-leaf", lambda: star_graph(300000, 77), 77),
    ("tree", lambda: binary_tree(70000), 0),
]


@pytest.mark.parametrize("regime", REGIMES)
@pytest.mark.parametrize("name,make,root", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(name, make, root, regime):
    ro, col, expect = make()
    with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
        check_root(g, ro, col, root, expect)


def test_kronecker_scale16_all_64_roots():
    ro, col = graphgen.kronecker(16, 16, 1)
    with gb.Graph(ro, col, mode=HYB) as g:
        for r in graphgen.pick_roots(ro, 64, 1):
            check_root(g, ro, col, r)


@pytest.mark.parametrize("regime", REGIMES)
def test_kronecker_and_erdos_renyi_regimes(regime):
    for kind, seed in (("kronecker", 3), ("erdos_renyi", 4)):
        ro, col = getattr(graphgen, kind)(15, 16, seed)
        with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
            for r in graphgen.pick_roots(ro, 6, seed):
                check_root(g, ro, col, r)


def test_cliques_and_shared_leaves():
    for n in (64, 1500):
        e = [(u, v) for u in range(n) for v in range(u + 1, n)]
        ro, col = csr_from_edges(n, e, False)
        for regime in ("default", "bottom_up", "alternate"):
            with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
                for r in (0, n - 1):
                    check_root(g, ro, col, r)
    leaves = 100_000
    e = [(0, 1)] + [(0, 2 + i) for i in range(leaves)] + [(1, 2 + i) for i in range(leaves)]
    ro, col = csr_from_edges(leaves + 2, e, False)
    for regime in REGIMES:
        with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
            for r in (0, 2, leaves + 1):
                check_root(g, ro, col, r)


@pytest.mark.parametrize("regime", REGIMES)
def test_directed_graph_bottom_up_on_in_edges(regime):
    """On a directed graph the bottom-up layers scan in-edges (a transposed
    CSR built on first use)."""
    rng = np.random.default_rng(3)
    n, ne = 5000, 40000
    src = rng.integers(0, n, ne).astype(np.int32)
    dst = rng.integers(0, n, ne).astype(np.int32)
    src[:50] = dst[:50]
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=False, drop_loops=False, dedup=False)
    with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
        for r in (0, 1234, 4999):
            check_root(g, ro, col, r)


def test_directed_star_reached_through_in_edges():
    """Edges hub -> leaf only: the leaves have no out-edge (they sort last in
    the degree order), so a bottom-up layer finds them by their in-edges alone."""
    leaves = 20000
    e = [(0, 1 + i) for i in range(leaves)] + [(1 + i, 1 + leaves) for i in range(0, leaves, 7)]
    ro, col = csr_from_edges(leaves + 2, e, True)
    for regime in ("bottom_up", "alternate", "default"):
        with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
            for r in (0, 1, 8):
                check_root(g, ro, col, r)


def test_directed_bottom_up_layers_ran():
    """Forced bottom-up on a directed Kronecker-shaped graph: some layer's
    examined edges differ from the top-down count, so the in-edge path ran."""
    tup_src, tup_dst = graphgen.rmat_tuples(14, 16, 37)
    n = 1 << 14
    ro, col = graphgen.csr_from_tuples(n, tup_src, tup_dst, symmetrize=False, drop_loops=True, dedup=True)
    with gb.Graph(ro, col, mode=HYB, layer_stats=1, **REGIMES["bottom_up"]) as g:
        for r in graphgen.pick_roots(ro, 3, 37):
            lv, _ = check_root(g, ro, col, r)
            v, e, t = g.layer_stats()
            ov, oe, ot = oracle.layer_profile(ro, lv)
            np.testing.assert_array_equal(v, ov)
            np.testing.assert_array_equal(t, ot)
            if len(e) > 1:
                assert (e != oe).any()


def test_uncleaned_symmetric_graph():
    """Self-loops and repeated edges, symmetric: bottom-up is allowed."""
    rng = np.random.default_rng(5)
    n, ne = 6000, 50000
    src = rng.integers(0, n, ne).astype(np.int32)
    dst = rng.integers(0, n, ne).astype(np.int32)
    src[:60] = dst[:60]
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=True, drop_loops=False, dedup=False)
    for regime in REGIMES:
        with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
            for r in (0, 77, 5999):
                check_root(g, ro, col, r)


def test_ragged_sizes_empty_and_isolated():
    for n in (1, 2, 31, 33, 1007, 4099):
        ro, col, expect = path_graph(n, n // 3)
        for regime in ("bottom_up", "alternate"):
            with gb.Graph(ro, col, mode=HYB, **REGIMES[regime]) as g:
                check_root(g, ro, col, n // 3, expect)
    ro = np.zeros(11, np.int32)
    with gb.Graph(ro, np.zeros(0, np.int32), mode=HYB) as g:
        expect = np.full(10, -1, np.int32)
        expect[4] = 0
        lv, pa = check_root(g, ro, np.zeros(0, np.int32), 4, expect)
        assert pa[4] == 4


@pytest.mark.parametrize("opts", [dict(block=256), dict(max_ctas=1), dict(max_ctas=7, block=256),
                                  dict(ctas_per_sm=1), dict(layer_stats=1)],
                         ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_options_keep_results_exact(opts):
    ro, col = graphgen.kronecker(14, 16, 6)
    for regime in ("default", "alternate"):
        with gb.Graph(ro, col, mode=HYB, **REGIMES[regime], **opts) as g:
            for r in graphgen.pick_roots(ro, 3, 6):
                check_root(g, ro, col, r)


@pytest.mark.parametrize("regime", REGIMES)
def test_layer_stats(regime):
    """Frontier sizes and new vertices per layer are the Table 1 columns of
    the oracle.  A layer examines either the frontier's edges (top-down) or
    at most the edges of the vertices still unvisited (bottom-up); top-down
    only gives the oracle's edge column, and the default regime examines
    fewer edges in total."""
    ro, col = graphgen.kronecker(16, 16, 1)
    deg = np.diff(ro).astype(np.int64)
    with gb.Graph(ro, col, layer_stats=1, mode=HYB, **REGIMES[regime]) as g:
        for r in graphgen.pick_roots(ro, 3, 1):
            lv, _ = check_root(g, ro, col, r)
            v, e, t = g.layer_stats()
            ov, oe, ot = oracle.layer_profile(ro, lv)
            np.testing.assert_array_equal(v, ov)
            np.testing.assert_array_equal(t, ot)
            for d in range(len(e)):
                unvisited = (lv > d) | (lv < 0)
                assert e[d] <= max(oe[d], deg[unvisited].sum()), d
            if regime == "top_down":
                np.testing.assert_array_equal(e, oe)
            if regime == "default":
                assert e.sum() < oe.sum()


def test_modes_alternate_on_one_graph():
    ro, col = graphgen.kronecker(15, 16, 5)
    roots = graphgen.pick_roots(ro, 8, 5)
    with gb.Graph(ro, col) as g:
        for i, r in enumerate(roots):
            g.set_option("mode", (HYB, 0, gb.MODE_RESTORE, HYB)[i % 4])
            check_root(g, ro, col, r)


def test_option_errors_and_timeout_recovery():
    ro, col = graphgen.kronecker(14, 16, 12)
    r = int(graphgen.pick_roots(ro, 1, 12)[0])
    with gb.Graph(ro, col, mode=HYB) as g:
        for name, val in (("alpha", -1), ("beta", 0), ("alpha", (1 << 30) + 1), ("mode", 5)):
            with pytest.raises(gb.BfsError):
                g.set_option(name, val)
        assert g.get_option("alpha") == 14 and g.get_option("beta") == 24
        g.set_option("block", 1024)
        with pytest.raises(gb.BfsError) as ei:
            g.run(r)
        assert ei.value.status == gb.BFS_ERR_INVALID_ARG
        g.set_option("block", 512)
        g.set_option("timeout_ns", 0)
        g.run(r)
        torch.cuda.synchronize()
        with pytest.raises(gb.BfsError) as ei:
            g.status()
        assert ei.value.status == gb.BFS_ERR_TIMEOUT
        g.set_option("timeout_ns", 4_000_000_000)
        check_root(g, ro, col, r)


def _gpu_run(g):
    def run(r):
        level, parent = g.run(int(r))
        torch.cuda.synchronize()
        assert g.status() == gb.BFS_OK, gb.last_error()
        return level.cpu().numpy(), parent.cpu().numpy()
    return run


@pytest.mark.parametrize("kind,scale,nroots", [("kronecker", 20, 64), ("kronecker", 22, 64),
                                                 ("kronecker", 24, 64), ("erdos_renyi", 24, 64)])
def test_full_size_every_root(kind, scale, nroots):
    """Mode 3 (direction-optimising): the benchmark's graphs and roots (64 seeded roots of degree
    >= 1, paper Sec. 5.3) in the benchmark's launch configuration; every
    root's levels equal the oracle's and its parents pass the validation."""
    ro, col = big_graph(kind, scale)
    roots = graphgen.pick_roots(ro, 64, 1)[:nroots]
    with gb.Graph(ro, col, mode=HYB) as g:
        fails = check_roots(_gpu_run(g), ro, col, roots)
    assert fails == [], fails[:5]
