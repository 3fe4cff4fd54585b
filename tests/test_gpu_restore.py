"""GPU parity of the atomic-free top-down BFS (mode 2: Alg. 3, Sec. 3.3.2).

Pass B sets the output bitmap with plain read-modify-writes, so bits of
vertices sharing a word are lost whenever two warps race on it; the
per-layer restoration pass must bring every one of them back from P.  The
results must be those of the atomic path: levels equal to the oracle's bit
for bit, parents passing the oracle's validation.  Graphs whose vertices
crowd into few bitmap words (cliques, stars, hubs) make the races frequent.
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

RST = gb.MODE_RESTORE


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


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_golden_fixtures(case):
    with gb.Graph(case["row_offsets"], case["col_idx"], mode=RST) as g:
        check_root(g, case["row_offsets"], case["col_idx"], case["root"], case["levels"])
        if case["bitmap"] is not None:  # the visited bitmap after restoration
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


@pytest.mark.parametrize("name,make,root", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(name, make, root):
    ro, col, expect = make()
    with gb.Graph(ro, col, mode=RST) as g:
        check_root(g, ro, col, root, expect)


def test_cliques_race_on_every_word():
    """In a clique every vertex of layer 1 is set by every warp that holds a
    slice of the root's list at once: all 32 bits of a word race."""
    for n in (64, 200, 1500):
        e = [(u, v) for u in range(n) for v in range(u + 1, n)]
        ro, col = csr_from_edges(n, e, False)
        with gb.Graph(ro, col, mode=RST) as g:
            for r in (0, 31, n - 1):
                check_root(g, ro, col, r)


def test_two_hubs_share_all_leaves():
    """Two adjacent hubs with the same 100,000 leaves: in layer 2 the
    leaves are set from both hubs' slices at once."""
    leaves = 100_000
    e = [(0, 1)] + [(0, 2 + i) for i in range(leaves)] + [(1, 2 + i) for i in range(leaves)]
    ro, col = csr_from_edges(leaves + 2, e, False)
    with gb.Graph(ro, col, mode=RST) as g:
        for r in (0, 2, leaves + 1):
            check_root(g, ro, col, r)


def test_kronecker_scale16_all_64_roots():
    ro, col = graphgen.kronecker(16, 16, 1)
    with gb.Graph(ro, col, mode=RST) as g:
        for r in graphgen.pick_roots(ro, 64, 1):
            check_root(g, ro, col, r)


def test_erdos_renyi_and_directed_graphs():
    ro, col = graphgen.erdos_renyi(16, 16, 2)
    with gb.Graph(ro, col, mode=RST) as g:
        for r in graphgen.pick_roots(ro, 8, 2):
            check_root(g, ro, col, r)
    rng = np.random.default_rng(3)
    n, ne = 5000, 40000
    src = rng.integers(0, n, ne).astype(np.int32)
    dst = rng.integers(0, n, ne).astype(np.int32)
    src[:50] = dst[:50]
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=False, drop_loops=False, dedup=False)
    with gb.Graph(ro, col, mode=RST) as g:
        for r in (0, 1234, 4999):
            check_root(g, ro, col, r)


def test_ragged_sizes_empty_and_isolated():
    for n in (1, 2, 31, 33, 1007, 4099):
        ro, col, expect = path_graph(n, n // 3)
        with gb.Graph(ro, col, mode=RST) as g:
            check_root(g, ro, col, n // 3, expect)
    ro = np.zeros(11, np.int32)
    with gb.Graph(ro, np.zeros(0, np.int32), mode=RST) as g:
        expect = np.full(10, -1, np.int32)
        expect[4] = 0
        lv, pa = check_root(g, ro, np.zeros(0, np.int32), 4, expect)
        assert pa[4] == 4


def test_units_boundaries():
    T = 320
    degs = [1, 2, 31, 32, 33, T - 1, T, T + 1, 2 * T - 1, 2 * T, 2 * T + 1, 5 * T + 3]
    edges, nxt = [], 1 + len(degs)
    for i, dgr in enumerate(degs):
        hub = 1 + i
        edges.append((0, hub))
        for _ in range(dgr - 1):
            edges.append((hub, nxt))
            nxt += 1
    ro, col = csr_from_edges(nxt, edges, False)
    for block in (256, 512):
        with gb.Graph(ro, col, block=block, mode=RST) as g:
            for r in (0, 3, nxt - 1):
                check_root(g, ro, col, r)


@pytest.mark.parametrize("opts", [
    dict(block=256), dict(block=512, ctas_per_sm=1), dict(max_ctas=1), dict(max_ctas=7, block=256),
    dict(layer_stats=1),
], ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_options_keep_results_exact(opts):
    ro, col = graphgen.kronecker(14, 16, 6)
    with gb.Graph(ro, col, mode=RST, **opts) as g:
        for r in graphgen.pick_roots(ro, 4, 6):
            check_root(g, ro, col, r)


def test_layer_stats_match_table1_columns():
    ro, col = graphgen.kronecker(16, 16, 1)
    with gb.Graph(ro, col, layer_stats=1, mode=RST) as g:
        for r in graphgen.pick_roots(ro, 3, 1):
            lv, _ = check_root(g, ro, col, r)
            v, e, t = g.layer_stats()
            ov, oe, ot = oracle.layer_profile(ro, lv)
            np.testing.assert_array_equal(v, ov)
            np.testing.assert_array_equal(e, oe)
            np.testing.assert_array_equal(t, ot)


def test_modes_alternate_on_one_graph():
    """Switching between the atomic and the restoration path reuses the
    graph's workspace; each run starts from its own initialisation."""
    ro, col = graphgen.kronecker(15, 16, 5)
    roots = graphgen.pick_roots(ro, 6, 5)
    with gb.Graph(ro, col) as g:
        for i, r in enumerate(roots):
            g.set_option("mode", (0, RST, 1)[i % 3])
            check_root(g, ro, col, r)


def test_rejects_block_1024_and_recovers_from_timeout():
    ro, col, _ = path_graph(10, 0)
    with gb.Graph(ro, col, block=1024, mode=RST) as g:
        with pytest.raises(gb.BfsError) as ei:
            g.run(0)
        assert ei.value.status == gb.BFS_ERR_INVALID_ARG
    ro, col = graphgen.kronecker(14, 16, 12)
    r = int(graphgen.pick_roots(ro, 1, 12)[0])
    with gb.Graph(ro, col, mode=RST) as g:
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
                                                 ("kronecker", 24, 64), ("erdos_renyi", 24, 16)])
def test_full_size_every_root(kind, scale, nroots):
    """Mode 2 (Alg. 3 restoration): the benchmark's graphs and roots (64 seeded roots of degree
    >= 1, paper Sec. 5.3) in the benchmark's launch configuration; every
    root's levels equal the oracle's and its parents pass the validation."""
    ro, col = big_graph(kind, scale)
    roots = graphgen.pick_roots(ro, 64, 1)[:nroots]
    with gb.Graph(ro, col, mode=RST) as g:
        fails = check_roots(_gpu_run(g), ro, col, roots)
    assert fails == [], fails[:5]
