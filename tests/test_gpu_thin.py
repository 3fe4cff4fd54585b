"""GPU parity of bfs_run mode 4 (thin warps) against the CPU oracle.

Mode 4 runs the layer step of Alg. 2 with the atomic visited bitmap of
Listing 1, like mode 0, but with more, lighter warps that read each work
item's adjacency straight from memory (lane -> list by ballots) and claim
each candidate at once.  Levels must equal the
oracle's bit for bit; parents (not unique, Sec. 3.2) must pass the oracle's
validation.  Everything goes through the C ABI.
"""
import numpy as np
import pytest

import graphgen
import oracle
from fixtures import (binary_tree, csr_from_edges, cycle_graph, golden_cases, grid_graph,
                      hypercube_graph, path_graph, star_graph)
from parity_pool import big_graph, check_roots

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1604_02844_gb300 as gb  # noqa: E402
from paper_1604_02844_gb300 import build as lib_build  # noqa: E402

THIN = 4


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
    with gb.Graph(case["row_offsets"], case["col_idx"], mode=THIN) as g:
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


@pytest.mark.parametrize("name,make,root", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(name, make, root):
    ro, col, expect = make()
    with gb.Graph(ro, col, mode=THIN) as g:
        check_root(g, ro, col, root, expect)


def test_units_slices_and_steps():
    """Degrees around the 32-entry step, the unit target and the hub slice
    length (320): unit cutting, slicing, the last partial slice and steps that
    span several lists."""
    T = 320
    degs = [1, 2, 31, 32, 33, 127, 128, 129, T - 1, T, T + 1, 2 * T - 1, 2 * T, 2 * T + 1, 5 * T + 3]
    edges, nxt = [], 1 + len(degs)
    for i, dgr in enumerate(degs):
        hub = 1 + i
        edges.append((0, hub))
        for _ in range(dgr - 1):
            edges.append((hub, nxt))
            nxt += 1
    ro, col = csr_from_edges(nxt, edges, False)
    with gb.Graph(ro, col, mode=THIN) as g:
        for r in (0, 3, 9, nxt - 1):
            check_root(g, ro, col, r)


def test_dense_clique_and_ragged_paths():
    n = 200
    ro, col = csr_from_edges(n, [(u, v) for u in range(n) for v in range(u + 1, n)], False)
    with gb.Graph(ro, col, mode=THIN) as g:
        for r in (0, 31, 199):
            check_root(g, ro, col, r)
    for n in (1, 2, 31, 33, 1007, 4099):
        ro, col, expect = path_graph(n, n // 3)
        with gb.Graph(ro, col, mode=THIN) as g:
            check_root(g, ro, col, n // 3, expect)


def test_directed_uncleaned_graph():
    rng = np.random.default_rng(5)
    n = 3000
    src = rng.integers(0, n, 20000).astype(np.int32)
    dst = rng.integers(0, n, 20000).astype(np.int32)
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=False, drop_loops=False, dedup=False)
    with gb.Graph(ro, col, mode=THIN) as g:
        for r in (0, 17, 2999):
            check_root(g, ro, col, r)


def test_kronecker_scale16_all_64_roots_and_layer_stats():
    ro, col = graphgen.kronecker(16, 16, 1)
    roots = graphgen.pick_roots(ro, 64, 1)
    with gb.Graph(ro, col, mode=THIN) as g:
        for r in roots:
            check_root(g, ro, col, r)
        g.set_option("layer_stats", 1)
        for r in roots[:3]:
            lv, _ = check_root(g, ro, col, r)
            v, e, t = g.layer_stats()
            ov, oe, ot = oracle.layer_profile(ro, lv)
            np.testing.assert_array_equal(v, ov)
            np.testing.assert_array_equal(e, oe)
            np.testing.assert_array_equal(t, ot)


def test_limited_grid_and_host_outputs():
    ro, col = graphgen.kronecker(15, 16, 3)
    roots = graphgen.pick_roots(ro, 4, 3)
    n = len(ro) - 1
    for opts in (dict(max_ctas=1), dict(max_ctas=7), dict(ctas_per_sm=1)):
        with gb.Graph(ro, col, mode=THIN, **opts) as g:
            for r in roots:
                check_root(g, ro, col, r)
    with gb.Graph(ro, col, mode=THIN) as g:
        lv = torch.empty(n, dtype=torch.int32).pin_memory()
        pa = torch.empty(n, dtype=torch.int32).pin_memory()
        gb.bfs_run(g.handle, int(roots[0]), lv, pa, None)
        torch.cuda.synchronize()
        g.status()
        ref = oracle.bfs(ro, col, int(roots[0]), want_parent=False)[0]
        np.testing.assert_array_equal(lv.numpy(), ref)
        assert oracle.validate(ro, col, int(roots[0]), lv.numpy(), pa.numpy(), ref)[0] == 0


def test_bounded_wait_times_out_and_recovers():
    ro, col = graphgen.kronecker(14, 16, 12)
    r = int(graphgen.pick_roots(ro, 1, 12)[0])
    with gb.Graph(ro, col, mode=THIN) as g:
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
    """The benchmark's graphs and roots (64 seeded roots of degree >= 1,
    paper Sec. 5.3): every root's levels equal the oracle's and its parents
    pass the validation."""
    ro, col = big_graph(kind, scale)
    roots = graphgen.pick_roots(ro, 64, 1)[:nroots]
    with gb.Graph(ro, col, mode=THIN) as g:
        fails = check_roots(_gpu_run(g), ro, col, roots)
    assert fails == [], fails[:5]
