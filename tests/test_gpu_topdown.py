"""GPU parity of the single-source top-down BFS against the CPU oracle.

Levels must equal the oracle's bit for bit; parents (not unique, Sec. 3.2
benign race) must pass the oracle's validation rules.  Everything goes
through the C ABI (libgbbfs.so via the ctypes binding).
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    lib_build.build()
    gb.load()


def gpu_bfs(g, root, want_parent=True):
    level, parent = g.run(int(root), want_parent=want_parent)
    torch.cuda.synchronize()
    assert g.status() == gb.BFS_OK, gb.last_error()
    return level.cpu().numpy(), (parent.cpu().numpy() if want_parent else None)


def check_root(g, ro, col, root, expect=None):
    lv, pa = gpu_bfs(g, root)
    ref = oracle.bfs(ro, col, int(root), want_parent=False)[0] if expect is None else expect
    np.testing.assert_array_equal(lv, ref, err_msg=f"levels differ, root {root}")
    rule, bad = oracle.validate(ro, col, int(root), lv, pa, ref)
    assert rule == 0, f"root {root}: {oracle.VALIDATE_RULES[rule]} at vertex {bad}"
    return lv, pa


@pytest.mark.parametrize("case", golden_cases(), ids=lambda c: c["name"])
def test_golden_fixtures(case):
    with gb.Graph(case["row_offsets"], case["col_idx"]) as g:
        check_root(g, case["row_offsets"], case["col_idx"], case["root"], case["levels"])
        if case["bitmap"] is not None:
            np.testing.assert_array_equal(g.visited_bitmap(), np.array(case["bitmap"], np.uint32))


def test_bitmap_layout_matches_levels():
    ro, col = graphgen.kronecker(12, 16, 4)
    r = int(graphgen.pick_roots(ro, 1, 4)[0])
    with gb.Graph(ro, col) as g:
        lv, _ = check_root(g, ro, col, r)
        words = g.visited_bitmap()
    bits = np.unpackbits(words.view(np.uint8), bitorder="little")[: len(lv)]
    np.testing.assert_array_equal(bits.astype(bool), lv >= 0)


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
    with gb.Graph(ro, col) as g:
        check_root(g, ro, col, root, expect)


def test_kronecker_scale16_all_64_roots():
    ro, col = graphgen.kronecker(16, 16, 1)
    roots = graphgen.pick_roots(ro, 64, 1)
    with gb.Graph(ro, col) as g:
        for r in roots:
            check_root(g, ro, col, r)


def test_erdos_renyi_scale16():
    ro, col = graphgen.erdos_renyi(16, 16, 2)
    with gb.Graph(ro, col) as g:
        for r in graphgen.pick_roots(ro, 8, 2):
            check_root(g, ro, col, r)


def test_units_boundaries():
    """Degrees around the unit target T = 2*BLOCK and the hub slice length:
    a root whose neighbours have degrees T-1, T, T+1, 2T, 2T+1, ... exercises
    unit cutting, hub slicing and the last partial slice."""
    for mode, block, T in ((0, 256, 320), (0, 512, 320), (1, 512, 1024)):
        degs = [1, 2, 31, 32, 33, T - 1, T, T + 1, 2 * T - 1, 2 * T, 2 * T + 1, 5 * T + 3]
        edges, nxt = [], 1 + len(degs)
        for i, dgr in enumerate(degs):
            hub = 1 + i
            edges.append((0, hub))
            for _ in range(dgr - 1):
                edges.append((hub, nxt))
                nxt += 1
        ro, col = csr_from_edges(nxt, edges, False)
        with gb.Graph(ro, col, block=block, mode=mode) as g:
            for r in (0, 3, nxt - 1):
                check_root(g, ro, col, r)


def test_dense_clique_shares_bitmap_words():
    n = 200
    e = [(u, v) for u in range(n) for v in range(u + 1, n)]
    ro, col = csr_from_edges(n, e, False)
    with gb.Graph(ro, col) as g:
        for r in (0, 31, 199):
            check_root(g, ro, col, r)


def test_ragged_sizes_and_tails():
    for n in (1, 2, 31, 33, 1000 + 7, 4099):
        ro, col, expect = path_graph(n, n // 3)
        with gb.Graph(ro, col) as g:
            check_root(g, ro, col, n // 3, expect)


def test_empty_graph_and_isolated_root():
    ro = np.zeros(11, np.int32)
    col = np.zeros(0, np.int32)
    with gb.Graph(ro, col) as g:
        lv, pa = gpu_bfs(g, 4)
    expect = np.full(10, -1, np.int32)
    expect[4] = 0
    np.testing.assert_array_equal(lv, expect)
    assert pa[4] == 4 and (pa[np.arange(10) != 4] == -1).all()
    ro, col = graphgen.kronecker(12, 16, 1)
    iso = int(np.where(np.diff(ro) == 0)[0][0])
    with gb.Graph(ro, col) as g:
        lv, pa = gpu_bfs(g, iso)
    assert (lv >= 0).sum() == 1 and lv[iso] == 0 and pa[iso] == iso


def test_directed_uncleaned_graph():
    rng = np.random.default_rng(3)
    n, ne = 5000, 40000
    src = rng.integers(0, n, ne).astype(np.int32)
    dst = rng.integers(0, n, ne).astype(np.int32)
    src[:50] = dst[:50]  # self-loops
    # keep repeats and self-loops: symmetrize=False, no cleaning
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=False, drop_loops=False, dedup=False)
    with gb.Graph(ro, col) as g:
        for r in (0, 1234, 4999):
            check_root(g, ro, col, r)


def test_long_path_many_layers():
    ro, col, expect = path_graph(3000, 0)
    with gb.Graph(ro, col) as g:
        check_root(g, ro, col, 0, expect)


@pytest.mark.parametrize("opts", [
    dict(block=256), dict(block=512, ctas_per_sm=1), dict(max_ctas=1), dict(max_ctas=7, block=256),
    dict(max_ctas=5), dict(layer_stats=1),
    dict(mode=1), dict(mode=1, block=256), dict(mode=1, block=1024), dict(mode=1, warp_degree=1),
    dict(mode=1, warp_degree=64), dict(mode=1, cta_degree=64, segment=256),
    dict(mode=1, cta_degree=100000), dict(mode=1, max_ctas=1), dict(mode=1, max_ctas=7, block=256),
    dict(mode=1, ctas_per_sm=1), dict(mode=1, layer_stats=1),
], ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_options_keep_results_exact(opts):
    ro, col = graphgen.kronecker(14, 16, 6)
    with gb.Graph(ro, col, **opts) as g:
        for k, v in opts.items():
            assert g.get_option(k) == v
        for r in graphgen.pick_roots(ro, 4, 6):
            check_root(g, ro, col, r)


def test_host_outputs_pageable_and_pinned():
    ro, col = graphgen.kronecker(13, 16, 8)
    r = int(graphgen.pick_roots(ro, 1, 8)[0])
    ref = oracle.bfs(ro, col, r, want_parent=False)[0]
    n = len(ro) - 1
    with gb.Graph(ro, col) as g:
        lv = np.empty(n, np.int32)
        pa = np.empty(n, np.int32)
        gb.bfs_run(g.handle, r, lv, pa)
        torch.cuda.synchronize()
        assert g.status() == gb.BFS_OK
        np.testing.assert_array_equal(lv, ref)
        assert oracle.validate(ro, col, r, lv, pa, ref)[0] == 0
        lvp = torch.empty(n, dtype=torch.int32).pin_memory()
        pap = torch.empty(n, dtype=torch.int32).pin_memory()
        gb.bfs_run(g.handle, r, lvp, pap)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(lvp.numpy(), ref)
        assert oracle.validate(ro, col, r, lvp.numpy(), pap.numpy(), ref)[0] == 0


def test_parent_output_optional():
    ro, col = graphgen.kronecker(12, 16, 9)
    r = int(graphgen.pick_roots(ro, 1, 9)[0])
    with gb.Graph(ro, col) as g:
        lv, _ = gpu_bfs(g, r, want_parent=False)
    np.testing.assert_array_equal(lv, oracle.bfs(ro, col, r, want_parent=False)[0])


def test_device_resident_inputs_and_streams():
    ro, col = graphgen.kronecker(13, 16, 10)
    roots = graphgen.pick_roots(ro, 3, 10)
    with gb.Graph(torch.from_numpy(ro).cuda(), torch.from_numpy(col).cuda()) as g:
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        outs = []
        for i, r in enumerate(roots):
            s = s1 if i % 2 == 0 else s2
            with torch.cuda.stream(s):
                lv, pa = g.run(int(r))
                outs.append((r, lv.clone(), pa.clone()))
        torch.cuda.synchronize()
        assert g.status() == gb.BFS_OK
    for r, lv, pa in outs:
        ref = oracle.bfs(ro, col, int(r), want_parent=False)[0]
        np.testing.assert_array_equal(lv.cpu().numpy(), ref)


@pytest.mark.parametrize("mode", [0, 1])
def test_layer_stats_match_table1_columns(mode):
    ro, col = graphgen.kronecker(16, 16, 1)
    with gb.Graph(ro, col, layer_stats=1, mode=mode) as g:
        for r in graphgen.pick_roots(ro, 3, 1):
            lv, _ = check_root(g, ro, col, r)
            v, e, t = g.layer_stats()
            ov, oe, ot = oracle.layer_profile(ro, lv)
            np.testing.assert_array_equal(v, ov)
            np.testing.assert_array_equal(e, oe)
            np.testing.assert_array_equal(t, ot)
            times = g.layer_times()
            assert len(times) == len(v) and np.all(np.diff(times) >= 0) and times[0] > 0


def test_warp_mode_rejects_block_1024():
    ro, col, _ = path_graph(10, 0)
    with gb.Graph(ro, col, block=1024, mode=0) as g:
        with pytest.raises(gb.BfsError) as ei:
            g.run(0)
        assert ei.value.status == gb.BFS_ERR_INVALID_ARG


@pytest.mark.parametrize("mode", [0, 1])
def test_modes_agree_on_kronecker_scale18(mode):
    ro, col = graphgen.kronecker(18, 16, 2)
    with gb.Graph(ro, col, mode=mode) as g:
        for r in graphgen.pick_roots(ro, 6, 2):
            check_root(g, ro, col, r)


def test_invalid_csr_rejected_on_device():
    good_ro = np.array([0, 2, 3, 4], np.int32)
    good_col = np.array([1, 2, 0, 0], np.int32)
    cases = {
        "column out of range": (good_ro, np.array([1, 3, 0, 0], np.int32)),
        "negative column": (good_ro, np.array([1, -1, 0, 0], np.int32)),
        "offsets decrease": (np.array([0, 3, 2, 4], np.int32), good_col),
        "first offset": (np.array([1, 2, 3, 4], np.int32), good_col),
        "last offset": (np.array([0, 2, 3, 3], np.int32), good_col),
    }
    for name, (ro, col) in cases.items():
        with pytest.raises(gb.BfsError) as ei:
            gb.bfs_graph_create(ro, col, 3, 4)
        assert ei.value.status == gb.BFS_ERR_INVALID_GRAPH, name
    h = gb.bfs_graph_create(good_ro, good_col, 3, 4)
    gb.bfs_graph_destroy(h)


def test_bad_root_and_options():
    ro, col, _ = path_graph(10, 0)
    with gb.Graph(ro, col) as g:
        out = torch.empty(10, dtype=torch.int32, device="cuda")
        for bad in (-1, 10):
            with pytest.raises(gb.BfsError) as ei:
                gb.bfs_run(g.handle, bad, out)
            assert ei.value.status == gb.BFS_ERR_INVALID_ARG
        for name, val in (("block", 300), ("cta_degree", 8), ("segment", 10), ("warp_degree", 0)):
            with pytest.raises(gb.BfsError):
                g.set_option(name, val)


def test_bounded_wait_times_out_and_recovers():
    """A barrier limit of 0 ns makes the grid barrier give up: the kernel
    returns, the status reads BFS_ERR_TIMEOUT, and the next run is exact."""
    ro, col = graphgen.kronecker(14, 16, 12)
    r = int(graphgen.pick_roots(ro, 1, 12)[0])
    with gb.Graph(ro, col) as g:
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
    """Mode 0 (the default top-down path): the benchmark's graphs and roots (64 seeded roots of degree
    >= 1, paper Sec. 5.3) in the benchmark's launch configuration; every
    root's levels equal the oracle's and its parents pass the validation."""
    ro, col = big_graph(kind, scale)
    roots = graphgen.pick_roots(ro, 64, 1)[:nroots]
    with gb.Graph(ro, col) as g:
        fails = check_roots(_gpu_run(g), ro, col, roots)
    assert fails == [], fails[:5]
