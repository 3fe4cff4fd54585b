"""The serving loop (bfs_server_*): continuous batching over resident graphs.

Each query's levels must be the same whether it ran alone or in a mixed
stream that arrived while other queries were on the GPU (exact: the search
is integer), and equal to the oracle's.
"""
import random
import threading
import time

import numpy as np
import pytest

import graphgen
import oracle

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


@pytest.fixture(scope="module")
def resident():
    specs = [("kron", 12, 8), ("kron", 14, 16), ("kron", 16, 16), ("er", 13, 16)]
    out = []
    for kind, scale, ef in specs:
        ro, col = (graphgen.kronecker if kind == "kron" else graphgen.erdos_renyi)(scale, ef, 50 + scale)
        out.append((ro, col, gb.Graph(ro, col)))
    yield out
    for _, _, g in out:
        g.close()


def make_queries(resident, k, seed):
    rng = random.Random(seed)
    qs = []
    for _ in range(k):
        gi = rng.randrange(len(resident))
        ro = resident[gi][0]
        r = int(graphgen.pick_roots(ro, 1, rng.randrange(1 << 30))[0])
        qs.append((gi, r))
    return qs


def run_alone(server, ids, resident, queries):
    res = []
    for gi, r in queries:
        buf = np.empty(len(resident[gi][0]) - 1, np.uint8)
        t = server.submit(ids[gi], r, buf)
        server.wait(t)
        res.append(buf)
    return res


def run_mixed(server, ids, resident, queries, seed):
    bufs = [np.empty(len(resident[gi][0]) - 1, np.uint8) for gi, _ in queries]
    tickets = [None] * len(queries)
    rng = random.Random(seed)

    def producer():
        for i, (gi, r) in enumerate(queries):
            tickets[i] = server.submit(ids[gi], r, bufs[i])
            if rng.random() < 0.3:
                time.sleep(rng.random() * 0.002)  # arrivals while others run

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    server.drain()
    for t in tickets:
        assert server.poll(t)
    return bufs, tickets


def test_alone_and_mixed_results_are_identical(resident):
    queries = make_queries(resident, 160, 1)
    with gb.Server() as s:
        ids = [s.add_graph(g) for _, _, g in resident]
        alone = run_alone(s, ids, resident, queries[:40])
        mixed, tickets = run_mixed(s, ids, resident, queries, 2)
        for i in range(40):
            np.testing.assert_array_equal(alone[i], mixed[i], err_msg=f"query {i}")
        for i, (gi, r) in enumerate(queries):
            ro, col, _ = resident[gi]
            ref = oracle.bfs_batch(ro, col, np.array([r], np.int32))[0]
            np.testing.assert_array_equal(mixed[i], ref, err_msg=f"query {i} graph {gi}")
        for t in tickets:
            t0, t1 = s.times(t)
            assert t1 >= t0 > 0


def test_tight_budget_admits_one_workspace_at_a_time(resident):
    # room for the largest workspace only: graphs take turns
    queries = make_queries(resident, 60, 3)
    budget = 14 << 20  # the scale-16 workspace (~13.7 MB) fits only alone
    with gb.Server(budget) as s:
        ids = [s.add_graph(g) for _, _, g in resident]
        mixed, _ = run_mixed(s, ids, resident, queries, 4)
    for i, (gi, r) in enumerate(queries):
        ro, col, _ = resident[gi]
        np.testing.assert_array_equal(mixed[i], oracle.bfs_batch(ro, col, np.array([r], np.int32))[0])


def test_submit_errors(resident):
    with gb.Server(1 << 20) as s:  # 1 MiB: no workspace fits
        gid = s.add_graph(resident[2][2])
        buf = np.empty(len(resident[2][0]) - 1, np.uint8)
        with pytest.raises(gb.BfsError) as ei:
            s.submit(gid, 0, buf)
        assert ei.value.status == gb.BFS_ERR_BUSY
        with pytest.raises(gb.BfsError):
            s.submit(gid + 5, 0, buf)
        with pytest.raises(gb.BfsError):
            gb.bfs_poll(s.handle, 12345)


def test_device_timeout_fails_queries_without_hanging():
    """Device waits limited to 0 ns: the graph's batched search gives up at
    its first grid barrier.  The server reports BFS_ERR_TIMEOUT for every
    query instead of leaving callers waiting, refuses new queries, and shuts
    down cleanly; no GPU fault is involved."""
    ro, col = graphgen.kronecker(12, 16, 61)
    roots = graphgen.pick_roots(ro, 4, 61)
    n = len(ro) - 1
    with gb.Graph(ro, col) as g:
        g.set_option("timeout_ns", 0)
        s = gb.Server()
        try:
            gid = s.add_graph(g)
            bufs = [np.empty(n, np.uint8) for _ in roots]
            tickets = [s.submit(gid, int(r), b) for r, b in zip(roots, bufs)]
            with pytest.raises(gb.BfsError) as ei:
                s.drain()
            assert ei.value.status == gb.BFS_ERR_TIMEOUT
            for t in tickets:
                with pytest.raises(gb.BfsError) as ei:
                    s.poll(t)
                assert ei.value.status == gb.BFS_ERR_TIMEOUT
            with pytest.raises(gb.BfsError):
                s.submit(gid, int(roots[0]), bufs[0])
        finally:
            s.close()


def test_graph_stats_after_drain(resident):
    """The monitoring counters: nothing waiting or running after a drain,
    rounds and iterations counted for the graphs that had queries, and every
    worker back to waiting for work."""
    queries = make_queries(resident, 40, 9)
    with gb.Server() as s:
        ids = [s.add_graph(g) for _, _, g in resident]
        run_mixed(s, ids, resident, queries, 10)
        for gi, gid in enumerate(ids):
            deadline = time.time() + 5.0
            st = s.graph_stats(gid)
            while st["phase"] != "waiting for work" and time.time() < deadline:
                time.sleep(0.01)  # the worker may still be leaving its last round
                st = s.graph_stats(gid)
            assert st["phase"] == "waiting for work", st
            assert st["waiting"] == 0 and st["running"] == 0, st
            if any(q[0] == gi for q in queries):
                assert st["rounds"] > 0 and st["iter"] > 0 and st["has_workspace"], st
        with pytest.raises(gb.BfsError):
            s.graph_stats(len(ids))


def test_registered_graph_cannot_be_destroyed_under_a_live_server():
    """A server's worker may search its graphs until the server is
    destroyed: bfs_graph_destroy refuses a registered graph with
    BFS_ERR_BUSY (nothing freed, the graph stays usable) and succeeds once
    the server is gone."""
    ro, col = graphgen.kronecker(12, 16, 71)
    r = int(graphgen.pick_roots(ro, 1, 71)[0])
    n = len(ro) - 1
    g = gb.Graph(ro, col)
    s = gb.Server()
    gid = s.add_graph(g)
    with pytest.raises(gb.BfsError) as ei:
        g.close()
    assert ei.value.status == gb.BFS_ERR_BUSY and g.handle
    buf = np.empty(n, np.uint8)
    s.wait(s.submit(gid, r, buf), timeout_s=60)
    np.testing.assert_array_equal(buf, oracle.bfs_batch(ro, col, np.array([r], np.int32))[0])
    s.close()
    g.close()
    assert g.handle is None


def test_continuous_batching_queries_join_a_running_search():
    """Continuous batching on the device: while a deep search (a 200-vertex
    path hanging off a Kronecker scale-14 graph, searched from the path's
    far end) is running, further queries on the same graph are admitted into
    free lanes of that search.  Their ticket records show that they joined a
    running search (lanes busy, join iteration > 0, admission before the deep
    query finished), and every result equals the oracle's and the same query
    run alone."""
    kro, kcol = graphgen.kronecker(14, 16, 81)
    nk = len(kro) - 1
    src = np.repeat(np.arange(nk, dtype=np.int32), np.diff(kro))
    hub = int(np.argmax(np.diff(kro)))
    path = np.arange(nk, nk + 200, dtype=np.int32)
    ps = np.concatenate([src, path[:-1], [path[0]]]).astype(np.int32)
    pd = np.concatenate([kcol, path[1:], [hub]]).astype(np.int32)
    ro, col = graphgen.csr_from_tuples(nk + 200, ps, pd)
    n = len(ro) - 1
    deep = int(path[-1])
    others = [int(r) for r in graphgen.pick_roots(kro, 24, 82)]
    with gb.Graph(ro, col) as g:
        with gb.Server() as s:
            gid = s.add_graph(g)
            bufs = {deep: np.empty(n, np.uint8)}
            t_deep = s.submit(gid, deep, bufs[deep])
            t0 = time.monotonic()
            while s.graph_stats(gid)["iter"] < 20 and time.monotonic() - t0 < 30:
                time.sleep(0.0005)
            assert s.graph_stats(gid)["iter"] >= 20 and not s.poll(t_deep)
            tickets = {}
            for r in others:
                bufs[r] = np.empty(n, np.uint8)
                tickets[r] = s.submit(gid, r, bufs[r])
            s.wait(t_deep, timeout_s=60)
            for t in tickets.values():
                s.wait(t, timeout_s=60)
            deep_rec = s.info(t_deep)
            joined = [s.info(t) for t in tickets.values()]
            assert deep_rec["join_iter"] == 0 and deep_rec["done_iter"] >= 200
            overlap = [r for r in joined if r["lanes_busy_at_join"] > 0 and r["join_iter"] >= 20
                       and r["t_admit_ns"] < deep_rec["t_done_ns"]]
            assert len(overlap) == len(others), joined[:3]
            assert len({r["lane"] for r in joined} | {deep_rec["lane"]}) == len(others) + 1
            # the same queries alone (one at a time on the same server)
            for r in [deep] + others[:6]:
                alone = np.empty(n, np.uint8)
                s.wait(s.submit(gid, r, alone), timeout_s=60)
                np.testing.assert_array_equal(alone, bufs[r], err_msg=f"root {r}: alone vs mixed")
    ref = oracle.bfs_batch(ro, col, np.array([deep] + others, np.int32))
    for i, r in enumerate([deep] + others):
        np.testing.assert_array_equal(bufs[r], ref[i], err_msg=f"root {r}")


def test_queries_ending_at_vertices_without_out_edges_complete():
    """A directed graph whose searches end at vertices without out-edges (a
    path into a sink, a star of sinks) and a root without edges: the last
    layer of such a query adds no frontier entry, and the query must still
    complete with the oracle's levels instead of waiting forever."""
    src = list(range(0, 9)) + [10] * 10 + [30, 31]
    dst = list(range(1, 10)) + list(range(11, 21)) + [31, 32]
    n = 40
    ro, col = graphgen.csr_from_tuples(n, np.array(src, np.int32), np.array(dst, np.int32), symmetrize=False)
    roots = [0, 10, 21, 5, 30, 9]
    with gb.Graph(ro, col) as g:
        with gb.Server() as s:
            gid = s.add_graph(g)
            for rnd in range(2):  # alone, then all at once
                bufs = [np.empty(n, np.uint8) for _ in roots]
                if rnd == 0:
                    for r, b in zip(roots, bufs):
                        s.wait(s.submit(gid, r, b), timeout_s=30)
                else:
                    ts = [s.submit(gid, r, b) for r, b in zip(roots, bufs)]
                    for t in ts:
                        s.wait(t, timeout_s=30)
                ref = oracle.bfs_batch(ro, col, np.array(roots, np.int32))
                for i, r in enumerate(roots):
                    np.testing.assert_array_equal(bufs[i], ref[i], err_msg=f"root {r}, round {rnd}")
