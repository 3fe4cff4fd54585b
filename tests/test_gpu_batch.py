"""GPU parity of the bit-parallel batched search (bfs_run_batch).

Every level of every source must equal the oracle's (uint8, 0xFF for
unreached), whatever the batch width, the output location or the number of
batches.
"""
import numpy as np
import pytest

import graphgen
import oracle
from fixtures import csr_from_edges, path_graph, star_graph

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


def batch_levels(g, roots, on_device=True):
    n = g.n
    if on_device:
        out = torch.empty((len(roots), n), dtype=torch.uint8, device="cuda")
        gb.bfs_run_batch(g.handle, roots, out)
        return out.cpu().numpy()
    out = np.empty((len(roots), n), np.uint8)
    gb.bfs_run_batch(g.handle, roots, out)
    return out


@pytest.mark.parametrize("k", [1, 7, 64, 100])
def test_kronecker_scale14_batches(k):
    ro, col = graphgen.kronecker(14, 16, 31)
    roots = graphgen.pick_roots(ro, k, 31)
    with gb.Graph(ro, col) as g:
        got = batch_levels(g, roots)
    np.testing.assert_array_equal(got, oracle.bfs_batch(ro, col, roots))


@pytest.mark.parametrize("width", [8, 24, 64])
def test_batch_width_and_host_output(width):
    ro, col = graphgen.kronecker(13, 16, 32)
    roots = graphgen.pick_roots(ro, 50, 32)
    with gb.Graph(ro, col, batch_width=width) as g:
        got_h = batch_levels(g, roots, on_device=False)
        got_d = batch_levels(g, roots, on_device=True)
    ref = oracle.bfs_batch(ro, col, roots)
    np.testing.assert_array_equal(got_h, ref)
    np.testing.assert_array_equal(got_d, ref)


@pytest.mark.parametrize("streams", [1, 2, 3, 4, 8])
def test_batches_in_flight_together(streams):
    """BATCH_STREAMS: batch b runs on stream b % streams with its own
    workspace and 1/streams of the grid.  Every row equals the oracle's for
    device and host outputs, with a partial last batch, fewer batches than
    streams, and a replay of the captured launch sequence with new sources."""
    ro, col = graphgen.kronecker(14, 16, 35)
    n = len(ro) - 1
    for k in (1, 70, 300):
        roots = graphgen.pick_roots(ro, k, 35 + k, distinct=False)
        ref = oracle.bfs_batch(ro, col, roots)
        with gb.Graph(ro, col, batch_streams=streams, batch_width=32 if k == 300 else 64) as g:
            np.testing.assert_array_equal(batch_levels(g, roots), ref)
            np.testing.assert_array_equal(batch_levels(g, roots, on_device=False), ref)
            out = torch.empty((k, n), dtype=torch.uint8, device="cuda")
            gb.bfs_run_batch(g.handle, roots, out)  # captured shape: replayed below
            roots2 = graphgen.pick_roots(ro, k, 99 + k, distinct=False)
            gb.bfs_run_batch(g.handle, roots2, out)
            np.testing.assert_array_equal(out.cpu().numpy(), oracle.bfs_batch(ro, col, roots2))


def test_batch_streams_with_a_tiny_grid():
    """MAX_CTAS below BATCH_STREAMS: fewer groups, each with at least one CTA,
    so the grids still add up to MAX_CTAS."""
    ro, col = graphgen.kronecker(12, 16, 36)
    roots = graphgen.pick_roots(ro, 200, 36, distinct=False)
    for cap in (1, 3):
        with gb.Graph(ro, col, batch_streams=8, max_ctas=cap) as g:
            np.testing.assert_array_equal(batch_levels(g, roots), oracle.bfs_batch(ro, col, roots))


def test_batch_streams_option_bounds():
    ro, col, _ = path_graph(10, 0)
    with gb.Graph(ro, col) as g:
        assert g.get_option("batch_streams") == 4
        for bad in (0, 9):
            with pytest.raises(gb.BfsError):
                g.set_option("batch_streams", bad)


def test_duplicate_isolated_and_directed_sources():
    rng = np.random.default_rng(4)
    n, ne = 3000, 12000
    src = rng.integers(0, n, ne).astype(np.int32)
    dst = rng.integers(0, n, ne).astype(np.int32)
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=False, drop_loops=False, dedup=False)
    iso = [int(v) for v in np.where(np.diff(ro) == 0)[0][:2]]
    roots = np.array([0, 0, 5, 2999] + iso + [5, 17], np.int32)  # repeats, degree-0 sources
    with gb.Graph(ro, col) as g:
        got = batch_levels(g, roots)
    np.testing.assert_array_equal(got, oracle.bfs_batch(ro, col, roots))


def test_hub_slices_and_erdos_renyi():
    ro, col, _ = star_graph(5000, 0)
    roots = np.array([0, 1, 4999], np.int32)
    with gb.Graph(ro, col) as g:
        np.testing.assert_array_equal(batch_levels(g, roots), oracle.bfs_batch(ro, col, roots))
    ro, col = graphgen.erdos_renyi(14, 16, 3)
    roots = graphgen.pick_roots(ro, 64, 3)
    with gb.Graph(ro, col) as g:
        np.testing.assert_array_equal(batch_levels(g, roots), oracle.bfs_batch(ro, col, roots))


def test_depth_limit():
    ro, col, _ = path_graph(300, 0)
    with gb.Graph(ro, col) as g:
        ok = batch_levels(g, np.array([150], np.int32))  # depth 150 fits uint8
        np.testing.assert_array_equal(ok, oracle.bfs_batch(ro, col, np.array([150], np.int32)))
        with pytest.raises(gb.BfsError) as ei:
            batch_levels(g, np.array([0], np.int32))
        assert ei.value.status == gb.BFS_ERR_DEPTH


def test_empty_and_bad_arguments():
    ro, col, _ = path_graph(10, 0)
    with gb.Graph(ro, col) as g:
        gb.bfs_run_batch(g.handle, np.zeros(0, np.int32), np.zeros((0, 10), np.uint8))
        with pytest.raises(gb.BfsError) as ei:
            batch_levels(g, np.array([3, 10], np.int32))
        assert ei.value.status == gb.BFS_ERR_INVALID_ARG


def test_batch_and_single_source_share_a_graph():
    ro, col = graphgen.kronecker(12, 16, 33)
    roots = graphgen.pick_roots(ro, 5, 33)
    with gb.Graph(ro, col) as g:
        b1 = batch_levels(g, roots)
        lv, _ = g.run(int(roots[2]))
        torch.cuda.synchronize()
        b2 = batch_levels(g, roots)
    np.testing.assert_array_equal(b1, b2)
    ref = lv.cpu().numpy()
    np.testing.assert_array_equal(np.where(ref < 0, 255, ref).astype(np.uint8), b1[2])


def test_scale20_1024_sources_sampled():
    """The batched workload: scale-20 Kronecker graph, 1,024 sources run in
    batches of 64; sampled rows are checked against the oracle."""
    ro, col = graphgen.kronecker(20, 16, 1)
    roots = graphgen.pick_roots(ro, 1024, 7)
    with gb.Graph(ro, col) as g:
        got = batch_levels(g, roots)
    for i in (0, 63, 64, 500, 1023):
        ref = oracle.bfs_batch(ro, col, roots[i:i + 1])[0]
        np.testing.assert_array_equal(got[i], ref, err_msg=f"row {i}")


def test_uneven_mix_of_six_graphs():
    """256 sources over six resident graphs of scales 12..22 (43/43/43/43/42/42)."""
    scales = [12, 14, 16, 18, 20, 22]
    counts = [43, 43, 43, 43, 42, 42]
    graphs = []
    try:
        for s, k in zip(scales, counts):
            ro, col = graphgen.kronecker(s, 16, 40 + s)
            g = gb.Graph(ro, col)
            graphs.append(g)
            roots = graphgen.pick_roots(ro, k, 40 + s)
            got = batch_levels(g, roots)
            for i in (0, k - 1):
                ref = oracle.bfs_batch(ro, col, roots[i:i + 1])[0]
                np.testing.assert_array_equal(got[i], ref, err_msg=f"scale {s} row {i}")
    finally:
        for g in graphs:
            g.close()


def test_pull_steps_and_push_steps_agree():
    """A symmetric graph with sorted rows takes pull steps in its heavy
    iterations; the same graph with every row reversed fails the exact
    symmetry test at creation and stays with push steps.  Both must match
    the oracle."""
    ro, col = graphgen.kronecker(15, 16, 34)
    col_rev = col.copy()
    for u in range(len(ro) - 1):
        col_rev[ro[u]:ro[u + 1]] = col[ro[u]:ro[u + 1]][::-1]
    roots = graphgen.pick_roots(ro, 64, 34)
    ref = oracle.bfs_batch(ro, col, roots)
    with gb.Graph(ro, col) as g:
        np.testing.assert_array_equal(batch_levels(g, roots), ref)
    with gb.Graph(ro, col_rev) as g:
        np.testing.assert_array_equal(batch_levels(g, roots), ref)


def test_repeated_calls_replay_the_captured_sequence():
    """The second call of a shape replays the launch sequence captured by the
    first, with the new roots; a changed option or output re-captures it."""
    ro, col = graphgen.kronecker(13, 16, 41)
    n = len(ro) - 1
    with gb.Graph(ro, col) as g:
        dev_out = torch.empty((100, n), dtype=torch.uint8, device="cuda")
        host_out = np.empty((100, n), np.uint8)
        for rep, seed in enumerate((41, 42, 43, 44)):
            roots = graphgen.pick_roots(ro, 100, seed)
            ref = oracle.bfs_batch(ro, col, roots)
            if rep == 2:
                g.set_option("batch_width", 32)
            gb.bfs_run_batch(g.handle, roots, dev_out)
            np.testing.assert_array_equal(dev_out.cpu().numpy(), ref, err_msg=f"device output, call {rep}")
            gb.bfs_run_batch(g.handle, roots, host_out)
            np.testing.assert_array_equal(host_out, ref, err_msg=f"host output, call {rep}")


def test_bounded_wait_times_out_and_next_call_is_exact():
    """Device waits limited to 0 ns: bfs_run_batch reports BFS_ERR_TIMEOUT;
    with the limit restored the next call on the same workspace is exact."""
    ro, col = graphgen.kronecker(12, 16, 62)
    roots = graphgen.pick_roots(ro, 70, 62)
    n = len(ro) - 1
    with gb.Graph(ro, col) as g:
        out = torch.empty((len(roots), n), dtype=torch.uint8, device="cuda")
        g.set_option("timeout_ns", 0)
        with pytest.raises(gb.BfsError) as ei:
            gb.bfs_run_batch(g.handle, roots, out)
        assert ei.value.status == gb.BFS_ERR_TIMEOUT
        g.set_option("timeout_ns", 4_000_000_000)
        gb.bfs_run_batch(g.handle, roots, out)
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.bfs_batch(ro, col, roots))
