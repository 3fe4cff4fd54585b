"""The autotuner (bfs_graph_autotune) only changes timing: after tuning, the
options hold values from the candidate sets, and every result is still the
oracle's (levels bit for bit, parents valid, batched levels bit for bit)."""
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


def check_roots(g, ro, col, roots):
    for r in roots:
        level, parent = g.run(int(r))
        torch.cuda.synchronize()
        assert g.status() == gb.BFS_OK
        lv, pa = level.cpu().numpy(), parent.cpu().numpy()
        ref = oracle.bfs(ro, col, int(r), want_parent=False)[0]
        np.testing.assert_array_equal(lv, ref)
        assert oracle.validate(ro, col, int(r), lv, pa, ref)[0] == 0


@pytest.mark.parametrize("mode", [0, 1, 2, 3, 4])
def test_single_source_tuning_keeps_results_exact(mode):
    ro, col = graphgen.kronecker(14, 16, 31)
    with gb.Graph(ro, col, mode=mode) as g:
        opts = g.autotune(gb.BFS_TUNE_SINGLE, samples=4)
        assert opts["mode"] == mode
        assert opts["block"] in ((256, 512, 1024) if mode == 1 else (256, 512))
        if mode == 4:
            assert opts["block"] == 512  # the thin warps' CTA size is fixed: nothing to tune
        if mode == 1:
            assert opts["warp_degree"] in (4, 8, 16, 32)
            assert opts["cta_degree"] in (256, 1024, 4096)
            assert opts["segment"] in (1024, 4096, 16384)
        if mode == 3:
            assert opts["alpha"] in (2, 4, 8, 14, 32, 64)
            assert opts["beta"] in (4, 8, 24, 64, 256)
        check_roots(g, ro, col, graphgen.pick_roots(ro, 4, 31))


def test_mode_tuning_picks_top_down_or_direction_optimising():
    for ro, col in (graphgen.kronecker(15, 16, 32), graphgen.erdos_renyi(14, 16, 33)):
        with gb.Graph(ro, col) as g:
            opts = g.autotune(gb.BFS_TUNE_MODE | gb.BFS_TUNE_SINGLE)
            assert opts["mode"] in (0, 3, 4)
            check_roots(g, ro, col, graphgen.pick_roots(ro, 3, 32))


def test_batch_tuning_keeps_results_exact():
    ro, col = graphgen.kronecker(14, 16, 34)
    roots = graphgen.pick_roots(ro, 100, 34)
    n = len(ro) - 1
    with gb.Graph(ro, col) as g:
        opts = g.autotune(gb.BFS_TUNE_BATCH, samples=16)
        assert opts["batch_width"] in (16, 32, 64) and opts["batch_block"] in (256, 512)
        out = torch.empty((len(roots), n), dtype=torch.uint8, device="cuda")
        gb.bfs_run_batch(g.handle, roots, out)
        np.testing.assert_array_equal(out.cpu().numpy(), oracle.bfs_batch(ro, col, roots))


def test_directed_and_tiny_graphs():
    rng = np.random.default_rng(35)
    n, ne = 3000, 20000
    src = rng.integers(0, n, ne).astype(np.int32)
    dst = rng.integers(0, n, ne).astype(np.int32)
    ro, col = graphgen.csr_from_tuples(n, src, dst, symmetrize=False, drop_loops=False, dedup=False)
    with gb.Graph(ro, col) as g:
        g.autotune(gb.BFS_TUNE_MODE | gb.BFS_TUNE_SINGLE | gb.BFS_TUNE_BATCH, samples=3)
        check_roots(g, ro, col, [0, 1234, 2999])
    ro = np.array([0, 1, 2], np.int32)
    col = np.array([1, 0], np.int32)
    with gb.Graph(ro, col) as g:
        g.autotune(gb.BFS_TUNE_SINGLE | gb.BFS_TUNE_BATCH, samples=1)
        check_roots(g, ro, col, [0, 1])


def test_bad_arguments_leave_options_unchanged():
    ro, col = graphgen.kronecker(10, 16, 36)
    with gb.Graph(ro, col, block=256) as g:
        for what, samples in ((0, 4), (8, 4), (gb.BFS_TUNE_SINGLE, -1), (gb.BFS_TUNE_SINGLE, 5000)):
            with pytest.raises(gb.BfsError) as ei:
                gb.bfs_graph_autotune(g.handle, what, samples)
            assert ei.value.status == gb.BFS_ERR_INVALID_ARG
        assert g.get_option("block") == 256
