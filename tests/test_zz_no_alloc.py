"""bfs_run_noalloc against bfs_run.

bfs_run_noalloc is for callers that cannot allocate GPU memory at the moment
they search (their device memory belongs to another allocator or a fixed
budget, or they run on a path that must not block in cudaMalloc/cudaFree).
It searches the caller's device CSR with scratch state kept in a fixed array
inside the library.  Its results must equal those of the ordinary entry
point and of the oracle: levels bit for bit, and parents that pass the
oracle's validation (the parent choice is not unique).

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""
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


def test_noalloc_matches_bfs_run_on_two_calls_in_a_row():
    ro, col = graphgen.kronecker(14, 16, 21)
    n, m = len(ro) - 1, len(col)
    assert n <= gb.NOALLOC_MAX_VERTICES and m <= gb.NOALLOC_MAX_EDGES
    d_ro = torch.from_numpy(ro).cuda()
    d_col = torch.from_numpy(col).cuda()
    roots = graphgen.pick_roots(ro, 2, 21)
    g = gb.Graph(ro, col)
    try:
        for r in roots:  # two calls in a row share the library's scratch array
            lv = torch.empty(n, dtype=torch.int32, device="cuda")
            pa = torch.empty(n, dtype=torch.int32, device="cuda")
            gb.bfs_run_noalloc(d_ro, d_col, int(r), lv, pa)
            ref_lv, ref_pa = g.run(int(r))
            torch.cuda.synchronize()
            assert g.status() == gb.BFS_OK
            lv, pa = lv.cpu().numpy(), pa.cpu().numpy()
            ref_lv, ref_pa = ref_lv.cpu().numpy(), ref_pa.cpu().numpy()
            np.testing.assert_array_equal(lv, ref_lv)
            # both against the oracle: levels bit for bit, parents validated
            # with the oracle's levels as the reached-set reference
            or_lv = oracle.bfs(ro, col, int(r), want_parent=False)[0]
            np.testing.assert_array_equal(lv, or_lv)
            assert oracle.validate(ro, col, int(r), lv, pa, or_lv)[0] == 0
            assert oracle.validate(ro, col, int(r), ref_lv, ref_pa, or_lv)[0] == 0
    finally:
        g.close()


def test_noalloc_takes_no_device_memory_per_call():
    ro, col = graphgen.kronecker(12, 16, 22)
    n = len(ro) - 1
    d_ro = torch.from_numpy(ro).cuda()
    d_col = torch.from_numpy(col).cuda()
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    r = int(graphgen.pick_roots(ro, 1, 22)[0])
    gb.bfs_run_noalloc(d_ro, d_col, r, lv)  # first call on the device: set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        gb.bfs_run_noalloc(d_ro, d_col, r, lv)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before
    np.testing.assert_array_equal(lv.cpu().numpy(), oracle.bfs(ro, col, r, want_parent=False)[0])


def test_noalloc_rejects_out_of_limit_and_host_arguments():
    ro = np.zeros(gb.NOALLOC_MAX_VERTICES + 2, np.int32)
    d_ro = torch.from_numpy(ro).cuda()
    lv = torch.empty(len(ro) - 1, dtype=torch.int32, device="cuda")
    with pytest.raises(gb.BfsError) as ei:
        gb.bfs_run_noalloc(d_ro, torch.zeros(1, dtype=torch.int32, device="cuda"), 0, lv, m=0)
    assert ei.value.status == gb.BFS_ERR_INVALID_ARG
    assert "131072" in str(ei.value)
    small = np.array([0, 1, 2], np.int32)
    with pytest.raises(gb.BfsError) as ei:  # host arrays are refused, not copied
        gb.bfs_run_noalloc(small, np.array([1, 0], np.int32), 0,
                           torch.empty(2, dtype=torch.int32, device="cuda"))
    assert ei.value.status == gb.BFS_ERR_INVALID_ARG
