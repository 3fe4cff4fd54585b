"""The bounds-checking build (-DBFS_BOUNDS_CHECK) on the GPU.

In that build every index of the kernels' main array accesses (adjacency,
row offsets, visited bitmap, level, parent, id maps, frontier queues, the
batched search's frontier, seen and level rows) is checked; the first one
out of range is recorded with its array and the call reports BFS_ERR_CUDA.
Here the checked library runs the searches of every mode, the batched
search, the allocation-free entry point and the serving loop on graphs that
exercise hubs, slices, long paths and tiny components, in a child process
(the binding loads one library per process, chosen by GBBFS_LIB).  Every
call must return BFS_OK, so no index left its array, and every result must
equal the oracle's (levels bit for bit, parents validated)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1604_02844_gb300 import build as lib_build  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r}); sys.path.insert(0, {tests!r})
import graphgen, oracle
import paper_1604_02844_gb300 as gb
from fixtures import path_graph, star_graph, grid_graph
lib = gb.load()
assert lib._name.endswith("libgbbfs_check.so"), lib._name

def check(ro, col, mode, roots):
    with gb.Graph(ro, col, mode=mode) as g:
        for r in roots:
            level, parent = g.run(int(r))
            torch.cuda.synchronize()
            assert g.status() == gb.BFS_OK, gb.last_error()
            lv, pa = level.cpu().numpy(), parent.cpu().numpy()
            ref = oracle.bfs(ro, col, int(r), want_parent=False)[0]
            assert np.array_equal(lv, ref), (mode, int(r))
            assert oracle.validate(ro, col, int(r), lv, pa, ref)[0] == 0, (mode, int(r))

graphs = [graphgen.kronecker(16, 16, 1), graphgen.erdos_renyi(15, 16, 2), path_graph(3000, 7)[:2],
          star_graph(100000, 0)[:2], grid_graph(200, 150, 99)[:2]]
for ro, col in graphs:
    roots = graphgen.pick_roots(ro, 4, 3)
    for mode in (0, 2, 3, 4):
        check(ro, col, mode, roots)

ro, col = graphgen.kronecker(14, 16, 5)
n = len(ro) - 1
srcs = graphgen.pick_roots(ro, 80, 5, distinct=False)
ref = oracle.bfs_batch(ro, col, srcs)
with gb.Graph(ro, col) as g:
    out = torch.empty((len(srcs), n), dtype=torch.uint8, device="cuda")
    gb.bfs_run_batch(g.handle, srcs, out)
    assert np.array_equal(out.cpu().numpy(), ref)
d_ro, d_col = torch.from_numpy(ro).cuda(), torch.from_numpy(col).cuda()
lv = torch.empty(n, dtype=torch.int32, device="cuda")
pa = torch.empty(n, dtype=torch.int32, device="cuda")
gb.bfs_run_noalloc(d_ro, d_col, int(srcs[0]), lv, pa)
torch.cuda.synchronize()
ref0 = oracle.bfs(ro, col, int(srcs[0]), want_parent=False)[0]
assert np.array_equal(lv.cpu().numpy(), ref0)
assert oracle.validate(ro, col, int(srcs[0]), lv.cpu().numpy(), pa.cpu().numpy(), ref0)[0] == 0

g = gb.Graph(ro, col)
server = gb.Server()
try:
    gid = server.add_graph(g)
    bufs = [np.empty(n, np.uint8) for _ in range(40)]
    tickets = [server.submit(gid, int(r), b) for r, b in zip(srcs[:40], bufs)]
    for t in tickets:
        server.wait(t, timeout_s=120)
    for i in range(40):
        assert np.array_equal(bufs[i], ref[i]), i
finally:
    server.close()
    g.close()
print("bounds-checked ok")
'''


def test_bounds_checking_build_runs_clean_and_matches_the_oracle():
    lib = lib_build.build_checked()
    env = dict(os.environ, GBBFS_LIB=lib)
    code = SCRIPT.format(root=ROOT, tests=os.path.join(ROOT, "tests"))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "bounds-checked ok" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
