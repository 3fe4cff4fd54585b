"""Run bench.py's own-arm flow (run_ours) end to end on a machine without a
GPU: torch.cuda is replaced by host stand-ins (CPU tensors, wall-clock
events) and the BFS library by one whose searches are the CPU oracle's, so
that every step of the bench -- bookkeeping, timed steps, roofline, e2e,
ablation, batched, uneven mix, serving with its stall handling, CPU baseline
-- runs and prints its JSON line.  Numbers from this run mean nothing; the
point is that the flow completes and the line has its keys.

    python run_with_stand_ins.py [stalling server numbers ...]

prints the bench's JSON line (rank 0 only), then one line "exit: <how the
bench ended>".  Under torch.distributed.run each rank runs it, and the ranks
meet over gloo.
"""
import contextlib
import io
import os
import sys
import time
import types

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch as real  # noqa: E402

import oracle  # noqa: E402

# ---- torch with host stand-ins for the CUDA parts ---------------------------
real.Tensor.pin_memory = lambda self: self


class _Torch(types.ModuleType):
    def __getattr__(self, name):
        return getattr(real, name)


class _Event:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return (other.t - self.t) * 1e3 + 1e-3


class _Stream:
    cuda_stream = 0

    def synchronize(self):
        pass


def _no_props(dev):
    raise RuntimeError("no device properties on the host")


def _empty(*a, **k):
    k.pop("device", None)
    return real.empty(*a, **k)


torch_sub = _Torch("torch")
torch_sub.device = lambda *a, **k: real.device("cpu")
torch_sub.empty = _empty
torch_sub.cuda = types.SimpleNamespace(set_device=lambda d: None, current_stream=lambda d=None: _Stream(),
                                       synchronize=lambda: None, Event=_Event,
                                       get_device_properties=_no_props, is_available=lambda: False)
sys.modules["torch"] = torch_sub

# ---- the library, with the oracle's searches ---------------------------------
import test_bench_host  # noqa: E402  (its stand-in server)

lib = types.ModuleType("paper_1604_02844_gb300")
lib.BFS_OK = 0
lib.BFS_TUNE_BATCH = 2
lib.OPTION_NAMES = {k: i for i, k in enumerate(["block", "mode", "alpha", "beta", "batch_width", "batch_block",
                                                     "batch_streams", "max_ctas"])}
lib.BfsError = test_bench_host._FakeBfsError
lib.last_error = lambda: ""
lib.load = lambda: None
_handles = {}


def _search(g, root, level, parent):
    lv, pa = oracle.bfs(g.ro, g.col, int(root))
    g.last_level = lv
    level.copy_(real.from_numpy(lv))
    if parent is not None:
        parent.copy_(real.from_numpy(pa))


class _Graph:
    def __init__(self, ro, col, **kw):
        self.ro, self.col = np.asarray(ro), np.asarray(col)
        self.n = len(ro) - 1
        self.opts = {"block": 512, "mode": 0, "alpha": 14, "beta": 24, "batch_width": 64, "batch_block": 256,
                     "batch_streams": 4, "max_ctas": 0}
        self.handle = id(self)
        _handles[self.handle] = self

    def set_option(self, k, v):
        self.opts[k] = v

    def get_option(self, k):
        return self.opts[k]

    def run(self, root, level, parent):
        _search(self, root, level, parent)
        return level, parent

    def status(self):
        return 0

    def layer_stats(self):
        return oracle.layer_profile(self.ro, self.last_level)

    def layer_times(self):
        v, _, _ = self.layer_stats()
        return np.cumsum(np.full(len(v), 1000, np.int64))

    def autotune(self, what, samples=0):
        return dict(self.opts)

    def close(self):
        pass


lib.Graph = _Graph
lib.bfs_run = lambda h, root, level, parent, stream: _search(_handles[h], root, level, parent)
lib.bfs_run_batch = lambda h, roots, out: out.zero_()
lib.bfs_graph_status = lambda h: 0
stub_gb, _ = test_bench_host._fake_gb(stall_servers=tuple(int(x) for x in sys.argv[1:]))
lib.Server = stub_gb.Server
sys.modules["paper_1604_02844_gb300"] = lib

# ---- the bench, on small sizes ----------------------------------------------
import bench  # noqa: E402

bench.L2_FLUSH_BYTES = 1 << 20
bench.SERVING_WAIT_S = 0.5
bench.SERVING_WAIT_PER_QUERY_S = 0.0
bench.UNEVEN_MIX_SCALES = (6, 7, 8)


class _Exited(Exception):
    pass


def _exit(code):
    raise _Exited(code)


os._exit = _exit
buf = io.StringIO()
how = None
with contextlib.redirect_stdout(buf):
    try:
        how = f"returned {bench.main(['--scale', '10', '--steps', '1', '--warmup', '3', '--batched-scale', '10', '--batched-sources', '64', '--serving-requests', '2000', '--serving-scales', '6,7', '--cpu-sample-roots', '4', '--other-workloads', 'erdos_renyi:9,kronecker:8'])}"
    except _Exited as e:
        how = f"direct exit {e.args[0]}"
lines = buf.getvalue().strip().splitlines()
if lines:  # ranks other than 0 print no line
    print(lines[-1])
print(f"exit: {how}")
sys.stdout.flush()
