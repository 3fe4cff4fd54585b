"""Host-side logic of bench.py that needs no GPU: the bounded wait on
serving tickets must return once every ticket is done and give up, with an
error, when one never completes."""
import time

import pytest

import bench


def test_wait_tickets_returns_when_all_done():
    done_at = {t: time.perf_counter() + 0.01 * t for t in range(5)}
    bench.wait_tickets(lambda t: time.perf_counter() >= done_at[t], list(range(5)), limit_s=5.0)


def test_wait_tickets_gives_up_on_a_lost_query():
    t0 = time.perf_counter()
    with pytest.raises(bench.ServingStuck, match="1 of 3 queries unfinished"):
        bench.wait_tickets(lambda t: t != 2, [0, 1, 2], limit_s=0.2)
    assert time.perf_counter() - t0 < 5.0


def test_wait_tickets_empty():
    bench.wait_tickets(lambda t: False, [], limit_s=0.0)


def test_algorithmic_bytes_hand_count():
    # path 0-1-2 (4 directed entries), all reached: adjacency 16 B, row_offsets
    # pairs 24 B, frontier ids 24 B, level+parent 24 B, bitmap 3/4 B
    assert bench.algorithmic_bytes(4, 3, 3) == 16 + 24 + 24 + 24 + 0.75


def test_harmonic_mean():
    assert abs(bench.harmonic_mean([1.0, 2.0, 4.0]) - 3.0 / 1.75) < 1e-12
    assert bench.harmonic_mean([5.0] * 64) == pytest.approx(5.0)


def test_clock_summary_parses_samples(tmp_path):
    s = bench.ClockSampler()
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()  # as if nvidia-smi had run
    rows = [
        "0, GPU-a, 345, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # idle: dropped
        "0, GPU-a, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, GPU-a, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, GPU-a, 2040, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active",
        "garbage line",
    ]
    open(s.path, "w").write("\n".join(rows) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2055 and out["sm_max_mhz"] == 2070
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 4


def test_clock_summary_flags_thermal_slowdown(tmp_path):
    s = bench.ClockSampler()
    s.path = str(tmp_path / "clocks.csv")
    s.proc = object()
    open(s.path, "w").write("0, GPU-a, 1500, 2070, 1000.0, 0x40, Not Active, Active, Not Active, Not Active\n")
    assert s.summary()["reasons"] == ["hw_thermal_slowdown"]


def test_profiled_traffic_only_for_the_profiled_kernel(tmp_path, monkeypatch):
    import argparse
    args = argparse.Namespace(graph="kronecker", scale=22)
    t = bench.profiled_traffic(args, {"mode": 0, "block": 512})
    assert t is None or t > 0  # present while the kernel sources match the summary
    assert bench.profiled_traffic(args, {"mode": 3, "block": 512}) is None
    assert bench.profiled_traffic(args, {"mode": 0, "block": 256}) is None
    # a changed kernel source invalidates the stored figure
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        p = root / f
        p.parent.mkdir(parents=True, exist_ok=True)
        p.write_text("changed\n")
    (root / "profiles" / "td_warp_kernel_kronecker_s22.txt").write_text(
        "traffic_bytes_per_launch: 123\nsource_sha256_16: 0000000000000000\n")
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_traffic(args, {"mode": 0, "block": 512}) is None


# ---- the serving measurement's control flow, on a stand-in library --------

class _FakeBfsError(Exception):
    def __init__(self, status, msg=""):
        super().__init__(msg)
        self.status = status


class _FakeGraph:
    fail_status = False  # every search reports a device timeout

    def __init__(self, ro, col):
        self.n = len(ro) - 1
        self.handle = object()
        self.closed = False

    def status(self):
        if _FakeGraph.fail_status:
            raise _FakeBfsError(-6, "a device-side wait ran out")
        return 0

    def close(self):
        self.closed = True


def _fake_gb(stall_servers, fail_servers=(), hang_close=False):
    """A stand-in for the library: servers numbered from 0; those listed in
    stall_servers never complete a query, those in fail_servers report every
    query as failed."""
    import time as _t
    import types
    state = {"servers": 0}

    class Server:
        def __init__(self):
            self.no = state["servers"]
            state["servers"] += 1
            self.stall = self.no in stall_servers
            self.fail = self.no in fail_servers
            self.graphs = []
            self._keep = {}
            self.t = {}
            self.gid = {}
            self.closed = False

        def add_graph(self, g):
            self.graphs.append(g)
            return len(self.graphs) - 1

        def submit(self, gid, root, buf):
            t = len(self.t) + 1
            self.t[t] = _t.monotonic_ns()
            self.gid[t] = gid
            return t

        def poll(self, t):
            if self.fail:
                raise _FakeBfsError(-6, "a device-side wait ran out")
            return not self.stall

        def times(self, t):
            return self.t[t], self.t[t] + 1000

        def info(self, t):
            return {"t_submit_ns": self.t[t], "t_admit_ns": self.t[t] + 400, "t_done_ns": self.t[t] + 1000,
                    "join_iter": 2, "done_iter": 5, "graph_id": self.gid[t], "lane": 0,
                    "lanes_busy_at_join": t % 2}

        def graph_stats(self, gid):
            return {"waiting": 1, "running": 0, "phase": "waiting for work"}

        def close(self):
            if hang_close:
                _t.sleep(3.0)
            self.closed = True

    return types.SimpleNamespace(Graph=_FakeGraph, Server=Server, BfsError=_FakeBfsError,
                                 bfs_run=lambda *a: None), state


def _fake_torch():
    import types
    import numpy as np

    class T:
        def __init__(self, n, dtype):
            self.a = np.zeros(n, dtype)

        def pin_memory(self):
            return self

        def numpy(self):
            return self.a

    class Stream:
        def synchronize(self):
            pass

    cuda = types.SimpleNamespace(current_stream=lambda dev=None: Stream())
    return types.SimpleNamespace(empty=lambda n, dtype=None: T(n, dtype), uint8=np.uint8, int32=np.int32, cuda=cuda)


def _serving_args():
    import argparse
    return argparse.Namespace(serving_scales="6,7", seed=1, serving_requests=1000)


@pytest.fixture
def short_deadline(monkeypatch):
    monkeypatch.setattr(bench, "SERVING_WAIT_S", 0.2)
    monkeypatch.setattr(bench, "SERVING_WAIT_PER_QUERY_S", 0.0)
    monkeypatch.setattr(bench, "SERVER_CLOSE_WAIT_S", 0.2)
    monkeypatch.setattr(bench, "_KEEP_ALIVE", [])


def test_serving_measurement_normal_run(short_deadline):
    pytest.importorskip("graphgen")
    gb, state = _fake_gb(stall_servers=())
    out = bench.serving_measurement(_serving_args(), gb, _fake_torch(), None)
    assert "error" not in out and "stalls_before_this_attempt" not in out
    assert out["queries_per_s"] > 0 and len(out["sweep"]) == len(bench.SERVING_SWEEP) and state["servers"] == 1
    assert out["sustainable_qps"] > 0 and out["offered_qps"] == pytest.approx(0.7 * out["sustainable_qps"])
    head = out["headline"]
    assert set(head["per_scale"]) == {"6", "7"} and head["queue_wait_p99_ms"] == pytest.approx(4e-4)
    assert head["in_search_p50_ms"] == pytest.approx(6e-4) and 0.4 < head["joined_running_search"] < 0.6


def test_serving_stats_hand_count():
    # four queries on two graphs (scales 10 and 20); times in ns
    recs = [dict(t_submit_ns=0, t_admit_ns=1_000_000, t_done_ns=3_000_000, graph_id=0, lanes_busy_at_join=0,
                 join_iter=0, done_iter=4),
            dict(t_submit_ns=1_000_000, t_admit_ns=1_000_000, t_done_ns=2_000_000, graph_id=1, lanes_busy_at_join=3,
                 join_iter=2, done_iter=5),
            dict(t_submit_ns=2_000_000, t_admit_ns=4_000_000, t_done_ns=5_000_000, graph_id=0, lanes_busy_at_join=1,
                 join_iter=4, done_iter=6),
            dict(t_submit_ns=4_000_000, t_admit_ns=4_000_000, t_done_ns=10_000_000, graph_id=1, lanes_busy_at_join=0,
                 join_iter=0, done_iter=8)]
    st = bench.serving_stats(recs, [10, 20])
    assert st["p50_ms"] == pytest.approx(3.0)          # latencies 3, 1, 3, 6 ms
    assert st["queue_wait_p50_ms"] == pytest.approx(0.5)  # waits 1, 0, 2, 0 ms
    assert st["joined_running_search"] == 0.5
    # steady window: submissions span 0..4 ms, window 1..4 ms; completions in it: 2, 3 ms
    assert st["steady_served_qps"] == pytest.approx(2 / 3e-3)
    assert st["per_scale"]["10"]["requests"] == 2 and st["per_scale"]["20"]["iterations_p50"] == pytest.approx(5.5)  # 3 and 8


def test_find_knee():
    pts = [{"offered_qps": 100, "steady_served_qps": 99}, {"offered_qps": 200, "steady_served_qps": 192},
           {"offered_qps": 300, "steady_served_qps": 240}]
    assert bench.find_knee(pts) == 200
    assert bench.find_knee([{"offered_qps": 100, "steady_served_qps": 50}]) is None
    # a sustained point above a missed one does not count
    pts.append({"offered_qps": 400, "steady_served_qps": 399})
    assert bench.find_knee(pts) == 200


def test_serving_measurement_retries_once_after_a_stall(short_deadline):
    pytest.importorskip("graphgen")
    gb, state = _fake_gb(stall_servers=(0,))
    out = bench.serving_measurement(_serving_args(), gb, _fake_torch(), None)
    assert "error" not in out and out["queries_per_s"] > 0
    (stall,) = out["stalls_before_this_attempt"]
    assert "unfinished" in stall["error"] and len(stall["graphs"]) == 2
    assert state["servers"] == 2 and len(bench._KEEP_ALIVE) == 1


def test_serving_measurement_reports_two_stalls(short_deadline):
    pytest.importorskip("graphgen")
    gb, state = _fake_gb(stall_servers=(0, 1))
    out = bench.serving_measurement(_serving_args(), gb, _fake_torch(), None)
    assert out["error"] == "serving measurement stopped twice" and len(out["stalls"]) == 2
    assert state["servers"] == 2


def test_serving_measurement_retries_after_failed_queries(short_deadline):
    pytest.importorskip("graphgen")
    gb, state = _fake_gb(stall_servers=(), fail_servers=(0,))
    out = bench.serving_measurement(_serving_args(), gb, _fake_torch(), None)
    assert "error" not in out and out["queries_per_s"] > 0
    (stall,) = out["stalls_before_this_attempt"]
    assert "device-side wait" in stall["error"] and state["servers"] == 2


def test_guarded_turns_an_exception_into_an_entry():
    assert bench.guarded("x", lambda: {"a": 1}) == {"a": 1}

    def boom():
        raise RuntimeError("device lost")

    out = bench.guarded("batched", boom)
    assert out == {"error": "batched: RuntimeError: device lost"}


def test_serving_measurement_stops_the_plain_path_at_a_failed_search(short_deadline, monkeypatch):
    pytest.importorskip("graphgen")
    monkeypatch.setattr(_FakeGraph, "fail_status", True)
    gb, state = _fake_gb(stall_servers=())
    out = bench.serving_measurement(_serving_args(), gb, _fake_torch(), None)
    assert out["queries_per_s"] > 0  # the serving numbers are kept
    assert out["plain_queries_per_s"] is None and "plain bfs_run 0 " in out["plain_error"]


def test_serving_measurement_bounds_the_server_close(short_deadline):
    pytest.importorskip("graphgen")
    gb, state = _fake_gb(stall_servers=(), hang_close=True)
    searched = []
    gb.bfs_run = lambda *a: searched.append(a)
    out = bench.serving_measurement(_serving_args(), gb, _fake_torch(), None)
    assert out["queries_per_s"] > 0 and "did not return" in out["close_error"]
    assert len(bench._KEEP_ALIVE) == 1
    # the server's workers may still use its graphs: none is searched or freed
    (server, graphs), = bench._KEEP_ALIVE
    assert graphs and not any(g.closed for _, g in graphs)
    assert searched == [] and out["plain_queries_per_s"] is None and "skipped" in out["plain_error"]


def test_bounded_reports_a_measurement_that_does_not_finish(monkeypatch):
    import time as _t
    monkeypatch.setattr(bench, "_KEEP_ALIVE", [])
    assert bench.bounded("quick", lambda: {"ok": 1}, 5.0) == {"ok": 1}
    seen = []
    out = bench.bounded("slow", lambda: _t.sleep(2.0), 0.1, setup=lambda: seen.append("setup"))
    assert out == {"error": "slow: did not finish within 0 s"} and seen == ["setup"]
    assert len(bench._KEEP_ALIVE) == 1
    assert bench.bounded("boom", lambda: 1 / 0, 5.0)["error"].startswith("boom: ZeroDivisionError")


def test_batched_algorithmic_bytes_hand_count():
    """Path 0-1-2, sources 0 and 2 in one group: iteration 0 reads vertices
    0 and 2 (4 B/entry + 24 B each: 28 + 28) and writes the row of vertex 1
    (64); iteration 1 reads vertex 1 (8 + 24) and writes rows 0 and 2 (128);
    iteration 2 reads vertices 0 and 2 (56)."""
    torch = pytest.importorskip("torch")
    import numpy as np
    lv = torch.tensor([[0, 1, 2], [2, 1, 0]], dtype=torch.uint8)
    assert bench.batched_algorithmic_bytes(torch, lv, np.array([1, 2, 1]), "cpu") == 56 + 64 + 32 + 128 + 56
    # an unreached vertex (0xFF) costs nothing
    lv2 = torch.tensor([[0, 1, 255]], dtype=torch.uint8)
    assert bench.batched_algorithmic_bytes(torch, lv2, np.array([1, 1, 0]), "cpu") == 28 + 64 + 28


def test_largest_component_stats():
    # roots 1 and 2 in the largest component (100 edges), root 3 in a 1-edge component
    mcc = {1: 100.0, 2: 100.0, 3: 1.0}
    runs = [(1, 1e-9), (2, 2e-9), (3, 1e-9)]
    st = bench.largest_component_stats(runs, mcc)
    assert st["roots_outside_largest_component"] == 1
    assert st["hm_gteps_largest_component"] == pytest.approx(bench.harmonic_mean([100.0, 50.0]))
