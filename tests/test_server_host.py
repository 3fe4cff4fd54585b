"""Host-only tests of the serving loop's scheduling (server.cu), no GPU.

server.cu holds no device code, so it is compiled here with g++ against
tests/server_host/fake_backend.cpp. That file stands in for the CUDA runtime
calls and for the batched-search entry points. In the stand-in, a lane's
search is a countdown, and its level row depends only on the graph, the root
and the vertex. The scenarios in tests/server_host/scenarios.cpp drive the
loop through its C ABI and check that:
- results reach their own buffers while lanes are recycled;
- graphs take turns under a tight HBM budget, and the device memory comes
  back at shutdown;
- when the device is out of memory, a graph waits while another holds a
  workspace, and fails when none does;
- the room limit holds;
- device timeouts and depth overflows fail the queries instead of hanging;
- the host backstops end a lane that never finishes, and a search that
  keeps lanes alive without running an iteration;
- the pull-phase hold is kept;
- a graph registered with a live server cannot be released;
- a query submitted during another's search joins it, and its record
  (bfs_ticket_info) says so;
- a query completes only once its result copy has landed (the stand-in's
  copy streams defer each copy until it is waited for).

The loop's wait for room is shortened to 1.5 s in this build. A stress
scenario mixes eight graphs, bursts of queries, steps of random length, the
hold and a budget for three workspaces. Every scenario also runs under
ThreadSanitizer, and under AddressSanitizer with UBSan. A last test plants mistakes in a copy of server.cu and
checks that each one is caught.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1604_02844_gb300", "csrc")
HOST = os.path.join(HERE, "server_host")
SCENARIOS = ["mixed", "tight_budget", "device_oom_wait", "device_oom_fail", "room_limit", "timeout",
             "depth_backstop", "kernel_depth", "pull_hold", "stress", "registration",
             "join_record", "no_progress"]


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime_api.h")):
            return os.path.join(base, "include")
    return None


def _build(server_src, out, extra=()):
    inc = _cuda_include()
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-pthread", *extra, "-DGBBFS_ROOM_WAIT_NS=1500000000",
           f"-I{CSRC}", f"-I{HOST}", f"-I{inc}",
           "-x", "c++", server_src, "-x", "none",
           os.path.join(HOST, "fake_backend.cpp"), os.path.join(HOST, "scenarios.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return out


def _run(exe, scenario, timeout=120):
    return subprocess.run([exe, scenario], capture_output=True, text=True, timeout=timeout)


@pytest.fixture(scope="module")
def server_host(tmp_path_factory):
    if shutil.which("g++") is None or _cuda_include() is None:
        pytest.skip("needs g++ and the CUDA runtime headers")
    d = tmp_path_factory.mktemp("server_host")
    return _build(os.path.join(CSRC, "server.cu"), str(d / "server_host"))


@pytest.mark.parametrize("scenario", SCENARIOS)
def test_scenario(server_host, scenario):
    r = _run(server_host, scenario)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def _sanitizer_usable(tmp_path, flag):
    probe = tmp_path / "probe.cpp"
    probe.write_text("int main() { return 0; }\n")
    return subprocess.run(["g++", f"-fsanitize={flag}", str(probe), "-o", str(tmp_path / "probe")],
                          capture_output=True).returncode == 0


@pytest.mark.parametrize("flag", ["thread", "address,undefined"])
def test_scenarios_under_sanitizers(tmp_path, flag):
    """Every scenario again, built with ThreadSanitizer (the worker threads,
    the submitting thread and the pollers share no unsynchronised state) or
    with AddressSanitizer and UBSan (no use of a workspace after eviction, no
    leak at shutdown, no undefined arithmetic)."""
    if shutil.which("g++") is None or _cuda_include() is None:
        pytest.skip("needs g++ and the CUDA runtime headers")
    if not _sanitizer_usable(tmp_path, flag):
        pytest.skip(f"g++ cannot build with -fsanitize={flag} here")
    extra = [f"-fsanitize={flag}", "-fno-omit-frame-pointer"]
    if "undefined" in flag:
        extra.append("-fno-sanitize-recover=undefined")
    exe = _build(os.path.join(CSRC, "server.cu"), str(tmp_path / "server_host_san"), extra)
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66", ASAN_OPTIONS="detect_leaks=1")
    for scenario in SCENARIOS:
        r = subprocess.run([exe, scenario], capture_output=True, text=True, timeout=300, env=env)
        assert r.returncode == 0 and r.stdout.strip() == "ok", f"{scenario}:\n{r.stdout}{r.stderr[-4000:]}"


# (name, text in server.cu, replacement, scenario that must then fail)
MUTANTS = [
    ("no pull-phase hold",
     "const bool hold = gs.running && gs.have_last && pull_phase(gs.g, gs.last, gs.running);",
     "const bool hold = false;", "pull_hold"),
    ("results to a neighbouring lane's buffer",
     "out = reqs[gs.lane_ticket[i] - 1]->out;",
     "out = reqs[gs.lane_ticket[i ^ 1] ? gs.lane_ticket[i ^ 1] - 1 : gs.lane_ticket[i] - 1]->out;", "mixed"),
    ("no room limit",
     "if (t - gs.room_wait_since <= kRoomWaitNs) return BFS_NOT_READY;",
     "return BFS_NOT_READY;", "room_limit"),
    ("a device allocation failure only ever waits",
     "    if (rc != BFS_OK) return rc;\n    gs.has_ws = true;",
     "    if (rc != BFS_OK) return BFS_NOT_READY;\n    gs.has_ws = true;", "device_oom_fail"),
    ("idle workspaces never given back",
     "        evict_idle(gs, need);\n", "", "tight_budget"),
    ("no backstop for a search without progress",
     "if (had_last && !add && st.iter == iter_before", "if (false && st.iter == iter_before", "no_progress"),
    ("queries completed before their result copy has landed",
     "const cudaError_t e = cudaEventSynchronize(gs.ev_copied);", "const cudaError_t e = cudaSuccess;", "mixed"),
]


@pytest.mark.parametrize("name,old,new,scenario", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_are_caught(server_host, tmp_path, name, old, new, scenario):
    src = open(os.path.join(CSRC, "server.cu")).read()
    assert src.count(old) == 1, f"mutant {name!r} no longer applies"
    mutated = tmp_path / "server.cu"
    mutated.write_text(src.replace(old, new))
    exe = _build(str(mutated), str(tmp_path / "server_host"))
    r = _run(exe, scenario, timeout=90)
    assert r.returncode != 0, f"{name}: scenario {scenario} still passes"


def test_planted_race_is_caught(tmp_path):
    """The race detector itself: a lane mask cleared outside the server's
    lock (other workers read it under the lock) must be reported."""
    if shutil.which("g++") is None or _cuda_include() is None:
        pytest.skip("needs g++ and the CUDA runtime headers")
    if not _sanitizer_usable(tmp_path, "thread"):
        pytest.skip("g++ cannot build with -fsanitize=thread here")
    src = open(os.path.join(CSRC, "server.cu")).read()
    old = "    std::lock_guard<std::mutex> lk(mu);\n    for (int i = 0; i < 64; ++i) {\n" \
          "        if (!((mask >> i) & 1ull)) continue;\n        gs.pending_ticket[i] = gs.lane_ticket[i];"
    assert src.count(old) == 1, "the planted race no longer applies"
    mutated = tmp_path / "server.cu"
    mutated.write_text(src.replace(old, "    gs.running &= ~mask;\n" + old))
    exe = _build(str(mutated), str(tmp_path / "racy"), ["-fsanitize=thread"])
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1 exitcode=66")
    r = subprocess.run([exe, "stress"], capture_output=True, text=True, timeout=300, env=env)
    assert r.returncode == 66 and "data race" in r.stderr
