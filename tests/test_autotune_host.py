"""Host-only tests of the autotuner (autotune.cu), no GPU.

autotune.cu is host code: it times sample searches and keeps the fastest
option values.  Here it is compiled with g++ against
tests/autotune_host/fake_runtime.cpp, whose searches "cost" a time given by
a cost model of the options with a known optimum (event times for bfs_run,
host sleeps for bfs_run_batch), so the choices the descent makes can be
checked exactly: each option's best value, the mode choice, candidates that
are refused or fail, the restoring of every option when a stage fails,
argument checks, and the sample roots.  A second test plants mistakes in a
copy of autotune.cu and checks that each is caught.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1604_02844_gb300", "csrc")
HOST = os.path.join(HERE, "autotune_host")
SCENARIOS = ["single_mode0", "mode_then_single", "mode_thin", "mode_stays", "binned", "rejected_value", "failing_value",
             "all_fail", "late_failure", "batch", "args", "samples"]


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime_api.h")):
            return os.path.join(base, "include")
    return None


def _build(src, out, extra=()):
    cmd = ["g++", "-std=c++17", "-O1", "-g", "-pthread", *extra, f"-I{CSRC}", f"-I{HOST}", f"-I{_cuda_include()}",
           "-x", "c++", src, "-x", "none",
           os.path.join(HOST, "fake_runtime.cpp"), os.path.join(HOST, "scenarios.cpp"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return out


@pytest.fixture(scope="module")
def autotune_host(tmp_path_factory):
    if shutil.which("g++") is None or _cuda_include() is None:
        pytest.skip("needs g++ and the CUDA runtime headers")
    d = tmp_path_factory.mktemp("autotune_host")
    return _build(os.path.join(CSRC, "autotune.cu"), str(d / "autotune_host"))


@pytest.mark.parametrize("scenario", SCENARIOS)
def test_scenario(autotune_host, scenario):
    r = subprocess.run([autotune_host, scenario], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr


def test_scenarios_under_address_and_ub_sanitizers(tmp_path):
    """Every scenario again, built with AddressSanitizer and UBSan."""
    if shutil.which("g++") is None or _cuda_include() is None:
        pytest.skip("needs g++ and the CUDA runtime headers")
    probe = tmp_path / "probe.cpp"
    probe.write_text("int main() { return 0; }\n")
    flags = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer"]
    if subprocess.run(["g++", *flags, str(probe), "-o", str(tmp_path / "probe")], capture_output=True).returncode:
        pytest.skip("g++ cannot build with the sanitizers here")
    exe = _build(os.path.join(CSRC, "autotune.cu"), str(tmp_path / "autotune_san"), flags)
    for scenario in SCENARIOS:
        r = subprocess.run([exe, scenario], capture_output=True, text=True, timeout=120,
                           env=dict(os.environ, ASAN_OPTIONS="detect_leaks=1"))
        assert r.returncode == 0 and r.stdout.strip() == "ok", f"{scenario}:\n{r.stdout}{r.stderr[-4000:]}"


# (name, text in autotune.cu, replacement, scenario that must then fail)
MUTANTS = [
    ("the slower candidate kept", "if (t < best_t) {", "if (t > best_t) {", "single_mode0"),
    ("options left changed after a failure", "if (code != BFS_OK) g->opt = saved;", "(void)saved;",
     "late_failure"),
    ("sample roots not spread over the degree order", "(int64_t)i * span / k", "(int64_t)i", "samples"),
    ("mode 3's switching thresholds not tuned", "{BFS_OPT_ALPHA, {2, 4, 8, 14, 32, 64}}, ", "",
     "mode_then_single"),
    ("a failing starting value ignored",
     "if (best_t == kFailed) return bfs_last_status() < 0 ? bfs_last_status() : BFS_ERR_CUDA;", "",
     "all_fail"),
]


@pytest.mark.parametrize("name,old,new,scenario", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistakes_are_caught(autotune_host, tmp_path, name, old, new, scenario):
    src = open(os.path.join(CSRC, "autotune.cu")).read()
    assert src.count(old) == 1, f"mutant {name!r} no longer applies"
    mutated = tmp_path / "autotune.cu"
    mutated.write_text(src.replace(old, new))
    exe = _build(str(mutated), str(tmp_path / "autotune_host"))
    r = subprocess.run([exe, scenario], capture_output=True, text=True, timeout=120)
    assert r.returncode != 0, f"{name}: scenario {scenario} still passes"
