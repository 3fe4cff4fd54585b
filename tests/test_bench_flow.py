"""bench.py's own-arm flow, end to end, on a machine without a GPU.

tests/bench_flow/run_with_stand_ins.py replaces torch.cuda with host
stand-ins and the BFS library with one whose searches are the CPU oracle's,
then runs bench.main on small sizes in a child process.  The JSON line must
carry every key the measurement contract asks for, and a serving attempt
that stalls must be reported and retried (or, twice stalled, reported as an
error) without losing the line.  The numbers of these runs mean nothing.
"""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HARNESS = os.path.join(HERE, "bench_flow", "run_with_stand_ins.py")
BENCH = os.path.join(os.path.dirname(HERE), "bench.py")


def _run(*stalling):
    r = subprocess.run([sys.executable, HARNESS, *stalling], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    lines = r.stdout.strip().splitlines()
    return json.loads(lines[-2]), lines[-1]


def _check_contract(line):
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e",
              "gpu_launches", "clocks"):
        assert k in line, k
    assert line["value"] > 0 and line["n_gpus"] == 1 and line["steps"] == 1 and line["warmup"] == 3
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["config"]["workload"] == "kronecker_scale10_ef16_64roots"
    roof = line["roofline"]
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s" and "traffic" in roof
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] > 0 and cpu["sample"]
    e2e = line["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] > 0 and e2e["d2h_bytes_per_step"] > 0
    assert line["gpu_launches"] == 64
    assert set(line["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
    assert len(line["ablation"]) == 4 and all("error" not in v for v in line["ablation"].values())
    assert line["batched"]["queries_per_s"] > 0 and line["batched"]["uneven_mix"]["queries_per_s"] > 0
    conc = line["batched"]["uneven_mix"]["concurrent"]
    assert conc["queries_per_s"] > 0 and conc["levels_match_sequential"] is True
    lp = line["layer_profile"]
    assert "error" not in lp and lp["roots"] == 64 and lp["layers"][0]["d"] == 0
    assert sum(x["edges_share"] for x in lp["layers"]) == pytest.approx(1.0)
    others = line["other_workloads"]
    assert set(others) == {"erdos_renyi_scale9_ef16_64roots", "kronecker_scale8_ef16_64roots"}
    for v in others.values():
        assert "error" not in v and v["hm_gteps"] > 0 and 0 < v["roofline"]["frac"]
        assert v["teps_stats"]["runs"] == 128 and v["mean_launch_us"] > 0


def test_flow_without_stalls():
    line, how = _run()
    _check_contract(line)
    assert how == "exit: returned 0"
    assert line["serving"]["queries_per_s"] > 0 and "stalls_before_this_attempt" not in line["serving"]


def test_flow_with_one_stalled_serving_attempt():
    line, how = _run("0")
    _check_contract(line)
    assert how == "exit: direct exit 0"  # the stalled server is left alive, so no destructors run
    assert line["serving"]["queries_per_s"] > 0
    assert len(line["serving"]["stalls_before_this_attempt"]) == 1


def test_flow_with_two_stalled_serving_attempts():
    line, how = _run("0", "1")
    _check_contract(line)
    assert line["serving"]["error"] == "serving measurement stopped twice"
    assert len(line["serving"]["stalls"]) == 2


def test_reference_arm_line():
    """--impl reference (the oracle on the host cores) on a small graph."""
    r = subprocess.run([sys.executable, BENCH, "--impl", "reference", "--scale", "10",
                        "--steps", "2", "--warmup", "3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-4000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "GTEPS"
    assert line["steps"] == 2 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["config"]["workload"] == "kronecker_scale10_ef16_64roots"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GTEPS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_no_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, BENCH, "--impl", "reference", "--scale", "10", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_flow_with_two_ranks_over_gloo(tmp_path):
    """Two replicas (ranks over gloo, as under torchrun): rank 0 prints one
    line whose value is the sum over the ranks, both ranks finish."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), HARNESS],
                       capture_output=True, text=True, timeout=900, cwd=str(tmp_path))
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    out = [ln for ln in r.stdout.splitlines() if ln.strip()]
    lines = [json.loads(ln) for ln in out if ln.startswith("{")]
    assert len(lines) == 1 and sum(ln.startswith("exit:") for ln in out) == 2
    line = lines[0]
    assert line["n_gpus"] == 2 and line["value"] > 0 and line["config"]["parallelism"] == "replicas"
