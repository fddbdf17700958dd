"""The bench's reference arm on CPU: `bench.py --impl reference` times the
oracle's operator apply on a bounded sample and prints one JSON line with the
keys of the contract; under torchrun only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
           "--cpu-sample-elems", "3"]
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    res = _run({})
    assert res.returncode == 0, res.stderr
    lines = [ln for ln in res.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "GDOF/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"] == dict(value=line["value"], unit="GDOF/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    assert line["config"]["W"] == 8 and line["config"]["n_elem"] == 512
    # the GPU arm's workload config, and the time of the step's sample
    assert line["config"]["rhs_per_gpu"] == 64 and line["config"]["dof_per_rhs"] == 512 * 9 ** 3
    assert line["config"]["workload"].startswith("varcoef -div(a grad u)=f")
    assert line["ms_per_step"] > 0


def test_reference_arm_other_ranks_print_nothing():
    res = _run({"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert res.returncode == 0, res.stderr
    assert res.stdout.strip() == ""
