"""The reference arm of the benchmark (`bench.py --impl reference`) runs the float64 oracle on the
host cores, so its JSON-line contract is checked here without a GPU: one line from rank 0 with the
arm's metric, unit and cpu_baseline, zero host-device bytes, and nothing from other ranks."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(env_extra, *args):
    env = dict(os.environ)
    env.update(env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return [l for l in r.stdout.splitlines() if l.strip()]


def test_reference_arm_prints_one_line_with_the_contract_keys():
    # 3 steps leave 50 s per step: the largest KH sample the rule allows (2048^2 on a few cores),
    # a few seconds per step
    lines = run_bench({"RANK": "0", "WORLD_SIZE": "1", "LOCAL_RANK": "0"}, "--steps", "3", "--warmup", "0")
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["higher_is_better"] is True and d["value"] > 0
    assert d["unit"] == "cell-stages/s" and d["steps"] == 3 and d["warmup"] == 0
    nproc = os.cpu_count() or 1
    want = 32
    for s in (64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536, 2048):
        if s * s * 3 * 1.0e-6 / nproc <= 150.0 / 3:
            want = s
    assert d["config"]["sample_side"] == want
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == nproc and cb["value"] == d["value"]
    assert f"{want}^2" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["ms_per_step"] > 0


def test_reference_arm_other_ranks_print_nothing():
    lines = run_bench({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--steps", "3", "--warmup", "0")
    assert lines == []
