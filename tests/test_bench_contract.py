"""The bench's JSON line (CPU): the reference arm, which times the oracle on
the host cores, prints one line with the contract's keys; a rank other than
0 of a multi-rank launch prints nothing and exits 0; the ncu-summary readers
give the committed figures only while the kernel sources match the capture.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _run(extra_env, *args):
    env = dict(os.environ, **extra_env)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({}, "--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert cb["one_core"]["cores"] == 1 and cb["one_core"]["value"] > 0
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}, "--impl", "reference", "--steps", "1",
             "--warmup", "0", "--gpus", "2")
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]


@pytest.mark.parametrize("path", [bench.PROFILE, bench.PROFILE_FULL_MODEL])
def test_profile_figures_follow_the_kernel_hash(path, tmp_path):
    fields = bench._profile_fields(path)
    traffic, note = bench.profiled_traffic(path)
    share = bench.profiled_fp64_share(path)
    inst = bench.profiled_inst_per_32(path)
    if fields.get("kernel_sources_sha256") == bench.kernel_sources_sha256():
        assert traffic == int(fields["traffic_bytes_per_launch"]) and traffic > 0
        assert share == pytest.approx(float(fields["fp64_pipe_pct_of_peak"]) / 100.0)
        if "warp_inst_per_32_evals" in fields:
            assert inst == pytest.approx(float(fields["warp_inst_per_32_evals"])) and inst > 0
    else:
        assert traffic is None and share is None and inst is None
    # a summary whose hash does not match gives no figures
    stale = tmp_path / "stale.md"
    stale.write_text(open(path).read().replace(fields["kernel_sources_sha256"], "0" * 64))
    assert bench.profiled_traffic(str(stale))[0] is None and bench.profiled_fp64_share(str(stale)) is None
