"""bench.py's host-side contract, on the CPU: the reference arm (the FP64
oracle timed on host cores) prints one JSON line with the keys the benchmark
contract names; ranks other than 0 print nothing; the variant workloads' reference
arm reports itself unavailable; and the GPU arm fails loudly without a CUDA device
(there is no CPU path)."""
import json
import os
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMALL = ["--views", "1", "--width", "96", "--height", "64", "--buckets", "32", "--n", "4"]


def bench(*args, env=None, timeout=300):
    e = dict(os.environ, **(env or {}))
    return subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, env=e, capture_output=True, text=True,
                          timeout=timeout)


def test_reference_arm_prints_one_contract_line():
    r = bench("--impl", "reference", "--steps", "2", "--warmup", "1", *SMALL)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "Gfrag/s" and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "Gfrag/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert "workload" in d["config"]
    # the measured time of the calls as run, and the rate from the backward's time scaled to the whole sample
    assert d["ms_per_step_normalised"] >= d["ms_per_step"] > 0
    assert d["cpu_baseline"]["fwd_gfrag_s_1_thread"] > 0 and d["cpu_baseline"]["cpu_model"]


def test_reference_arm_other_ranks_stay_silent():
    r = bench("--impl", "reference", "--steps", "1", "--warmup", "0", *SMALL,
              env={"RANK": "1", "LOCAL_RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


@pytest.mark.parametrize("workload", ["world", "shadow"])
def test_variant_reference_arm_is_unavailable(workload):
    r = bench("--workload", workload, "--impl", "reference", "--steps", "1", "--warmup", "0")
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads(r.stdout.strip())
    assert d["impl"] == "reference" and "unavailable" in d


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the behaviour without a CUDA device")
def test_gpu_arm_fails_loudly_without_cuda():
    r = bench("--steps", "1", "--warmup", "1", *SMALL)
    assert r.returncode != 0
    assert "CUDA" in (r.stderr + r.stdout)


def test_step_form_flags():
    """The timed step is the fused launch unless --separate asks for the three launches;
    --fused names the default, the two exclude each other, and --no-fused-line is the
    older name of --no-other-step."""
    sys.path.insert(0, ROOT)
    import bench as b

    assert b.parse_args([]).fused is True
    assert b.parse_args(["--fused"]).fused is True
    assert b.parse_args(["--separate"]).fused is False
    with pytest.raises(SystemExit):
        b.parse_args(["--fused", "--separate"])
    assert b.parse_args(["--no-fused-line"]).no_other_step is True
    assert b.parse_args(["--no-other-step"]).no_other_step is True
    assert b.parse_args([]).no_other_step is False
