"""A short bench.py run on the GPU prints one JSON line with every key of the
benchmark contract: the metric on the 256^3 workload, the roofline block of the
step kernel, the oracle CPU baseline, the end-to-end block with its copied
bytes, the kernel launch count of the timed region and the clock record."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "12", "--warmup", "3",
                        "--e2e-steps", "1", "--no-extra"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["unit"] == "MLUPS" and d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 12 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["dtype"] == "f32"
    assert d["data"] == "synthetic" and "256^3" in d["config"]["workload"]
    assert d["gpu_launches"] == 12
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    assert "traffic" in rf
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["unit"] == "MLUPS" and e2e["value"] > 0
    assert e2e["h2d_bytes_per_step"] == e2e["d2h_bytes_per_step"] == 10 * 256 ** 3 * 4
    ck = d["clocks"]
    assert ck["sm_mhz"] > 0 and ck["sm_max_mhz"] > 0 and isinstance(ck["reasons"], list)
    assert d["parity"]["fp32"]["pass"] is True
