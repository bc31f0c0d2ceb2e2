"""The JSON line of bench.py's reference arm (the oracle on the host cores):
the keys the launch contract needs, on a tiny bounded sample (CPU only)."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "3000",
                          "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["value"] > 0
    assert j["cpu_baseline"]["kind"] == "oracle" and j["cpu_baseline"]["value"] == j["value"]
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["e2e"]["d2h_bytes_per_step"] == 0
    assert j["config"]["workload"] == "rng-1m-d128"


def test_clock_sampler_summary(tmp_path, monkeypatch):
    """The clock sampler's summary (median SM clock, maximum, the throttle
    reasons seen active) from a stand-in sampler that prints the query's
    CSV fields; its temporary file is removed afterwards."""
    import time
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\n"
                    "i=0\n"
                    "while true; do\n"
                    "  if [ $i = 2 ]; then r='Active'; else r='Not Active'; fi\n"
                    "  echo \"0, 1900, 2070, 700.5, 0x0, Not Active, Not Active, Not Active, $r\"\n"
                    "  i=$((i+1)); sleep 0.03\n"
                    "done\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}:{os.environ['PATH']}")
    sys.path.insert(0, ROOT)
    import bench
    c = bench.Clocks(0)
    c.start()
    time.sleep(0.4)
    r = c.stop()
    assert r["sm_mhz"] == 1900.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"] and r["samples"] >= 3
    assert not os.path.exists(c.path)
