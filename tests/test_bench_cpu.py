"""The benchmark's reference arm on the host: the JSON line keeps the
contract (impl, metric, unit, steps, warm-up, cpu_baseline, e2e with zero
copies), carries the GPU arm's unit and dtype strings (so that the two
lines can be divided), and its value is the oracle's own throughput on all
host cores over the timed steps."""
from __future__ import annotations

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run(
        [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
         "--steps", "2", "--warmup", "1", "--workload", "quant-small"],
        capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["steps"] == 2 and line["warmup"] == 1 and line["n_gpus"] == 1
    assert line["unit"] == "GB/s (input bytes compressed per second)"
    assert line["higher_is_better"] is True
    assert line["dtype"] == "u8/u32 symbols (integer/byte path, lossless)"
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == (os.cpu_count() or 1)
    assert cb["value"] == line["value"] and cb["unit"] == line["unit"] and cb["cpu_model"]
    assert "uint16 quant codes" in cb["sample"] and "2 timed steps" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    # a step compresses whole chunks (or the whole input when it is shorter)
    n = int(cb["sample"].split("first ")[1].split(" bytes")[0])
    assert n > 0 and (n % 4096 == 0 or n == 1 << 20)


def test_issue_roofline_from_committed_profiles():
    """The issue roofline divides the ncu instruction count by the live time
    and 4 warp instructions per SM per cycle; a profile taken on other
    sources gives no figure."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench._issue_roofline("compress_kernel", "compress_kernel_quant-256MiB.md",
                              bench.KERNEL_SOURCES, 2.0, 1 << 20, 152, 2000.0)
    assert r["peak"] == 152 * 4 * 2000e6 / 1e9
    if r["achieved"] is not None:  # the profile matches the sources
        assert abs(r["achieved"] - r["warp_inst_per_launch"] / 2e-3 / 1e9) < 0.1
        assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
        assert r["warp_inst_per_symbol"] == round(r["warp_inst_per_launch"] / (1 << 20), 2)
    other = bench._issue_roofline("decompress_kernel", "decompress_kernel_quant-256MiB.md",
                                  bench.KERNEL_SOURCES, 1.0, 1 << 20, 152, 2000.0)
    assert other["achieved"] is None and other["frac"] is None
