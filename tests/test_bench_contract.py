"""The benchmark's reference arm (the CPU oracle timed as the reference, the
one part of bench.py that runs without a GPU) prints one JSON line with the
contract's keys, for every operation."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("op", ["dilate", "erode", "fill_holes", "dt"])
def test_reference_arm_json_line(op):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--op", op,
                          "--workload", "single512", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, check=True).stdout
    lines = [l for l in out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["config"]["op"] == op
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_kernel_hash_ignores_comments_only():
    """The staleness check of the committed ncu counters: a comment or blank
    line does not change the kernel's code hash, a code change does."""
    sys.path.insert(0, ROOT)
    import bench
    files = {}

    def read(f):
        return files[f]

    base = {f: open(os.path.join(ROOT, f)).read() for f in
            ("paper_1311_0378_gb300/csrc/recon_kernels.cu", "paper_1311_0378_gb300/csrc/recon_internal.h")}
    files.update(base)
    h0 = bench.kernel_hash(read)
    assert h0 == bench.kernel_hash()
    k = "paper_1311_0378_gb300/csrc/recon_kernels.cu"
    files[k] = "// a new comment\n\n/* and a block\n comment */\n" + base[k]
    assert bench.kernel_hash(read) == h0
    files[k] = base[k].replace("constexpr unsigned FULL = 0xFFFFFFFFu;", "constexpr unsigned FULL = 0xFFFFFFFEu;")
    assert bench.kernel_hash(read) != h0
