"""bench.py's command line and the reference arm's JSON line (CPU only).

The reference arm times the CPU oracle on a bounded sample of the bench
workload; its line must carry the keys the JSON contract names, with the
oracle described as the baseline and no host<->device bytes.
"""
import json
import subprocess
import sys
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def test_reference_arm_line():
    # a scale-12 R-MAT of the bench recipe keeps the CPU suite short (the box runs scale 24)
    out = subprocess.run([sys.executable, str(ROOT / "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "3", "--graph-scale", "12"], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [line for line in out.stdout.splitlines() if line.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["value"] > 0 and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == "rmat12_sssp" and d["config"]["queries_per_step"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["unit"] == d["unit"]


@pytest.mark.parametrize("flag", ["--configs", "--serving", "--ablation", "--ncp", "--ll", "--bc", "--walks",
                                  "--local-ppr", "--grid"])
def test_every_mode_flag_parses(flag, monkeypatch):
    sys.path.insert(0, str(ROOT))
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py", flag])
    args = bench.parse()
    assert getattr(args, flag[2:].replace("-", "_")) is True
    assert args.gpus == 1 and args.impl == "fg"


def test_step_sources_cover_the_list_before_repeating():
    sys.path.insert(0, str(ROOT))
    import numpy as np
    import bench
    srcs = np.arange(1000, dtype=np.int32)
    seen = []
    for step in range(5):
        for rank in range(2):
            b = bench.step_sources(srcs, rank, 2, step, 100)
            assert len(b) == 100 and b.flags["C_CONTIGUOUS"]
            seen.append(b)
    allv = np.concatenate(seen)
    assert len(np.unique(allv)) == 1000  # ten blocks of 100, each once
    assert np.array_equal(bench.step_sources(srcs, 0, 2, 5, 100), seen[0])  # then the list wraps


def test_traffic_record_matches_code_not_comments(tmp_path, monkeypatch):
    """The committed ncu traffic record is used only for the kernel code it was
    taken from (a comment edit keeps it, a code edit drops it) and only for the
    captured launch (sources per launch, group size)."""
    sys.path.insert(0, str(ROOT))
    import bench
    csrc = tmp_path / "paper_2103_14915_gb300" / "csrc"
    csrc.mkdir(parents=True)
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = csrc / "k.cu"
    src.write_text("// header\n__global__ void k(int *p) {\n  p[0] = 1;  // store\n}\n")
    sha = bench.code_sha256_16(src)
    (prof / "t.txt").write_text(f"# note: a: b\nsource_sha256_16: {sha}\ncapture_sources: 256\ncapture_group: 64\n"
                                "dram_bytes_per_launch: 1000\n")
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    assert bench.kernel_traffic("t.txt", "k.cu", 256, 64) == 1000.0
    assert bench.kernel_traffic("t.txt", "k.cu", 128, 64) is None
    assert bench.kernel_traffic("t.txt", "k.cu", 256, 32) is None
    src.write_text("// another header\n\n__global__ void k(int *p) {\n  p[0] = 1;\n}\n")  # comments only
    assert bench.kernel_traffic("t.txt", "k.cu", 256, 64) == 1000.0
    src.write_text("__global__ void k(int *p) {\n  p[0] = 2;\n}\n")  # the code changed
    assert bench.kernel_traffic("t.txt", "k.cu", 256, 64) is None
