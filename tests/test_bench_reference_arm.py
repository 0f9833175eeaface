"""The benchmark's reference arm (the CPU oracle timed on host cores): its JSON line.

`bench.py --impl reference` runs the oracle on bounded samples of the FT-DGEMM workload and
prints one line with the same metric, unit and config keys as the GPU arm, plus the
`cpu_baseline` and a zero-copy `e2e`. Under a multi-rank launch rank 0 alone runs and prints;
the other ranks exit 0 without work. Both launches run on the CPU here, at a small size.
Also the fingerprint that ties a committed DRAM capture to the kernel code it measured.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REQUIRED = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
            "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
            "cpu_baseline", "e2e"}


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check_line(line, n, steps, warmup, gpus):
    assert REQUIRED <= set(line)
    assert line["impl"] == "reference"
    assert line["unit"] == "TFLOP/s" and line["higher_is_better"] is True
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (gpus, steps, warmup)
    assert line["value"] > 0 and line["ms_per_step"] > 0
    cfg = line["config"]
    assert cfg["workload"] == f"ft_dgemm_fp64_col_major_{n}x{n}x{n}"
    assert (cfg["M"], cfg["N"], cfg["K"]) == (n, n, n)
    assert "within" in cfg["l2"]  # a 512^3 problem's operands fit in L2, and the line says so
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
    assert cb["unit"] == line["unit"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def _env():
    env = dict(os.environ)
    env["PYTHONPATH"] = ROOT + os.pathsep + env.get("PYTHONPATH", "")
    env["CUDA_VISIBLE_DEVICES"] = ""
    return env


def test_reference_arm_one_rank():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--size", "512",
                        "--steps", "2", "--warmup", "3"],
                       cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=240)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 512, 2, 3, 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.timeout(300)
def test_reference_arm_two_ranks_rank0_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           "bench.py", "--impl", "reference", "--gpus", "2", "--size", "512", "--steps", "1",
           "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=_env(), capture_output=True, text=True, timeout=280)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 512, 1, 3, 2)


def test_profile_fingerprint_ignores_comments_and_catches_code_changes(tmp_path, monkeypatch):
    """A committed DRAM capture stays valid while only comments or layout change, and is
    voided by any change of code."""
    monkeypatch.syspath_prepend(ROOT)
    import bench
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    src = tmp_path / "k.cu"
    src.write_text("// header\n__global__ void k(float* x) {\n  x[0] = 1.0f;  // store\n}\n")
    h0 = bench.sources_sha256(["k.cu"])
    src.write_text("/* a new\n   block comment */\n// header, reworded\n\n__global__ void k(float* x) {\n"
                   "    x[0] = 1.0f;\n}\n")
    assert bench.sources_sha256(["k.cu"]) == h0
    src.write_text("// header\n__global__ void k(float* x) {\n  x[0] = 2.0f;  // store\n}\n")
    assert bench.sources_sha256(["k.cu"]) != h0
