"""bench.py's reference arm (the FP64 oracle timed on the host cores) on the CPU: one JSON line
with the headline's metric, unit and workload, the oracle as its kind, no host-device copies;
under a two-rank launch only rank 0 runs and prints, and every rank exits 0."""
import json
import os
import socket
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _check_line(line, n_gpus):
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT and line["higher_is_better"] is True
    assert line["n_gpus"] == n_gpus and line["steps"] == 1 and line["warmup"] == 3
    assert line["value"] > 0 and line["ms_per_step"] > 0
    # the headline arm's config (the full LWA-like configuration), key for key
    cfg = line["config"]
    assert cfg["workload"] == "LWA-like: 256 ant, 128 chan, 2 pol, T=1024, 128x128 image, ci4"
    assert (cfg["antennas"], cfg["time_samples"], cfg["channels"], cfg["pols"]) == (256, 1024, 128, 2)
    assert cfg["grid"] == "64x64 padded to 128x128" and cfg["images_per_step"] == 262144
    assert cfg["parallelism"] == ("1 GPU" if n_gpus == 1 else "independent replicas per GPU")
    # ms_per_step is the measured time of the bounded sample step, not an extrapolation: the
    # timed steps fit well inside the run
    assert line["ms_per_step"] < 60e3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 1)


def test_reference_arm_two_ranks():
    pytest.importorskip("torch")
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port),
           "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    _check_line(lines[0], 2)
