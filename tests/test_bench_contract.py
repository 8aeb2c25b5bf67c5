"""The benchmark's JSON-line contract on the CPU: the reference arm (the CPU
oracle timed on the host) prints one line with the contract's keys, and under a
two-process launch only rank 0 prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
        "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"}


def _json_lines(text):
    out = []
    for line in text.splitlines():
        line = line.strip()
        if line.startswith("{"):
            out.append(json.loads(line))
    return out


def _run(args, **kw):
    r = subprocess.run([sys.executable, *args], cwd=ROOT, capture_output=True, text=True, timeout=600, **kw)
    assert r.returncode == 0, r.stderr[-2000:]
    return _json_lines(r.stdout)


def _check_reference_line(d, steps, warmup, gpus=1):
    assert KEYS <= set(d), KEYS - set(d)
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["unit"] == "tests/s" and d["higher_is_better"] is True
    assert d["n_gpus"] == gpus and d["steps"] == steps and d["warmup"] == warmup
    assert d["ms_per_step"] > 0 and d["data"] == "synthetic" and d["vs_baseline"] is None
    assert isinstance(d["config"].get("workload"), str)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_line():
    lines = _run(["bench.py", "--impl", "reference", "--workload", "small1k", "--steps", "2", "--warmup", "1"])
    assert len(lines) == 1
    _check_reference_line(lines[0], 2, 1)


def test_reference_arm_mcs_order():
    lines = _run(["bench.py", "--impl", "reference", "--workload", "small1k", "--order", "mcs", "--steps", "1",
                  "--warmup", "0"])
    assert len(lines) == 1
    _check_reference_line(lines[0], 1, 0)
    assert "MCS" in lines[0]["config"]["order"]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_reference_arm_under_two_ranks_prints_once():
    pytest.importorskip("torch")
    lines = _run(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                  "--master-port", str(_free_port()), "bench.py", "--impl", "reference", "--gpus", "2",
                  "--workload", "small1k", "--steps", "1", "--warmup", "0"])
    assert len(lines) == 1
    _check_reference_line(lines[0], 1, 0, gpus=2)
