"""Host-side pieces of the benchmark, on the CPU: the clock sampler against a
fake nvidia-smi (throttle reasons reported, none invented), the measured-peak
loader, and the algorithmic byte counts of the roofline (each pivot row once,
plus row v and row p(v) per vertex; CSR adds the position gathers)."""
import os
import stat
import time

import numpy as np

import bench
import graphgen as gg

FAKE = """#!/bin/sh
echo "2070, 2070, 500.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active"
echo "2065, 2070, 700.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active"
echo "1200, 2070, 900.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active"
echo "[N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]"
exec sleep 30
"""


def _fake_smi(tmp_path, body):
    d = tmp_path / "bin"
    d.mkdir()
    p = d / "nvidia-smi"
    p.write_text(body)
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(d)


def test_clock_sampler_reads_clocks_and_reasons(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, FAKE) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    c = s.stop()
    assert c["samples"] == 3                        # the unparsable line is skipped
    assert c["sm_mhz"] == 2065.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_clock_sampler_quiet_gpu(tmp_path, monkeypatch):
    quiet = "#!/bin/sh\n" + 'echo "2070, 2070, 300.0, 0x0, Not Active, Not Active, Not Active, Not Active"\n' * 3 + \
        "exec sleep 30\n"
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, quiet) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(0)
    s.start()
    time.sleep(0.5)
    c = s.stop()
    assert c["reasons"] == [] and c["sm_mhz"] == 2070.0


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(0)
    s.start()
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_measured_peaks_loaded():
    peaks, kind = bench.load_peaks()
    if os.path.exists(os.path.join(bench.ROOT, "MEASURED_PEAKS.json")):
        assert kind == "measured" and peaks["hbm_gbs"] > 0
    else:
        assert kind == "fallback" and peaks["hbm_gbs"] == 6800.0


def test_algorithmic_bytes():
    g = gg.subtree_dense(100, 20, 1)
    assert bench.algorithmic_bytes(g) == 3 * g.n * g.words * 4
    c = gg.dense_to_csr(g)
    nnz = int(c.row_ptr[-1])
    assert c.nnz == nnz == int(np.unpackbits(g.rows.view(np.uint8)).sum())
    assert bench.algorithmic_bytes(c) == 3 * (8 * c.n + 4 * nnz) + 4 * nnz


def test_traffic_figure_follows_the_kernel_sources(tmp_path):
    """The roofline's traffic is read from the kept ncu summary only while the
    kernel's sources hash to the value recorded at capture time."""
    summary, srcs = bench.TRAFFIC_SUMMARIES["dense16k"]
    for p in srcs:
        (tmp_path / os.path.dirname(p)).mkdir(parents=True, exist_ok=True)
        (tmp_path / p).write_bytes(open(os.path.join(bench.ROOT, p), "rb").read())
    (tmp_path / "profiles").mkdir()
    digest = bench.sources_sha256(srcs, str(tmp_path))
    (tmp_path / summary).write_text(f"kernel: x\nsource_sha256: {digest}\ndram_bytes_per_launch: 69120000\n")
    assert bench.ncu_traffic("dense16k", root=str(tmp_path))[0] == 69120000.0
    (tmp_path / summary).write_text(f"source_sha256: {'0' * 64}\ndram_bytes_per_launch: 69120000\n")
    t, note = bench.ncu_traffic("dense16k", root=str(tmp_path))
    assert t is None and "changed" in note
    (tmp_path / summary).write_text("dram_bytes_per_launch: 1\n")
    assert bench.ncu_traffic("dense16k", root=str(tmp_path))[0] is None
    assert bench.ncu_traffic("batch4096", root=str(tmp_path))[0] is None
