"""bench.py's host-side logic, on the CPU: the reference arm's JSON line (the
oracle timed on the host cores -- the driver runs this arm every round), the
gating of the recorded DRAM traffic by the kernel sources' digest and its
scaling to n, and the reading of the clock record (throttle reasons, median
SM clock)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("workload", ["real-fp32-tan64", "real-fp32-rerun", "complex64"])
def test_reference_arm_prints_one_complete_line(workload):
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", workload,
                        "--steps", "1", "--warmup", "0"], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    W = bench.WORKLOADS[workload]
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "matrices/s" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 1 and d["warmup"] == 0 and d["n_gpus"] == 1
    assert d["dtype"] == W["dtype"] and d["config"]["workload"] == W["desc"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "matrices/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] - d["config"]["sample_per_step"] / d["value"] * 1e3) \
        <= 1e-6 * d["ms_per_step"]


def test_recorded_traffic_needs_the_recorded_digest_and_scales_with_n(monkeypatch):
    w = "real-fp32-tan64"
    with open(os.path.join(ROOT, "profiles", "dram_traffic.txt")) as f:
        row = next(ln.split() for ln in f if ln.split()[:1] == [w])
    digest, n_cap, rd, wr = row[1], int(row[3]), float(row[4]), float(row[5])
    # sources with the recorded digest: the capture scaled to n
    monkeypatch.setattr(bench, "sources_digest", lambda workload: digest)
    assert bench.recorded_traffic(w, n_cap) == pytest.approx(rd + wr, rel=1e-12)
    assert bench.recorded_traffic(w, 4 * n_cap) == pytest.approx(4 * (rd + wr), rel=1e-12)
    # the traffic of a kernel whose sources changed is not reported
    monkeypatch.setattr(bench, "sources_digest", lambda workload: "0000000000000000")
    assert bench.recorded_traffic(w, n_cap) is None


class _Done:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampled(lines):
    c = bench.ClockSampler(0)
    c.proc = _Done()
    c.lines = list(lines)
    return c.stop()


def test_clock_record_reasons_and_median():
    na, act = "Not Active", "Active"
    rows = [f"0, {mhz}, 2070, 950.0, 0x0, {na}, {na}, {na}, {cap}"
            for mhz, cap in ((2070, na), (2055, act), (2070, na), (1980, na), (2070, act))]
    r = _sampled(rows + ["garbage", "0, [N/A], 2070, 1, 0x0, a, b, c, d"])
    assert r["samples"] == 5 and r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    r = _sampled([f"0, 1500, 2070, 900.0, 0x0, {act}, {na}, {act}, {na}"])
    assert r["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"] and r["sm_mhz"] == 1500.0


def test_clock_record_without_nvidia_smi():
    c = bench.ClockSampler(0)
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]
