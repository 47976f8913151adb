"""Host helpers of bench.py, on the CPU: the recorded DRAM traffic is only reported for the
kernel source and launch mode it was captured on, and the peaks fall back when the
measured file is missing."""
import bench


def _write(tmp_path, name, text):
    d = tmp_path / "profiles"
    d.mkdir(exist_ok=True)
    (d / name).write_text(text)


def test_recorded_traffic_needs_matching_source_and_launch(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc123")
    _write(tmp_path, "a.md", "notes\n\ntraffic_kernel: mac\ntraffic_launch: multi\nsource_hash: abc123\n"
                             "traffic_workload: bert-large-n8192\ntraffic_bytes_per_launch: 4699534194\n")
    _write(tmp_path, "b.md", "traffic_kernel: mac\ntraffic_launch: groups\nsource_hash: old999\n"
                             "traffic_workload: bert-large-n8192\ntraffic_bytes_per_launch: 1\n")
    assert bench.recorded_traffic("mac", "multi") == 4699534194.0
    assert bench.recorded_traffic("mac", "multi", "bert-base") is None  # captured on another workload
    assert bench.recorded_traffic("mac", "groups") is None  # captured on another source
    assert bench.recorded_traffic("ntt", "multi") is None   # no record for that kernel
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    assert bench.recorded_traffic("mac", "multi") is None   # the kernel changed since


def test_committed_traffic_record_is_well_formed():
    """A committed summary names a kernel, a launch mode, a workload, a 16-hex-digit fingerprint
    and a byte count (whether it matches the current source is the bench's business)."""
    import re

    recs = [p for p in (bench.ROOT / "profiles").glob("*.md") if "traffic_kernel:" in p.read_text()]
    assert recs
    for p in recs:
        t = p.read_text()
        assert re.search(r"^source_hash: [0-9a-f]{16}$", t, re.M), p
        assert re.search(r"^traffic_launch: (multi|groups)$", t, re.M), p
        assert re.search(r"^traffic_workload: (%s)$" % "|".join(bench.WORKLOADS), t, re.M), p
        assert float(re.search(r"^traffic_bytes_per_launch: ([0-9.eE+]+)$", t, re.M).group(1)) > 0


def test_peaks_fall_back_without_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", tmp_path)
    pk, src = bench.peaks()
    assert src == "fallback" and pk["hbm_gbs"] == 6800.0
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6749.7, "bf16_tflops": 1901.0}')
    pk, src = bench.peaks()
    assert src == "measured" and pk["hbm_gbs"] == 6749.7


def test_clock_summary_parses_nvidia_smi_rows():
    s = bench.ClockSampler(0)
    s.out = "\n".join([
        "0, 2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2062, 2070, 1210.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 345, 2070, 120.0, 0x0000000000000001, Not Active, Not Active, Not Active, Not Active",  # idle
        "garbage line",
    ])
    c = s.summary()
    assert c["samples"] == 3 and c["sm_max_mhz"] == 2070.0
    assert c["sm_mhz"] == 2066.0  # median over the loaded samples (idle ones dropped)
    assert c["reasons"] == ["sw_power_cap"]
    s.out = "0, 1800, 2070, 1300.0, 0x48, Active, Not Active, Active, Not Active"
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.out = ""
    assert s.summary() is None
