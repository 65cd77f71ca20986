"""Host-side logic of bench.py on the CPU: the clock sampler against a fake
nvidia-smi, the per-kernel work model, and the traffic lookup's digest key."""
import os
import stat
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

UUID0 = "GPU-00000000-1111-2222-3333-444444444444"
UUID1 = "GPU-99999999-1111-2222-3333-444444444444"


def _fake_smi(tmp_path, rows):
    """An nvidia-smi that prints `rows` (CSV, no header) every 20 ms until killed."""
    body = "\n".join(f"echo '{r}'" for r in rows)
    script = tmp_path / "nvidia-smi"
    script.write_text(textwrap.dedent("""\
        #!/bin/bash
        trap 'exit 0' TERM
        while true; do
        {body}
        sleep 0.02
        done
        """).format(body=body))
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


def _sample(tmp_path, monkeypatch, rows, uuid):
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, rows) + os.pathsep + os.environ["PATH"])
    s = bench.ClockSampler(uuid)
    s.start()
    return s.stop()


def test_clock_sampler_reads_its_own_gpu(tmp_path, monkeypatch):
    rows = [f"0, {UUID0}, 1965, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
            f"1, {UUID1}, 345, 2070, 90.0, 0x0000000000000000, Active, Not Active, Not Active, Not Active"]
    c = _sample(tmp_path, monkeypatch, rows, UUID0)
    assert c["sm_mhz"] == 1965.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] >= 1
    c = _sample(tmp_path, monkeypatch, rows, UUID1)
    assert c["sm_mhz"] == 345.0 and c["reasons"] == ["hw_slowdown"]


def test_clock_sampler_median_and_bad_fields(tmp_path, monkeypatch):
    rows = [f"0, {UUID0}, 2000, 2070, 700, 0x0, Not Active, Not Active, Not Active, Not Active",
            f"0, {UUID0}, 1900, 2070, 700, 0x0, Not Active, Not Active, Active, Not Active",
            f"0, {UUID0}, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]",
            "garbage line"]
    c = _sample(tmp_path, monkeypatch, rows, UUID0)
    assert c["sm_mhz"] in (1900.0, 1950.0, 2000.0)  # median over whole cycles of the four rows
    assert c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_thermal_slowdown"]


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    s = bench.ClockSampler(UUID0)
    s.start()
    c = s.stop()
    assert c["sm_mhz"] is None and c["reasons"] == ["nvidia-smi unavailable"]


def test_kernel_work_model():
    st = {"positions": 1000, "pass1_marks": 80, "pass2_marks": 50}
    m, n, tb = 1024, 3, 1 << 20
    assert bench.kernel_work("pass1_insert", st, m, n, tb) == (1000, "rand_or")
    assert bench.kernel_work("pass1_probe", st, m, n, tb) == (1000, "rand_read")
    assert bench.kernel_work("partition_count", st, m, n, tb) == (1000, "rand_read")
    assert bench.kernel_work("pass2_insert", st, m, n, tb) == (80, "rand_or")
    assert bench.kernel_work("pass2_classify", st, m, n, tb) == (80, "rand_read")
    assert bench.kernel_work("pack", st, m, n, tb) == (m + m / 4, "hbm")
    assert bench.kernel_work("class_map", st, m, n, tb) == (m / 4 + m, "hbm")
    assert bench.kernel_work("table_clear", st, m, n, tb) == (tb, "hbm")
    assert bench.kernel_work("emit", st, m, n, tb) == (m / 8 + 8 * 50, "hbm")
    assert bench.kernel_work("table_setup", st, m, n, tb) == (None, None)
    # the region-ordered first pass, 4 rounds: records and ranks per member, planes per round
    assert bench.kernel_work("ord_scatter", st, m, n, tb, 4) == (4 * (2 * m + m / 4) + 10 * 1000, "hbm")
    assert bench.kernel_work("ord_or", st, m, n, tb, 4) == (1000, "l2_or")
    assert bench.kernel_work("ord_probe", st, m, n, tb, 4) == (1000, "l2_read")
    assert bench.kernel_work("ord_classify", st, m, n, tb, 4) == (80, "l2_read")
    assert bench.kernel_work("ord_gather", st, m, n, tb, 4) == \
        (4 * (2 * m + m / 8) + 2 * 1000 + 1000 / 8 + 8 * 80, "hbm")


def test_roofline_of_an_ordered_kernel_takes_the_l2_peak():
    st = {"positions": 10**9, "pass1_marks": 80, "pass2_marks": 50}
    prof = {"ord_or": {"launches": 4, "ms": 8.0}, "ord_probe": {"launches": 4, "ms": 4.0}}
    peaks = {"or": 25e9, "read": 40e9, "buffer_bytes": 1 << 33, "l2_or": 200e9, "l2_read": 300e9,
             "l2_bytes": 32 << 20}
    r = bench.roofline(prof, st, 1024, 3, 1 << 20, peaks, 6000.0, {}, "wl", False, 1, 4)
    assert r["kernel"] == "ord_or" and r["bound"] == "l2" and r["unit"] == "Gaccess/s"
    assert abs(r["achieved"] - 125.0) < 1e-6 and abs(r["frac"] - 125.0 / 200.0) < 1e-9


def test_roofline_takes_the_dominant_modelled_kernel_per_launch():
    st = {"positions": 10**9, "pass1_marks": 80, "pass2_marks": 50}
    prof = {"pass1_insert": {"launches": 4, "ms": 8.0}, "table_setup": {"launches": 4, "ms": 100.0},
            "pass1_probe": {"launches": 4, "ms": 4.0}}
    peaks = {"or": 250e9, "read": 400e9, "buffer_bytes": 1 << 30}
    r = bench.roofline(prof, st, 1024, 3, 1 << 20, peaks, 6000.0, {}, "wl", False, 1)
    assert r["kernel"] == "pass1_insert" and r["bound"] == "hbm_random"
    # 1e9 positions over 4 launches of 2 ms each: 2.5e8 / 2 ms = 125 G/s against 250 G/s
    assert abs(r["achieved"] - 125.0) < 1e-6 and abs(r["frac"] - 0.5) < 1e-9
    # the same per launch when the profile sums two steps (8 launches, 16 ms)
    prof2 = {k: {"launches": 2 * v["launches"], "ms": 2 * v["ms"]} for k, v in prof.items()}
    r2 = bench.roofline(prof2, st, 1024, 3, 1 << 20, peaks, 6000.0, {}, "wl", False, 2)
    assert abs(r2["achieved"] - 125.0) < 1e-6


def test_traffic_lookup_is_keyed_by_workload_kernel_and_code(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    src = tmp_path / "paper_1602_05856_gb300" / "csrc"
    src.mkdir(parents=True)
    (src / "twopaco_kernels.cu").write_text("int f() { return 1; }\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    d = bench.kernel_code_digest()
    (prof / "dram_traffic_x.md").write_text(
        f"dram-traffic wl pass1_probe 123456 sha256:{d}\n"
        f"dram-traffic wl pass1_insert 777 sha256:{'0' * 64}\n")
    assert bench.ncu_traffic("wl", "pass1_probe") == 123456
    assert bench.ncu_traffic("wl", "pass1_insert") is None  # captured on other code
    assert bench.ncu_traffic("other", "pass1_probe") is None
    (src / "twopaco_kernels.cu").write_text("// a comment\nint f() { return 1; }\n\n")
    assert bench.ncu_traffic("wl", "pass1_probe") == 123456  # comments do not count
    (src / "twopaco_kernels.cu").write_text("int f() { return 2; }\n")
    assert bench.ncu_traffic("wl", "pass1_probe") is None


def test_workload_config_names_the_workload():
    c = bench.workload_config("bacterial_set", 35_000_000)
    assert c["workload"].startswith("bacterial_set") and c["k"] == 25
    assert c["filter_bits"] == 1 << 28 and c["rounds"] == 1 and "flushed" in c["l2"]
    assert "model" not in c
    c = bench.workload_config("mammal_set", 24_000_000_000)
    assert c["workload"].startswith("mammal_set") and c["filter_bits"] == 1 << 36
    assert c["rounds"] == 4 and "no flush" in c["l2"]
