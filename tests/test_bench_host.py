"""bench.py host logic on CPU: the DRAM-traffic record is used only for the kernel, lattice and
hop sources it was captured with; the host and clock records, the peaks lookup, the GFLOP/s
convention and the warm-up floor."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _write(tmp_path, sha, kernel="hop_f16n", lattice="64,32,32,32"):
    p = tmp_path / "traffic.txt"
    p.write_text(f"# comment\nkernel={kernel}\nlattice={lattice}\nbytes_per_launch=123456\nsource_sha256={sha}\n")
    return str(p)


def test_record_matches_current_sources(tmp_path):
    p = _write(tmp_path, bench.hop_source_hash())
    assert bench.recorded_traffic("hop_f16n", (64, 32, 32, 32), p) == 123456.0


def test_record_rejected_when_sources_kernel_or_lattice_differ(tmp_path):
    assert bench.recorded_traffic("hop_f16n", (64, 32, 32, 32), _write(tmp_path, "0" * 64)) is None
    good = _write(tmp_path, bench.hop_source_hash())
    assert bench.recorded_traffic("hop_f32", (64, 32, 32, 32), good) is None
    assert bench.recorded_traffic("hop_f16n", (96, 48, 48, 48), good) is None
    assert bench.recorded_traffic("hop_f16n", (64, 32, 32, 32), str(tmp_path / "missing.txt")) is None


def test_hash_covers_every_hop_source():
    for f in bench.HOP_SOURCES:
        assert os.path.exists(os.path.join(ROOT, "paper_2502_02490_gb300", "csrc", f))
    assert bench.hop_source_hash() == bench.hop_source_hash()


def test_host_cpu_record():
    import bench

    h = bench.host_cpu()
    assert h and f"{os.cpu_count()} logical cores" in h


def test_dslash_gflops_convention():
    import bench

    g = bench.dslash_gflops("hop_f16n", 10, 1.0, 1 << 20)  # 10 launches of 2^20 sites in 1 ms
    assert g["value"] == 1824 * (1 << 20) * 10 / 1e-3 / 1e9 and g["unit"] == "GFLOP/s"
    assert bench.dslash_gflops("hop_f16n", 0, 0.0, 8)["value"] is None


def test_host_cpu_names_arm_parts(tmp_path):
    import bench

    f = tmp_path / "cpuinfo"
    f.write_text("processor\t: 0\nBogoMIPS\t: 2000.00\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n\n"
                 "processor\t: 1\nCPU implementer\t: 0x41\nCPU part\t: 0xd4f\n")
    assert "implementer 0x41 part 0xd4f" in bench.host_cpu(str(f))
    assert "logical cores" in bench.host_cpu(str(tmp_path / "missing"))


def test_clock_summary_reports_median_and_throttle_reasons():
    import bench

    c = bench.Clocks(0)
    assert c.summary()["reasons"] == ["unsampled"]
    row = "0, {sm}, 2070, 900.5, 0x0000000000000004, Not Active, Not Active, Not Active, {cap}"
    c.rows = [[x.strip() for x in row.format(sm=s, cap=cap).split(",")]
              for s, cap in ((2070, "Not Active"), (1965, "Active"), (2070, "Not Active"))]
    s = c.summary()
    assert s["sm_mhz"] == 2070 and s["sm_max_mhz"] == 2070 and s["samples"] == 3
    assert s["reasons"] == ["sw_power_cap"]
    c.rows[0][5] = "Active"  # a hardware slowdown in one sample is reported
    assert bench.Clocks.summary(c)["reasons"] == ["hw_slowdown", "sw_power_cap"]


def test_measured_peaks_reads_the_copy_bandwidth_or_falls_back(tmp_path):
    import bench

    f = tmp_path / "peaks.json"
    f.write_text('{"hbm_gbs": 6785.9, "bf16_tflops": 1901.2}')
    assert bench.measured_peaks(str(f)) == (6785.9, "measured")
    for bad in ('{"bf16_tflops": 1901.2}', "not json", '[1, 2]', '{"hbm_gbs": -1}'):
        f.write_text(bad)
        assert bench.measured_peaks(str(f)) == (6800.0, "fallback"), bad
    assert bench.measured_peaks(str(tmp_path / "missing.json")) == (6800.0, "fallback")


def test_bench_rejects_fewer_than_three_warmup_steps():
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--warmup", "2"], capture_output=True,
                       text=True, timeout=120)
    assert r.returncode != 0 and "--warmup must be >= 3" in r.stderr


def test_cpu_apply_c1_record():
    """The CPU baseline's 4^4 apply of the oracle's D: a positive rate on the 2112 B/site
    convention, consistent with its own time per apply."""
    r = bench.cpu_apply_c1(reps=2)
    assert r["seconds_per_apply"] > 0 and r["processes"] == 1
    assert abs(r["sites_per_s"] * r["seconds_per_apply"] - 256) < 1e-6
    assert abs(r["GBps_2112B_per_site"] - r["sites_per_s"] * 2112 / 1e9) < 1e-9
