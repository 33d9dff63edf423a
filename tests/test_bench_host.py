"""bench.py's host-side logic on the CPU: the tracker-source hash that keys the
committed DRAM-traffic figure (blind to comments and blank lines, not to
code), the traffic lookup, the clock sampler's parsing of nvidia-smi samples,
and the peak-bandwidth file with its fallback."""
import json

import bench


def make_tree(root, render_src, device_src, profile=None):
    csrc = root / "paper_2504_04564_gb300" / "csrc"
    csrc.mkdir(parents=True, exist_ok=True)
    (csrc / "render.cu").write_text(render_src)
    (csrc / "vdbc_device.cuh").write_text(device_src)
    if profile is not None:
        (root / "profiles").mkdir(exist_ok=True)
        (root / "profiles" / "k_pt_vdb_turbulence512.md").write_text(profile)


def test_source_hash_ignores_comments_and_blank_lines_not_code(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    make_tree(tmp_path, "int a;  // a note\n/* a block\n   comment */\nint b;\n", "int c;\n")
    h = bench.kernel_source_hash()
    make_tree(tmp_path, "// another note\n\nint a;\n\n\nint b;   /* x */\n", "int c; // y\n")
    assert bench.kernel_source_hash() == h
    make_tree(tmp_path, "int a;\nint b = 1;\n", "int c;\n")
    assert bench.kernel_source_hash() != h
    make_tree(tmp_path, "int a;\nint b;\n", "int d;\n")
    assert bench.kernel_source_hash() != h


def test_traffic_is_reported_only_for_the_profiled_source(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    make_tree(tmp_path, "int a;\n", "int c;\n")
    assert bench.profiled_traffic() is None                    # no summary committed
    h = bench.kernel_source_hash()
    make_tree(tmp_path, "int a;\n", "int c;\n",
              "# k_pt\n\nkernel_source_sha256_16: %s\ndram_bytes_per_launch_full_size: 1234500\n" % h)
    assert bench.profiled_traffic() == 1234500.0
    make_tree(tmp_path, "int a = 2;\n", "int c;\n")            # the kernel changed since the capture
    assert bench.profiled_traffic() is None


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0

    def kill(self):
        pass


def test_clock_sampler_takes_the_median_and_throttle_reasons_of_the_timed_region():
    cs = bench.ClockSampler()
    cs.proc = _FakeProc()
    row = "0, {sm}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, {pc}"
    cs.lines = [row.format(sm=1000, hw="Active", pc="Not Active")]          # before the region: skipped
    cs.skip = 1
    cs.lines += [row.format(sm=s, hw="Not Active", pc=pc) for s, pc in
                 ((2070, "Not Active"), (1980, "Active"), (2070, "Not Active"), ("bad", "Not Active"))]
    r = cs.stop()
    assert r["sm_mhz"] == 2070.0 and r["sm_max_mhz"] == 2070.0 and r["samples"] == 3
    assert r["reasons"] == ["sw_power_cap"]                    # hw_slowdown only before the region
    empty = bench.ClockSampler()
    assert empty.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_peaks_come_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6780.7, "bf16_tflops": 1900.0}))
    assert bench.measured_peaks() == (6780.7, "measured")
