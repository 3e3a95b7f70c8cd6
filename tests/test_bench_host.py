"""Host logic of the bench line (no GPU).  `roofline.traffic`: the DRAM bytes
of the committed ncu summary are reported only for the captured kernel
variant and L2 prefetch distance and only while the kernel sources still
match the digests recorded with the capture."""
import hashlib
import os
import shutil

import bench

NAME = "k_stream_collide_micropost_filter_256x128x64_f32.md"
SRCS = ("lattice_kernels.cu", "lbibm_internal.cuh")


def _tree(tmp_path):
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    (root / "paper_1110_0995_gb300" / "csrc").mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", NAME), root / "profiles" / NAME)
    for f in SRCS:
        shutil.copy(os.path.join(bench.ROOT, "paper_1110_0995_gb300", "csrc", f),
                    root / "paper_1110_0995_gb300" / "csrc" / f)
    # digests of the copied sources, so that this tests the logic whether or
    # not the committed summary is current
    prof = root / "profiles" / NAME
    digests = " ".join(f"{f} {hashlib.sha256((root / 'paper_1110_0995_gb300' / 'csrc' / f).read_bytes()).hexdigest()}"
                       for f in SRCS)
    prof.write_text("\n".join(f"kernel_source_sha256: {digests}" if l.startswith("kernel_source_sha256: ") else l
                              for l in prof.read_text().splitlines()) + "\n")
    return root


def _recorded():
    text = open(os.path.join(bench.ROOT, "profiles", NAME)).read()
    line = [l for l in text.splitlines() if l.startswith("dram_bytes_per_launch: ")][0]
    return int(line.split(": ")[1])


def test_traffic_only_for_the_captured_kernel(tmp_path, monkeypatch):
    root = _tree(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(root))
    wl, st, var = "micropost_filter_256x128x64", "f32", {"npt": 1, "bs": 128, "pf": 65536}
    assert bench.profiled_traffic(wl, st, var) == _recorded()
    assert bench.profiled_traffic(wl, st, {"npt": 2, "bs": 256, "pf": 65536}) is None   # another variant
    assert bench.profiled_traffic(wl, st, {"npt": 1, "bs": 128, "pf": 0}) is None       # another prefetch distance
    assert bench.profiled_traffic(wl, "f16", var) is None                      # no summary for it
    src = root / "paper_1110_0995_gb300" / "csrc" / SRCS[1]
    src.write_text(src.read_text() + "\n")                                      # the kernel changed
    assert bench.profiled_traffic(wl, st, var) is None


def test_clock_summary_from_nvidia_smi_lines():
    """The clocks object of the bench line from sampled nvidia-smi CSV rows:
    median SM clock of the busy samples, the maximum, every active throttle
    reason; no samples -> 'unavailable'."""
    s = bench.ClockSampler(0)
    s.lines = ["1965, 2070, Not Active, Not Active, Not Active, Not Active",
               "2070, 2070, Not Active, Not Active, Not Active, Active",
               "2070, 2070, Not Active, Not Active, Not Active, Not Active",
               "2055, 2070, Not Active, Not Active, Not Active, Not Active",
               "[N/A], 2070, Not Active, Not Active, Not Active, Not Active",
               "garbage"]
    out = s.summary()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 4}
    s.lines = ["600, 2070, Active, Not Active, Active, Not Active"] * 3
    assert s.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    s.lines = []
    assert s.summary()["reasons"] == ["unavailable"]


def test_workloads_and_oracle_samples():
    """The bench's named workloads have the sizes they are named for, an
    unknown name is refused, and the oracle's bounded sample is the largest
    filter instance within the node budget."""
    import pytest

    (f,) = bench.make_workload("micropost_filter_256x128x64")
    assert f.dims == (256, 128, 64) and len(f.meshes) == 62
    (c,) = bench.make_workload("channel_32x16x64_1rbc")
    assert c.dims == (32, 16, 64) and len(c.meshes) == 1
    with pytest.raises(ValueError):
        bench.make_workload("no_such_workload")
    for budget, dims in ((256 * 128 * 64, (256, 128, 64)), (256 * 128 * 64 - 1, (128, 64, 64)),
                         (64 * 64 * 64, (64, 64, 64)), (10, (32, 32, 16))):
        sc, n = bench.oracle_sample_scene(budget)
        assert sc.dims == dims and n == dims[0] * dims[1] * dims[2]


def test_peak_from_the_measured_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peak() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6791.0, "bf16_tflops": 1873.4}')
    assert bench.measured_peak() == (6791.0, "measured")
