"""Host logic of bench.py on CPU: the classify kernel's source key, the
algorithmic byte counts behind the roofline, and the clock sampler's reading
of nvidia-smi rows."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_kernel_key_covers_the_classify_section_only(tmp_path, monkeypatch):
    key = bench.kernel_sha()
    assert len(key) == 16 and int(key, 16) >= 0
    # an edit outside the classify section keeps the key, one inside changes it
    src = open(bench.KERNEL_FILE).read()
    a = src.index("// a2..a5: persistent streaming classification")
    outside = tmp_path / "outside.cu"
    outside.write_text(src + "\n// another kernel's comment\n")
    inside = tmp_path / "inside.cu"
    inside.write_text(src[:a + 60] + "// a classify comment\n" + src[a + 60:])
    monkeypatch.setattr(bench, "KERNEL_FILE", str(outside))
    assert bench.kernel_sha() == key
    monkeypatch.setattr(bench, "KERNEL_FILE", str(inside))
    assert bench.kernel_sha() != key


def test_traffic_profile_is_ignored_for_other_sources(tmp_path, monkeypatch):
    prof = tmp_path / "traffic.txt"
    prof.write_text("# comment\nkernel_sha = 0000000000000000\nworkload = large\n"
                    "bytes_per_launch = 123\n")
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(prof))
    assert bench.profiled_traffic("large") is None
    prof.write_text(f"kernel_sha = {bench.kernel_sha()}\nworkload = large\nbytes_per_launch = 123\n")
    assert bench.profiled_traffic("large") == 123.0
    assert bench.profiled_traffic("7dof") is None


def test_algorithmic_bytes():
    info = {"record_bytes": 1000, "num_edges": 10, "num_tiles": 3, "round_filter": 0}
    # every record once and 8 B of pass bits per edge
    assert bench.algorithmic_bytes(info) == 1000 + 80
    assert bench.algorithmic_bytes(info, 400) == 1000 + 80      # unfiltered: counter ignored
    f = dict(info, round_filter=1)
    # filtered: the copied record bytes, the pass bits and 28 B per round slot (32 per tile)
    assert bench.algorithmic_bytes(f, 400) == 400 + 80 + (28 * 32 + 24) * 3


def test_clock_sampler_summary(tmp_path):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    rows = [
        "0, 1200, 2070, 150.0, 0x0, Not Active, Not Active, Not Active, Not Active, 3996, 40",
        "0, 2070, 2070, 600.0, 0x4, Not Active, Not Active, Not Active, Active, 3996, 50",
        "0, 2070, 2070, 610.0, 0x0, Not Active, Not Active, Not Active, Not Active, 3996, 51",
        "0, 2055, 2070, 620.0, 0x0, Not Active, Not Active, Not Active, Not Active, 3996, 52",
    ]
    open(s.path, "w").write("\n".join(rows) + "\n")
    s.proc = object()        # a sampler that ran
    s.skip = 1               # its first row was written before the timed region
    out = s.summary()
    assert out["samples"] == 3
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["mem_mhz"] == 3996.0
    assert not os.path.exists(s.path)     # the sampler's file is removed


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_sjf_groups_order_and_counts():
    sizes = [50, 10, 40, 10, 30, 20, 60, 5]
    g = bench.sjf_groups(sizes, 3)
    flat = [k for grp in g for k in grp]
    assert sorted(flat) == list(range(len(sizes)))               # each roadmap once
    assert [sizes[k] for k in flat] == sorted(sizes)             # smallest first
    assert [len(x) for x in g] == [3, 2, 3]                      # (nearly) equal counts
    assert bench.sjf_groups(sizes, 100) == [[k] for k in flat]   # at most one per roadmap
    assert bench.sjf_groups([7], 8) == [[0]]


def test_issue_roofline_uses_four_schedulers_per_sm_at_the_sampled_clock():
    r = bench.issue_roofline({"inst_per_launch": 4e9, "issue_active": 0.8}, 2.0, 2000.0, 100)
    assert r["peak_warp_inst_per_s"] == 100 * 4 * 2000e6
    assert abs(r["achieved_warp_inst_per_s"] - 2e12) < 1.0
    assert abs(r["frac"] - 2.5) < 1e-12
    assert bench.issue_roofline({}, 2.0, 2000.0, 100) is None
    assert bench.issue_roofline({"inst_per_launch": 4e9}, 2.0, None, 100) is None
