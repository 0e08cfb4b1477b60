"""Host logic of bench.py that the bench line's figures rest on.

- algorithmic bytes per node of the step kernels: 16 Q + 1 (D2Q9: 145 B) and
  16 Q + 9 (D3Q27: 441 B, with rho and phi of the moments pass);
- the HBM roofline (achieved = algorithmic bytes / kernel time, frac =
  achieved / peak) and the issue roofline (152 SMs x 4 warp instructions per
  clock at the sampled SM clock);
- the committed ncu counters are reported only while the kernel sources hash
  to the recorded value;
- the clock sampler's summary of nvidia-smi rows (median SM clock, largest
  maximum, active throttle reasons);
- the oracle's bounded sample of the headline lattice: a centred column of
  full depth.
"""
import json
import os

import numpy as np

import bench


def test_algorithmic_bytes_per_node():
    assert bench.algorithmic_bytes(9, 1) == 145
    assert bench.algorithmic_bytes(27, 1) == 441
    assert bench.algorithmic_bytes(27, 192 * 192 * 128) == 441 * 4718592


def test_hbm_roofline_arithmetic():
    N, ms, peak = 4718592, 0.766, 6783.1
    r = bench.roofline(27, N, ms, peak, "measured", "step_batch_kernel", "c2_lubricated_d3q27_192x192x128")
    achieved = 441 * N / (ms * 1e-3) / 1e9
    assert abs(r["achieved"] - achieved) < 0.06 and abs(r["frac"] - achieved / peak) < 1e-4
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == peak
    assert r["algorithmic_bytes_per_launch"] == 441 * N
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    assert r["traffic"] == t["traffic_bytes_per_launch"]["c2_lubricated_d3q27_192x192x128"]


def test_issue_roofline_arithmetic():
    name = "c2_lubricated_d3q27_192x192x128"
    r = bench.issue_roofline(name, 0.766, 2070.0)
    inst = bench.measured_instructions(name)
    assert inst and r["warp_instructions_per_launch"] == inst
    assert abs(r["peak"] - 152 * 4 * 2070e6 / 1e9) < 0.06
    assert abs(r["frac"] - (inst / 0.766e-3 / 1e9) / (152 * 4 * 2.07)) < 1e-4
    assert bench.issue_roofline(name, 0.766, None) is None


def test_counters_withdrawn_when_the_sources_change(monkeypatch):
    assert bench.measured_traffic("c1_capillary_d2q9_1024x64")
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0" * 64)
    assert bench.measured_traffic("c1_capillary_d2q9_1024x64") is None
    assert bench.measured_instructions("c1_capillary_d2q9_1024x64") is None
    r = bench.roofline(9, 65536, 0.0152, 6783.1, "measured", "k", "c1_capillary_d2q9_1024x64")
    assert r["traffic"] is None


def test_clock_summary():
    c = bench.ClockSampler(0)
    assert c.summary()["reasons"] == ["unsampled"]
    c.samples = [["2070", "2070", "900.1", "Not Active", "Not Active", "Not Active", "Not Active"],
                 ["2055", "2070", "1010.0", "Not Active", "Not Active", "Not Active", "Active"],
                 ["1980", "2070", "1100.4", "Not Active", "Not Active", "Not Active", "Active"],
                 ["[N/A]", "2070", "1000.0", "Not Active", "Not Active", "Not Active", "Not Active"]]
    s = c.summary()
    assert s["sm_mhz"] == 2055.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 4
    c.samples.append(["1500", "2070", "1200", "Not Active", "Active", "Not Active", "Not Active"])
    assert bench.ClockSampler.summary(c)["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_oracle_sample_is_a_centred_full_depth_column():
    from paper_1904_06881_gb300 import workloads as W

    wl = W.c2_lubricated(nx=64, ny=56, nz=40, R=10.0, lub=4, gap=2, kw_rho=0.02)
    s = bench.oracle_sample(wl, n=16)
    assert (s["nx"], s["ny"], s["nz"]) == (16, 16, 40)
    x0, y0 = (64 - 16) // 2, (56 - 16) // 2
    for k in ("mask", "rho", "phi"):
        assert s[k].flags["C_CONTIGUOUS"]
        assert np.array_equal(s[k], wl[k][:, y0:y0 + 16, x0:x0 + 16])
    assert s["params"] == wl["params"]
    d2 = W.c0_sessile_drop()
    assert bench.oracle_sample(d2) is d2
