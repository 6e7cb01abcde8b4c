"""Host-side arithmetic of bench.py, without a GPU: the algorithmic bytes behind the
headline roofline (the distinct delay planes of a push, counted here independently
by brute force), the roofline fraction, and the clock-record summary on a fake
nvidia-smi sample list."""
import datetime
import os

import numpy as np

import bench
import synth
from oracle import lpf_oracle as O


def _delays(spec):
    return O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)


def test_algorithmic_bytes_of_the_aartfaac_push():
    spec = synth.spec_aartfaac(dtype="fp32")
    delays = _delays(spec)
    # brute force: every (subband, frames-back) plane some trial of a full push reads
    planes = {(f, int(delays[d].max() - delays[d, f])) for d in range(len(spec.dm_grid)) for f in range(spec.F)}
    nb = bench.algorithmic_bytes(spec, delays, "fp32")
    assert nb["U"] == len(planes) == 401
    HW = spec.H * spec.W
    assert nb["ring_reads"] == 401 * HW * 4 == 1_681_915_904
    assert nb["ingest"] == spec.F * HW * (4 + 4)
    assert nb["path"] == 1_816_133_632
    nb16 = bench.algorithmic_bytes(synth.spec_aartfaac(dtype="fp16"), delays, "fp16")
    assert nb16["U"] == 401 and nb16["path"] == 401 * HW * 2 + spec.F * HW * 6 == 941_621_248


def test_path_roofline_fraction():
    spec = synth.spec_aartfaac(dtype="fp32")
    r = bench.path_roofline(spec, "fp32", _delays(spec), 1.0, 6499.3, "of measured", traffic=123)
    assert abs(r["achieved"] - 1816.133632) < 1e-9          # GB/s at 1 ms per step
    assert abs(r["frac"] - r["achieved"] / 6499.3) < 1e-15
    assert r["traffic"] == 123 and r["bound"] == "hbm" and r["unit"] == "GB/s"


def _row(t, sm, mx, reasons=()):
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    flags = ["Active" if n in reasons else "Not Active" for n in names]
    return [t, "0", str(sm), str(mx), "900.0", "0x0"] + flags


def test_clock_summary_median_reasons_and_window():
    c = bench.Clocks(0)
    c.p = object()                                           # as if the sampler had run
    t0 = datetime.datetime(2026, 1, 1).timestamp()
    c.rows = [_row(t0 + 0.01 * i, 2032 if i != 3 else 1500, 2032) for i in range(10)]
    c.rows.append(_row(t0 + 0.05, 2032, 2032, ("sw_power_cap",)))
    s = c.summary(t0, t0 + 1.0)
    assert s["sm_mhz"] == 2032.0 and s["sm_max_mhz"] == 2032.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 11 and s["window"] == "timed region"
    # a timed region shorter than three samples takes the samples within 0.5 s of it
    s = c.summary(t0 + 0.2, t0 + 0.201)
    assert s["samples"] == 11 and s["window"].startswith("timed region +- 0.5 s")
    # no sampler: stated, not invented
    c2 = bench.Clocks(0)
    assert c2.summary(t0, t0 + 1)["reasons"] == ["nvidia-smi unavailable"]
    for k in (c, c2):                                        # the unused sample files
        k.f.close()
        os.unlink(k.f.name)


def test_kernel_traffic_goes_stale_with_any_source(tmp_path):
    """A capture's counters are used only while every file its kernel is compiled
    from is unchanged (hashed together, in order)."""
    srcs = ["paper_2103_15418_b300/csrc/lpf_dedisperse.cuh", "paper_2103_15418_b300/csrc/lpf_kernels.cuh"]
    rec = {"a": {"dram_bytes_per_launch": 7, "source": srcs, "sha256": bench.sources_sha256(srcs)},
           "b": {"dram_bytes_per_launch": 8, "source": srcs[0], "sha256": bench.sources_sha256(srcs[:1])},
           "c": {"dram_bytes_per_launch": 9, "source": srcs[::-1], "sha256": bench.sources_sha256(srcs)}}
    import json
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    got = bench.kernel_traffic(path=str(p))
    assert got == {"a": 7, "b": 8, "c": None}
    # the committed record: every kernel's sources exist and the hashes are well formed
    committed = json.load(open(os.path.join(bench.ROOT, "profiles", "traffic.json")))
    for k, v in committed.items():
        assert len(v["sha256"]) == 64 and bench.sources_sha256(v["source"]), k
