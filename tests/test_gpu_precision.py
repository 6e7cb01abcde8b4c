"""Reduced-precision ring storage: parity and the precision report.

Parity: FP16/BF16 storage against the oracle run on what the rings hold: the
storage-rounded frames (for D) and the storage-rounded per-subband residuals
X - C(X) (for D - C); the CUDA path computes in FP32 from those values.  Report: S/N error
and candidate-set difference against the oracle on the unrounded FP32 frames,
on the 2048^2 precision workload's bands and DM grid (501 trials, depth 48)
at 512^2.  FP16 must stay within 2e-3 relative S/N error.
"""
import json

import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
from tests.parity import cached_frames, cached_residuals, compare_push, ambiguous_mask

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

DMS = [0, 7, 120, 333, 500]


def precision_vs_unrounded(gpu, frame_at, T, delays, r, kappa, dms):
    """max relative S/N error over candidates found by both, and the symmetric difference
    (excluding pixels within 1e-3 of kappa or at an FP32-undecidable local-max tie)."""
    _, _, maps = O.search_push(frame_at, T, delays, r, kappa, dms=dms, keep_maps=True)
    worst, sym, matched = 0.0, 0, 0
    F = delays.shape[1]
    for d in dms:
        m = maps[d]
        amb = ambiguous_mask(m, F, kappa)
        o = set(zip(*np.nonzero(m["mask"])))
        g = {(int(c["y"]), int(c["x"])): float(c["snr"]) for c in gpu[gpu["dm_idx"] == d]}
        for p, snr in g.items():
            if p in o:
                worst = max(worst, abs(snr - m["snr"][p]) / abs(m["snr"][p]))
                matched += 1
        sym += sum(1 for p in set(g) ^ o if not amb[p])
    return worst, sym, matched


def test_precision_report(lib, capsys):
    spec = synth.spec_precision(H=512, W=512, n_pulses=12, n_frames=60, n_sources=120)
    st = synth.SyntheticStream(spec, seed=44)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    T = int(delays.max()) + 2
    unrounded = cached_frames(st, "fp32")
    report = {}
    for dtype in ("fp32", "fp16", "bf16"):
        with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                        box_r=spec.box_r, dtype=dtype) as s:
            for t in range(T + 1):
                s.push(torch.from_numpy(st.frame(t)).cuda(), t)
                _, c, n, _ = s.poll(timeout_ms=60000)
            # parity against the oracle on the values the ring holds
            compare_push(c, cached_frames(st, dtype), T, delays, spec.box_r, spec.kappa, dms=DMS,
                         gpu_stats=s.stats(),
                         res_at=None if dtype == "fp32" else cached_residuals(st, dtype, spec.box_r))
            worst, sym, matched = precision_vs_unrounded(c, unrounded, T, delays, spec.box_r,
                                                         spec.kappa, DMS)
            report[dtype] = dict(max_rel_snr_err=worst, sym_diff=sym, matched=matched, n_total=n)
    with capsys.disabled():
        print("\nPRECISION_REPORT " + json.dumps(report))
    assert report["fp32"]["max_rel_snr_err"] < 1e-4
    assert report["fp16"]["max_rel_snr_err"] <= 2e-3
    assert report["fp16"]["matched"] > 100
