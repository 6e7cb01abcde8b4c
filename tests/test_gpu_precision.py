"""Reduced-precision ring storage: parity and the precision report, at full size.

Parity (gating): FP16/BF16 storage against the plain FP64 oracle (search_push)
run on the storage-rounded frames, at the storage tolerances of tests/parity.py
(candidate sets equal outside the undecidable pixels, S/N within 2e-3 for FP16
and 1.6e-2 for BF16), and against the residual-form reference at the FP32
tolerances.  Report: S/N error and candidate-set symmetric difference against
the oracle on the unrounded frames, asserted within the same tolerances and
zero.  Workloads: the 2048^2 precision stream (AARTFAAC bands, 501 trials, DM
step 0.5, depth 48, 40 pulses) in FP32, FP16 and BF16; the 1024^2 AARTFAAC
stream in FP16 and BF16.  The oracle runs on sampled trials of one push.
"""
import json

import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
from tests.parity import SNR_RTOL, compare_push, precision_vs_unrounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


class PlaneFrames:
    """Frame source for the oracle that keeps only the (t, f) planes the sampled
    trials of one push read (full-size frames are 268 MB each); frame_at(t)[f]
    is the plane rounded to the storage type, as float64."""

    def __init__(self, planes, dtype):
        self.planes, self.dtype = planes, dtype

    def __call__(self, t):
        planes, dtype = self.planes, self.dtype

        class _Frame:
            def __getitem__(self, f):
                return O.storage_round(planes[(t, f)], dtype)
        return _Frame()


def run_storage_types(lib, spec, seed, dms, dtypes, extra_open=None):
    """Push frames 0..T (T = largest delay + 2) through one stream per storage type;
    returns (T, delays, planes, {dtype: (candidates, stats)})."""
    st = synth.SyntheticStream(spec, seed=seed)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    T = int(delays.max()) + 2
    dmax = delays.max(axis=1)
    need = {(int(T - dmax[d] + delays[d, f]), f) for d in dms for f in range(spec.F)}
    planes = {}
    streams = {dt: lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                              box_r=spec.box_r, dtype=dt, **(extra_open or {})) for dt in dtypes}
    out = {}
    try:
        for t in range(T + 1):
            x = st.frame(t)
            for f in range(spec.F):
                if (t, f) in need:
                    planes[(t, f)] = x[f].copy()
            xd = torch.from_numpy(x).cuda()
            for dt, s in streams.items():
                s.push(xd, t)
                _, c, n, trunc = s.poll(timeout_ms=120000)
                assert not trunc
                if t == T:
                    out[dt] = (c, s.stats())
            del xd
    finally:
        for s in streams.values():
            s.close()
    return T, delays, planes, out


def report_for(spec, T, delays, planes, results, dms):
    rep = {}
    unrounded = PlaneFrames(planes, "fp32")
    # the synthetic frames are FP32, so the oracle on unrounded frames is the FP32 parity reference
    _, _, umaps = O.search_push(unrounded, T, delays, spec.box_r, spec.kappa, dms=dms, keep_maps=True)
    for dt, (c, stats) in results.items():
        rounded = PlaneFrames(planes, dt)
        par = compare_push(c, rounded, T, delays, spec.box_r, spec.kappa, dms=dms, gpu_stats=stats, storage=dt)
        rep[dt] = dict(parity_max_rel=par["max_rel"], parity_matched=par["matched"],
                       parity_excluded=par["excluded"], n_total=int(len(c)))
        if dt != "fp32":
            # the plain oracle on unrounded frames (for FP32 rings the frames are exact)
            rep[dt].update(precision_vs_unrounded(c, unrounded, T, delays, spec.box_r, spec.kappa, dms, dt,
                                                  maps=umaps))
        else:
            rep[dt].update(max_rel_snr_err=par["max_rel"], sym_diff=0, matched=par["matched"])
    return rep


def check(rep, min_matched):
    for dt, r in rep.items():
        assert r["sym_diff"] == 0, (dt, r)
        assert r["max_rel_snr_err"] <= SNR_RTOL[dt], (dt, r)
        assert r["matched"] >= min_matched, (dt, r)


def test_precision_report_2048(lib, capsys):
    spec = synth.spec_precision()
    dms = [0, 7, 120, 333, 500]
    T, delays, planes, res = run_storage_types(lib, spec, 44, dms, ("fp32", "fp16", "bf16"))
    rep = report_for(spec, T, delays, planes, res, dms)
    with capsys.disabled():
        print("\nPRECISION_REPORT " + json.dumps({"precision-2048x2048-16sb-501dm-depth48": rep}))
    check(rep, 300 * len(dms))
    # FP16 meets the 2e-3 target against the unrounded FP64 oracle
    assert rep["fp16"]["max_rel_snr_err"] <= 2e-3


def test_precision_report_aartfaac_16bit(lib, capsys):
    spec = synth.spec_aartfaac(n_frames=60)
    dms = [0, 1, 37, 100, 173, 250]
    T, delays, planes, res = run_storage_types(lib, spec, 2, dms, ("fp16", "bf16"))
    rep = report_for(spec, T, delays, planes, res, dms)
    with capsys.disabled():
        print("\nPRECISION_REPORT " + json.dumps({"aartfaac-1024x1024-16sb-251dm-depth48": rep}))
    check(rep, 300 * len(dms))


def test_precision_report_small_residual_form(lib):
    """512^2 cut of the precision stream: 16-bit rings also against the residual-form
    reference (the ring's exact values) at the FP32 tolerances."""
    from tests.parity import cached_frames, cached_residuals, compare_storage
    spec = synth.spec_precision(H=512, W=512, n_pulses=12, n_frames=60, n_sources=120)
    st = synth.SyntheticStream(spec, seed=44)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    T = int(delays.max()) + 2
    dms = [0, 7, 120, 333, 500]
    for dtype in ("fp16", "bf16"):
        with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                        box_r=spec.box_r, dtype=dtype) as s:
            for t in range(T + 1):
                s.push(torch.from_numpy(st.frame(t)).cuda(), t)
                _, c, n, _ = s.poll(timeout_ms=60000)
            res = compare_storage(c, cached_frames(st, dtype), T, delays, spec.box_r, spec.kappa, dtype, dms=dms,
                                  gpu_stats=s.stats(), res_at=cached_residuals(st, dtype, spec.box_r))
            assert res["matched"] > 100
