"""Stress workload: 2048^2 px, 32 subbands (57.6-63.85 MHz), 1001 DM trials, FP16 ring.

The sweep of DM 500 spans 113 frames, so the ring needs depth 114 (depth 96 is
rejected, see test_abi_cpu).  12 synthetic frames (dispersed pulses, 1% RFI
stripes) are cycled to fill the ring; the oracle reads the same cycle.  Checks
sampled trials against the oracle and the 32 x 64 FP32 dynamic spectra of the
frame's candidates against direct indexing of the frames.
"""
import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
import json

from tests.parity import SNR_RTOL, assert_sorted_unique, compare_storage, precision_vs_unrounded

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_stress_sampled_trials_and_dynspec(lib, capsys):
    spec = synth.spec_stress(depth=114)
    st = synth.SyntheticStream(spec, seed=50)
    pool = [st.frame(t) for t in range(12)]
    pool[5][:, 1000, :] += 10.0                      # one broadband RFI stripe in the cycle
    raw_pool = [O.storage_round(p, "fp16") for p in pool]
    res_pool = [O.storage_round(O.residual_frame(p, spec.box_r), "fp16") for p in raw_pool]
    frame_at = lambda t: raw_pool[t % 12]
    res_at = lambda t: res_pool[t % 12]
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    T = int(delays.max()) + 3
    dev_pool = [torch.from_numpy(p).cuda() for p in pool]
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                    box_r=spec.box_r, dtype="fp16") as s:
        for t in range(T + 1):
            s.push(dev_pool[t % 12], t)
            _, c, n, trunc = s.poll(timeout_ms=120000)
        assert not trunc
        assert_sorted_unique(c)
        # trials with candidates (the two with the most) beside fixed ones, so that the
        # comparisons below cover crossings and not only empty trials
        counts = np.bincount(np.asarray(c["dm_idx"], dtype=np.int64), minlength=len(spec.dm_grid)) if len(c) else []
        busy = [int(d) for d in np.argsort(-np.asarray(counts))[:2] if len(c) and counts[d] > 0]
        dms = sorted(set([0, 1, 400, 1000] + busy))
        compare_storage(c, frame_at, T, delays, spec.box_r, spec.kappa, "fp16", dms=dms,
                        gpu_stats=s.stats(), res_at=res_at)
        # precision report against the oracle on the unrounded frames
        rep = precision_vs_unrounded(c, lambda t: pool[t % 12], T, delays, spec.box_r, spec.kappa, dms, "fp16")
        with capsys.disabled():
            print("\nPRECISION_REPORT " + json.dumps({"stress-2048x2048-32sb-1001dm-depth114": {"fp16": rep}}))
        assert rep["sym_diff"] == 0 and rep["max_rel_snr_err"] <= SNR_RTOL["fp16"], rep
        assert not busy or rep["matched"] > 0, rep
        Tw = 64
        ds = s.dynspec(c, Tw)                              # contiguous [n][32][64] FP32 batch
        assert ds.shape == (len(c), 32, Tw) and ds.is_contiguous()
        pick = np.linspace(0, len(c) - 1, min(len(c), 50)).astype(int) if len(c) else []
        if len(c):
            ref = O.dynspec(frame_at, T, Tw, [(int(c["y"][i]), int(c["x"][i])) for i in pick])
            np.testing.assert_array_equal(ds.cpu().numpy()[pick], ref.astype(np.float32))
