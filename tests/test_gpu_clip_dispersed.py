"""Iterated sigma clipping in the dispersed search (Sec. 2.1.1, clip_iters > 1),
through the C ABI, against the FP64 oracle: for every active DM trial, the
oracle dedisperses the (storage-rounded) frames (App. B.2) and runs clip_detect
on D_d with the 3x3 maximum; candidates, S/N and per-trial statistics must match
at the FP32 tolerances (the clipping path sums D from the raw ring, so a 16-bit
ring adds no rounding beyond the stored frames)."""
import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
from tests.parity import assert_sorted_unique, cached_frames, check_stats, compare_trial

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


class PlantedStream:
    """The tiny stream plus steady bright point sources, each with a faint compact
    neighbour 5 px away that the one-pass filter misses (the bright source inflates
    the spread of its window); identical in every subband and frame."""

    def __init__(self, spec, seed):
        self.st = synth.SyntheticStream(spec, seed=seed)
        yy, xx = np.mgrid[:spec.H, :spec.W]
        self.add = np.zeros((spec.H, spec.W), np.float32)
        for (y0, x0) in [(20, 24), (60, 90), (30, 100), (80, 40)]:
            self.add[y0, x0] += 40.0
            self.add += (4.0 * np.exp(-((yy - y0) ** 2 + (xx - x0 - 5) ** 2) / 2.0)).astype(np.float32)

    def frame(self, t):
        return (self.st.frame(t) + self.add[None]).astype(np.float32)


@pytest.mark.parametrize("dtype,iters", [("fp32", 4), ("fp16", 3), ("fp32", 2)])
def test_dispersed_clipping_matches_oracle(lib, dtype, iters):
    spec = synth.spec_tiny(H=96, W=128, n_sources=0, box_r=7, kappa=6.0)
    st = PlantedStream(spec, 41)
    fa = cached_frames(st, dtype)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    T_checks = {int(delays.max()), int(delays.max()) + 2}
    matched = more = 0
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                    box_r=spec.box_r, dtype=dtype, clip_iters=iters) as s:
        for T in range(max(T_checks) + 1):
            s.push(torch.from_numpy(st.frame(T)).cuda(), T)
            _, c, n, trunc = s.poll(timeout_ms=60000)
            assert not trunc and n == len(c)
            if T not in T_checks:
                continue
            assert_sorted_unique(c)
            gstats = s.stats()
            for d in O.active_trials(delays, T):
                t0, D = O.dedisperse(fa, T, delays, d)
                m = O.clip_detect(D, spec.box_r, spec.kappa, 1, iters)
                m["abs_sum"] = O.abs_sum(fa, T, delays, d)
                sel = c[c["dm_idx"] == d]
                assert np.all(sel["t0"] == t0)
                nm, _, _ = compare_trial(sel, m, spec.F, spec.kappa)
                matched += nm
                mean, rms, nv = O.frame_stats(m["snr"], m["valid"])
                check_stats(gstats, {d: (mean, rms, nv)}, d, "fp32")
                one = O.clip_detect(D, spec.box_r, spec.kappa, 1, 1)
                more += int(m["mask"].sum() - one["mask"].sum())
    assert matched > 0
    assert more > 0          # the iterations find the faint neighbours one pass misses
