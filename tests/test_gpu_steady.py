"""Opt-in steady-source suppression (suppress_steady = K) on the GPU.

The tiny stream has three steady 20-sigma sources, which at kappa 4 are
candidates at every trial of every push, and one pulse.  A stream with
suppression runs beside one without, on the same frames:
  * per push, its candidates equal the unsuppressed stream's candidates after the
    oracle's SteadyMask / suppress_steady (same kernels otherwise, so the S/N is
    bit-identical), its n_out counts them, and they stay sorted;
  * FP32: against the full oracle pipeline (search_push, the mask, the drop
    rule), the sets agree outside the 1e-3 band around kappa;
  * the source pixels lose every dispersed-trial candidate from the K-th push on.
"""
import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
from tests.parity import assert_sorted_unique

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _keys(c):
    return {(int(r["t0"]), int(r["dm_idx"]), int(r["y"]), int(r["x"])): float(r["snr"]) for r in c}


@pytest.mark.parametrize("dtype", ["fp32", "fp16"])
def test_steady_suppression_against_the_oracle(lib, dtype):
    spec = synth.spec_tiny(kappa=4.0)
    st = synth.SyntheticStream(spec, seed=3)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    dmax = delays.max(axis=1)
    src = {(y, x) for y, x, _ in st.sources}
    K = 3
    gpu_mask, ora_mask = O.SteadyMask(K), O.SteadyMask(K)
    frame_at = lambda t: O.storage_round(st.frame(t), dtype)
    dropped_total = 0
    band = 1e-3                                           # undecidable S/N band around kappa (FP32)
    kw = dict(kappa=spec.kappa, box_r=spec.box_r, dtype=dtype)
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, suppress_steady=K, **kw) as s, \
         lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, **kw) as s0:
        for T in range(20):
            x = torch.from_numpy(st.frame(T)).cuda()
            s.push(x, T)
            s0.push(x, T)
            _, c, n, trunc = s.poll(timeout_ms=60000)
            _, c0, n0, _ = s0.poll(timeout_ms=60000)
            assert not trunc and n == len(c)
            assert_sorted_unique(c)
            got, all0 = _keys(c), _keys(c0)
            # the drop rule on the unsuppressed stream's own candidates
            steady = gpu_mask.update({(k[2], k[3]) for k in all0 if dmax[k[1]] == 0})
            recs0 = [k + (v,) for k, v in all0.items()]
            want = {r[:4]: r[4] for r in O.suppress_steady(recs0, dmax, steady)}
            assert got == want, (T, set(got) ^ set(want))
            dropped_total += n0 - n
            if T >= K - 1:
                assert not [k for k in got if dmax[k[1]] > 0 and (k[2], k[3]) in src], T
            if dtype != "fp32":
                continue                                  # 16-bit parity itself: test_gpu_parity
            # the full oracle pipeline, outside the band around kappa
            ref, _, maps = O.search_push(lambda t: frame_at(t).astype(np.float64), T, delays, spec.box_r,
                                         spec.kappa, keep_maps=True)
            ora_steady = ora_mask.update({(r[2], r[3]) for r in ref if dmax[r[1]] == 0})
            ora = {r[:4] for r in O.suppress_steady(ref, dmax, ora_steady)}
            for k in set(got) ^ ora:
                assert abs(maps[k[1]]["snr"][k[2], k[3]] - spec.kappa) < band, (T, k)
            assert ora_steady == steady or any(
                abs(maps[d]["snr"][p] - spec.kappa) < band for p in ora_steady ^ steady for d in np.flatnonzero(dmax == 0)
            ), (T, ora_steady ^ steady)
    assert dropped_total > 0


def test_steady_suppression_on_the_tiled_path_and_with_a_full_list(lib):
    """The same drop rule on the tiled filter path (records emitted by the filter
    itself), and with a candidate list too small for most pushes: the mask state
    is that of the full candidate sets (marks do not depend on the list), the
    returned records are a sorted subset of the suppressed full set, truncation is
    reported, and n_out is the number of records returned (the records past the
    list were never checked against the mask)."""
    spec = synth.spec_tiny(kappa=4.0)
    st = synth.SyntheticStream(spec, seed=3)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    dmax = delays.max(axis=1)
    K = 2
    mask = O.SteadyMask(K)
    kw = dict(kappa=spec.kappa, box_r=spec.box_r)
    saw_trunc = saw_drop = False
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, **kw) as full, \
         lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, suppress_steady=K,
                    filter_impl="tiled", **kw) as tiled, \
         lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, suppress_steady=K,
                    cand_cap=24, **kw) as small:
        for T in range(16):
            x = torch.from_numpy(st.frame(T)).cuda()
            for s in (full, tiled, small):
                s.push(x, T)
            _, c0, n0, _ = full.poll(timeout_ms=60000)
            _, ct, nt, trunc_t = tiled.poll(timeout_ms=60000)
            _, cs, ns, trunc_s = small.poll(timeout_ms=60000)
            all0 = {(int(r["t0"]), int(r["dm_idx"]), int(r["y"]), int(r["x"])) for r in c0}
            steady = mask.update({(k[2], k[3]) for k in all0 if dmax[k[1]] == 0})
            want = {r[:4] for r in O.suppress_steady([k + (0.0,) for k in all0], dmax, steady)}
            got_t = {(int(r["t0"]), int(r["dm_idx"]), int(r["y"]), int(r["x"])) for r in ct}
            # the tiled filter computes the same S/N within FP32 rounding: the sets
            # agree (the tiny stream has no pixel within 1e-3 of kappa here)
            assert not trunc_t and nt == len(ct) and got_t == want, (T, got_t ^ want)
            got_s = [(int(r["t0"]), int(r["dm_idx"]), int(r["y"]), int(r["x"])) for r in cs]
            assert_sorted_unique(cs)
            # the marks come from every zero-delay candidate found, stored or not,
            # so the capped stream follows the same mask: its records are kept ones
            assert set(got_s) <= want and len(got_s) == min(ns, 24), (T, set(got_s) - want)
            if n0 > 24:
                # the list overflowed: the drop saw only the stored records, and
                # n_out counts the kept ones among them (all returned)
                assert trunc_s and ns == len(got_s)
                saw_trunc = True
                saw_drop |= ns < 24                         # a stored record was dropped
            else:
                assert not trunc_s and set(got_s) == want and ns == len(want), T
    assert saw_trunc and saw_drop


def test_steady_suppression_on_the_clipping_path(lib):
    """The marks set by the clipping emit (dispersed search, two clipping
    iterations): per push, the suppressed stream's candidates are the unsuppressed
    clipping stream's candidates after the oracle's mask and drop rule."""
    spec = synth.spec_tiny(kappa=4.0)
    st = synth.SyntheticStream(spec, seed=3)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    dmax = delays.max(axis=1)
    K = 2
    mask = O.SteadyMask(K)
    kw = dict(kappa=spec.kappa, box_r=spec.box_r, clip_iters=2)
    dropped = 0
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, suppress_steady=K, **kw) as s, \
         lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, **kw) as s0:
        for T in range(10):
            x = torch.from_numpy(st.frame(T)).cuda()
            s.push(x, T)
            s0.push(x, T)
            _, c, n, trunc = s.poll(timeout_ms=60000)
            _, c0, n0, _ = s0.poll(timeout_ms=60000)
            assert not trunc and n == len(c)
            assert_sorted_unique(c)
            got, all0 = _keys(c), _keys(c0)
            steady = mask.update({(k[2], k[3]) for k in all0 if dmax[k[1]] == 0})
            want = {r[:4]: r[4] for r in O.suppress_steady([k + (v,) for k, v in all0.items()], dmax, steady)}
            assert got == want, (T, set(got) ^ set(want))
            dropped += n0 - n
    assert dropped > 0
