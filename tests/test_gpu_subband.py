"""The paper's per-subband detector (stream mode "subband") against the FP64
oracle, through the C ABI: candidates (band, y, x, S/N) and per-band statistics
of every band image of each frame, 7x7 maximum filter."""
import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
from tests.parity import assert_sorted_unique, compare_trial

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def residual_form(x, res, r, kappa, k):
    """One band image as a reduced-precision ring holds it: S/N from its stored
    residual X - C(X) (box mean of the squared residual), the maximum on X."""
    cnt = O.window_count(*x.shape, r)
    S = O.box_sum(res * res, r) / cnt
    snr = np.zeros_like(x)
    ok = S > 0
    snr[ok] = res[ok] / np.sqrt(S[ok])
    q = O.local_max_mask(x, k)
    return dict(snr=snr, valid=ok, mask=(snr > kappa) & q & ok, lmax_margin=x - O.neighbour_max(x, k))


@pytest.mark.parametrize("dtype", ["fp32", "fp16"])
def test_subband_detector_matches_oracle(lib, dtype):
    spec = synth.spec_aartfaac(H=96, W=136, n_sources=25, n_pulses=2, box_r=15, n_frames=8)
    st = synth.SyntheticStream(spec, seed=4)
    k, matched = 3, 0
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, None, 2, cadence_s=spec.cadence_s, kappa=spec.kappa,
                    box_r=spec.box_r, dtype=dtype, mode="subband", lmax_r=k) as s:
        assert s.info()["n_distinct"] == spec.F and s.info()["max_delay"] == 0
        for T in range(6):
            frame = st.frame(T)
            s.push(torch.from_numpy(frame).cuda(), T)
            Tp, c, n, trunc = s.poll(timeout_ms=60000)
            assert Tp == T and not trunc and n == len(c)
            assert np.all(c["t0"] == T) and np.all((c["dm_idx"] >= 0) & (c["dm_idx"] < spec.F))
            assert_sorted_unique(c)
            x = O.storage_round(frame, dtype)
            if dtype == "fp32":
                _, stats, maps = O.subband_detect(x, spec.box_r, spec.kappa, k)
            else:
                res = O.storage_round(O.residual_frame(x, spec.box_r), dtype)
                maps = {b: residual_form(x[b], res[b], spec.box_r, spec.kappa, k) for b in range(spec.F)}
                stats = {b: O.frame_stats(maps[b]["snr"], maps[b]["valid"]) for b in range(spec.F)}
            gstats = s.stats()
            for b in range(spec.F):
                maps[b]["abs_sum"] = np.abs(x[b])        # one plane: the tie band of a stored value
                nm, _, _ = compare_trial(c[c["dm_idx"] == b], maps[b], 1, spec.kappa)
                matched += nm
                mean, rms, _ = stats[b]
                assert abs(gstats[b][0] - mean) <= 1e-4 * abs(mean) + 1e-6, (b, gstats[b], mean)
                assert abs(gstats[b][1] - rms) <= 1e-4 * abs(rms) + 1e-6, (b, gstats[b], rms)
    assert matched > 50


def test_subband_detector_7x7_deblends(lib):
    """Pairs of compact sources 3 px apart in band 0: the 3x3 window reports both
    peaks of a pair, the 7x7 window only the brighter (Sec. 2.1.2 deblending);
    every 7x7 maximum above the threshold is also a 3x3 one."""
    spec = synth.spec_aartfaac(H=128, W=128, n_sources=0, n_pulses=0, box_r=15, n_frames=4)
    st = synth.SyntheticStream(spec, seed=9)
    x = st.frame(0)
    yy, xx = np.mgrid[:spec.H, :spec.W]
    pairs = [(30, 30), (30, 90), (90, 34), (96, 96)]
    for (y0, x0) in pairs:
        x[0] += 24.0 * np.exp(-((yy - y0) ** 2 + (xx - x0) ** 2) / 2.0)
        x[0] += 20.0 * np.exp(-((yy - y0) ** 2 + (xx - x0 - 3) ** 2) / 2.0)
    frame = torch.from_numpy(x.astype(np.float32)).cuda()
    got = {}
    for k in (1, 3):
        with lib.Stream(spec.H, spec.W, spec.freqs_mhz, None, 1, kappa=spec.kappa, box_r=spec.box_r,
                        mode="subband", lmax_r=k) as s:
            s.push(frame, 0)
            _, c, _, _ = s.poll(timeout_ms=60000)
            got[k] = set(zip(c["dm_idx"].tolist(), c["y"].tolist(), c["x"].tolist()))
    assert got[3] <= got[1]
    for (y0, x0) in pairs:
        assert (0, y0, x0) in got[3] and (0, y0, x0) in got[1]
        assert (0, y0, x0 + 3) in got[1] and (0, y0, x0 + 3) not in got[3]


def clip_frame(spec, st, T):
    """The noise-and-gradient stream with planted bright point sources, each with a
    faint compact source 5 px away that the one-pass filter misses (band-dependent
    positions)."""
    x = st.frame(T)
    yy, xx = np.mgrid[:spec.H, :spec.W]
    for b in range(spec.F):
        for j, (y0, x0) in enumerate([(20, 24), (60, 90), (30, 100), (80, 40)]):
            y0 = (y0 + 3 * b + 7 * T) % (spec.H - 20) + 10
            x0 = (x0 + 5 * b + 11 * T) % (spec.W - 30) + 10
            x[b, y0, x0] += 300.0
            x[b] += 10.0 * np.exp(-((yy - y0) ** 2 + (xx - x0 - 5) ** 2) / 2.0)
    return x.astype(np.float32)


@pytest.mark.parametrize("dtype", ["fp32", "fp16"])
def test_subband_clipping_matches_oracle(lib, dtype):
    spec = synth.spec_aartfaac(H=96, W=128, n_sources=0, n_pulses=0, box_r=7, n_frames=6)
    st = synth.SyntheticStream(spec, seed=31)
    k, iters, more = 3, 4, 0
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, None, 1, kappa=spec.kappa, box_r=spec.box_r, dtype=dtype,
                    mode="subband", lmax_r=k, clip_iters=iters) as s:
        for T in range(3):
            frame = clip_frame(spec, st, T)
            s.push(torch.from_numpy(frame).cuda(), T)
            _, c, n, trunc = s.poll(timeout_ms=60000)
            assert not trunc and n == len(c) and np.all(c["t0"] == T)
            assert_sorted_unique(c)
            x = O.storage_round(frame, dtype)
            gstats = s.stats()
            for b in range(spec.F):
                m = O.clip_detect(x[b], spec.box_r, spec.kappa, k, iters)
                m["abs_sum"] = np.abs(x[b])
                compare_trial(c[c["dm_idx"] == b], m, 1, spec.kappa)
                one = O.clip_detect(x[b], spec.box_r, spec.kappa, k, 1)
                more += int(m["mask"].sum() - one["mask"].sum())
                mean, rms, _ = O.frame_stats(m["snr"], m["valid"])
                assert abs(gstats[b][0] - mean) <= 1e-4 * abs(mean) + 1e-6, (b, gstats[b], mean)
                assert abs(gstats[b][1] - rms) <= 1e-4 * abs(rms) + 1e-6, (b, gstats[b], rms)
    assert more > 0          # clipping found sources the one-pass filter missed


@pytest.mark.parametrize("dtype,iters,r,H,W", [("fp32", 1, 9, 96, 128), ("fp32", 3, 15, 96, 128),
                                               ("fp16", 1, 15, 96, 128), ("bf16", 3, 7, 96, 128),
                                               ("fp32", 2, 7, 97, 531), ("fp32", 2, 15, 45, 70),
                                               ("fp32", 2, 1, 64, 77), ("fp16", 1, 16, 96, 128)])
def test_subband_gaussian_kernel_matches_oracle(lib, dtype, iters, r, H, W):
    """The per-subband detector with the Gaussian background kernel of Sec. 2.1.1
    (s = 3 px on the (2r+1)^2 window, r from 1 to 16), one pass and clipping
    iterations, against
    clip_detect(..., s): candidates, S/N and per-band statistics; ragged sizes
    (a second 512-column segment, partial 32 x 64 tiles, windows wider than the
    image) included."""
    # a 3 x 3 Gaussian window caps a lone source's S/N near sqrt(Z) = 2.9: a lower threshold there
    spec = synth.spec_aartfaac(H=H, W=W, n_sources=0, n_pulses=0, box_r=r, n_frames=6,
                               kappa=6.0 if r > 2 else 2.5)
    st = synth.SyntheticStream(spec, seed=37)
    s_px, k, matched = 3.0, 3, 0
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, None, 1, kappa=spec.kappa, box_r=spec.box_r, dtype=dtype,
                    mode="subband", lmax_r=k, clip_iters=iters, kernel="gauss", gauss_sigma=s_px) as s:
        for T in range(3):
            frame = clip_frame(spec, st, T)
            s.push(torch.from_numpy(frame).cuda(), T)
            _, c, n, trunc = s.poll(timeout_ms=60000)
            assert not trunc and n == len(c) and np.all(c["t0"] == T)
            assert_sorted_unique(c)
            x = O.storage_round(frame, dtype)
            gstats = s.stats()
            for b in range(spec.F):
                m = O.clip_detect(x[b], spec.box_r, spec.kappa, k, iters, s=s_px)
                m["abs_sum"] = np.abs(x[b])
                nm, _, _ = compare_trial(c[c["dm_idx"] == b], m, 1, spec.kappa)
                matched += nm
                mean, rms, _ = O.frame_stats(m["snr"], m["valid"])
                assert abs(gstats[b][0] - mean) <= 1e-4 * abs(mean) + 1e-6, (b, gstats[b], mean)
                assert abs(gstats[b][1] - rms) <= 1e-4 * abs(rms) + 1e-6, (b, gstats[b], rms)
    assert matched > 2 * spec.F
