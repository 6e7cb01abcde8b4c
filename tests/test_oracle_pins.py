"""Pins of the FP64 oracle against facts independent of its own code.

Each test checks one step of the method against something the paper or the
mathematics fixes: a physical constant derived from CODATA values, closed forms,
brute-force loops on tiny inputs, invariants, and the Gaussian false-alarm law
of App. B.1.  The last group plants plausible mistakes in copies of oracle
functions and checks that a pin catches each of them.
"""
import math
from decimal import Decimal, getcontext, ROUND_HALF_UP

import numpy as np
import pytest

from oracle import lpf_oracle as O
import synth


# ----------------------------------------------------------------- helpers
def brute_box_mean(img, r):
    H, W = img.shape
    out = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            s, n = 0.0, 0
            for yy in range(y - r, y + r + 1):
                for xx in range(x - r, x + r + 1):
                    if 0 <= yy < H and 0 <= xx < W:
                        s += img[yy, xx]
                        n += 1
            out[y, x] = s / n
    return out


def brute_spread(img, C, r):
    H, W = img.shape
    out = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            s, n = 0.0, 0
            for yy in range(y - r, y + r + 1):
                for xx in range(x - r, x + r + 1):
                    if 0 <= yy < H and 0 <= xx < W:
                        s += (img[yy, xx] - C[yy, xx]) ** 2
                        n += 1
            out[y, x] = s / n
    return out


def brute_local_max(img, k=1):
    H, W = img.shape
    out = np.zeros((H, W), bool)
    for y in range(H):
        for x in range(W):
            m = -math.inf
            for yy in range(y - k, y + k + 1):
                for xx in range(x - k, x + k + 1):
                    if 0 <= yy < H and 0 <= xx < W:
                        m = max(m, img[yy, xx])
            out[y, x] = img[y, x] == m
    return out


def phi(x):
    return 0.5 * math.erfc(-x / math.sqrt(2.0))


# ----------------------------------------------------------------- a1 delay table
def test_dispersion_constant_from_codata():
    """Sec. 3.2: C_DM = e^2 pc / (8 pi^2 eps0 m_e c) * 1e-6 (s MHz^2 cm^3/pc)."""
    e, eps0, me, c = 1.602176634e-19, 8.8541878128e-12, 9.1093837015e-31, 299792458.0
    pc = 3.0856775814913673e16
    derived = e ** 2 / (8 * math.pi ** 2 * eps0 * me * c) * pc * 1e-6
    assert abs(O.C_DM_S - derived) / derived < 1e-6
    # the paper prints 4148.806 (with a garbled unit)
    assert abs(O.C_DM_S - 4148.806) < 0.01


def test_delay_table_high_precision_rounding():
    """Same delays from 40-digit decimal arithmetic with round-half-up."""
    getcontext().prec = 40
    freqs = synth.AARTFAAC_BANDS
    dms = np.arange(0, 251, 7, dtype=np.float64)
    tab = O.delay_table(freqs, dms, 1.0)
    C = Decimal(repr(O.C_DM_S))
    ref = Decimal(repr(float(max(freqs))))
    for d, dm in enumerate(dms):
        for f, nu in enumerate(freqs):
            nu = Decimal(repr(float(nu)))
            x = C * Decimal(repr(float(dm))) * (1 / (nu * nu) - 1 / (ref * ref))
            assert int(x.quantize(Decimal(1), rounding=ROUND_HALF_UP)) == tab[d, f]


def test_delay_table_invariants():
    freqs = synth.AARTFAAC_BANDS
    dms = np.arange(251, dtype=np.float64)
    tab = O.delay_table(freqs, dms, 1.0)
    ref = int(np.argmax(freqs))
    assert np.all(tab[:, ref] == 0)                 # no delay at nu_ref
    assert np.all(tab >= 0)
    assert np.all(tab[0] == 0)                      # DM 0: no delay
    assert np.all(np.diff(tab, axis=0) >= 0)        # monotone in DM
    order = np.argsort(freqs)                       # lower frequency arrives later
    assert np.all(np.diff(tab[:, order], axis=1) <= 0)
    # linear in DM / cadence up to rounding: halving the cadence doubles the delay (+-1)
    tab2 = O.delay_table(freqs, dms, 0.5)
    assert np.all(np.abs(tab2 - 2 * tab) <= 1)
    # the rounding is well conditioned on the benchmark grids (ties far from FP64 error)
    assert O.delay_fraction_margin(freqs, dms, 1.0) > 1e-6
    assert O.delay_fraction_margin(freqs, np.arange(501) * 0.5, 1.0) > 1e-6


def test_delay_textbook_magnitude():
    """Lorimer & Kramer: ~4.15 ms * DM * nu_GHz^-2; DM 100 at 100 MHz vs infinity = 41.5 s."""
    tab = O.delay_table([100.0, 1e9], [100.0], 1e-3)      # cadence 1 ms
    assert abs(tab[0, 0] - 41488) <= 1
    assert tab[0, 1] == 0


# ----------------------------------------------------------------- a3 shift-sum
def _frames_from_array(arr):
    return lambda t: arr[t]


def test_dm0_trial_is_plain_subband_sum():
    rng = np.random.default_rng(0)
    arr = rng.standard_normal((10, 5, 7, 9))
    delays = np.zeros((1, 5), np.int64)
    t0, D = O.dedisperse(_frames_from_array(arr), 6, delays, 0)
    assert t0 == 6
    np.testing.assert_allclose(D, arr[6].sum(axis=0), rtol=0, atol=1e-12)


def test_shift_sum_impulse_lands_at_t0():
    """A unit impulse at (f, t) reaches trial d exactly when t = t0 + delay[d][f]."""
    F, T_len = 4, 12
    delays = np.array([[0, 0, 0, 0], [3, 2, 1, 0], [5, 3, 1, 0], [4, 4, 0, 0]], np.int64)
    for f in range(F):
        for t in range(T_len):
            arr = np.zeros((T_len, F, 3, 4))
            arr[t, f, 1, 2] = 1.0
            for d in range(delays.shape[0]):
                dmax = int(delays[d].max())
                for T in range(dmax, T_len):
                    t0, D = O.dedisperse(_frames_from_array(arr), T, delays, d)
                    expect = 1.0 if t == t0 + delays[d, f] else 0.0
                    assert D[1, 2] == expect and D.sum() == expect


def test_shift_sum_linearity():
    rng = np.random.default_rng(1)
    a = rng.standard_normal((8, 3, 5, 6))
    b = rng.standard_normal((8, 3, 5, 6))
    delays = np.array([[2, 1, 0]], np.int64)
    _, Da = O.dedisperse(_frames_from_array(a), 5, delays, 0)
    _, Db = O.dedisperse(_frames_from_array(b), 5, delays, 0)
    _, Dab = O.dedisperse(_frames_from_array(2 * a - b), 5, delays, 0)
    np.testing.assert_allclose(Dab, 2 * Da - Db, atol=1e-12)


# ----------------------------------------------------------------- a4 / a5 box filter
@pytest.mark.parametrize("r", [1, 2, 3])
def test_box_filter_matches_brute_force(r):
    rng = np.random.default_rng(2 + r)
    img = rng.standard_normal((11, 17)) * 3 + np.arange(17)[None] * 0.5   # non-square, sloped
    C = O.local_centre(img, r)
    np.testing.assert_allclose(C, brute_box_mean(img, r), rtol=0, atol=1e-12)
    S = O.local_spread(img, C, r)
    np.testing.assert_allclose(S, brute_spread(img, brute_box_mean(img, r), r), rtol=0, atol=1e-12)


def test_window_count_closed_form():
    H, W, r = 9, 14, 3
    n = O.window_count(H, W, r)
    for y in range(H):
        for x in range(W):
            ny = min(y + r, H - 1) - max(y - r, 0) + 1
            nx = min(x + r, W - 1) - max(x - r, 0) + 1
            assert n[y, x] == ny * nx


def test_constant_image_has_zero_spread():
    img = np.full((20, 30), 7.25)
    C = O.local_centre(img, 5)
    S = O.local_spread(img, C, 5)
    np.testing.assert_allclose(C, 7.25, atol=1e-12)
    np.testing.assert_allclose(S, 0.0, atol=1e-20)
    res = O.detect(img, 5, 1.0)
    assert not res["mask"].any() and np.all(res["snr"] == 0)


def test_snr_affine_invariance():
    rng = np.random.default_rng(4)
    img = rng.standard_normal((24, 21))
    a = O.detect(img, 4, 2.0)
    b = O.detect(3.5 * img - 11.0, 4, 2.0)
    np.testing.assert_allclose(a["snr"], b["snr"], atol=1e-9)
    assert np.array_equal(a["mask"], b["mask"])


# ----------------------------------------------------------------- a6 detection
def test_local_max_matches_brute_force():
    rng = np.random.default_rng(5)
    img = rng.integers(0, 4, (13, 10)).astype(float)     # many ties
    assert np.array_equal(O.local_max_mask(img), brute_local_max(img))


def test_plateau_ties_all_emitted():
    img = np.zeros((9, 9))
    img[4, 4] = img[4, 5] = 10.0
    q = O.local_max_mask(img)
    assert q[4, 4] and q[4, 5]
    assert not q[3, 4]


def test_iid_noise_local_max_fraction_is_one_ninth():
    rng = np.random.default_rng(6)
    img = rng.standard_normal((400, 400))
    frac = O.local_max_mask(img)[1:-1, 1:-1].mean()
    n = 398 * 398
    sigma = math.sqrt((1 / 9) * (8 / 9) / n) * 3    # neighbouring maxima are dependent
    assert abs(frac - 1 / 9) < 5 * sigma


def test_threshold_is_strict():
    rng = np.random.default_rng(7)
    img = rng.standard_normal((31, 31))
    img[15, 15] = 9.0
    base = O.detect(img, 5, 0.0)
    k = base["snr"][15, 15]
    assert O.detect(img, 5, k)["mask"][15, 15] == False          # noqa: E712  (x > kappa)
    assert O.detect(img, 5, np.nextafter(k, -np.inf))["mask"][15, 15]


def test_noise_false_alarm_rate_follows_gaussian_tail():
    """App. B.1: Pr(type-1 error) = 1 - Phi(kappa) for pure N(0, n^2) noise."""
    rng = np.random.default_rng(8)
    H = W = 64
    frames = 600
    counts = {3.5: 0, 4.0: 0}
    delays = np.zeros((1, 16), np.int64)            # DM 0: independent frames
    for t in range(frames):
        cube = rng.standard_normal((16, H, W))
        _, D = O.dedisperse(lambda _t, c=cube: c, 0, delays, 0)
        snr = O.detect(D, 15, 99.0)["snr"]
        for k in counts:
            counts[k] += int((snr > k).sum())
    for k, got in counts.items():
        expect = H * W * frames * (1 - phi(k))
        tol = 5 * math.sqrt(expect) + 0.10 * expect
        assert abs(got - expect) < tol, (k, got, expect)


def test_injected_pulse_recovered_at_pixel_and_dm():
    """A dispersed pulse (paper's Sec. 3.2 model) is found at its pixel, in a trial whose
    rounded delay row is that of the injected DM."""
    spec = synth.spec_aartfaac(H=96, W=96, n_sources=0, gradient_amp=0.0, n_pulses=0,
                               n_frames=80, dm_grid=np.arange(0, 161, dtype=np.float64))
    pulse = synth.Pulse(y=40, x=57, t0=20.0, dm=100.0, width=1.0, alpha=0.0, amp=8.0)
    st = synth.SyntheticStream(spec, seed=3, pulses=[pulse])
    frame_at = lambda t: st.frame(t).astype(np.float64)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, 1.0)
    T = 20 + int(delays.max(axis=1)[100])
    true_row = delays[100]
    best = None
    for d in range(len(spec.dm_grid)):
        if int(delays[d].max()) != T - 20:
            continue                      # only trials whose t0 is the pulse's
        _, D = O.dedisperse(frame_at, T, delays, d)
        res = O.detect(D, spec.box_r, spec.kappa)
        if best is None or res["snr"][40, 57] > best[0]:
            best = (res["snr"][40, 57], d, res["mask"][40, 57])
    snr, d_best, det = best
    assert det and snr > 15
    assert np.array_equal(delays[d_best], true_row) or abs(d_best - 100) <= 1


# ----------------------------------------------------------------- a7 stats
def test_frame_stats_against_fsum():
    rng = np.random.default_rng(9)
    snr = rng.standard_normal((50, 40)) * 1e3 + 1e-3
    valid = rng.random((50, 40)) > 0.2
    mean, rms, n = O.frame_stats(snr, valid)
    v = snr[valid].tolist()
    assert n == len(v)
    assert abs(mean - math.fsum(v) / n) <= 1e-12 * abs(math.fsum(v) / n) + 1e-15
    assert abs(rms - math.sqrt(math.fsum(x * x for x in v) / n)) <= 1e-12 * rms


# ----------------------------------------------------------------- a8 dynspec
def test_dynspec_is_direct_indexing_of_frames():
    spec = synth.spec_tiny()
    st = synth.SyntheticStream(spec, seed=11)
    T, Tw = 20, 6
    cands = [(0, 0), (10, 63), (33, 17)]
    out = O.dynspec(lambda t: st.frame(t), T, Tw, cands, 0)
    for n, (y, x) in enumerate(cands):
        for tau in range(Tw):
            np.testing.assert_array_equal(out[n, :, tau], st.frame(T - Tw + 1 + tau)[:, y, x])
    outb = O.dynspec(lambda t: st.frame(t), T, Tw, cands, 1)
    fr = st.frame(T)
    assert outb[1, 3, Tw - 1] == max(fr[3, yy, xx] for yy in (9, 10, 11) for xx in (62, 63))


# ----------------------------------------------------------------- storage rounding
def test_storage_round_ties_to_even():
    x = np.array([1.0 + 2.0 ** -11, 1.0 + 3 * 2.0 ** -11, 65504.0, 1.0 + 2.0 ** -8])
    h = O.storage_round(x, "fp16")
    assert h[0] == 1.0 and h[1] == 1.0 + 2 * 2.0 ** -10 and h[2] == 65504.0
    b = O.storage_round(x, "bf16")
    assert b[3] == 1.0                     # 1 + 2^-8 is a tie in bf16 -> even (1.0)


# ----------------------------------------------------------------- whole push
def test_search_push_warmup_and_order():
    spec = synth.spec_tiny()
    st = synth.SyntheticStream(spec, seed=12)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    dmax = delays.max(axis=1)
    fa = lambda t: st.frame(t).astype(np.float64)
    # at T = 0 only the trials without delay are active
    cands, stats, _ = O.search_push(fa, 0, delays, spec.box_r, spec.kappa)
    assert set(stats) == {d for d in range(spec.n_dm) if dmax[d] == 0}
    cands, stats, _ = O.search_push(fa, 5, delays, spec.box_r, spec.kappa)
    assert set(stats) == set(range(spec.n_dm))
    keys = [(c[0], c[1], c[2], c[3]) for c in cands]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    # the injected DM-7 pulse is detected at its pixel in the push that completes its sweep
    p = st.pulses[0]
    t0 = int(round(p.t0))
    hits = []
    for T in range(t0, t0 + int(dmax.max()) + 1):
        cs, _, _ = O.search_push(fa, T, delays, spec.box_r, spec.kappa)
        hits += [c for c in cs if (c[2], c[3]) == (p.y, p.x) and c[0] == t0]
    assert hits and max(c[4] for c in hits) > 8


@pytest.mark.parametrize("r", [2, 7])
def test_lone_delta_snr_closed_form(r):
    """Two-pass chain on a lone delta over a zero background: C = A/n on the window,
    S(p) = A^2 (n-1)/n^2, hence snr(p) = sqrt(n - 1) for any amplitude A."""
    size = 4 * r + 9
    for A in (1.0, 37.5):
        img = np.zeros((size, size))
        c = size // 2
        img[c, c] = A
        res = O.detect(img, r, 0.0)
        n = (2 * r + 1) ** 2
        assert abs(res["snr"][c, c] - math.sqrt(n - 1)) < 1e-9
        assert res["mask"][c, c] and res["mask"].sum() == 1


# ----------------------------------------------------------------- planted mistakes
def _pins_box(centre, spread):
    rng = np.random.default_rng(21)
    img = rng.standard_normal((9, 13)) + np.arange(13)[None] * 0.3
    C = centre(img, 2)
    ok = np.allclose(C, brute_box_mean(img, 2), atol=1e-12)
    ok &= np.allclose(spread(img, C, 2), brute_spread(img, brute_box_mean(img, 2), 2), atol=1e-12)
    return ok


def test_pins_catch_planted_box_mistakes():
    assert _pins_box(O.local_centre, O.local_spread)
    full_norm = lambda D, r: O.box_sum(D, r) / (2 * r + 1) ** 2
    assert not _pins_box(full_norm, O.local_spread)                      # no edge truncation
    one_pass = lambda D, C, r: O.local_centre(D * D, r) - C * C
    assert not _pins_box(O.local_centre, one_pass)                       # E[x^2]-E[x]^2
    short = lambda D, r: O.window_sum_1d(O.window_sum_1d(D, r, 1), r - 1, 0) / O.window_count(*D.shape, r)
    assert not _pins_box(short, O.local_spread)                          # wrong radius on one axis
    centre_here = lambda D, C, r: O.box_sum(D * D, r) / O.window_count(*D.shape, r) - 2 * C * O.local_centre(D, r) + C * C
    assert not _pins_box(O.local_centre, centre_here)


def test_pins_catch_planted_shift_sign():
    def wrong_dedisperse(frame_at, T, delays, d):
        row = delays[d]
        t0 = T - int(row.max())
        D = 0
        for f in range(len(row)):
            D = D + frame_at(t0 + int(row.max() - row[f]))[f]      # reversed shift
        return t0, D
    delays = np.array([[3, 2, 1, 0]], np.int64)
    arr = np.zeros((8, 4, 2, 2))
    arr[6, 1, 0, 0] = 1.0                       # impulse at f=1, t=6 -> t0 = 4 at T = 7
    _, D = wrong_dedisperse(_frames_from_array(arr), 7, delays, 0)
    _, Dok = O.dedisperse(_frames_from_array(arr), 7, delays, 0)
    assert Dok[0, 0] == 1.0 and D[0, 0] != 1.0


def test_residual_form_equals_direct_form():
    """Linearity of the local centre: sum_f (X_f - C(X_f)) shifted = D - C (Sec. 2.1.1)."""
    spec = synth.spec_tiny(H=40, W=52, box_r=5, kappa=3.0, n_sources=6)
    st = synth.SyntheticStream(spec, seed=31)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    raw = lambda t: st.frame(t).astype(np.float64)
    res = lambda t: O.residual_frame(raw(t), spec.box_r)
    for T in (3, 9):
        a, sa, ma = O.search_push(raw, T, delays, spec.box_r, spec.kappa, keep_maps=True)
        b, sb, mb = O.search_push_residual(raw, res, T, delays, spec.box_r, spec.kappa, keep_maps=True)
        assert [c[:4] for c in a] == [c[:4] for c in b] and len(a) > 0
        for d in ma:
            np.testing.assert_allclose(ma[d]["snr"], mb[d]["snr"], rtol=0, atol=1e-9)
            assert abs(sa[d][1] - sb[d][1]) < 1e-12


# ----------------------------------------------------------------- quality control (App. A)
def _bands(means, H=4, W=4):
    return np.stack([np.full((H, W), float(v)) for v in means])


def test_qc_band_scores_closed_forms():
    """Median and median absolute deviation worked by hand (App. A z-scores)."""
    # odd count: median 3, |dev| = 2 1 0 1 97 -> MAD 1
    assert np.allclose(O.qc_band_scores(_bands([1, 2, 3, 4, 100])), [-2, -1, 0, 1, 97])
    # even count: median 2.5, |dev| = 1.5 .5 .5 1.5 -> MAD 1
    assert np.allclose(O.qc_band_scores(_bands([1, 2, 3, 4])), [-1.5, -0.5, 0.5, 1.5])
    # MAD = 0: the bands at the median score 0, the other +inf
    z = O.qc_band_scores(_bands([5, 5, 5, 9]))
    assert list(z[:3]) == [0, 0, 0] and z[3] == np.inf
    # the band mean is over all pixels of the band image
    f = _bands([0, 0, 0, 0, 0])
    f[4, 0, 0] = 16.0                        # mean 1 over 16 pixels
    assert np.allclose(O.qc_band_scores(f), [0, 0, 0, 0, np.inf])


def _qc_history(seed=3, T=40, F=6, H=8, W=9):
    rng = np.random.default_rng(seed)
    # band levels differ (as real band images do), so noise alone keeps |z| small
    level = 0.5 * np.arange(F)[:, None, None]
    frames = [level + rng.standard_normal((F, H, W)) * (1 + 0.1 * np.arange(F))[:, None, None] for _ in range(T)]
    frames[17][2] += 40.0                    # a corrupted band (global offset)
    frames[25][4, 3, 3] += 500.0             # an RFI spike in one band
    return frames


def test_qc_running_statistics_equal_batch_statistics():
    """Welford state = mean and sample variance of exactly the kept band images."""
    frames = _qc_history()
    F, H, W = frames[0].shape
    st = O.QCState(F, H, W)
    kept = [[] for _ in range(F)]
    for x in frames:
        _, disc, _, _ = O.qc_frame(x, st, z_thr=5.0, zeta_thr=20.0, min_frames=10)
        for f in range(F):
            if not disc[f]:
                kept[f].append(x[f])
    for f in range(F):
        h = np.array(kept[f])
        assert st.n[f] == len(h)
        assert np.allclose(st.mean[f], h.mean(axis=0), atol=1e-12)
        assert np.allclose(st.m2[f] / (len(h) - 1), h.var(axis=0, ddof=1), atol=1e-11)


def test_qc_discards_corrupted_band_and_spike_only():
    frames = _qc_history()
    F, H, W = frames[0].shape
    st = O.QCState(F, H, W)
    seen = {}
    for t, x in enumerate(frames):
        out, disc, z, zeta = O.qc_frame(x, st, z_thr=5.0, zeta_thr=20.0, min_frames=10)
        seen[t] = disc.copy()
        assert np.all(out[disc] == 0) and np.array_equal(out[~disc], x[~disc])
    assert seen[17][2] and seen[17].sum() == 1           # band offset: |z| large
    assert seen[25][4] and seen[25].sum() == 1           # spike: |zeta| large
    assert sum(int(v.sum()) for v in seen.values()) == 2  # nothing else


def test_qc_pixel_score_uses_the_previous_statistics():
    """zeta of the spike frame is computed from the 25 frames before it (band 4 of
    none of them discarded), by hand."""
    frames = _qc_history()
    F, H, W = frames[0].shape
    st = O.QCState(F, H, W)
    for x in frames[:25]:
        O.qc_frame(x, st, z_thr=5.0, zeta_thr=20.0, min_frames=10)
    hist = np.array([x[4] for x in frames[:25]])
    s = hist.std(axis=0, ddof=1)
    expect = np.max(np.abs(frames[25][4] - hist.mean(axis=0)) / s)
    _, _, _, zeta = O.qc_frame(frames[25], st, z_thr=5.0, zeta_thr=20.0, min_frames=10)
    assert np.isclose(zeta[4], expect, rtol=1e-12)
    # and below min_frames no band is pixel-tested
    st2 = O.QCState(F, H, W)
    for x in frames[:5]:
        _, _, _, zeta = O.qc_frame(x, st2, z_thr=5.0, zeta_thr=20.0, min_frames=10)
        assert np.all(zeta == 0)


def test_pins_catch_planted_qc_mistakes():
    # a mean in place of the median moves every score of the worked example
    def mean_centre(frame):
        b = frame.reshape(frame.shape[0], -1).mean(axis=1)
        c = b.mean()
        return (b - c) / np.median(np.abs(b - c))
    assert not np.allclose(mean_centre(_bands([1, 2, 3, 4, 100])), [-2, -1, 0, 1, 97])

    # folding the frame in before scoring it hides the spike (the test above would fail)
    frames = _qc_history()
    F, H, W = frames[0].shape
    st = O.QCState(F, H, W)
    for x in frames[:25]:
        O.qc_frame(x, st, z_thr=5.0, zeta_thr=20.0, min_frames=10)
    n, mean, m2 = st.n[4] + 1, st.mean[4].copy(), st.m2[4].copy()
    x = frames[25][4]
    d = x - mean
    mean += d / n
    m2 += d * (x - mean)
    zeta_after = np.max(np.abs(x - mean) / np.sqrt(m2 / (n - 1)))
    _, _, _, zeta = O.qc_frame(frames[25], st, z_thr=5.0, zeta_thr=20.0, min_frames=10)
    assert zeta[4] > 20.0 and zeta_after < zeta[4] / 1.5



# ----------------------------------------------------------------- per-subband detector (Sec. 2.1.1-2.1.2)
def test_local_max_radius_3_matches_brute_force():
    rng = np.random.default_rng(15)
    img = rng.integers(0, 6, (17, 14)).astype(float)     # ties and clipped windows
    assert np.array_equal(O.local_max_mask(img, 3), brute_local_max(img, 3))
    assert np.array_equal(O.local_max_mask(img, 1), brute_local_max(img, 1))


def test_iid_noise_local_max_fraction_radius_3_is_one_49th():
    rng = np.random.default_rng(16)
    img = rng.standard_normal((600, 600))
    frac = O.local_max_mask(img, 3)[3:-3, 3:-3].mean()
    n = 594 * 594
    sigma = math.sqrt((1 / 49) * (48 / 49) / n) * 7     # overlapping windows are dependent
    assert abs(frac - 1 / 49) < 5 * sigma


def test_subband_detect_finds_a_source_in_one_band_only():
    """A compact source in band 2 only (31x31 box, so its own flux does not swamp
    its spread): one candidate there, none in the other bands.  A side lobe 3 px
    away is above the threshold and a 3x3 maximum, but the 7x7 maximum filter
    merges it into the source (the deblending of Sec. 2.1.2)."""
    rng = np.random.default_rng(17)
    F, H, W = 4, 48, 48
    x = rng.standard_normal((F, H, W)) * 0.1
    yy, xx = np.mgrid[:H, :W]
    x[2] += 20.0 * np.exp(-((yy - 20) ** 2 + (xx - 30) ** 2) / (2 * 1.5 ** 2))
    x[2, 20, 33] += 14.0                                # the side lobe
    cands, stats, maps = O.subband_detect(x, 15, 6.0, k=3)
    assert [(b, y, xq) for b, y, xq, _ in cands] == [(2, 20, 30)]
    three = O.detect(x[2], 15, 6.0, 1)
    assert three["mask"][20, 33] and three["mask"][20, 30]   # the 3x3 window keeps both
    assert set(stats) == {0, 1, 2, 3}


def test_subband_detect_is_detect_per_band():
    rng = np.random.default_rng(18)
    x = rng.standard_normal((3, 20, 24))
    x[1, 5, 7] += 30.0
    cands, _, maps = O.subband_detect(x, 5, 4.0, k=2)
    for b in range(3):
        ref = O.detect(x[b], 5, 4.0, 2)
        assert np.array_equal(maps[b]["mask"], ref["mask"])
        got = sorted((y, xq) for bb, y, xq, _ in cands if bb == b)
        assert got == sorted(zip(*np.nonzero(ref["mask"])))


# ----------------------------------------------------------------- iterated sigma clipping (Sec. 2.1.1)
def test_clip_one_iteration_is_the_one_pass_filter():
    rng = np.random.default_rng(19)
    D = rng.standard_normal((30, 34))
    D[10, 12] += 25.0
    a = O.clip_detect(D, 5, 4.0, k=1, iters=1)
    b = O.detect(D, 5, 4.0, 1)
    assert np.array_equal(a["mask"], b["mask"]) and np.allclose(a["snr"], b["snr"], atol=1e-12)


def test_clip_masked_means_by_brute_force():
    """Second iteration: C and S at every pixel from the unflagged window pixels only."""
    rng = np.random.default_rng(20)
    D = rng.standard_normal((14, 15))
    D[6, 7] += 40.0
    r = 2                                    # a lone delta reaches sqrt(24) = 4.9 in a 5x5 window
    first = O.clip_detect(D, r, 4.0, iters=1)
    flags = first["snr"] > 4.0
    assert flags[6, 7] and flags.sum() == 1
    second = O.clip_detect(D, r, 4.0, iters=2)
    H, W = D.shape
    for y in range(H):
        for x in range(W):
            vals = [D[yy, xx] for yy in range(max(0, y - r), min(H, y + r + 1))
                    for xx in range(max(0, x - r), min(W, x + r + 1)) if not flags[yy, xx]]
            c = sum(vals) / len(vals)
            assert abs(second["C"][y, x] - c) < 1e-12
    # S uses C at each window pixel (two-pass), over the same pixels
    y, x = 6, 7
    terms = [(D[yy, xx] - second["C"][yy, xx]) ** 2 for yy in range(y - r, y + r + 1)
             for xx in range(x - r, x + r + 1) if not flags[yy, xx]]
    assert abs(second["S"][y, x] - sum(terms) / len(terms)) < 1e-12


def test_clip_unmasks_a_faint_source_beside_a_bright_one():
    """One pass: a bright point source inflates the spread around it and hides a
    faint source 6 px away; once the bright pixel is flagged (first pass) and left
    out of C and S (second pass) the faint one crosses the threshold; a third pass
    flags nothing new and the loop stops."""
    rng = np.random.default_rng(22)
    D = rng.standard_normal((64, 64))
    yy, xx = np.mgrid[:64, :64]
    D[30, 30] += 400.0
    D += 9.0 * np.exp(-((yy - 30) ** 2 + (xx - 36) ** 2) / (2 * 1.0 ** 2))
    one = O.clip_detect(D, 7, 6.0, k=1, iters=1)
    many = O.clip_detect(D, 7, 6.0, k=1, iters=6)
    assert not one["mask"][30, 36] and many["mask"][30, 36]
    assert many["mask"][30, 30]
    # the loop stops once nothing new is flagged: more iterations change nothing
    more = O.clip_detect(D, 7, 6.0, k=1, iters=12)
    assert np.array_equal(more["mask"], many["mask"]) and np.array_equal(more["flags"], many["flags"])


# ----------------------------------------------------------------- Gaussian kernel G(n, m, s) (Sec. 2.1.1)
def test_gauss_kernel_delta_response_is_the_normalised_kernel():
    """A unit delta at p0: wherever the window lies inside the image, C(p) =
    exp(-|p - p0|^2 / (2 s^2)) / Z, Z the unnormalised kernel summed over the
    (2r+1)^2 window (the 2-D form, not its factors); zero beyond r."""
    H, W, r, s = 41, 37, 5, 1.7
    D = np.zeros((H, W))
    y0, x0 = 20, 18
    D[y0, x0] = 1.0
    Z = sum(math.exp(-(i * i + j * j) / (2 * s * s)) for i in range(-r, r + 1) for j in range(-r, r + 1))
    C = O.clip_detect(D, r, 1e9, iters=1, s=s)["C"]
    for dy in range(-r - 2, r + 3):
        for dx in range(-r - 2, r + 3):
            inside = abs(dy) <= r and abs(dx) <= r
            want = math.exp(-(dy * dy + dx * dx) / (2 * s * s)) / Z if inside else 0.0
            assert abs(C[y0 + dy, x0 + dx] - want) < 1e-15 + 1e-12 * want, (dy, dx)


def test_gauss_kernel_reproduces_an_affine_image_inside():
    """G is symmetric, so G * (a + b y + c x) is the image itself wherever the window
    is whole, and S = 0 where every window pixel's C is exact; at an edge the
    truncated window is lopsided and C departs from the image."""
    H, W, r, s = 40, 44, 4, 2.5
    yy, xx = np.mgrid[:H, :W]
    D = 3.0 + 0.7 * yy - 1.3 * xx
    res = O.clip_detect(D, r, 6.0, iters=1, s=s)
    inner = (slice(r, H - r), slice(r, W - r))
    assert np.allclose(res["C"][inner], D[inner], rtol=0, atol=1e-10)
    core = (slice(2 * r, H - 2 * r), slice(2 * r, W - 2 * r))
    assert np.all(res["S"][core] < 1e-18)
    assert abs(res["C"][0, 20] - D[0, 20]) > 0.5


def test_gauss_kernel_masked_means_by_brute_force():
    """Second iteration with the Gaussian kernel, image edges included: C and S at
    every pixel are the means over the unflagged in-image window pixels, each
    weighted by exp(-(dy^2 + dx^2) / (2 s^2)) taken whole.  A lone delta reaches
    at most sqrt(Z) = 3.47 here, hence kappa = 3."""
    rng = np.random.default_rng(23)
    D = rng.standard_normal((13, 11))
    D[5, 4] += 60.0
    D[9, 8] += 45.0
    r, s, kappa = 3, 1.4, 3.0
    first = O.clip_detect(D, r, kappa, iters=1, s=s)
    flags = first["snr"] > kappa
    assert flags[5, 4] and flags[9, 8] and flags.sum() == 2
    second = O.clip_detect(D, r, kappa, iters=2, s=s)
    H, W = D.shape

    def wmean(y, x, val):
        num = den = 0.0
        for yy in range(max(0, y - r), min(H, y + r + 1)):
            for xx in range(max(0, x - r), min(W, x + r + 1)):
                if not flags[yy, xx]:
                    w = math.exp(-((yy - y) ** 2 + (xx - x) ** 2) / (2 * s * s))
                    num += w * val(yy, xx)
                    den += w
        return num / den

    for y in range(H):
        for x in range(W):
            assert abs(second["C"][y, x] - wmean(y, x, lambda a, b: D[a, b])) < 1e-12
            sq = wmean(y, x, lambda a, b: (D[a, b] - second["C"][a, b]) ** 2)
            assert abs(second["S"][y, x] - sq) < 1e-12 * max(1.0, sq)


def test_gauss_kernel_wide_limit_is_the_box():
    """s -> infinity: every weight tends to 1 and the Gaussian detector becomes the
    box detector (masks equal, S/N to 1e-9), through three clipping iterations."""
    rng = np.random.default_rng(24)
    D = rng.standard_normal((30, 26))
    D[12, 9] += 30.0
    D[20, 18] += 12.0
    a = O.clip_detect(D, 4, 4.0, k=2, iters=3, s=1e7)
    b = O.clip_detect(D, 4, 4.0, k=2, iters=3)
    assert np.array_equal(a["mask"], b["mask"]) and a["mask"].any()
    assert np.allclose(a["snr"], b["snr"], rtol=0, atol=1e-9)


def _factor_sum(img, g, rx, ry):
    """sum of img over the window clipped to the image, weights g[|dx|] g[|dy|] (a test copy)."""
    out = np.asarray(img, np.float64)
    for axis, r in ((1, rx), (0, ry)):
        a, n = out, out.shape[axis]
        out = np.zeros_like(a)
        for k in range(-r, r + 1):
            dst, src = [slice(None)] * 2, [slice(None)] * 2
            dst[axis] = slice(max(-k, 0), n - max(k, 0))
            src[axis] = slice(max(k, 0), n - max(-k, 0))
            out[tuple(dst)] += g[abs(k)] * a[tuple(src)]
    return out


def _gauss_pins_hold(centre):
    """The Gaussian kernel's pins for a centre estimate centre(D, m, r, s): the
    delta response (2-D normalised kernel inside the image) and the masked means
    with whole 2-D weights at the image edges."""
    r, s = 4, 1.7
    D = np.zeros((21, 19))
    D[10, 9] = 1.0
    Z = sum(math.exp(-(i * i + j * j) / (2 * s * s)) for i in range(-r, r + 1) for j in range(-r, r + 1))
    C = centre(D, np.ones_like(D), r, s)
    ok = all(abs(C[10 + dy, 9 + dx] - math.exp(-(dy * dy + dx * dx) / (2 * s * s)) / Z) < 1e-12
             for dy in range(-r, r + 1) for dx in range(-r, r + 1))
    rng = np.random.default_rng(25)
    X = rng.standard_normal((9, 11))
    m = np.ones_like(X)
    m[0, 0] = m[4, 5] = m[8, 3] = 0.0
    r2, s2 = 3, 1.4
    C2 = centre(X, m, r2, s2)
    for y in range(9):
        for x in range(11):
            num = den = 0.0
            for yy in range(max(0, y - r2), min(9, y + r2 + 1)):
                for xx in range(max(0, x - r2), min(11, x + r2 + 1)):
                    w = m[yy, xx] * math.exp(-((yy - y) ** 2 + (xx - x) ** 2) / (2 * s2 * s2))
                    num += w * X[yy, xx]
                    den += w
            ok &= abs(C2[y, x] - num / den) < 1e-12
    return bool(ok)


def test_pins_catch_planted_gauss_mistakes():
    oracle = lambda D, m, r, s: O.kernel_sum(D * m, r, s) / O.kernel_sum(m, r, s)
    assert _gauss_pins_hold(oracle)
    fac = lambda r, s, den: np.exp(-np.arange(r + 1) ** 2 / den(s))
    # s in place of s^2 in the exponent
    bad_width = lambda D, m, r, s: (_factor_sum(D * m, fac(r, s, lambda s: 2 * s), r, r)
                                    / _factor_sum(m, fac(r, s, lambda s: 2 * s), r, r))
    assert not _gauss_pins_hold(bad_width)
    # normalised by the whole window's weight (no truncation at the edges, no mask)
    full_z = lambda D, m, r, s: O.kernel_sum(D * m, r, s) / (O.kernel_factors(r, s).sum() ** 2)
    assert not _gauss_pins_hold(full_z)
    # flagged pixels left in the normaliser
    unmasked = lambda D, m, r, s: O.kernel_sum(D * m, r, s) / O.kernel_sum(np.ones_like(m), r, s)
    assert not _gauss_pins_hold(unmasked)
    # control: the test's own weighted sums with the right factors pass
    g = lambda r, s: fac(r, s, lambda s: 2 * s * s)
    assert _gauss_pins_hold(lambda D, m, r, s: _factor_sum(D * m, g(r, s), r, r) / _factor_sum(m, g(r, s), r, r))
    # one axis a pixel short
    short = lambda D, m, r, s: _factor_sum(D * m, g(r, s), r, r - 1) / _factor_sum(m, g(r, s), r, r - 1)
    assert not _gauss_pins_hold(short)


def _clip_pin_holds(clip):
    """The masked-means pin of iterated clipping for an implementation
    clip(D, r, kappa, iters) -> (C, S): the second iteration's C and S are the
    means over the window pixels the first iteration left unflagged."""
    rng = np.random.default_rng(20)
    D = rng.standard_normal((14, 15))
    D[6, 7] += 40.0
    r, kappa = 2, 4.0
    flags = O.clip_detect(D, r, kappa, iters=1)["snr"] > kappa
    C, S = clip(D, r, kappa, 2)
    H, W = D.shape
    ok = True
    for y in range(H):
        for x in range(W):
            win = [(yy, xx) for yy in range(max(0, y - r), min(H, y + r + 1))
                   for xx in range(max(0, x - r), min(W, x + r + 1)) if not flags[yy, xx]]
            c = sum(D[q] for q in win) / len(win)
            sq = sum((D[q] - C[q]) ** 2 for q in win) / len(win)
            ok &= abs(C[y, x] - c) < 1e-12 and abs(S[y, x] - sq) < 1e-12
    return bool(ok)


def test_pins_catch_planted_clip_mistakes():
    def oracle(D, r, kappa, iters):
        m = O.clip_detect(D, r, kappa, iters=iters)
        return m["C"], m["S"]
    assert _clip_pin_holds(oracle)

    def first_pass_only(D, r, kappa, iters):              # never re-estimates
        return oracle(D, r, kappa, 1)
    assert not _clip_pin_holds(first_pass_only)

    def full_count(D, r, kappa, iters):                   # masked sums over the whole window's count
        flags = O.clip_detect(D, r, kappa, iters=1)["snr"] > kappa
        m = (~flags).astype(float)
        n = O.window_count(*D.shape, r)
        C = O.box_sum(D * m, r) / n
        return C, O.box_sum((D - C) ** 2 * m, r) / n
    assert not _clip_pin_holds(full_count)


# ---------------------------------------------------------------------------
# opt-in steady-source suppression (a reading of Sec. 2.2 / 2.3 removal)

def test_steady_mask_needs_k_pushes_in_a_row():
    m = O.SteadyMask(3)
    a, b = (5, 7), (9, 1)
    seq = [{a}, {a, b}, {a, b}, {b}, {a, b}, {a, b}, {a}]
    got = [m.update(s) for s in seq]
    # a: runs 1, 2, 3, 0, 1, 2, 3 -> steady at the third and the seventh push
    # b: runs 0, 1, 2, 3, 4, 5, 0 -> steady at the fourth to the sixth push
    assert got == [set(), set(), {a}, {b}, {b}, {b}, {a}]


def test_suppress_steady_drops_only_dispersed_trials_at_steady_pixels():
    dmax = np.array([0, 0, 3, 5])                    # trials 0 and 1: zero delay rows
    cands = [(10, 0, 5, 5, 9.0), (10, 1, 5, 5, 9.0), (7, 2, 5, 5, 8.0), (5, 3, 5, 5, 7.0),
             (7, 2, 6, 6, 8.0), (5, 3, 1, 2, 7.0)]
    kept = O.suppress_steady(cands, dmax, {(5, 5)})
    assert kept == [(10, 0, 5, 5, 9.0), (10, 1, 5, 5, 9.0), (7, 2, 6, 6, 8.0), (5, 3, 1, 2, 7.0)]
    assert O.suppress_steady(cands, dmax, set()) == cands


def test_steady_sources_suppressed_and_pulse_kept_on_a_stream():
    """On the tiny stream (three steady 20-sigma sources, one pulse at DM 7,
    kappa 4): once the sources have been zero-delay candidates K pushes in a row,
    no dispersed trial keeps a candidate at a source pixel, and the pulse's
    candidates are untouched."""
    spec = synth.spec_tiny(kappa=4.0)
    st = synth.SyntheticStream(spec, seed=3)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    dmax = delays.max(axis=1)
    assert (dmax == 0).any() and (dmax > 0).any()
    src = {(y, x) for y, x, _ in st.sources}
    frame_at = lambda t: st.frame(t).astype(np.float64)
    K = 3
    mask = O.SteadyMask(K)
    dropped_at_sources = 0
    for T in range(20):
        cands, _, _ = O.search_push(frame_at, T, delays, spec.box_r, spec.kappa)
        steady = mask.update({(c[2], c[3]) for c in cands if dmax[c[1]] == 0})
        kept = O.suppress_steady(cands, dmax, steady)
        if T >= K - 1:
            assert src <= steady, (T, src - steady)
            assert not [c for c in kept if dmax[c[1]] > 0 and (c[2], c[3]) in src]
        dropped_at_sources += sum(1 for c in cands if dmax[c[1]] > 0 and (c[2], c[3]) in src)
        # nothing outside the steady pixels is dropped
        assert [c for c in cands if (c[2], c[3]) not in steady] == [c for c in kept if (c[2], c[3]) not in steady]
    assert dropped_at_sources > 0
