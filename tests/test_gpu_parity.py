"""Parity of the CUDA path (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
from tests.parity import assert_sorted_unique, cached_frames, cached_residuals, compare_push, compare_storage

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _open(lib, spec, dtype=None, **kw):
    return lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth,
                      cadence_s=spec.cadence_s, kappa=spec.kappa, box_r=spec.box_r,
                      dtype=dtype or spec.dtype, **kw)


def _push(s, st, T):
    s.push(torch.from_numpy(st.frame(T)).cuda(), T)


def test_tiny_stream_every_frame(lib):
    spec = synth.spec_tiny()
    st = synth.SyntheticStream(spec, seed=5)
    fa = cached_frames(st)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    matched = 0
    with _open(lib, spec) as s:
        assert np.array_equal(s.delay_table(), delays)          # bit-exact integer table
        for T in range(spec.n_frames):
            _push(s, st, T)
            Tp, c, n, trunc = s.poll(timeout_ms=60000)
            assert Tp == T and not trunc and n == len(c)
            assert_sorted_unique(c)
            res = compare_push(c, fa, T, delays, spec.box_r, spec.kappa, gpu_stats=s.stats())
            matched += res["matched"]
    assert matched > 0          # the injected DM-7 pulse is found


@pytest.mark.parametrize("dtype", ["fp32", "fp16", "bf16"])
def test_aartfaac_bands_256px(lib, dtype):
    """AARTFAAC band layout and DM grid (251 trials, depth 48) on a 256x256 image."""
    spec = synth.spec_aartfaac(H=256, W=256, n_sources=40, n_pulses=6, n_frames=80)
    st = synth.SyntheticStream(spec, seed=7)
    fa = cached_frames(st, dtype)
    ra = None if dtype == "fp32" else cached_residuals(st, dtype, spec.box_r)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    checks = {10, 47, 48, 61}
    with _open(lib, spec, dtype=dtype) as s:
        assert np.array_equal(s.delay_table(), delays)
        for T in range(62):
            _push(s, st, T)
            Tp, c, n, trunc = s.poll(timeout_ms=60000)
            assert Tp == T and not trunc
            if T in checks:
                assert_sorted_unique(c)
                res = compare_storage(c, fa, T, delays, spec.box_r, spec.kappa, dtype, gpu_stats=s.stats(),
                                      res_at=ra)
                assert res["matched"] > 0


@pytest.mark.parametrize("r", [5, 7])
def test_ragged_sizes_and_small_box(lib, r):
    """Image not a multiple of the tile/strip or of 4 pixels, 5 subbands (tiled r=5, streaming r=7)."""
    spec = synth.spec_tiny(H=70, W=93, freqs_mhz=synth.subband_centres([60.0], 5),
                           dm_grid=np.arange(0, 40, 3, dtype=np.float64), depth=12, box_r=r,
                           kappa=4.0, n_sources=4)
    st = synth.SyntheticStream(spec, seed=9)
    fa = cached_frames(st)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    assert delays.max() + 1 <= spec.depth
    with _open(lib, spec) as s:
        for T in range(20):
            _push(s, st, T)
            _, c, n, _ = s.poll(timeout_ms=60000)
            assert_sorted_unique(c)
            compare_push(c, fa, T, delays, spec.box_r, spec.kappa, gpu_stats=s.stats())


@pytest.mark.parametrize("F,dtype", [(32, "fp32"), (32, "fp16"), (24, "bf16"), (17, "fp32")])
def test_more_than_16_subbands(lib, F, dtype):
    """More than 16 subbands (the shift-sum with 8 bytes of each plane per thread;
    24 and 17 take the instantiation for F below its maximum), FP32 and 16-bit
    rings, a 66 x 90 image (rows not a multiple of 4 pixels)."""
    spec = synth.spec_tiny(H=66, W=90, freqs_mhz=synth.subband_centres([57.6], F),
                           dm_grid=np.arange(0, 40, 2.0), depth=24, box_r=7, kappa=4.0, n_sources=4)
    st = synth.SyntheticStream(spec, seed=13)
    fa = cached_frames(st, dtype)
    ra = None if dtype == "fp32" else cached_residuals(st, dtype, spec.box_r)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    assert delays.max() + 1 <= spec.depth
    matched = 0
    with _open(lib, spec, dtype=dtype) as s:
        for T in range(int(delays.max()) + 6):
            _push(s, st, T)
            _, c, n, trunc = s.poll(timeout_ms=60000)
            assert not trunc
            if T >= delays.max():
                assert_sorted_unique(c)
                res = compare_storage(c, fa, T, delays, spec.box_r, spec.kappa, dtype, gpu_stats=s.stats(),
                                      res_at=ra)
                matched += res["matched"]
    assert matched > 0


@pytest.mark.parametrize("r", [1, 8, 16])
def test_box_radius_extremes(lib, r):
    spec = synth.spec_tiny(H=80, W=72, box_r=r, kappa=4.0, n_frames=8)
    st = synth.SyntheticStream(spec, seed=10 + r)
    fa = cached_frames(st)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    with _open(lib, spec) as s:
        for T in range(4):
            _push(s, st, T)
            _, c, _, _ = s.poll(timeout_ms=60000)
            compare_push(c, fa, T, delays, r, spec.kappa, gpu_stats=s.stats())


@pytest.mark.parametrize("impl", ["tiled", "streaming"])
def test_filter_kernels_agree_at_r15(lib, impl):
    """Both filter kernels on the AARTFAAC bands at 320x288 (strip and tile tails), kappa 4."""
    spec = synth.spec_aartfaac(H=320, W=288, n_sources=60, n_pulses=4, n_frames=52, kappa=4.0)
    st = synth.SyntheticStream(spec, seed=17)
    fa = cached_frames(st)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    with _open(lib, spec, filter_impl=impl) as s:
        for T in range(49):
            _push(s, st, T)
            _, c, n, trunc = s.poll(timeout_ms=60000)
        res = compare_push(c, fa, 48, delays, spec.box_r, spec.kappa, dms=[0, 3, 50, 120, 200, 250],
                           gpu_stats=s.stats())
        assert res["matched"] > 100


def test_aartfaac_full_size_sampled_trials(lib):
    """1024^2 x 16 subbands x 251 trials, depth 48: every candidate of sampled trials."""
    spec = synth.spec_aartfaac(n_frames=60)
    st = synth.SyntheticStream(spec, seed=2)
    fa = cached_frames(st)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    with _open(lib, spec) as s:
        for T in range(50):
            _push(s, st, T)
            _, c, n, trunc = s.poll(timeout_ms=120000)
            assert not trunc
        assert_sorted_unique(c)
        # steady sources are found at every trial: about 500 candidates per trial
        assert n > 250 * 251
        dms = [0, 1, 37, 100, 173, 250]
        res = compare_push(c, fa, 49, delays, spec.box_r, spec.kappa, dms=dms, gpu_stats=s.stats())
        assert res["matched"] > 300 * len(dms)


def test_dynspec_matches_direct_indexing(lib):
    for dtype in ("fp32", "fp16"):
        for box in (0, 1):
            spec = synth.spec_tiny()
            st = synth.SyntheticStream(spec, seed=3)
            fa = cached_frames(st, dtype)
            with _open(lib, spec, dtype=dtype, dyn_box_r=box) as s:
                for T in range(20):
                    _push(s, st, T)
                    _, c, _, _ = s.poll(timeout_ms=60000)
                extra = np.zeros(3, dtype=c.dtype)
                extra["y"] = [0, 63, 17]
                extra["x"] = [0, 63, 40]
                cands = np.concatenate([c, extra])
                out = s.dynspec(cands, 12).cpu().numpy()
                ref = O.dynspec(fa, 19, 12, list(zip(cands["y"].tolist(), cands["x"].tolist())), box)
                np.testing.assert_array_equal(out, ref.astype(np.float32))


def test_errors_and_edge_cases(lib):
    spec = synth.spec_tiny()
    st = synth.SyntheticStream(spec, seed=4)
    with pytest.raises(lib.LpfError) as e:
        lib.Stream(64, 64, spec.freqs_mhz, np.array([0.0, 400.0]), 4)
    assert e.value.code == lib.LPF_E_DEPTH
    with _open(lib, spec, result_slots=2) as s:
        _push(s, st, 0)
        with pytest.raises(lib.LpfError) as e:
            _push(s, st, 2)
        assert e.value.code == lib.LPF_E_ORDER
        _push(s, st, 1)
        with pytest.raises(lib.LpfError) as e:
            _push(s, st, 2)
        assert e.value.code == lib.LPF_E_BUSY
        assert s.poll(timeout_ms=60000)[0] == 0
        assert s.poll(timeout_ms=60000)[0] == 1
        with pytest.raises(lib.LpfError) as e:
            s.poll(timeout_ms=0)
        assert e.value.code == lib.LPF_E_NODATA
        # dynspec: window beyond the first frame, pixel outside the image, Tw > depth
        with pytest.raises(lib.LpfError) as e:
            s.dynspec(np.zeros(1, dtype=lib.CANDIDATE_DTYPE), 5)
        assert e.value.code == lib.LPF_E_STALE
        bad = np.zeros(1, dtype=lib.CANDIDATE_DTYPE)
        bad["y"] = 64
        with pytest.raises(lib.LpfError) as e:
            s.dynspec(bad, 1)
        assert e.value.code == lib.LPF_E_ARG
        with pytest.raises(lib.LpfError) as e:
            s.dynspec(bad, 17)
        assert e.value.code == lib.LPF_E_DEPTH
    # frames overwritten in the ring -> stale (frame 2 polled, then 16 more pushed, depth 16)
    with _open(lib, spec, result_slots=16) as s:
        for T in range(3):
            _push(s, st, T)
            s.poll(timeout_ms=60000)
        s.dynspec(np.zeros(1, dtype=lib.CANDIDATE_DTYPE), 1)
        for T in range(3, 19):
            _push(s, st, T)
        with pytest.raises(lib.LpfError) as e:
            s.dynspec(np.zeros(1, dtype=lib.CANDIDATE_DTYPE), 1)
        assert e.value.code == lib.LPF_E_STALE
        for T in range(3, 19):
            s.poll(timeout_ms=60000)


def test_truncation_reports_true_count(lib):
    spec = synth.spec_aartfaac(H=128, W=128, n_sources=30, n_pulses=0, n_frames=50)
    st = synth.SyntheticStream(spec, seed=8)
    with _open(lib, spec) as full, _open(lib, spec, cand_cap=100) as small:
        for T in range(49):
            f = torch.from_numpy(st.frame(T)).cuda()
            full.push(f, T)
            small.push(f, T)
            _, c_full, n_full, tr_full = full.poll(timeout_ms=60000)
            _, c_small, n_small, tr_small = small.poll(timeout_ms=60000)
            assert n_small == n_full and not tr_full
            assert tr_small == (n_full > 100)
            assert len(c_small) == min(100, n_full)
            assert_sorted_unique(c_small)
            assert set(map(tuple, c_small[["dm_idx", "y", "x"]].tolist())) <= \
                set(map(tuple, c_full[["dm_idx", "y", "x"]].tolist()))
    # poll with a small host cap
    with _open(lib, spec) as s:
        for T in range(48):
            _push(s, st, T)
            s.poll(timeout_ms=60000)
        _push(s, st, 48)
        _, c, n, tr = s.poll(cap=7, timeout_ms=60000)
        assert tr and len(c) == 7 and n > 7


def test_empty_and_constant_frames(lib):
    spec = synth.spec_tiny()
    with _open(lib, spec) as s:
        for T in range(20):
            s.push(torch.full((spec.F, spec.H, spec.W), 3.0, device="cuda"), T)
            _, c, n, _ = s.poll(timeout_ms=60000)
            assert n == 0 and len(c) == 0
        st = s.stats()
        assert np.all(st[:, 0] == 0) and np.all(st[:, 1] == 0)     # no valid pixel: S = 0


def test_deterministic_repeat(lib):
    spec = synth.spec_aartfaac(H=192, W=160, n_sources=60, n_frames=52)
    st = synth.SyntheticStream(spec, seed=12)
    outs = []
    for _ in range(2):
        with _open(lib, spec) as s:
            for T in range(50):
                _push(s, st, T)
                _, c, _, _ = s.poll(timeout_ms=60000)
            outs.append((c.tobytes(), s.stats().tobytes()))
    assert outs[0] == outs[1]


def test_host_push_matches_device_push(lib):
    spec = synth.spec_tiny()
    st = synth.SyntheticStream(spec, seed=13)
    with _open(lib, spec) as a, _open(lib, spec) as b:
        for T in range(20):
            fr = st.frame(T)
            a.push(torch.from_numpy(fr).cuda(), T)
            b.push_host(torch.from_numpy(fr).pin_memory(), T)
            ca = a.poll(timeout_ms=60000)[1]
            cb = b.poll(timeout_ms=60000)[1]
            assert ca.tobytes() == cb.tobytes()


def test_crossing_list_overflow_resolves_every_crossing(lib):
    """kappa = 0.5: about a third of all pixels of every delay row cross the
    threshold, more than the crossing list holds (max(cand_cap, rows x pixels /
    32)); the overflowing warps resolve their crossings inside the filter and
    the candidates and their count still match the oracle exactly."""
    spec = synth.spec_aartfaac(H=320, W=320, dm_grid=np.arange(64, dtype=np.float64), depth=16,
                               box_r=7, kappa=0.5, n_sources=10, n_pulses=0, n_frames=20)
    st = synth.SyntheticStream(spec, seed=21)
    fa = cached_frames(st)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    T = int(delays.max()) + 2
    with _open(lib, spec) as s:
        for t in range(T + 1):
            _push(s, st, t)
            _, c, n, trunc = s.poll(timeout_ms=60000)
        assert not trunc and n == len(c)
        assert_sorted_unique(c)
        n_rows = s.info()["n_distinct"]
        xcap = max(1 << 20, n_rows * spec.H * spec.W // 32)
        _, _, maps = O.search_push(fa, T, delays, spec.box_r, spec.kappa, keep_maps=True)
        rows = {}
        for d in range(len(delays)):
            rows.setdefault(tuple(delays[d]), d)
        crossings = sum(int((maps[d]["snr"] > spec.kappa).sum()) for d in rows.values())
        assert crossings > xcap, (crossings, xcap)        # the overflow path ran
        res = compare_push(c, fa, T, delays, spec.box_r, spec.kappa, gpu_stats=s.stats())
        assert res["matched"] > 100000
