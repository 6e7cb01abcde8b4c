"""Serving loop: concurrent streams under an HBM budget (C++ worker, through the C ABI).

Each stream's candidates must be the same served alone, served in a mix of
four streams of different sizes and DM grids, and run directly on an
lpf_stream; streams that do not fit the budget wait and are admitted when
another closes.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def mix_specs():
    """The serving mix (FP16 storage) at a quarter of its image sizes."""
    out = []
    for sp in synth.spec_serving_mix():
        sp.H //= 4
        sp.W //= 4
        sp.n_frames = 60
        out.append(sp)
    return out


def kw(sp):
    return dict(kappa=sp.kappa, box_r=sp.box_r, dtype=sp.dtype, cadence_s=sp.cadence_s)


def direct_run(lib, sp, st, n):
    res = {}
    with lib.Stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **kw(sp)) as s:
        for T in range(n):
            s.push(torch.from_numpy(st.frame(T)).cuda(), T)
            Tp, c, _, _ = s.poll(timeout_ms=60000)
            res[Tp] = c.tobytes()
    return res


def serve(lib, specs, streams, n, budget, order_seed=0):
    """Submit n frames of every stream, interleaved in a seeded random order."""
    rng = np.random.default_rng(order_seed)
    out = {i: {} for i in range(len(specs))}
    lat = []
    with lib.Server(budget, max_streams=8) as srv:
        ids = [srv.open_stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **kw(sp)) for sp in specs]
        nxt = [0] * len(specs)
        while min(nxt) < n or any(len(out[i]) < n for i in range(len(specs))):
            live = [i for i in range(len(specs)) if nxt[i] < n]
            if live:
                i = int(rng.choice(live))
                if srv.submit(ids[i], streams[i].frame(nxt[i]), nxt[i]) == lib.LPF_OK:
                    nxt[i] += 1
                    continue
            # every stream busy or fully submitted: collect one result of the stream most behind
            i = min(range(len(specs)), key=lambda k: len(out[k]) - nxt[k])
            if len(out[i]) < nxt[i]:
                T, c, _, l = srv.fetch(ids[i], timeout_ms=120000)
                out[i][T] = c.tobytes()
                lat.append(l)
        st = srv.stats()
        for i in ids:
            srv.close_stream(i)
    return out, st, lat


def test_same_result_alone_in_mix_and_direct(lib):
    specs = mix_specs()
    streams = [synth.SyntheticStream(sp, seed=30 + i) for i, sp in enumerate(specs)]
    n = 52
    budget = 80 << 30
    alone = serve(lib, [specs[1]], [streams[1]], n, budget)[0][0]
    mix, stats, lat = serve(lib, specs, streams, n, budget, order_seed=5)
    assert mix[1] == alone
    for i, sp in enumerate(specs):
        direct = direct_run(lib, sp, streams[i], n)
        assert mix[i] == direct, sp.name
    assert stats["frames"] == 4 * n
    assert stats["p99_ms"] > 0 and stats["pixel_dm_per_s"] > 0
    assert any(len(np.frombuffer(v, dtype=lib.CANDIDATE_DTYPE)) for v in mix[0].values())


def test_admission_waits_for_budget(lib):
    specs = mix_specs()
    a, b, c = specs[1], specs[2], specs[3]
    fps = [lib.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **kw(sp)) for sp in (a, b, c)]
    budget = fps[0] + fps[1] + (1 << 20)           # c fits only after a or b leaves
    st_c = synth.SyntheticStream(c, seed=41)
    with lib.Server(budget, max_streams=4) as srv:
        ia = srv.open_stream(a.H, a.W, a.freqs_mhz, a.dm_grid, a.depth, **kw(a))
        ib = srv.open_stream(b.H, b.W, b.freqs_mhz, b.dm_grid, b.depth, **kw(b))
        ic = srv.open_stream(c.H, c.W, c.freqs_mhz, c.dm_grid, c.depth, **kw(c))
        import time
        t0 = time.time()
        while (srv.state(ia) != lib.SERVE_ACTIVE or srv.state(ib) != lib.SERVE_ACTIVE) and time.time() - t0 < 60:
            time.sleep(0.01)
        assert srv.state(ia) == lib.SERVE_ACTIVE and srv.state(ib) == lib.SERVE_ACTIVE
        # c queues frames while it waits for budget
        for T in range(3):
            assert srv.submit(ic, st_c.frame(T), T) == lib.LPF_OK
        time.sleep(0.2)
        assert srv.state(ic) == lib.SERVE_PENDING
        assert srv.stats()["used_bytes"] <= budget
        srv.close_stream(ia)
        got = {}
        for T in range(3):
            Tp, cands, _, _ = srv.fetch(ic, timeout_ms=120000)
            got[Tp] = cands.tobytes()
        assert srv.state(ic) == lib.SERVE_ACTIVE
        assert srv.state(ia) == lib.SERVE_CLOSED
    assert got == direct_run(lib, c, st_c, 3)


def test_stream_larger_than_budget_is_refused(lib):
    sp = mix_specs()[0]
    with lib.Server(1 << 20) as srv:
        with pytest.raises(lib.LpfError) as e:
            srv.open_stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **kw(sp))
        assert e.value.code == lib.LPF_E_BUDGET


def test_footprint_matches_allocation(lib):
    for sp in mix_specs()[:3]:
        fp = lib.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **kw(sp))
        with lib.Stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **kw(sp)) as s:
            assert s.info()["device_bytes"] == fp


def test_served_suppression_with_a_full_list_matches_direct(lib):
    """A stream with steady-source suppression and a 50-record candidate list,
    served and direct.  Frames that fit the list give the same records and count;
    which records an overflowed list holds is unspecified, so for those frames n_found
    is the number of sorted records returned.  The mask state does not depend on
    the list, so frames after an overflow agree again."""
    from tests.parity import assert_sorted_unique
    sp = synth.spec_tiny(kappa=4.0)
    st = synth.SyntheticStream(sp, seed=3)
    cap = 50
    opts = dict(kappa=sp.kappa, box_r=sp.box_r, suppress_steady=2, cand_cap=cap)
    n = 12
    direct = {}
    with lib.Stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **opts) as s:
        for T in range(n):
            s.push(torch.from_numpy(st.frame(T)).cuda(), T)
            Tp, c, nf, trunc = s.poll(timeout_ms=60000)
            direct[Tp] = (c.tobytes(), nf, trunc)
    flags = [v[2] for v in direct.values()]
    assert any(flags) and not all(flags)
    with lib.Server(8 << 30, max_streams=2) as srv:
        sid = srv.open_stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, **opts)
        for T in range(n):
            assert srv.submit(sid, st.frame(T), T) == lib.LPF_OK
            Tp, c, nf, _ = srv.fetch(sid, timeout_ms=60000)
            assert Tp == T
            if direct[T][2]:
                assert_sorted_unique(c)
                assert nf == len(c) <= cap, T
            else:
                assert (c.tobytes(), nf) == direct[T][:2], T
        srv.close_stream(sid)
