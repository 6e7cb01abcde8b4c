"""Quality control on the GPU (App. A) against the FP64 oracle, through the C ABI:
the bands each frame discards, their scores, and the candidates of the search on
the imputed frames."""
import numpy as np
import pytest

import synth
from oracle import lpf_oracle as O
from tests.parity import assert_sorted_unique, compare_storage

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

QC = dict(qc_z=5.0, qc_zeta=12.0, qc_min_frames=20)


def corrupted_frames(st, n):
    """The synthetic stream with planted corruptions: a band offset (frame 30,
    band 5), an RFI spike (frame 34, band 9) and both at once (frame 36)."""
    out = []
    for t in range(n):
        x = st.frame(t).astype(np.float32)
        if t in (30, 36):
            x[5] += 3.0
        if t in (34, 36):
            x[9, 40, 50] += 200.0
        out.append(x)
    return out


@pytest.mark.parametrize("dtype", ["fp32", "fp16"])
def test_quality_control_matches_oracle(lib, dtype):
    spec = synth.spec_aartfaac(H=128, W=128, dm_grid=np.arange(32, dtype=np.float64), depth=8, box_r=7,
                               n_sources=20, n_pulses=3, n_frames=48)
    st = synth.SyntheticStream(spec, seed=12)
    frames = corrupted_frames(st, 44)
    state = O.QCState(spec.F, spec.H, spec.W)
    qc_out, disc_ref, z_ref = [], [], []
    for x in frames:
        out, disc, z, _ = O.qc_frame(x.astype(np.float64), state, QC["qc_z"], QC["qc_zeta"], QC["qc_min_frames"])
        qc_out.append(O.storage_round(out, dtype))
        disc_ref.append(disc)
        z_ref.append(z)
    assert disc_ref[30][5] and disc_ref[34][9] and disc_ref[36][5] and disc_ref[36][9]
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    fa = lambda t: qc_out[t]
    ra = None
    if dtype != "fp32":
        ra = lambda t: O.storage_round(O.residual_frame(qc_out[t], spec.box_r), dtype)
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, cadence_s=spec.cadence_s,
                    kappa=spec.kappa, box_r=spec.box_r, dtype=dtype, qc=True, **QC) as s:
        for T, x in enumerate(frames):
            s.push(torch.from_numpy(x).cuda(), T)
            Tp, c, n, _ = s.poll(timeout_ms=60000)
            Tq, disc, z = s.qc()
            assert Tp == T and Tq == T
            assert np.array_equal(disc, disc_ref[T]), (T, disc, disc_ref[T])
            fin = np.isfinite(z_ref[T])
            assert np.allclose(z[fin], z_ref[T][fin], rtol=1e-4, atol=1e-3), T
            if T in (33, 37, 43):               # windows holding the imputed bands
                assert_sorted_unique(c)
                compare_storage(c, fa, T, delays, spec.box_r, spec.kappa, dtype, gpu_stats=s.stats(), res_at=ra)


def test_quality_control_off_leaves_frames_untouched(lib):
    """qc = 0 (the default): the same candidates as a stream without the option, and
    no quality-control record."""
    spec = synth.spec_tiny()
    st = synth.SyntheticStream(spec, seed=2)
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                    box_r=spec.box_r) as a, \
         lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                    box_r=spec.box_r, qc=False, qc_z=1.0) as b:
        for T in range(20):
            f = torch.from_numpy(st.frame(T)).cuda()
            a.push(f, T)
            b.push(f, T)
            assert a.poll(timeout_ms=60000)[1].tobytes() == b.poll(timeout_ms=60000)[1].tobytes()
        with pytest.raises(lib.LpfError) as e:
            b.qc()
        assert e.value.code == lib.LPF_E_NODATA
