"""The parameter-inference network (Sec. 2.3) on the GPU (tcgen05 implicit-GEMM
convolutions), through the C ABI, against the FP64 oracle that rounds weights
and activations to BF16 at the same points.

Tolerance: the network's FP32 sums and the oracle's FP64 ones can round an
activation to neighbouring BF16 values (a change of 2^-8 relative in one of
thousands of activations, averaged by the pooling); the outputs agree within
2e-3 absolute plus 2e-3 relative."""
import numpy as np
import pytest

import synth
from oracle import cnn_oracle as C

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RTOL = ATOL = 2e-3


def spectra(n, F, Tw, seed):
    """Noise plus, per spectrum, a dispersed sweep (a slanted track of a few sigma)
    and sometimes a steady bright subband row."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, F, Tw)).astype(np.float32)
    for i in range(n):
        t0, slope, amp = rng.integers(0, Tw // 2), rng.uniform(0.0, 2.0), rng.uniform(2.0, 12.0)
        for f in range(F):
            t = int(t0 + slope * (F - 1 - f))
            if t < Tw:
                x[i, f, t] += amp
        if i % 3 == 0:
            x[i, rng.integers(0, F)] += rng.uniform(1.0, 5.0)
    return x


@pytest.mark.parametrize("F,Tw,n", [(32, 64, 37), (32, 64, 1), (16, 64, 5), (8, 16, 21)])
def test_cnn_matches_oracle(lib, F, Tw, n):
    params = synth.cnn_params(11)
    x = spectra(n, F, Tw, seed=F + Tw + n)
    ref = C.forward(x.astype(np.float64), params)
    with lib.Cnn(F, Tw, params, max_batch=64) as net:
        got = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        # a second call on the same buffers gives the same outputs
        again = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, again)
    assert got.shape == (n, 5) and np.all(np.isfinite(got))
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=ATOL)
    assert np.all(got[:, 2] > 0) and np.all(got[:, 4] > 0)         # L has a positive diagonal
    assert np.ptp(ref[:, 0]) > 10 * ATOL or n == 1                  # the inputs move the outputs


def test_cnn_batch_spans_many_spectra_per_cta(lib):
    """700 spectra of 32 x 64: more than one spectrum per CTA of the one-kernel
    network (at most two CTAs per SM).  Sampled spectra from every position of the
    persistent loop against the oracle, a repeat bit-identical, and a spectrum's
    outputs independent of the batch it is in."""
    params = synth.cnn_params(7)
    n = 700
    x = spectra(n, 32, 64, seed=5)
    with lib.Cnn(32, 64, params, max_batch=n) as net:
        got = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        again = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
        part = net.forward(torch.from_numpy(x[290:330].copy()).cuda()).cpu().numpy()
    np.testing.assert_array_equal(got, again)
    np.testing.assert_array_equal(got[290:330], part)
    idx = [0, 1, 147, 148, 295, 296, 297, 443, 591, 592, 593, 699]
    ref = C.forward(x[idx].astype(np.float64), params)
    np.testing.assert_allclose(got[idx], ref, rtol=RTOL, atol=ATOL)
    assert np.all(np.isfinite(got))


def test_cnn_on_gathered_dynamic_spectra(lib):
    """The network as the consumer of the dynamic-spectrum gather: the candidates
    of a tiny stream, their 8 x 16 spectra gathered on the GPU, then the network."""
    spec = synth.spec_tiny(kappa=4.0)
    st = synth.SyntheticStream(spec, seed=21)
    params = synth.cnn_params(2)
    Tw = 16
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                    box_r=spec.box_r) as s:
        for T in range(20):
            s.push(torch.from_numpy(st.frame(T)).cuda(), T)
            _, cands, n, _ = s.poll(timeout_ms=60000)
        assert len(cands) > 3
        ds = s.dynspec(cands, Tw)                                   # [n][8][16] FP32 on the GPU
    with lib.Cnn(spec.F, Tw, params, max_batch=len(cands)) as net:
        got = net.forward(ds).cpu().numpy()
    ref = C.forward(ds.cpu().numpy().astype(np.float64), params)
    np.testing.assert_allclose(got, ref, rtol=RTOL, atol=ATOL)


def test_cnn_batch_limits(lib):
    params = synth.cnn_params(1)
    with lib.Cnn(8, 16, params, max_batch=4) as net:
        with pytest.raises(lib.LpfError):
            net.forward(torch.zeros((5, 8, 16), device="cuda"))
        out = net.forward(torch.zeros((0, 8, 16), device="cuda"))
        assert out.shape == (0, 5)
    # the one-kernel network copies each 32 x 64 spectrum in 16-byte pieces: a
    # misaligned batch is refused before any work is enqueued
    with lib.Cnn(32, 64, params, max_batch=2) as net:
        buf = torch.zeros(2 * 32 * 64 + 1, device="cuda")
        with pytest.raises(lib.LpfError):
            net.forward(buf[1:].view(2, 32, 64))
        assert np.all(np.isfinite(net.forward(buf[:-1].view(2, 32, 64)).cpu().numpy()))
