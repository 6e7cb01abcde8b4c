"""Pins of the FP64 oracle of the parameter-inference network (Sec. 2.3) against
facts independent of its own code: a library cross-correlation, the closed form of
a delta's response, hand-computed means and activations, the Cholesky-factor
property of the head, and planted mistakes that each fail a pin."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import synth
from oracle import cnn_oracle as C


def lib_conv3x3(x, w, b):
    """The same layer through scipy's 2-D cross-correlation (zero fill, 'same')."""
    out = np.empty((w.shape[0],) + x.shape[1:])
    for o in range(w.shape[0]):
        acc = np.full(x.shape[1:], b[o], dtype=np.float64)
        for i in range(x.shape[0]):
            acc += correlate2d(x[i], w[o, i], mode="same", boundary="fill", fillvalue=0.0)
        out[o] = acc
    return out


def test_conv_matches_library_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 8, 12))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    np.testing.assert_allclose(C.conv3x3(x, w, b), lib_conv3x3(x, w, b), rtol=1e-12, atol=1e-12)


def test_conv_of_a_delta_is_the_rotated_kernel():
    """Cross-correlation: a unit impulse at (y0, x0) gives out[y0 - dy][x0 - dx] = w[1 + dy][1 + dx]."""
    x = np.zeros((1, 7, 9))
    x[0, 3, 4] = 1.0
    w = np.arange(9, dtype=np.float64).reshape(1, 1, 3, 3) + 1.0
    out = C.conv3x3(x, w, np.zeros(1))[0]
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            assert out[3 - dy, 4 - dx] == w[0, 0, 1 + dy, 1 + dx]
    assert np.count_nonzero(out) == 9


def test_conv_is_linear_and_padding_is_zero():
    rng = np.random.default_rng(2)
    x1, x2 = rng.standard_normal((2, 2, 5, 6))
    w = rng.standard_normal((3, 2, 3, 3))
    z = np.zeros(3)
    np.testing.assert_allclose(C.conv3x3(2.0 * x1 - x2, w, z), 2.0 * C.conv3x3(x1, w, z) - C.conv3x3(x2, w, z),
                               atol=1e-12)
    # a constant image: the corner output sums the 2x2 of taps inside the image
    ones = np.ones((1, 4, 4))
    k = np.arange(9, dtype=np.float64).reshape(1, 1, 3, 3)
    out = C.conv3x3(ones, k, np.zeros(1))[0]
    assert out[0, 0] == k[0, 0, 1:, 1:].sum() and out[1, 1] == k.sum()


def test_pool_leaky_relu_and_bf16():
    x = np.arange(16, dtype=np.float64).reshape(1, 4, 4)
    np.testing.assert_array_equal(C.pool2x2(x)[0], [[2.5, 4.5], [10.5, 12.5]])
    np.testing.assert_array_equal(C.leaky_relu(np.array([-2.0, 0.0, 3.0])), [-0.02, 0.0, 3.0])
    # BF16 keeps 8 significant bits, ties to even
    assert C.bf16(np.array([1.0 + 2.0 ** -9]))[0] == 1.0
    assert C.bf16(np.array([1.0 + 3 * 2.0 ** -9]))[0] == 1.0 + 2.0 ** -7
    assert C.bf16(np.array([257.0]))[0] == 256.0


def test_head_is_a_cholesky_factor():
    out = np.array([C.head(np.array([0.3, -1.0, 0.0, 0.0, 0.0])), C.head(np.array([0.0, 0.0, -2.0, 5.0, 1.5]))])
    np.testing.assert_array_equal(out[0], [0.3, -1.0, 1.0, 0.0, 1.0])        # L = I
    sig = C.covariance(out)
    np.testing.assert_allclose(sig[0], np.eye(2))
    for s in sig:
        assert np.allclose(s, s.T) and np.all(np.linalg.eigvalsh(s) > 0)
        L = np.linalg.cholesky(s)
        assert np.all(np.diag(L) > 0)
    np.testing.assert_allclose(np.linalg.cholesky(sig[1]), [[np.exp(-2.0), 0.0], [5.0, np.exp(1.5)]])


def test_forward_shapes_and_layer_composition():
    """forward() equals the layers composed by hand with the library correlation."""
    p = synth.cnn_params(5)
    P = C.unpack(p)
    x = np.random.default_rng(3).standard_normal((8, 16))
    h = C.pool2x2(C.leaky_relu(lib_conv3x3(x[None], P["conv1.w"], P["conv1.b"])))
    h = C.bf16(h)
    h = C.pool2x2(C.leaky_relu(lib_conv3x3(h, C.bf16(P["conv2.w"]), P["conv2.b"])))
    h = C.bf16(h)
    f = C.leaky_relu(lib_conv3x3(h, C.bf16(P["conv3.w"]), P["conv3.b"])).mean(axis=(1, 2))
    z = P["head.w"] @ f + P["head.b"]
    want = np.array([z[0], z[1], np.exp(z[2]), z[3], np.exp(z[4])])
    np.testing.assert_allclose(C.forward(x[None], p)[0], want, rtol=1e-12, atol=1e-12)
    assert p.size == C.param_count() == 23621


@pytest.mark.parametrize("mistake", ["convolution", "no_pad_zero", "pool_max"])
def test_planted_mistakes_fail_a_pin(mistake):
    """Plausible slips in the layer code: a true convolution (flipped kernel), edge
    replication instead of zero padding, a max instead of a mean pool."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 6, 6))
    w = rng.standard_normal((2, 2, 3, 3))
    b = np.zeros(2)

    def bad_conv(x, w, b):
        if mistake == "convolution":
            return C.conv3x3(x, w[:, :, ::-1, ::-1], b)
        if mistake == "no_pad_zero":
            pad = np.pad(x, ((0, 0), (1, 1), (1, 1)), mode="edge")
            out = np.zeros((w.shape[0],) + x.shape[1:])
            for o in range(w.shape[0]):
                for i in range(x.shape[0]):
                    for ky in range(3):
                        for kx in range(3):
                            out[o] += w[o, i, ky, kx] * pad[i, ky:ky + x.shape[1], kx:kx + x.shape[2]]
            return out
        return C.conv3x3(x, w, b)

    if mistake == "pool_max":
        y = np.arange(16, dtype=np.float64).reshape(1, 4, 4)
        pooled = y.reshape(1, 2, 2, 2, 2).max(axis=(2, 4))
        assert not np.array_equal(pooled[0], [[2.5, 4.5], [10.5, 12.5]])
    else:
        assert not np.allclose(bad_conv(x, w, b), lib_conv3x3(x, w, b))
