"""FP64 CPU oracle of the parameter-inference network (Sec. 2.3).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this module.  It imports
nothing from the product, and the product never imports it.

The paper fixes the network's form, not its layers (Sec. 2.3): convolutions
whose hidden states are h = phi(x^T w + b) with the Leaky ReLU phi(h) = h for
h >= 0 and alpha h otherwise (alpha a small positive value), a final linear
layer without activation, and an output (mu, L) with L lower triangular with a
positive diagonal, the Cholesky factor of the covariance Sigma = L L^T of
p(theta | x).  Readings (no architecture or weights are given; the network is
measured for throughput, with fixed random weights):

  * input: one dynamic spectrum x [F][Tw] (subbands x frames) as one channel;
  * conv1: 3x3, 1 -> 16 channels, zero padding 1, bias, Leaky ReLU, then the
    mean of each 2x2 block                                  -> [16][F/2][Tw/2]
  * conv2: 3x3, 16 -> 32, the same                         -> [32][F/4][Tw/4]
  * conv3: 3x3, 32 -> 64, bias, Leaky ReLU, mean over all pixels    -> [64]
  * head: linear 64 -> 5; mu = (z0, z1), L = [[exp z2, 0], [z3, exp z4]]
    (theta two-dimensional, e.g. DM and fluence); alpha = 0.01;
  * storage: the network's weights of conv2 and conv3 and its activations
    after conv1 and conv2 are BF16 (the tensor-core operand type of the CUDA
    path), arithmetic FP32 there; this oracle rounds the same values to BF16
    at the same points and computes in FP64.

A convolution here is the cross-correlation of the CNN literature:
out[o][y][x] = b[o] + sum_{i,ky,kx} w[o][i][ky][kx] in[i][y+ky-1][x+kx-1].

Parameter vector (float32, the layout lpf_cnn_open takes):
  conv1.w [16][1][3][3], conv1.b [16], conv2.w [32][16][3][3], conv2.b [32],
  conv3.w [64][32][3][3], conv3.b [64], head.w [5][64], head.b [5].
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

ALPHA = 0.01
LAYERS: List[Tuple[str, Tuple[int, ...]]] = [
    ("conv1.w", (16, 1, 3, 3)), ("conv1.b", (16,)),
    ("conv2.w", (32, 16, 3, 3)), ("conv2.b", (32,)),
    ("conv3.w", (64, 32, 3, 3)), ("conv3.b", (64,)),
    ("head.w", (5, 64)), ("head.b", (5,)),
]


def param_count() -> int:
    return sum(int(np.prod(s)) for _, s in LAYERS)


def unpack(params: np.ndarray) -> Dict[str, np.ndarray]:
    """The flat parameter vector as named FP64 arrays."""
    out, o = {}, 0
    p = np.asarray(params, dtype=np.float64).ravel()
    for name, shape in LAYERS:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    assert o == p.size, "parameter vector has the wrong length"
    return out


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to BF16 (nearest, ties to even), returned as float64."""
    import torch  # plain CPU conversion
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def leaky_relu(h: np.ndarray, alpha: float = ALPHA) -> np.ndarray:
    return np.where(h >= 0.0, h, alpha * h)


def conv3x3(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x [C][H][W], w [O][C][3][3], b [O] -> [O][H][W], zero padding 1."""
    C, H, W = x.shape
    pad = np.zeros((C, H + 2, W + 2))
    pad[:, 1:-1, 1:-1] = x
    out = np.empty((w.shape[0], H, W))
    for o in range(w.shape[0]):
        acc = np.full((H, W), b[o], dtype=np.float64)
        for i in range(C):
            for ky in range(3):
                for kx in range(3):
                    acc = acc + w[o, i, ky, kx] * pad[i, ky:ky + H, kx:kx + W]
        out[o] = acc
    return out


def pool2x2(x: np.ndarray) -> np.ndarray:
    """Mean of each 2x2 block: [C][H][W] -> [C][H/2][W/2]."""
    C, H, W = x.shape
    return x.reshape(C, H // 2, 2, W // 2, 2).mean(axis=(2, 4))


def head(z: np.ndarray) -> np.ndarray:
    """Linear output z [5] -> (mu0, mu1, L00, L10, L11): the diagonal of L is exp of
    its outputs, so it is positive and L a Cholesky factor."""
    return np.array([z[0], z[1], np.exp(z[2]), z[3], np.exp(z[4])])


def forward_one(x: np.ndarray, p: Dict[str, np.ndarray]) -> np.ndarray:
    """One spectrum x [F][Tw] -> [5]."""
    h = pool2x2(leaky_relu(conv3x3(np.asarray(x, np.float64)[None], p["conv1.w"], p["conv1.b"])))
    h = bf16(h)
    h = pool2x2(leaky_relu(conv3x3(h, bf16(p["conv2.w"]), p["conv2.b"])))
    h = bf16(h)
    h = leaky_relu(conv3x3(h, bf16(p["conv3.w"]), p["conv3.b"])).mean(axis=(1, 2))
    return head(p["head.w"] @ h + p["head.b"])


def forward(xs: np.ndarray, params: np.ndarray) -> np.ndarray:
    """Batch [n][F][Tw] -> [n][5] (mu0, mu1, L00, L10, L11)."""
    p = unpack(params)
    return np.stack([forward_one(x, p) for x in np.asarray(xs)]) if len(xs) else np.zeros((0, 5))


def covariance(out: np.ndarray) -> np.ndarray:
    """Sigma = L L^T of each output row [n][5] -> [n][2][2]."""
    L = np.zeros((len(out), 2, 2))
    L[:, 0, 0], L[:, 1, 0], L[:, 1, 1] = out[:, 2], out[:, 3], out[:, 4]
    return L @ np.transpose(L, (0, 2, 1))
