"""Seeded synthetic sky-image streams for the dispersed-transient search.

This module is the one input source shared by the FP64 oracle and the CUDA
path.  It draws noise and paints steady sources and dispersed pulses; it holds
none of the search's arithmetic (no delay table, no shift-sum, no filter).

Every frame is a pure function of (spec, seed, t): the noise of frame t comes
from a Philox counter-based generator keyed by (seed, t), so any frame can be
regenerated on its own, in any order, by either side.

Content model (stand-in for AARTFAAC data, which is not available):
  * i.i.d. N(0, 1) noise per pixel, subband and frame;
  * an optional smooth 2-D cosine background (same in every subband/frame);
  * steady point sources with a Gaussian point-spread function (flat spectrum);
  * dispersed pulses following the paper's simulation recipe (Sec. 3.2):
    a Gaussian profile f(t) = exp(-((t - t_nu)/w)^2) whose arrival time in
    subband nu is t_nu = t0 + C * DM * (nu^-2 - nu_ref^-2) (continuous time,
    not rounded), scaled by A * (nu / nu_ref)^alpha.  Pulses are unresolved:
    they are painted on a single pixel;
  * optional broadband RFI stripes (a full image row or column at fixed
    amplitude in every subband of one frame).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

SUBBAND_MHZ = 0.1953125          # LOFAR subband width (195.3125 kHz)
# Cold-plasma dispersion constant of the injected-pulse physics, s MHz^2 cm^3/pc.
SIM_DISPERSION_S = 4.148808e3


def subband_centres(lows_mhz, n_per_group: int, width: float = SUBBAND_MHZ) -> np.ndarray:
    """Centre frequencies of contiguous subband groups starting at each lower edge."""
    out = []
    for lo in lows_mhz:
        out.extend(lo + (i + 0.5) * width for i in range(n_per_group))
    return np.asarray(out, dtype=np.float64)


@dataclass
class Pulse:
    y: int
    x: int
    t0: float        # arrival frame at the highest frequency
    dm: float
    width: float     # w of exp(-((t - t_nu)/w)^2), in frames
    alpha: float     # spectral index
    amp: float       # peak amplitude A at nu_ref, in noise sigma


@dataclass
class StreamSpec:
    name: str
    H: int
    W: int
    freqs_mhz: np.ndarray
    dm_grid: np.ndarray
    depth: int
    n_frames: int
    box_r: int
    kappa: float
    cadence_s: float = 1.0
    gradient_amp: float = 0.0
    n_sources: int = 0
    source_flux: Tuple[float, float] = (20.0, 20.0)   # log-uniform range, sigma
    psf_sigma: float = 1.5
    n_pulses: int = 0
    pulse_dm: Tuple[float, float] = (7.0, 7.0)
    pulse_width: Tuple[float, float] = (1.0, 1.0)
    pulse_alpha: Tuple[float, float] = (0.0, 0.0)
    pulse_peak: Optional[Tuple[float, float]] = (8.0, 8.0)     # peak amplitude, or
    pulse_fluence: Optional[Tuple[float, float]] = None        # fluence A*w*sqrt(pi)
    rfi_fraction: float = 0.0
    rfi_amp: float = 10.0
    dtype: str = "fp32"

    @property
    def F(self) -> int:
        return len(self.freqs_mhz)

    @property
    def n_dm(self) -> int:
        return len(self.dm_grid)


class SyntheticStream:
    """Deterministic frame source: ``frame(t)`` -> float32 [F, H, W]."""

    def __init__(self, spec: StreamSpec, seed: int = 1, pulses: Optional[List[Pulse]] = None):
        self.spec = spec
        self.seed = int(seed)
        rng = np.random.Generator(np.random.Philox(key=[self.seed, 0xC0FFEE]))
        H, W = spec.H, spec.W
        # steady sky: gradient + Gaussian-PSF point sources (identical in every subband)
        sky = np.zeros((H, W), np.float64)
        if spec.gradient_amp:
            py, px = rng.uniform(0, 2 * np.pi, 2)
            yy = np.cos(np.pi * np.arange(H) / H + py)
            xx = np.cos(np.pi * np.arange(W) / W + px)
            sky += spec.gradient_amp * yy[:, None] * xx[None, :]
        self.sources = []
        if spec.n_sources:
            lo, hi = spec.source_flux
            sy = rng.integers(4, H - 4, spec.n_sources)
            sx = rng.integers(4, W - 4, spec.n_sources)
            flux = np.exp(rng.uniform(np.log(lo), np.log(hi), spec.n_sources))
            rad = int(np.ceil(5 * spec.psf_sigma))
            oy, ox = np.mgrid[-rad:rad + 1, -rad:rad + 1]
            psf = np.exp(-(oy ** 2 + ox ** 2) / (2 * spec.psf_sigma ** 2))
            for y, x, s in zip(sy, sx, flux):
                y0, y1 = max(y - rad, 0), min(y + rad + 1, H)
                x0, x1 = max(x - rad, 0), min(x + rad + 1, W)
                sky[y0:y1, x0:x1] += s * psf[y0 - y + rad:y1 - y + rad, x0 - x + rad:x1 - x + rad]
                self.sources.append((int(y), int(x), float(s)))
        self.sky = sky.astype(np.float32)
        # dispersed pulses
        if pulses is None:
            pulses = []
            for _ in range(spec.n_pulses):
                w = float(rng.uniform(*spec.pulse_width))
                if spec.pulse_fluence is not None:
                    amp = float(rng.uniform(*spec.pulse_fluence)) / (w * np.sqrt(np.pi))
                else:
                    amp = float(rng.uniform(*spec.pulse_peak))
                dm = float(rng.uniform(*spec.pulse_dm))
                # keep the whole sweep inside the stream
                sweep = self._arrival_offsets(dm).max()
                t_lo = 2.0 + 3 * w
                t_hi = max(t_lo, spec.n_frames - 2 - sweep - 3 * w)
                pulses.append(Pulse(int(rng.integers(2, H - 2)), int(rng.integers(2, W - 2)),
                                    float(rng.uniform(t_lo, t_hi)), dm, w,
                                    float(rng.uniform(*spec.pulse_alpha)), amp))
        self.pulses = pulses
        # RFI stripes: a deterministic subset of frames
        self.rfi = {}
        if spec.rfi_fraction > 0:
            n = max(1, int(round(spec.rfi_fraction * spec.n_frames)))
            ts = rng.choice(spec.n_frames, n, replace=False)
            for t in ts:
                horizontal = bool(rng.integers(0, 2))
                pos = int(rng.integers(0, H if horizontal else W))
                self.rfi[int(t)] = (horizontal, pos)

    def _arrival_offsets(self, dm: float) -> np.ndarray:
        """Continuous arrival offsets (frames) of the injected pulse per subband."""
        f = self.spec.freqs_mhz
        ref = f.max()
        return SIM_DISPERSION_S * dm * (f ** -2.0 - ref ** -2.0) / self.spec.cadence_s

    def noise(self, t: int) -> np.ndarray:
        sp = self.spec
        g = np.random.Generator(np.random.Philox(key=[self.seed, 1 + int(t)]))
        return g.standard_normal((sp.F, sp.H, sp.W), dtype=np.float32)

    def frame(self, t: int) -> np.ndarray:
        """float32 [F, H, W] frame at integer time t (t >= 0)."""
        sp = self.spec
        x = self.noise(t)
        x += self.sky[None]
        f = sp.freqs_mhz
        ref = f.max()
        for p in self.pulses:
            tnu = p.t0 + self._arrival_offsets(p.dm)
            prof = np.exp(-((t - tnu) / p.width) ** 2)
            prof[np.abs(t - tnu) > 6 * p.width] = 0.0
            x[:, p.y, p.x] += (p.amp * (f / ref) ** p.alpha * prof).astype(np.float32)
        if int(t) in self.rfi:
            horizontal, pos = self.rfi[int(t)]
            if horizontal:
                x[:, pos, :] += sp.rfi_amp
            else:
                x[:, :, pos] += sp.rfi_amp
        return x


# --------------------------------------------------------------------------
# The workloads: tiny, AARTFAAC-shaped, precision, serving mix, stress.
# --------------------------------------------------------------------------
AARTFAAC_BANDS = subband_centres([57.6, 61.2], 8)     # 16 subbands in two groups


def spec_tiny(**kw) -> StreamSpec:
    """64x64 px, 8 subbands from 58.0 MHz, DM 0..15, depth 16, 32 frames."""
    d = dict(name="tiny", H=64, W=64, freqs_mhz=subband_centres([58.0], 8),
             dm_grid=np.arange(16, dtype=np.float64), depth=16, n_frames=32, box_r=7,
             kappa=6.0, n_sources=3, source_flux=(20.0, 20.0), psf_sigma=1.5, n_pulses=1,
             pulse_dm=(7.0, 7.0), pulse_width=(1.0, 1.0), pulse_peak=(8.0, 8.0))
    d.update(kw)
    return StreamSpec(**d)


def spec_aartfaac(**kw) -> StreamSpec:
    """1024x1024 px, 16 subbands in two groups, DM 0..250 step 1, depth 48."""
    d = dict(name="aartfaac", H=1024, W=1024, freqs_mhz=AARTFAAC_BANDS.copy(),
             dm_grid=np.arange(251, dtype=np.float64), depth=48, n_frames=600, box_r=15,
             kappa=6.0, gradient_amp=3.0, n_sources=500, source_flux=(5.0, 500.0),
             psf_sigma=1.5, n_pulses=20, pulse_dm=(5.0, 240.0), pulse_width=(1.0, 4.0),
             pulse_alpha=(-2.0, 2.0), pulse_peak=None, pulse_fluence=(6.0, 30.0))
    d.update(kw)
    return StreamSpec(**d)


def spec_precision(dtype: str = "fp16", **kw) -> StreamSpec:
    """2048x2048 px, AARTFAAC bands, DM 0..250 step 0.5 (501 trials), depth 48, 300 frames."""
    d = dict(name="precision-" + dtype, H=2048, W=2048, freqs_mhz=AARTFAAC_BANDS.copy(),
             dm_grid=np.arange(501, dtype=np.float64) * 0.5, depth=48, n_frames=300, box_r=15,
             kappa=6.0, gradient_amp=3.0, n_sources=500, source_flux=(5.0, 500.0),
             psf_sigma=1.5, n_pulses=40, pulse_dm=(5.0, 240.0), pulse_width=(1.0, 4.0),
             pulse_alpha=(-2.0, 2.0), pulse_peak=None, pulse_fluence=(6.0, 30.0), dtype=dtype)
    d.update(kw)
    return StreamSpec(**d)


def spec_serving_mix() -> List[StreamSpec]:
    """Four concurrent FP16 streams of different sizes and DM grids (content as the tiny stream)."""
    common = dict(kappa=6.0, n_sources=3, source_flux=(20.0, 20.0), psf_sigma=1.5, n_pulses=1,
                  pulse_dm=(7.0, 7.0), pulse_width=(1.0, 1.0), pulse_peak=(8.0, 8.0),
                  n_frames=600, dtype="fp16")
    return [
        StreamSpec(name="mix-2048", H=2048, W=2048, freqs_mhz=AARTFAAC_BANDS.copy(),
                   dm_grid=np.arange(501, dtype=np.float64) * 0.5, depth=48, box_r=15, **common),
        StreamSpec(name="mix-1024", H=1024, W=1024, freqs_mhz=AARTFAAC_BANDS.copy(),
                   dm_grid=np.arange(251, dtype=np.float64), depth=48, box_r=15, **common),
        StreamSpec(name="mix-512a", H=512, W=512, freqs_mhz=subband_centres([58.0], 8),
                   dm_grid=np.arange(128, dtype=np.float64), depth=8, box_r=7, **common),
        StreamSpec(name="mix-512b", H=512, W=512, freqs_mhz=subband_centres([58.0], 8),
                   dm_grid=np.arange(128, dtype=np.float64), depth=8, box_r=7, **common),
    ]


def spec_stress(depth: int = 114, **kw) -> StreamSpec:
    """2048x2048 px, 32 subbands from 57.6 MHz, DM 0..500 step 0.5 (1001 trials), FP16."""
    d = dict(name="stress", H=2048, W=2048, freqs_mhz=subband_centres([57.6], 32),
             dm_grid=np.arange(1001, dtype=np.float64) * 0.5, depth=depth, n_frames=600,
             box_r=15, kappa=6.0, gradient_amp=3.0, n_sources=0, source_flux=(5.0, 500.0),
             psf_sigma=1.5, n_pulses=200, pulse_dm=(5.0, 480.0), pulse_width=(1.0, 4.0),
             pulse_alpha=(-2.0, 2.0), pulse_peak=None, pulse_fluence=(6.0, 30.0),
             rfi_fraction=0.01, rfi_amp=10.0, dtype="fp16")
    d.update(kw)
    return StreamSpec(**d)


def cnn_params(seed: int = 3) -> np.ndarray:
    """Fixed random weights of the parameter-inference network, float32, in the
    order conv1.w [16][1][3][3], conv1.b [16], conv2.w [32][16][3][3], conv2.b [32],
    conv3.w [64][32][3][3], conv3.b [64], head.w [5][64], head.b [5]: normal
    draws scaled by sqrt(2 / fan_in) for the convolutions, 1/8 for the head, and
    0.1 for the biases (seeded)."""
    rng = np.random.Generator(np.random.Philox(key=[int(seed), 0xC44]))
    parts = []
    for shape, scale in [((16, 1, 3, 3), np.sqrt(2.0 / 9)), ((16,), 0.1),
                         ((32, 16, 3, 3), np.sqrt(2.0 / 144)), ((32,), 0.1),
                         ((64, 32, 3, 3), np.sqrt(2.0 / 288)), ((64,), 0.1),
                         ((5, 64), 0.125), ((5,), 0.1)]:
        parts.append((rng.standard_normal(shape) * scale).astype(np.float32).ravel())
    return np.concatenate(parts)
