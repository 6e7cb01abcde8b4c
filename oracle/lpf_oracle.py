"""FP64 CPU oracle for the image-plane dispersed-transient search.

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
cpu_baseline / reference leg of bench.py may import this module.  The product
path (the CUDA library and its Python binding) never imports or calls it, and
this module imports nothing from the product.

Plain, slow, obviously correct NumPy float64 code, one function per step of the
method, each citing the passage of Ruhe et al. (arXiv 2103.15418) it follows:

  delay_table      Sec. 3.2, dispersion delay t_nu = t0 + C_DM DM (nu^-2 - nu0^-2)
  dedisperse       App. B.2, "perfect dedispersion": sum over subbands after the shift
  local_centre     Sec. 2.1.1, C := G * X with the uniform kernel, normalised (Z)
  local_spread     Sec. 2.1.1, S := G * (X - C)^2, square taken element-wise first
  snr_map          Sec. 2.1.1, threshold y = I(x > c + kappa sqrt(s)) written as S/N
  local_max_mask   Sec. 2.1.2, q = I(x = max over the (2k+1)^2 window), here k = 1
  detect           Sec. 2.1.2, p = q AND y
  frame_stats      mean / RMS of S/N over valid pixels (diagnostic noise level)
  dynspec          Sec. 2.2, flux measurement + backward fill from cached images
  search_push_residual  the same search with D - C as a shift-sum of per-subband
                   residuals X - C(X) (linearity of the local centre); reference
                   for rings that store those residuals in reduced precision
  subband_detect   Sec. 2.1.1-2.1.2 on every band image, (2k+1)^2 maximum (k = 3)
  clip_detect      Sec. 2.1.1 iterated: C and S re-estimated from the pixels not
                   yet flagged, until no new flag or the iteration limit; the
                   uniform box or the Gaussian kernel G(n, m, s) (kernel_sum)
  qc_band_scores   App. A, z = (b - median(b)) / MAD(b) of the band-image means
  QCState, qc_frame  App. A, per-pixel running mean / standard deviation
                   (Welford) and scores zeta; bands over either threshold are
                   imputed with zeros
  SteadyMask, suppress_steady  an opt-in reading of the steady-source removal
                   the paper leaves to association (Sec. 2.2) and the network
                   (Sec. 2.3): a pixel that was a candidate of a zero-delay trial
                   in each of the K most recent pushes is steady, and the
                   candidates of the other trials there are dropped

Readings where the paper is silent or garbled (Sec. 2.1.1-2.1.2, Sec. 3.2, App. A):
  * C_DM = 4.148808e3 s MHz^2 cm^3 / pc (the printed unit "ms" is garbled; with
    nu in MHz the delay is in seconds); nu_ref = the highest frequency, so every
    delay is >= 0; delays are rounded half up, floor(x + 0.5), in FP64.
  * The kernel is the square uniform box of radius r, truncated at the image
    edge and normalised by the number of in-image pixels (Z of Sec. 2.1.1).
    The Gaussian kernel G(n, m, s) (per-subband detector) has the same square
    (2r+1)^2 support (the window of Z's double sum) and is normalised by the
    sum of its weights over the in-image window pixels.
  * The spread is two-pass: (D - C)^2 uses C at each window pixel.
  * The local maximum is taken on the dedispersed image over the 3x3 window
    clipped to the image; ties count as maxima (x = max).
  * Strict threshold (snr > kappa); pixels with S = 0 are never candidates and
    carry snr = 0.
  * A candidate's t0 is its arrival frame at nu_ref; it is produced by the push
    of frame T = t0 + max_f delay[d][f].
  * Quality control (App. A): MAD is the median absolute deviation from the
    median (the text's expansion "mean absolute deviation" is garbled; the
    statistics are robust ones); both thresholds apply to |z| and |zeta|; the
    pixel scores use the running statistics before the current frame, with the
    sample standard deviation, once a band has min_frames frames folded in,
    and only where that deviation is positive; only kept band images are
    folded into the running statistics.

Functions with no independent pin: none (see tests/test_oracle_pins.py).
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import numpy as np

# Sec. 3.2: C_DM = e^2 pc / (8 pi^2 eps0 m_e c) * 1e-6, in s MHz^2 cm^3 / pc.
C_DM_S = 4.148808e3

FrameFn = Callable[[int], np.ndarray]   # t -> [F, H, W] float64


# --------------------------------------------------------------------- a1
def delay_table(freqs_mhz: Sequence[float], dm_grid: Sequence[float],
                cadence_s: float) -> np.ndarray:
    """Integer delay in frames of subband f for DM trial d (Sec. 3.2, t_nu equation).

    delay[d][f] = floor(C_DM * DM_d * (nu_f^-2 - nu_ref^-2) / cadence + 1/2),
    nu_ref = max_f nu_f.  Returned as int64 [n_dm, F].
    """
    freqs = [float(v) for v in freqs_mhz]
    ref = max(freqs)
    out = np.zeros((len(dm_grid), len(freqs)), dtype=np.int64)
    for d, dm in enumerate(dm_grid):
        for f, nu in enumerate(freqs):
            seconds = C_DM_S * float(dm) * (nu ** -2 - ref ** -2)
            out[d, f] = math.floor(seconds / cadence_s + 0.5)
    return out


def delay_fraction_margin(freqs_mhz, dm_grid, cadence_s) -> float:
    """Smallest distance of an unrounded delay (in frames) to a rounding tie (.5)."""
    freqs = np.asarray(freqs_mhz, np.float64)
    ref = freqs.max()
    x = C_DM_S * np.asarray(dm_grid, np.float64)[:, None] * (freqs[None] ** -2 - ref ** -2) / cadence_s
    return float(np.min(np.abs((x - np.floor(x)) - 0.5)))


# --------------------------------------------------------------------- a3
def dedisperse(frame_at: FrameFn, T: int, delays: np.ndarray, d: int) -> Tuple[int, np.ndarray]:
    """Shift-and-sum for DM trial d completed by frame T (App. B.2, un-normalised mean).

    D_d = sum_f X_f(t0 + delay[d][f]),  t0 = T - max_f delay[d][f].
    Returns (t0, D) with D float64 [H, W].
    """
    row = delays[d]
    t0 = T - int(row.max())
    D = None
    for f in range(len(row)):
        plane = np.asarray(frame_at(t0 + int(row[f]))[f], dtype=np.float64)
        D = plane.copy() if D is None else D + plane
    return t0, D


def abs_sum(frame_at: FrameFn, T: int, delays: np.ndarray, d: int) -> np.ndarray:
    """sum_f |X_f(t0 + delay[d][f])|: scale of the FP32 rounding error of D_d."""
    row = delays[d]
    t0 = T - int(row.max())
    acc = None
    for f in range(len(row)):
        plane = np.abs(np.asarray(frame_at(t0 + int(row[f]))[f], dtype=np.float64))
        acc = plane if acc is None else acc + plane
    return acc


# --------------------------------------------------------------------- a4 / a5
def window_sum_1d(a: np.ndarray, r: int, axis: int) -> np.ndarray:
    """sum_{k=-r..r} a[i+k] along one axis, terms outside the array omitted."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[axis]
    out = np.zeros_like(a)
    for k in range(-r, r + 1):
        dst = [slice(None)] * a.ndim
        src = [slice(None)] * a.ndim
        if k >= 0:
            dst[axis] = slice(0, max(n - k, 0))
            src[axis] = slice(k, n)
        else:
            dst[axis] = slice(-k, n)
            src[axis] = slice(0, max(n + k, 0))
        out[tuple(dst)] += a[tuple(src)]
    return out


def box_sum(img: np.ndarray, r: int) -> np.ndarray:
    """sum over the (2r+1)^2 square window clipped to the image (double sum, rows then columns)."""
    return window_sum_1d(window_sum_1d(img, r, axis=1), r, axis=0)


def kernel_factors(r: int, s: Optional[float] = None) -> np.ndarray:
    """g(i), i = -r..r: the Gaussian kernel of Sec. 2.1.1 on the (2r+1)^2 window is
    G(n, m, s) = g(n) g(m) / Z with g(i) = exp(-i^2 / (2 s^2)), since
    exp(-(n^2 + m^2) / (2 s^2)) factorises; s = None is the uniform box (g = 1)."""
    i = np.arange(-r, r + 1, dtype=np.float64)
    if s is None:
        return np.ones_like(i)
    return np.exp(-(i * i) / (2.0 * float(s) * float(s)))


def kernel_sum(img: np.ndarray, r: int, s: Optional[float] = None) -> np.ndarray:
    """sum_q g(qy - py) g(qx - px) img(q) over the (2r+1)^2 window clipped to the
    image, unnormalised (rows then columns); s = None gives box_sum."""
    g = kernel_factors(r, s)
    out = np.asarray(img, dtype=np.float64)
    for axis in (1, 0):
        a = out
        n = a.shape[axis]
        out = np.zeros_like(a)
        for k in range(-r, r + 1):
            dst = [slice(None)] * a.ndim
            src = [slice(None)] * a.ndim
            if k >= 0:
                dst[axis] = slice(0, max(n - k, 0))
                src[axis] = slice(k, n)
            else:
                dst[axis] = slice(-k, n)
                src[axis] = slice(0, max(n + k, 0))
            out[tuple(dst)] += g[k + r] * a[tuple(src)]
    return out


def window_count(H: int, W: int, r: int) -> np.ndarray:
    """Number of in-image pixels of each clipped window (the normaliser Z of Sec. 2.1.1)."""
    return box_sum(np.ones((H, W)), r)


def local_centre(D: np.ndarray, r: int) -> np.ndarray:
    """C := G * D with the uniform box kernel, normalised per pixel (Sec. 2.1.1)."""
    return box_sum(D, r) / window_count(*D.shape, r)


def local_spread(D: np.ndarray, C: np.ndarray, r: int) -> np.ndarray:
    """S := G * (D - C)^2, the square element-wise before the second filter (Sec. 2.1.1)."""
    return box_sum((D - C) ** 2, r) / window_count(*D.shape, r)


# --------------------------------------------------------------------- a6
def snr_map(D: np.ndarray, C: np.ndarray, S: np.ndarray) -> np.ndarray:
    """(D - C)/sqrt(S) where S > 0, else 0 (Sec. 2.1.1 threshold, as S/N)."""
    out = np.zeros_like(D)
    ok = S > 0
    out[ok] = (D[ok] - C[ok]) / np.sqrt(S[ok])
    return out


def neighbour_max(D: np.ndarray, k: int = 1) -> np.ndarray:
    """Max of the other pixels of the (2k+1)^2 window inside the image (-inf where
    there are none)."""
    H, W = D.shape
    pad = np.full((H + 2 * k, W + 2 * k), -np.inf)
    pad[k:k + H, k:k + W] = D
    best = np.full((H, W), -np.inf)
    for dy in range(-k, k + 1):
        for dx in range(-k, k + 1):
            if dy == 0 and dx == 0:
                continue
            best = np.maximum(best, pad[k + dy:k + dy + H, k + dx:k + dx + W])
    return best


def local_max_mask(D: np.ndarray, k: int = 1) -> np.ndarray:
    """q = I(D = max over the (2k+1)^2 window clipped to the image) (Sec. 2.1.2;
    the dispersed search uses k = 1, the paper's per-subband detector k = 3)."""
    return D >= neighbour_max(D, k)


def detect(D: np.ndarray, r: int, kappa: float, k: int = 1) -> Dict[str, np.ndarray]:
    """Full per-image chain: C, S, snr, threshold AND local max (Sec. 2.1.1-2.1.2)."""
    C = local_centre(D, r)
    S = local_spread(D, C, r)
    snr = snr_map(D, C, S)
    above = snr > kappa                     # y: x > c + kappa sqrt(s), S > 0
    q = local_max_mask(D, k)
    return dict(C=C, S=S, snr=snr, valid=S > 0, mask=above & q & (S > 0),
                lmax_margin=D - neighbour_max(D, k))


# --------------------------------------------------------------------- a7
def frame_stats(snr: np.ndarray, valid: np.ndarray) -> Tuple[float, float, int]:
    """(mean, RMS) of S/N over the valid pixels, FP64, and the pixel count."""
    v = snr[valid]
    n = int(v.size)
    if n == 0:
        return 0.0, 0.0, 0
    return float(v.sum() / n), float(math.sqrt(float((v * v).sum()) / n)), n


# --------------------------------------------------------------------- whole push
def active_trials(delays: np.ndarray, T: int, T_first: int = 0) -> List[int]:
    """DM trials whose whole sweep has been pushed by frame T."""
    dmax = delays.max(axis=1)
    return [d for d in range(delays.shape[0]) if T - int(dmax[d]) >= T_first]


def search_push(frame_at: FrameFn, T: int, delays: np.ndarray, r: int, kappa: float,
                T_first: int = 0, dms: Optional[Sequence[int]] = None,
                keep_maps: bool = False):
    """All candidates (t0, d, y, x, snr) produced by the push of frame T.

    Returns (cands, stats, maps): cands sorted by (t0, d, y, x); stats maps
    d -> (mean, rms, n); maps (if keep_maps) d -> detect() dict plus D, abs_sum.
    """
    cands = []
    stats = {}
    maps = {}
    for d in (active_trials(delays, T, T_first) if dms is None else dms):
        t0, D = dedisperse(frame_at, T, delays, d)
        res = detect(D, r, kappa)
        ys, xs = np.nonzero(res["mask"])
        for y, x in zip(ys, xs):
            cands.append((t0, d, int(y), int(x), float(res["snr"][y, x])))
        stats[d] = frame_stats(res["snr"], res["valid"])
        if keep_maps:
            res["D"] = D
            res["abs_sum"] = abs_sum(frame_at, T, delays, d)
            res["t0"] = t0
            maps[d] = res
    cands.sort(key=lambda c: (c[0], c[1], c[2], c[3]))
    return cands, stats, maps


# --------------------------------------------------------------------- residual form
def residual_frame(frame: np.ndarray, r: int) -> np.ndarray:
    """X - C(X) for every subband plane of one frame (Sec. 2.1.1 local centre per plane)."""
    frame = np.asarray(frame, dtype=np.float64)
    return np.stack([frame[f] - local_centre(frame[f], r) for f in range(frame.shape[0])])


def search_push_residual(raw_at: FrameFn, res_at: FrameFn, T: int, delays: np.ndarray, r: int,
                         kappa: float, T_first: int = 0, dms: Optional[Sequence[int]] = None,
                         keep_maps: bool = False):
    """The search with D - C formed as the shift-sum of per-subband residuals.

    The local centre is linear and the same clipped window serves every plane,
    so D_d - C_d = sum_f (X_f - C(X_f)) at the shifted frames (Sec. 2.1.1,
    App. B.2); S = box mean of (D - C)^2, snr = (D - C)/sqrt(S); the local
    maximum is taken on D from raw_at.  With res_at = residual_frame(raw_at)
    this equals search_push exactly (up to rounding order); a ring that stores
    the residuals in reduced precision is reproduced by rounding res_at.
    """
    cands, stats, maps = [], {}, {}
    for d in (active_trials(delays, T, T_first) if dms is None else dms):
        t0, D = dedisperse(raw_at, T, delays, d)
        _, Rd = dedisperse(res_at, T, delays, d)
        S = box_sum(Rd * Rd, r) / window_count(*Rd.shape, r)
        snr = np.zeros_like(Rd)
        ok = S > 0
        snr[ok] = Rd[ok] / np.sqrt(S[ok])
        q = local_max_mask(D)
        mask = (snr > kappa) & q & ok
        ys, xs = np.nonzero(mask)
        for y, x in zip(ys, xs):
            cands.append((t0, d, int(y), int(x), float(snr[y, x])))
        stats[d] = frame_stats(snr, ok)
        if keep_maps:
            maps[d] = dict(D=D, S=S, snr=snr, valid=ok, mask=mask, lmax_margin=D - neighbour_max(D),
                           abs_sum=abs_sum(raw_at, T, delays, d), t0=t0)
    cands.sort(key=lambda c: (c[0], c[1], c[2], c[3]))
    return cands, stats, maps


# --------------------------------------------------------------------- a8
def dynspec(frame_at: FrameFn, T: int, Tw: int, cands: Sequence[Tuple[int, int]],
            box_r: int = 0) -> np.ndarray:
    """Dynamic spectra [n, F, Tw]: the flux at each candidate pixel in the Tw frames
    ending at T (Sec. 2.2 backward fill); with box_r > 0 the maximum pixel of the
    (2 box_r + 1)^2 box clipped to the image (Sec. 2.2 flux measurement)."""
    frames = [np.asarray(frame_at(T - Tw + 1 + tau), np.float64) for tau in range(Tw)]
    F, H, W = frames[0].shape
    out = np.zeros((len(cands), F, Tw))
    for n, (y, x) in enumerate(cands):
        y0, y1 = max(y - box_r, 0), min(y + box_r + 1, H)
        x0, x1 = max(x - box_r, 0), min(x + box_r + 1, W)
        for tau in range(Tw):
            out[n, :, tau] = frames[tau][:, y0:y1, x0:x1].reshape(F, -1).max(axis=1)
    return out


# --------------------------------------------------------------------- storage
def storage_round(x: np.ndarray, dtype: str) -> np.ndarray:
    """Values as stored in a reduced-precision ring (round to nearest even), as float64."""
    import torch  # plain CPU conversion
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32))
    if dtype == "fp32":
        return t.double().numpy()
    if dtype == "fp16":
        return t.to(torch.float16).double().numpy()
    if dtype == "bf16":
        return t.to(torch.bfloat16).double().numpy()
    raise ValueError(dtype)


# --------------------------------------------------------------------- quality control
def qc_band_scores(frame: np.ndarray) -> np.ndarray:
    """z_b = (b_b - median(b)) / MAD(b) with b_b the mean of band image b (App. A).

    MAD(b) = median(|b - median(b)|).  Where MAD = 0 a band equal to the median
    scores 0 and any other band +-inf.
    """
    F = frame.shape[0]
    b = np.asarray(frame, np.float64).reshape(F, -1).mean(axis=1)
    med = np.median(b)
    mad = np.median(np.abs(b - med))
    dev = b - med
    if mad > 0:
        return dev / mad
    return np.where(dev == 0, 0.0, np.copysign(np.inf, dev))


class QCState:
    """Running per-pixel statistics of the kept band images (App. A, Welford):
    per band the number n of frames folded in, per pixel the mean and the sum of
    squared deviations m2 (sample variance m2 / (n - 1))."""

    def __init__(self, F: int, H: int, W: int):
        self.n = np.zeros(F, np.int64)
        self.mean = np.zeros((F, H, W))
        self.m2 = np.zeros((F, H, W))


def qc_pixel_scores(frame: np.ndarray, state: QCState, min_frames: int) -> np.ndarray:
    """Per band the largest |zeta| = |x - mean| / s over pixels with s > 0, using the
    statistics before this frame; 0 for a band with fewer than min_frames frames."""
    F = frame.shape[0]
    out = np.zeros(F)
    for f in range(F):
        n = int(state.n[f])
        if n < max(min_frames, 2):
            continue
        s = np.sqrt(state.m2[f] / (n - 1))
        ok = s > 0
        if ok.any():
            out[f] = float(np.max(np.abs(np.asarray(frame[f], np.float64)[ok] - state.mean[f][ok]) / s[ok]))
    return out


def qc_frame(frame: np.ndarray, state: QCState, z_thr: float, zeta_thr: float, min_frames: int):
    """Quality control of one image cube (App. A): band image b is discarded
    (imputed with zeros) when |z_b| > z_thr or any |zeta_bij| > zeta_thr; the
    kept band images are then folded into the running statistics.

    Returns (frame after imputation, discarded [F] bool, z [F], max |zeta| [F]).
    """
    x = np.asarray(frame, np.float64)
    z = qc_band_scores(x)
    zeta = qc_pixel_scores(x, state, min_frames)
    discard = (np.abs(z) > z_thr) | (zeta > zeta_thr)
    out = x.copy()
    out[discard] = 0.0
    for f in np.nonzero(~discard)[0]:
        state.n[f] += 1
        delta = x[f] - state.mean[f]
        state.mean[f] += delta / state.n[f]
        state.m2[f] += delta * (x[f] - state.mean[f])
    return out, discard, z, zeta


# --------------------------------------------------------------------- per-subband detector
def subband_detect(frame: np.ndarray, r: int, kappa: float, k: int = 3):
    """The paper's per-bandpass detector on one image cube (Sec. 2.1.1-2.1.2): the
    one-pass centre / spread filter and threshold on every band image X_b, the
    (2k+1)^2 maximum filter on X_b (k = 3 in the paper), P_b = q AND y.

    Returns (cands sorted by (b, y, x) as (b, y, x, snr), stats b -> (mean, rms, n),
    maps b -> detect() dict).
    """
    x = np.asarray(frame, np.float64)
    cands, stats, maps = [], {}, {}
    for b in range(x.shape[0]):
        res = detect(x[b], r, kappa, k)
        ys, xs = np.nonzero(res["mask"])
        for y, xx in zip(ys, xs):
            cands.append((b, int(y), int(xx), float(res["snr"][y, xx])))
        stats[b] = frame_stats(res["snr"], res["valid"])
        maps[b] = res
    cands.sort(key=lambda c: (c[0], c[1], c[2]))
    return cands, stats, maps


def clip_detect(D: np.ndarray, r: int, kappa: float, k: int = 1, iters: int = 1,
                s: Optional[float] = None) -> Dict[str, np.ndarray]:
    """Iterated sigma clipping of one image (Sec. 2.1.1): at each iteration C and S
    are the kernel-weighted means over the window pixels not yet flagged (the
    kernel weight of those pixels normalises: Z restricted to them), y = I(snr >
    kappa) is added to the flags, and the loop stops when an iteration flags no
    new pixel or after iters iterations.  The peaks are the (2k+1)^2 maxima of D
    among the flagged pixels (Sec. 2.1.2); the S/N is that of the last iteration.
    The kernel is the Gaussian G(n, m, s) on the (2r+1)^2 window, or the uniform
    box for s = None; iters = 1 with the box is detect().
    """
    D = np.asarray(D, np.float64)
    flags = np.zeros(D.shape, bool)
    C = S = snr = None
    n = None
    for _ in range(max(int(iters), 1)):
        m = (~flags).astype(np.float64)
        n = kernel_sum(m, r, s)
        ok = n > 0
        C = np.zeros_like(D)
        C[ok] = kernel_sum(D * m, r, s)[ok] / n[ok]
        S = np.zeros_like(D)
        S[ok] = kernel_sum((D - C) ** 2 * m, r, s)[ok] / n[ok]
        snr = snr_map(D, C, S)
        above = snr > kappa
        new = above & ~flags
        flags |= above
        if not new.any():
            break
    q = local_max_mask(D, k)
    return dict(C=C, S=S, snr=snr, valid=S > 0, flags=flags, mask=flags & q & (S > 0),
                lmax_margin=D - neighbour_max(D, k))


# ---------------------------------------------------------------------------
# Opt-in steady-source suppression.  The paper removes steady sources after the
# search: association with the previous catalogue (Sec. 2.2) and the DM the
# network infers (Sec. 2.3).  Reading: a steady source is bright without
# dispersion in every frame, so a pixel counts as steady once it has been a
# candidate of a zero-delay trial (max_f delay = 0, the newest frame alone) in
# each of the K most recent pushes; a dispersed pulse can cross at zero delay in
# the frame its last subband arrives, but not K frames in a row for K above its
# width.  The candidates of every trial with a nonzero delay row at a steady
# pixel are dropped; the zero-delay trials keep theirs.

class SteadyMask:
    """Run length, per pixel, of consecutive pushes in which the pixel was a
    candidate of a zero-delay trial (saturating at 255)."""

    def __init__(self, K: int):
        self.K = int(K)
        self.run: Dict[Tuple[int, int], int] = {}

    def update(self, zero_delay_pixels) -> set:
        """Fold in one push (the set of (y, x) of its zero-delay candidates) and
        return the steady pixels after it (run >= K)."""
        hit = set(zero_delay_pixels)
        self.run = {p: min(self.run.get(p, 0) + 1, 255) for p in hit}
        return {p for p, n in self.run.items() if n >= self.K}


def suppress_steady(cands, max_delay_of_trial, steady: set):
    """The candidates (t0, d, y, x, snr) without those of trials whose delay row
    is not all zero at steady pixels."""
    return [c for c in cands if max_delay_of_trial[c[1]] == 0 or (c[2], c[3]) not in steady]
