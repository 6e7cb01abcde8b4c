"""Comparison of CUDA-path candidates with the FP64 oracle (test helper).

Parity rule (element by element, per DM trial), against the plain oracle
(search_push, Sec. 2.1-2.1.2 and App. B.2) run on the frames as the ring stores
them (storage_round):
  * candidate sets equal after excluding the pixels the arithmetic cannot
    decide: an S/N within a band of kappa, or a 3x3 local-maximum margin
    |D(p) - max_nbr D| below tau = 4 F 2^-24 max_nbr sum_f |X_f|, the FP32
    summation bound of the shift-sum over the pixel's neighbourhood;
  * S/N of matched candidates within SNR_RTOL[storage] relative;
  * per-trial mean and RMS of the S/N within STATS_RTOL[storage].

FP32 rings: band 1e-3 around kappa, S/N within 1e-4.  FP16/BF16 rings hold
the per-subband residuals X - C(X) rounded to the storage type, a second
rounding the plain oracle on rounded frames does not make; its S/N error is
bounded by the storage unit roundoff u times sum_f |X_f - C(X_f)| / |D - C|.
The tolerance is the stated precision target (FP16: 2e-3; BF16: 1.6e-2, the
FP16 figure scaled by the ratio 8 of the two unit roundoffs), and the band of
undecidable threshold decisions is kappa times that tolerance.

The residual-form reference (search_push_residual fed storage-rounded
residuals) reproduces the ring's values exactly; compare_push(res_at=...)
checks the CUDA arithmetic against it at the FP32 tolerances, in addition to
the plain-oracle comparison.

Against the oracle on unrounded frames (the precision report) the storage
rounding of X also moves D, so local-maximum margins below
2 u max_nbr sum_f |X_f| are undecidable too (storage_tau).
"""
from __future__ import annotations

import functools
from typing import Dict, Tuple

import numpy as np

from oracle import lpf_oracle as O

KAPPA_BAND = 1e-3
SNR_RTOL = {"fp32": 1e-4, "fp16": 2e-3, "bf16": 1.6e-2}
STATS_RTOL = {"fp32": 1e-4, "fp16": 1e-3, "bf16": 8e-3}
UNIT_ROUNDOFF = {"fp32": 0.0, "fp16": 2.0 ** -11, "bf16": 2.0 ** -8}


def cached_frames(stream, dtype: str = "fp32", maxsize: int = 256):
    @functools.lru_cache(maxsize=maxsize)
    def frame_at(t: int):
        return O.storage_round(stream.frame(t), dtype)
    return frame_at


def cached_residuals(stream, dtype: str, r: int, maxsize: int = 256):
    """Per-subband residuals X - C(X) of the storage-rounded frames, rounded to the
    storage type: what a reduced-precision residual ring holds."""
    raw = cached_frames(stream, dtype, maxsize)

    @functools.lru_cache(maxsize=maxsize)
    def res_at(t: int):
        return O.storage_round(O.residual_frame(raw(t), r), dtype)
    return res_at


def neighbourhood_max(a: np.ndarray) -> np.ndarray:
    H, W = a.shape
    pad = np.full((H + 2, W + 2), -np.inf)
    pad[1:-1, 1:-1] = a
    out = np.full((H, W), -np.inf)
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            out = np.maximum(out, pad[1 + dy:1 + dy + H, 1 + dx:1 + dx + W])
    return out


def kappa_band(kappa: float, storage: str) -> float:
    return KAPPA_BAND if storage == "fp32" else abs(kappa) * SNR_RTOL[storage]


def ambiguous_mask(m: dict, F: int, kappa: float, storage: str = "fp32",
                   storage_tau: bool = False) -> np.ndarray:
    """Pixels whose candidate decision the arithmetic cannot settle (see the module
    docstring); storage_tau: against unrounded frames, add the storage rounding of D."""
    scale = 4.0 * F * 2.0 ** -24 + (2.0 * UNIT_ROUNDOFF[storage] if storage_tau else 0.0)
    tau = scale * neighbourhood_max(m["abs_sum"])
    near_k = np.abs(m["snr"] - kappa) < kappa_band(kappa, storage)
    near_tie = np.abs(m["lmax_margin"]) <= tau
    return near_k | near_tie


def compare_trial(gpu: np.ndarray, m: dict, F: int, kappa: float,
                  storage: str = "fp32") -> Tuple[int, int, float]:
    """gpu: candidate records of one trial.  Returns (n_matched, n_excluded, max_rel_err)."""
    amb = ambiguous_mask(m, F, kappa, storage)
    o_set = set(zip(*np.nonzero(m["mask"])))
    g = {(int(c["y"]), int(c["x"])): float(c["snr"]) for c in gpu}
    assert len(g) == len(gpu), "duplicate pixel in one trial"
    only_g = [p for p in g if p not in o_set]
    only_o = [p for p in o_set if p not in g]
    bad_g = [p for p in only_g if not amb[p]]
    bad_o = [p for p in only_o if not amb[p]]
    assert not bad_g, f"GPU-only candidates {bad_g[:5]} (oracle snr {[m['snr'][p] for p in bad_g[:5]]})"
    assert not bad_o, f"oracle-only candidates {bad_o[:5]} (oracle snr {[m['snr'][p] for p in bad_o[:5]]})"
    worst = 0.0
    n = 0
    for p, s in g.items():
        if p in o_set:
            ref = m["snr"][p]
            rel = abs(s - ref) / abs(ref)
            worst = max(worst, rel)
            n += 1
    assert worst <= SNR_RTOL[storage], f"snr relative error {worst} ({storage})"
    return n, len(only_g) + len(only_o), worst


def check_stats(gpu_stats: np.ndarray, stats: dict, d: int, storage: str):
    """Per-trial mean and RMS of the S/N (FP32: relative to each; 16-bit rings:
    relative to the RMS, since the mean of noise S/N is near zero)."""
    mean, rms, _ = stats[d]
    gm, gr = gpu_stats[d]
    tol = STATS_RTOL[storage]
    if storage == "fp32":
        assert abs(gm - mean) <= tol * abs(mean) + 1e-6, (d, gm, mean)
    else:
        assert abs(gm - mean) <= tol * abs(rms) + 1e-6, (d, gm, mean, storage)
    assert abs(gr - rms) <= tol * abs(rms) + 1e-6, (d, gr, rms, storage)


def compare_push(gpu: np.ndarray, frame_at, T: int, delays: np.ndarray, r: int, kappa: float,
                 dms=None, T_first: int = 0, gpu_stats: np.ndarray = None,
                 res_at=None, storage: str = "fp32") -> Dict[str, float]:
    """Compare all trials (or the listed ones) of one push with the plain oracle on
    frame_at (the storage-rounded frames) at the tolerances of the storage type;
    with res_at: against the residual-form reference of a reduced-precision ring
    at the FP32 tolerances instead."""
    F = delays.shape[1]
    if dms is None:
        dms = O.active_trials(delays, T, T_first)
        # every GPU candidate must belong to an active trial
        assert set(np.unique(gpu["dm_idx"]).tolist()) <= set(dms)
    dmax = delays.max(axis=1)
    if res_at is None:
        _, stats, maps = O.search_push(frame_at, T, delays, r, kappa, T_first=T_first, dms=dms,
                                       keep_maps=True)
        tol = storage
    else:
        _, stats, maps = O.search_push_residual(frame_at, res_at, T, delays, r, kappa,
                                                T_first=T_first, dms=dms, keep_maps=True)
        tol = "fp32"
    tot_n = tot_x = 0
    worst = 0.0
    for d in dms:
        sel = gpu[gpu["dm_idx"] == d]
        assert np.all(sel["t0"] == T - dmax[d])
        n, x, w = compare_trial(sel, maps[d], F, kappa, tol)
        tot_n += n
        tot_x += x
        worst = max(worst, w)
        if gpu_stats is not None:
            check_stats(gpu_stats, stats, d, tol)
    return dict(matched=tot_n, excluded=tot_x, max_rel=worst)


def compare_storage(gpu: np.ndarray, frame_at, T: int, delays: np.ndarray, r: int, kappa: float,
                    storage: str, dms=None, gpu_stats: np.ndarray = None, res_at=None) -> Dict[str, float]:
    """A reduced-precision ring: the gating comparison with the plain oracle on the
    storage-rounded frames, plus (res_at given) the residual-form check."""
    out = compare_push(gpu, frame_at, T, delays, r, kappa, dms=dms, gpu_stats=gpu_stats, storage=storage)
    if res_at is not None and storage != "fp32":
        compare_push(gpu, frame_at, T, delays, r, kappa, dms=dms, gpu_stats=gpu_stats, res_at=res_at)
    return out


def precision_vs_unrounded(gpu: np.ndarray, frame_at, T: int, delays: np.ndarray, r: int, kappa: float,
                           dms, storage: str, maps=None) -> Dict[str, float]:
    """The precision report against the oracle on the unrounded frames: the largest
    relative S/N error over candidates both find, and the symmetric difference of
    the candidate sets outside the undecidable pixels (storage band around kappa,
    FP32 plus storage local-maximum margins).  maps: the oracle's maps of those
    trials on the unrounded frames, if already computed."""
    if maps is None:
        _, _, maps = O.search_push(frame_at, T, delays, r, kappa, dms=dms, keep_maps=True)
    worst, sym, matched = 0.0, 0, 0
    F = delays.shape[1]
    for d in dms:
        m = maps[d]
        amb = ambiguous_mask(m, F, kappa, storage, storage_tau=True)
        o = set(zip(*np.nonzero(m["mask"])))
        g = {(int(c["y"]), int(c["x"])): float(c["snr"]) for c in gpu[gpu["dm_idx"] == d]}
        for p, snr in g.items():
            if p in o:
                worst = max(worst, abs(snr - m["snr"][p]) / abs(m["snr"][p]))
                matched += 1
        sym += sum(1 for p in set(g) ^ o if not amb[p])
    return dict(max_rel_snr_err=worst, sym_diff=sym, matched=matched)


def assert_sorted_unique(c: np.ndarray):
    keys = list(zip(c["t0"].tolist(), c["dm_idx"].tolist(), c["y"].tolist(), c["x"].tolist()))
    assert keys == sorted(keys), "candidates not sorted by (t0, dm_idx, y, x)"
    assert len(set(keys)) == len(keys), "duplicate candidates"
