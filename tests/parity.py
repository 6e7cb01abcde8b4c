"""Comparison of CUDA-path candidates with the FP64 oracle (test helper).

Parity rule (element by element, per DM trial):
  * candidate sets equal after excluding pixels the FP32 arithmetic cannot
    decide: |snr_oracle - kappa| < 1e-3, or a 3x3 local-maximum margin
    |D(p) - max_nbr D| below tau = 4 F 2^-24 max_nbr sum_f |X_f|, the FP32
    summation bound of the shift-sum over the pixel's neighbourhood;
  * S/N of matched candidates within 1e-4 relative;
  * per-trial mean / RMS of snr within 1e-4 relative (absolute floor 1e-6).
"""
from __future__ import annotations

import functools
from typing import Dict, Tuple

import numpy as np

from oracle import lpf_oracle as O

SNR_RTOL = 1e-4
KAPPA_BAND = 1e-3


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


def ambiguous_mask(m: dict, F: int, kappa: float) -> np.ndarray:
    tau = 4.0 * F * 2.0 ** -24 * neighbourhood_max(m["abs_sum"])
    near_k = np.abs(m["snr"] - kappa) < KAPPA_BAND
    near_tie = np.abs(m["lmax_margin"]) <= tau
    return near_k | near_tie


def compare_trial(gpu: np.ndarray, m: dict, F: int, kappa: float) -> Tuple[int, int, float]:
    """gpu: candidate records of one trial.  Returns (n_matched, n_excluded, max_rel_err)."""
    amb = ambiguous_mask(m, F, kappa)
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
    assert worst <= SNR_RTOL, f"snr relative error {worst}"
    return n, len(only_g) + len(only_o), worst


def compare_push(gpu: np.ndarray, frame_at, T: int, delays: np.ndarray, r: int, kappa: float,
                 dms=None, T_first: int = 0, gpu_stats: np.ndarray = None,
                 res_at=None) -> Dict[str, float]:
    """Compare all trials (or the listed ones) of one push with the oracle
    (with res_at: the residual-form reference of a reduced-precision ring)."""
    F = delays.shape[1]
    if dms is None:
        dms = O.active_trials(delays, T, T_first)
        # every GPU candidate must belong to an active trial
        assert set(np.unique(gpu["dm_idx"]).tolist()) <= set(dms)
    dmax = delays.max(axis=1)
    if res_at is None:
        _, stats, maps = O.search_push(frame_at, T, delays, r, kappa, T_first=T_first, dms=dms,
                                       keep_maps=True)
    else:
        _, stats, maps = O.search_push_residual(frame_at, res_at, T, delays, r, kappa,
                                                T_first=T_first, dms=dms, keep_maps=True)
    tot_n = tot_x = 0
    worst = 0.0
    for d in dms:
        sel = gpu[gpu["dm_idx"] == d]
        assert np.all(sel["t0"] == T - dmax[d])
        n, x, w = compare_trial(sel, maps[d], F, kappa)
        tot_n += n
        tot_x += x
        worst = max(worst, w)
        if gpu_stats is not None:
            mean, rms, _ = stats[d]
            gm, gr = gpu_stats[d]
            assert abs(gm - mean) <= 1e-4 * abs(mean) + 1e-6, (d, gm, mean)
            assert abs(gr - rms) <= 1e-4 * abs(rms) + 1e-6, (d, gr, rms)
    return dict(matched=tot_n, excluded=tot_x, max_rel=worst)


def assert_sorted_unique(c: np.ndarray):
    keys = list(zip(c["t0"].tolist(), c["dm_idx"].tolist(), c["y"].tolist(), c["x"].tolist()))
    assert keys == sorted(keys), "candidates not sorted by (t0, dm_idx, y, x)"
    assert len(set(keys)) == len(keys), "duplicate candidates"
