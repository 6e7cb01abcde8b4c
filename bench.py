#!/usr/bin/env python
"""Throughput of the image-plane dispersed-transient search on the AARTFAAC-shaped
workload: 1024x1024 px, 16 subbands (two groups of 8 at 57.6 and 61.2 MHz),
251 DM trials (0..250 step 1), ring depth 48, 31x31 background box, kappa 6.

One step = one push of a new frame through the whole path (ingest, shift-sum,
box centre / spread, S/N threshold + 3x3 local maximum, candidate ordering,
per-trial stats).  Metric: pixel * DM-trials per second (H*W*N_DM per frame).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype fp32|fp16|bf16]
  python bench.py --impl reference ...     # the FP64 CPU oracle on the same metric

Under torchrun (N > 1) every rank runs an independent stream on its own GPU
(weak scaling, no collective on the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

RESULT_SLOTS = 4                # result slots: up to 3 frames ahead of the oldest unpolled one
METRIC = "pixel*DM-trials/s"
WORKLOAD = "aartfaac-1024x1024-16sb-251dm-depth48-box31"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--pool", type=int, default=12, help="distinct synthetic frames cycled")
    ap.add_argument("--clip-iters", type=int, default=1,
                    help="subband workload: sigma-clip iterations (1 = one pass)")
    ap.add_argument("--gauss-sigma", type=float, default=0.0,
                    help="subband workload: Gaussian background kernel of this width in pixels on the "
                         "31x31 window (0 = the uniform box)")
    ap.add_argument("--qc", action="store_true",
                    help="quality control of every frame before the search (band and pixel scores)")
    ap.add_argument("--workload", default="aartfaac", choices=["aartfaac", "serving", "subband", "stress"],
                    help="serving: four concurrent FP16 streams through the C++ serving loop")
    ap.add_argument("--cadence", type=float, default=1.0, help="serving: frame cadence in seconds")
    ap.add_argument("--frames", type=int, default=60, help="serving: frames per stream")
    return ap.parse_args()


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time); identity without a process group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def workload_spec(dtype):
    return synth.spec_aartfaac(dtype=dtype)


# Minimal FP32 work of the filter per pixel and distinct trial, given D - C: square,
# horizontal and vertical sliding sums (add + subtract each), normalise, rsqrt,
# multiply (S/N), threshold compare, two statistics accumulations.
FILTER_OPS_PER_PIXEL_TRIAL = 11


def kernel_traffic(field="dram_bytes_per_launch"):
    """A per-launch counter (DRAM bytes, or executed warp instructions) from the
    committed ncu capture, or None where the kernel's source has changed since the
    counters were taken or the capture has no such counter."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return {}
    out = {}
    for k, v in rec.items():
        src = os.path.join(ROOT, v["source"])
        try:
            sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
        except Exception:
            continue
        out[k] = v.get(field) if sha == v["sha256"] else None
    return out


def algorithmic_bytes(spec, delays, n_distinct):
    """Bytes a push must move at minimum, per stage, with storage type of b bytes."""
    b = 4 if spec.dtype == "fp32" else 2
    HW = spec.H * spec.W
    lags = delays.max(axis=1)[:, None] - delays
    U = sum(len(np.unique(lags[:, f])) for f in range(spec.F))
    ring_reads = U * HW * b
    return dict(
        path=ring_reads + spec.F * HW * (4 + b),
        ingest=spec.F * HW * (4 + b),
        dedisperse=ring_reads + n_distinct * HW * 4,
        filter_detect=n_distinct * HW * 4,
        U=U,
    )


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def oracle_sample(spec, frame_at, T, delays, dms):
    from oracle import lpf_oracle as O
    t = time.perf_counter()
    O.search_push(frame_at, T, delays, spec.box_r, spec.kappa, dms=dms)
    return time.perf_counter() - t


def cpu_baseline(spec, st, delays, n_dm=36):
    """The FP64 oracle (as it stands, one process) on a bounded sample of one push."""
    import functools
    fa = functools.lru_cache(maxsize=64)(lambda t: st.frame(t).astype(np.float64))
    T = int(delays.max())
    dms = [int(d) for d in np.linspace(0, spec.n_dm - 1, n_dm).round()]
    fa_warm = [fa(T - k) for k in range(int(delays.max()) + 1)]  # generation outside the timing
    del fa_warm
    secs = oracle_sample(spec, fa, T, delays, dms)
    val = spec.H * spec.W * len(dms) / secs
    return {"value": val, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"one push (T={T}) of the {spec.H}x{spec.W} stream, {len(dms)} of "
                      f"{spec.n_dm} DM trials, FP64 NumPy single process, {secs:.1f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    spec = workload_spec(args.dtype)
    from oracle import lpf_oracle as O
    import functools
    st = synth.SyntheticStream(spec, seed=1)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    fa = functools.lru_cache(maxsize=128)(lambda t: O.storage_round(st.frame(t), spec.dtype))
    T0 = int(delays.max())
    per_step = 2    # DM trials per step: the oracle's bounded sample of one push
    for w in range(args.warmup):
        for k in range(int(delays.max()) + 1):
            fa(T0 + w - k)
    tot = 0.0
    for k in range(args.steps):
        T = T0 + (k % 4)
        for j in range(int(delays.max()) + 1):
            fa(T - j)
        dms = [(k * per_step + j) % spec.n_dm for j in range(per_step)]
        tot += oracle_sample(spec, fa, T, delays, dms)
    val = spec.H * spec.W * per_step * args.steps / tot
    sample = (f"each step: {per_step} of {spec.n_dm} DM trials of one push of the "
              f"{spec.H}x{spec.W} stream, FP64 NumPy single process")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "storage": args.dtype,
                                            "sample_dm_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import paper_2103_15418_b300 as lpf

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    spec = workload_spec(args.dtype)
    st = synth.SyntheticStream(spec, seed=1 + rank)
    pool = [torch.from_numpy(st.frame(t)) for t in range(args.pool)]
    pool_dev = [p.to(dev) for p in pool]
    pool_pin = [p.pin_memory() for p in pool]
    cur = torch.cuda.Stream(dev)            # the search stream (the timing events are recorded on it)
    s = lpf.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                   box_r=spec.box_r, dtype=args.dtype, result_slots=RESULT_SLOTS, cuda_stream=cur,
                   qc=args.qc, qc_min_frames=16)
    info = s.info()
    delays = s.delay_table()
    nbytes = algorithmic_bytes(spec, delays, info["n_distinct"])
    depth = spec.depth
    T = 0
    polled = []

    def push(T):
        s.push(pool_dev[T % args.pool], T)

    def poll():
        _, c, n, _ = s.poll(timeout_ms=600000)
        polled.append(n)

    # fill the ring so every trial is active, then warm up
    for _ in range(depth + args.warmup):
        push(T)
        T += 1
        poll()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clocks = Clocks(local)
    clocks.start()
    s.kernel_times(reset=True)
    s.set_profiling(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # result_slots - 1 pushes ahead of the oldest unpolled frame, as in the
    # end-to-end loop below
    ahead = max(1, RESULT_SLOTS - 1)
    ev0.record(cur)
    for k in range(args.steps):
        push(T)
        T += 1
        if k >= ahead:
            poll()
    for _ in range(ahead):
        poll()
    ev1.record(cur)
    torch.cuda.synchronize()
    clk = clocks.stop()
    s.set_profiling(False)
    elapsed = ev0.elapsed_time(ev1) / 1e3
    ktimes = s.kernel_times(reset=True)
    elapsed = max_over_ranks(elapsed, dist, dev)
    ncand = float(np.mean(polled[-args.steps:]))
    pix_dm = spec.H * spec.W * spec.n_dm
    value = pix_dm * args.steps * ws / elapsed

    # end to end through the C ABI with host buffers: H2D of the frame, D2H of the
    # candidates, as a user streams frames: push frame T, then poll the oldest
    # frame once result_slots - 1 frames are in flight (the upload of T overlaps
    # the search of T - 1); latency is push call -> poll return of the same frame
    lat = []
    e2e_cands = []
    t_push = {}
    inflight = max(1, RESULT_SLOTS - 1)

    def poll_host():
        Tp, c, n, _ = s.poll(timeout_ms=600000)
        e2e_cands.append(n)
        lat.append(time.perf_counter() - t_push.pop(Tp))

    torch.cuda.synchronize()
    t_e0 = time.perf_counter()
    for k in range(args.e2e_steps):
        t_push[T] = time.perf_counter()
        s.push_host(pool_pin[T % args.pool], T)
        T += 1
        if len(t_push) >= inflight + 1:
            poll_host()
    while t_push:
        poll_host()
    e2e_s = time.perf_counter() - t_e0
    e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e_value = pix_dm * args.e2e_steps * ws / e2e_s
    s.close()

    if rank != 0:
        return
    # per-kernel rooflines from the CUDA-event stage times (on the launching stream)
    names = list(ktimes)
    per_push = {n: ktimes[n][0] / max(ktimes[n][1], 1) for n in names}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    peak_src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = peaks.get("sm_max_mhz", 2032.0)
    alu_peak = sms * 128 * sm_mhz * 1e6 / 1e12          # one FP32 op per lane per clock
    traffic = kernel_traffic()
    HW = spec.H * spec.W
    nd = info["n_distinct"]
    n_dd = 1                                              # residual ring -> D - C
    dd_ms = per_push["dedisperse"] / n_dd
    dd_bytes = nbytes["dedisperse"]
    dd_ach = dd_bytes / (dd_ms / 1e3) / 1e9
    f_ms = per_push["filter_detect"]
    f_ops = FILTER_OPS_PER_PIXEL_TRIAL * HW * nd
    f_ach = f_ops / (f_ms / 1e3) / 1e12
    roof_dd = {"kernel": "k_dedisperse (shift-sum)", "bound": "hbm", "achieved": dd_ach, "peak": hbm_peak,
               "unit": "GB/s", "frac": dd_ach / hbm_peak, "peak_source": peak_src,
               "traffic": traffic.get("k_dedisperse_" + args.dtype),
               "algorithmic_bytes_per_launch": dd_bytes, "avg_launch_ms": dd_ms, "launches_per_step": n_dd}
    roof_f = {"kernel": "k_filter_res<15> (box spread, S/N, threshold, stats)", "bound": "alu",
              "achieved": f_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": f_ach / alu_peak,
              "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz",
              "traffic": traffic.get("k_filter_res"),
              "algorithmic_flop_per_launch": f_ops, "avg_launch_ms": f_ms, "launches_per_step": 1}
    # the filter is bound by instruction issue: executed warp instructions per launch
    # (ncu) over the event-timed launch, against 4 schedulers per SM at the clock
    f_inst = kernel_traffic("warp_inst_per_launch").get("k_filter_res")
    issue_peak = sms * 4 * sm_mhz * 1e6 / 1e12
    roof_f_issue = {"kernel": "k_filter_res<15> (instruction issue)", "bound": "issue",
                    "achieved": f_inst / (f_ms / 1e3) / 1e12 if f_inst else None, "peak": issue_peak,
                    "unit": "T warp-instructions/s",
                    "frac": f_inst / (f_ms / 1e3) / 1e12 / issue_peak if f_inst else None,
                    "peak_source": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz",
                    "warp_instructions_per_launch": f_inst, "avg_launch_ms": f_ms}
    roof = roof_f if f_ms >= dd_ms else roof_dd
    # quality control + ingest (k_qc_scan, k_qc_decide, k_residual, k_ingest_qc): the
    # QC passes read the frame and the running mean and m2 twice and write them once
    b = 4 if args.dtype == "fp32" else 2
    qc_bytes = spec.F * HW * (12 + 20 + b)
    qc_ms = per_push["ingest"] + per_push.get("ring_write", 0.0)
    roof_qc = {"kernel": "quality control + ingest (k_qc_scan, k_qc_decide, k_ingest_qc, k_residual)",
               "bound": "hbm", "achieved": qc_bytes / (qc_ms / 1e3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
               "frac": qc_bytes / (qc_ms / 1e3) / 1e9 / hbm_peak, "peak_source": peak_src, "traffic": None,
               "algorithmic_bytes_per_launch": qc_bytes, "avg_launch_ms": qc_ms, "launches_per_step": 1,
               "note": "the stage also runs k_residual (per-subband X - C(X)), not counted in the bytes"}
    path_ach = nbytes["path"] / (elapsed / args.steps) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded AARTFAAC-shaped stream: noise, 3-sigma cosine gradient, "
                "500 Gaussian-PSF sources, 20 dispersed pulses)",
        "config": {"workload": WORKLOAD, "H": spec.H, "W": spec.W, "subbands": spec.F,
                   "dm_trials": spec.n_dm, "depth": depth, "box": 2 * spec.box_r + 1,
                   "storage": args.dtype, "distinct_delay_rows": info["n_distinct"],
                   "quality_control": bool(args.qc),
                   "l2": "inputs larger than L2 (ring %.2f GB)" % (info["ring_bytes"] / 1e9),
                   "parallelism": f"{ws} independent stream(s), one per GPU"},
        "e2e": {"value": e2e_value, "unit": METRIC,
                "h2d_bytes_per_step": spec.F * spec.H * spec.W * 4,
                "d2h_bytes_per_step": int(np.mean(e2e_cands) * 24 + spec.n_dm * 16)},
        "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                       "p99": 1e3 * float(np.percentile(lat, 99)),
                       "what": f"push_frame_host -> poll of the same frame, up to {RESULT_SLOTS} frames in flight"},
        # per push: ingest + residual, counter reset, shift-sum, filter, 3x3 maximum,
        # 3 per sort pass, format, stats
        "gpu_launches": int(args.steps * (8 + 3 * _passes(spec) + (2 if args.qc else 0))),
        "roofline": roof,
        "rooflines": [roof_f, roof_f_issue, roof_dd] + ([roof_qc] if args.qc else []),
        "path_roofline": {"bound": "hbm", "achieved": path_ach, "peak": hbm_peak, "unit": "GB/s",
                          "frac": path_ach / hbm_peak,
                          "algorithmic_bytes_per_step": nbytes["path"],
                          "note": "sum over subbands of distinct delay planes read once + ingest"},
        "kernel_ms_per_step": per_push,
        "candidates_per_step": ncand,
        "clocks": clk,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, st, delays)
    print(json.dumps(line), flush=True)


def _passes(spec):
    bits = lambda v: max(1, int(np.ceil(np.log2(v))))
    return (bits(spec.W) + bits(spec.H) + bits(spec.n_dm) + 7) // 8


def run_subband(args):
    """The paper's per-subband detector on the AARTFAAC stream (1024^2, 16 bands,
    31x31 window, uniform box or Gaussian kernel, 7x7 maximum): every band image of
    every frame, device-timed."""
    import torch
    import paper_2103_15418_b300 as lpf
    import synth
    spec = synth.spec_aartfaac(dtype=args.dtype)
    st = synth.SyntheticStream(spec, seed=0)
    pool = [torch.from_numpy(st.frame(t)).cuda() for t in range(args.pool)]
    cur = torch.cuda.Stream()               # the search stream (the timing events are recorded on it)
    s = lpf.Stream(spec.H, spec.W, spec.freqs_mhz, None, 2, kappa=spec.kappa, box_r=spec.box_r,
                   dtype=args.dtype, result_slots=RESULT_SLOTS, cuda_stream=cur, mode="subband", lmax_r=3,
                   clip_iters=args.clip_iters, kernel="gauss" if args.gauss_sigma > 0 else "box",
                   gauss_sigma=args.gauss_sigma)
    T = 0
    for _ in range(args.warmup + 2):
        s.push(pool[T % args.pool], T)
        T += 1
        s.poll(timeout_ms=600000)
    s.set_profiling(True)
    s.kernel_times(reset=True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(cur)
    ncand = []
    for k in range(args.steps):
        s.push(pool[T % args.pool], T)
        T += 1
        if k >= RESULT_SLOTS - 1:
            ncand.append(s.poll(timeout_ms=600000)[2])
    while len(ncand) < args.steps:
        ncand.append(s.poll(timeout_ms=600000)[2])
    ev1.record(cur)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    kt = s.kernel_times(reset=True)
    s.close()
    per_push = {n: kt[n][0] / max(kt[n][1], 1) for n in kt}
    px = spec.H * spec.W * spec.F
    print(json.dumps({
        "metric": "pixel*bands/s", "value": px * args.steps / elapsed, "unit": "pixel*bands/s",
        "workload": "subband-detector-1024x1024-16bands-" +
                    (f"gauss{args.gauss_sigma:g}-window31" if args.gauss_sigma > 0 else "box31") + "-max7x7",
        "storage": args.dtype, "clip_iters": args.clip_iters,
        "steps": args.steps, "ms_per_step": 1e3 * elapsed / args.steps,
        "kernel_ms_per_step": per_push, "candidates_per_step": float(np.mean(ncand)),
        "data": "synthetic (seeded AARTFAAC-shaped stream)"}), flush=True)


def run_serving(args):
    """Serving mix: 2048^2/16/501, 1024^2/16/251 and 2 x 512^2/8/128 FP16 streams, frames
    submitted at the cadence with +-5% jitter; p50/p99 submit -> finish latency and the
    aggregate pixel*DM-trials/s of the finished frames."""
    import threading
    import torch
    import paper_2103_15418_b300 as lpf
    specs = synth.spec_serving_mix()
    pools = []
    for i, sp in enumerate(specs):
        st = synth.SyntheticStream(sp, seed=60 + i)
        pools.append([st.frame(t) for t in range(4)])
    budget = 80 << 30
    n = args.frames
    jit = np.random.default_rng(7)
    with lpf.Server(budget, max_streams=8) as srv:
        ids = [srv.open_stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, kappa=sp.kappa,
                               box_r=sp.box_r, dtype=sp.dtype) for sp in specs]
        counts = {i: 0 for i in ids}

        def drain(i):
            while counts[i] < n:
                srv.fetch(i, timeout_ms=600000)
                counts[i] += 1
        threads = [threading.Thread(target=drain, args=(i,)) for i in ids]
        for th in threads:
            th.start()
        t0 = time.perf_counter()
        # staggered, jittered arrivals: stream k's frame T is due at (T + k/4) * cadence +- 5%
        events = sorted((T + k / len(ids) + jit.uniform(-0.05, 0.05)) * args.cadence for T in range(n)
                        for k in range(len(ids)))
        order = sorted(((T + k / len(ids)) * args.cadence, k, T) for T in range(n) for k in range(len(ids)))
        for (due, k, T), ev in zip(order, events):
            wait = t0 + ev - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            while srv.submit(ids[k], pools[k][T % 4], T) == lpf.LPF_E_BUSY:
                time.sleep(0.0005)
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        stats = srv.stats()
        per = {specs[i].name: srv.stats(ids[i]) for i in range(len(ids))}
    pixdm = sum(sp.H * sp.W * sp.n_dm for sp in specs) * n
    line = {"metric": METRIC, "workload": "serving-mix-4-streams-fp16", "cadence_s": args.cadence,
            "frames_per_stream": n, "p50_ms": stats["p50_ms"], "p99_ms": stats["p99_ms"],
            "max_ms": stats["max_ms"], "pixel_dm_per_s_served": stats["pixel_dm_per_s"],
            "offered_pixel_dm_per_s": pixdm / wall,
            "per_stream_p99_ms": {k: v["p99_ms"] for k, v in per.items()},
            "hbm_budget_bytes": budget, "peak_used_bytes": stats["used_bytes"]}
    print(json.dumps(line), flush=True)


def run_stress(args):
    """Stress workload: 2048^2 px, 32 subbands (57.6-63.85 MHz), 1001 DM trials, FP16
    ring of depth 114 (the DM 500 sweep spans 113 frames).  Each step pushes a frame,
    polls the oldest unpolled one and gathers the 32 x 64 FP32 dynamic spectra of its
    candidates; frames per second against the 1 s cadence is the real-time factor.
    The candidate load of about 1e4 per frame comes from 10 bright steady sources
    (each a candidate at every one of the 1001 trials): the 200 pulses give about 2."""
    import torch
    import paper_2103_15418_b300 as lpf
    spec = synth.spec_stress(depth=114, n_sources=10, source_flux=(40.0, 400.0))
    st = synth.SyntheticStream(spec, seed=50)
    npool = 4
    pool = [torch.from_numpy(st.frame(t)).cuda() for t in range(npool)]
    cur = torch.cuda.Stream()               # the search stream (the timing events are recorded on it)
    s = lpf.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                   box_r=spec.box_r, dtype="fp16", result_slots=RESULT_SLOTS, cuda_stream=cur)
    info = s.info()
    Tw, T = 64, 0
    ncand, nds, gev = [], [], []
    gbuf = torch.empty((16384, spec.F, Tw), dtype=torch.float32, device="cuda")   # reused output batch

    def poll_and_gather():
        Tp, c, n, _ = s.poll(timeout_ms=600000)
        g = 0
        if len(c) and Tp >= Tw - 1:         # once Tw frames exist
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e[0].record(cur)
            c = c[: gbuf.shape[0]]
            s.dynspec(c, Tw, out=gbuf[: len(c)], sync=False)   # [n, 32, 64] FP32 on the search stream
            e[1].record(cur)
            gev.append(e)
            g = len(c)
        ncand.append(n)
        nds.append(g)

    for _ in range(spec.depth + args.warmup):
        s.push(pool[T % npool], T)
        T += 1
        poll_and_gather()
    ahead = max(1, RESULT_SLOTS - 1)
    s.set_profiling(True)
    s.kernel_times(reset=True)
    torch.cuda.synchronize()
    ncand.clear()
    nds.clear()
    gev.clear()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(cur)
    for k in range(args.steps):
        s.push(pool[T % npool], T)
        T += 1
        if k >= ahead:
            poll_and_gather()
    for _ in range(ahead):
        poll_and_gather()
    ev1.record(cur)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    kt = s.kernel_times(reset=True)
    s.close()
    per_push = {n: kt[n][0] / max(kt[n][1], 1) for n in kt}
    per_push["dynspec_gather"] = float(np.mean([a.elapsed_time(b) for a, b in gev])) if gev else 0.0
    fps = args.steps / elapsed
    print(json.dumps({
        "metric": METRIC, "value": spec.H * spec.W * spec.n_dm * fps, "unit": METRIC,
        "workload": "stress-2048x2048-32sb-1001dm-depth114-fp16-dynspec32x64", "steps": args.steps,
        "ms_per_step": 1e3 * elapsed / args.steps, "frames_per_s": fps, "real_time_factor": fps * spec.cadence_s,
        "n_distinct": info["n_distinct"], "max_delay": info["max_delay"],
        "device_bytes": info.get("device_bytes"), "kernel_ms_per_step": per_push,
        "candidates_per_step": float(np.mean(ncand)), "dynspec_records_per_step": float(np.mean(nds)),
        "data": "synthetic (seeded: noise, gradient, 200 dispersed pulses, 1% RFI stripes, "
                "10 steady sources for the candidate load)"}), flush=True)


def main():
    args = parse()
    if args.workload == "stress":
        run_stress(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload == "subband":
        run_subband(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
