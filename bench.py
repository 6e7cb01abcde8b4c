#!/usr/bin/env python
"""Throughput of the image-plane dispersed-transient search on the AARTFAAC-shaped
workload: 1024x1024 px, 16 subbands (two groups of 8 at 57.6 and 61.2 MHz),
251 DM trials (0..250 step 1), ring depth 48, 31x31 background box, kappa 6.

One step = one push of a new frame through the whole path (ingest, shift-sum,
box centre / spread, S/N threshold + 3x3 local maximum, candidate ordering,
per-trial stats).  Metric: pixel * DM-trials per second (H*W*N_DM per frame).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--dtype fp32|fp16|bf16]
  python bench.py --impl reference ...     # the FP64 CPU oracle on the same metric
  python bench.py --workload serving|subband|stress

The default line also carries an FP16-storage measurement of the same workload
("fp16") and a short replay of the four-stream serving mix ("serving").

Under torchrun (N > 1) every rank runs an independent stream on its own GPU
(weak scaling, no collective on the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import datetime
import json
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

RESULT_SLOTS = 8                # result slots: up to 7 frames ahead of the oldest unpolled one
METRIC = "pixel*DM-trials/s"
WORKLOAD = "aartfaac-1024x1024-16sb-251dm-depth48-box31"
DTYPE_NAME = {"fp32": "f32", "fp16": "f16", "bf16": "bf16"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dtype", default="fp32", choices=["fp32", "fp16", "bf16"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp16", action="store_true", help="skip the FP16-storage sub-measurement")
    ap.add_argument("--serve-seconds", type=float, default=12.0,
                    help="length of the serving-mix replay in the default line (0: skip)")
    ap.add_argument("--pool", type=int, default=12, help="distinct synthetic frames cycled")
    ap.add_argument("--clip-iters", type=int, default=1,
                    help="subband workload: sigma-clip iterations (1 = one pass)")
    ap.add_argument("--gauss-sigma", type=float, default=0.0,
                    help="subband workload: Gaussian background kernel of this width in pixels on the "
                         "31x31 window (0 = the uniform box)")
    ap.add_argument("--suppress-steady", type=int, default=0,
                    help="steady-source suppression: K pushes in a row at zero delay (0 = off)")
    ap.add_argument("--qc", action="store_true",
                    help="quality control of every frame before the search (band and pixel scores)")
    ap.add_argument("--workload", default="aartfaac", choices=["aartfaac", "serving", "subband", "stress"],
                    help="serving: the four-stream FP16 mix through the C++ serving loop")
    ap.add_argument("--cadence", type=float, default=1.0, help="serving: frame cadence in seconds")
    ap.add_argument("--seconds", type=float, default=600.0, help="serving: length of the replay")
    ap.add_argument("--jitter", type=float, default=0.05, help="serving: arrival jitter, +- seconds")
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


def sources_sha256(sources):
    """SHA-256 of the files a kernel is compiled from (one path or a list, read in
    order and hashed as one byte string), relative to the repository root."""
    import hashlib
    h = hashlib.sha256()
    for src in [sources] if isinstance(sources, str) else sources:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def kernel_traffic(field="dram_bytes_per_launch", path=None):
    """A per-launch counter (DRAM bytes, or executed warp instructions) from the
    committed ncu capture, or None where a source of the kernel has changed since
    the counters were taken or the capture has no such counter."""
    path = path or os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return {}
    out = {}
    for k, v in rec.items():
        try:
            sha = sources_sha256(v["source"])
        except OSError:
            continue
        out[k] = v.get(field) if sha == v["sha256"] else None
    return out


def algorithmic_bytes(spec, delays, dtype):
    """Bytes a push must move at minimum (algorithmic count): the ring
    reads sum_f U_f H W b (every distinct delay plane read once) plus the ingest of
    the frame (F H W FP32 read, F H W b written); b = storage bytes."""
    b = 4 if dtype == "fp32" else 2
    HW = spec.H * spec.W
    lags = delays.max(axis=1)[:, None] - delays
    U = sum(len(np.unique(lags[:, f])) for f in range(spec.F))
    ring_reads = U * HW * b
    ingest = spec.F * HW * (4 + b)
    return dict(path=ring_reads + ingest, ring_reads=ring_reads, ingest=ingest, U=U)


class Clocks:
    """nvidia-smi sampling (10 ms) of SM clocks and throttle reasons, started before
    the ring fill; summary() keeps the samples taken inside a wall-clock window."""
    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        self.rows = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "10"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return
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
                if len(parts) < 10:
                    continue
                try:
                    ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                except ValueError:
                    continue
                rows.append([ts] + parts[1:])
        os.unlink(self.f.name)
        self.rows = rows

    def summary(self, t0, t1):
        """Samples inside [t0, t1]; if that window is shorter than the sampling period,
        the samples within 0.5 s of it (the same pushes, warm-up and e2e loop)."""
        if self.p is None or self.rows is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        win = "timed region"
        rows = [r for r in self.rows if t0 <= r[0] <= t1]
        if len(rows) < 3:
            rows = [r for r in self.rows if t0 - 0.5 <= r[0] <= t1 + 0.5]
            win = "timed region +- 0.5 s (warm-up and end-to-end pushes of the same stream)"
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        num = lambda v: v.replace(".", "", 1).isdigit()
        sm = [float(r[2]) for r in rows if num(r[2])]
        mx = [float(r[3]) for r in rows if num(r[3])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "window": win, "period_ms": 10}


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores (cpu_baseline and the reference arm): one
# spawned worker process per core; each step hands every worker DM trials of one
# push, the workers build the frames they read (untimed), meet at a barrier and
# run the oracle's search_push on their trials (timed).  The step's time is the
# first start to the last finish.
class _PlaneFrame:
    def __init__(self, planes, t):
        self.planes, self.t = planes, t

    def __getitem__(self, f):
        return self.planes[(self.t, f)]


def _oracle_worker(wid, dtype, seed, barrier, tasks, results):
    import synth as S
    from oracle import lpf_oracle as O
    spec = S.spec_aartfaac(dtype=dtype)
    st = S.SyntheticStream(spec, seed=seed)
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    dmax = delays.max(axis=1)
    while True:
        task = tasks.get()
        if task is None:
            return
        T, dms = task
        need = {}
        for d in dms:
            for f in range(spec.F):
                need.setdefault(int(T - dmax[d] + delays[d, f]), set()).add(f)
        planes = {}
        for t, fs in need.items():
            x = st.frame(t)
            for f in fs:
                planes[(t, f)] = O.storage_round(x[f], dtype) if dtype != "fp32" else x[f].astype(np.float64)
        barrier.wait()
        t_a = time.time()
        if dms:
            O.search_push(lambda t: _PlaneFrame(planes, t), T, delays, spec.box_r, spec.kappa, dms=dms)
        t_b = time.time()
        results.put((wid, t_a, t_b, len(dms)))


class OraclePool:
    def __init__(self, dtype, seed=1, max_workers=48):
        avail = len(os.sched_getaffinity(0))
        try:
            mem_gb = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES") / 2 ** 30
        except (ValueError, OSError):
            mem_gb = 16.0
        # about 0.5 GB per worker at 1024^2 (its planes and the oracle's temporaries)
        self.n = max(1, min(avail, max_workers, int(mem_gb / 0.5)))
        ctx = mp.get_context("spawn")
        self.barrier = ctx.Barrier(self.n)
        self.tasks = [ctx.Queue() for _ in range(self.n)]
        self.results = ctx.Queue()
        self.procs = [ctx.Process(target=_oracle_worker, args=(i, dtype, seed, self.barrier, self.tasks[i],
                                                               self.results), daemon=True)
                      for i in range(self.n)]
        for p in self.procs:
            p.start()

    def step(self, T, trials):
        """trials: one list of DM trials per worker.  Returns (seconds, trials run)."""
        for q, tr in zip(self.tasks, trials):
            q.put((int(T), [int(d) for d in tr]))
        res = [self.results.get(timeout=1800) for _ in range(self.n)]
        return max(r[2] for r in res) - min(r[1] for r in res), sum(r[3] for r in res)

    def close(self):
        for q in self.tasks:
            q.put(None)
        for p in self.procs:
            p.join(timeout=30)


def spread_trials(n_dm, n_workers, per_worker, offset=0):
    """per_worker DM trials for each worker, spread over the grid."""
    k = n_workers * per_worker
    picks = [int(v) % n_dm for v in np.linspace(0, n_dm - 1, k).round() + offset]
    return [picks[i::n_workers] for i in range(n_workers)]


def cpu_baseline(spec, delays, per_worker=2):
    """The FP64 oracle (as it stands) on the host cores: one push, per_worker DM trials
    per worker process."""
    pool = OraclePool(spec.dtype)
    try:
        T = int(delays.max())
        secs, n = pool.step(T, spread_trials(spec.n_dm, pool.n, per_worker))
    finally:
        pool.close()
    return {"value": spec.H * spec.W * n / secs, "unit": METRIC, "cores": pool.n, "kind": "oracle",
            "sample": f"one push (T={T}) of the {spec.H}x{spec.W} stream: {n} of {spec.n_dm} DM trials, "
                      f"{per_worker} per process, FP64 NumPy in {pool.n} spawned processes on "
                      f"{pool.n} host cores, {secs:.1f} s wall"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    spec = workload_spec(args.dtype)
    from oracle import lpf_oracle as O
    delays = O.delay_table(spec.freqs_mhz, spec.dm_grid, spec.cadence_s)
    T0 = int(delays.max())
    pool = OraclePool(spec.dtype)
    # one DM trial per worker per step; fewer workers per step for long runs, so that
    # the whole run stays within a few minutes
    per_step = pool.n if args.steps <= 40 else max(1, pool.n * 40 // args.steps)
    try:
        def trials(k):
            sel = spread_trials(spec.n_dm, per_step, 1, offset=k)
            return sel + [[] for _ in range(pool.n - per_step)]
        for w in range(args.warmup):
            pool.step(T0, trials(w))
        tot, n_tot = 0.0, 0
        for k in range(args.steps):
            secs, n = pool.step(T0 + (k % 4), trials(k))
            tot += secs
            n_tot += n
    finally:
        pool.close()
    val = spec.H * spec.W * n_tot / tot
    sample = (f"each step: {per_step} of {spec.n_dm} DM trials of one push of the {spec.H}x{spec.W} stream, "
              f"one per process, FP64 NumPy in {pool.n} spawned processes on {pool.n} host cores")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": METRIC, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "storage": args.dtype,
                                            "sample_dm_per_step": per_step},
            "cpu_baseline": {"value": val, "unit": METRIC, "cores": pool.n, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
def measure(lpf, torch, dev, spec, dtype, steps, warmup, pool_n, seed, qc=False, e2e_steps=0, dist=None,
            suppress_steady=0):
    """Device-timed steps of one stream (and, with e2e_steps, the end-to-end loop with
    host buffers).  The ring is filled first, so every trial is active."""
    st = synth.SyntheticStream(spec, seed=seed)
    pool = [torch.from_numpy(st.frame(t)) for t in range(pool_n)]
    pool_dev = [p.to(dev) for p in pool]
    pool_pin = [p.pin_memory() for p in pool] if e2e_steps else []
    cur = torch.cuda.Stream(dev)            # the search stream (the timing events are recorded on it)
    s = lpf.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                   box_r=spec.box_r, dtype=dtype, result_slots=RESULT_SLOTS, cuda_stream=cur,
                   qc=qc, qc_min_frames=16, suppress_steady=suppress_steady)
    out = {"info": s.info(), "delays": s.delay_table()}
    T = 0
    polled = []

    def push(T):
        s.push(pool_dev[T % pool_n], T)

    def poll():
        _, c, n, _ = s.poll(timeout_ms=600000, copy=False)   # records read in place
        polled.append(n)

    for _ in range(spec.depth + warmup):
        push(T)
        T += 1
        poll()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    s.kernel_times(reset=True)
    s.set_profiling(True)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    # result_slots - 1 pushes ahead of the oldest unpolled frame, as in the
    # end-to-end loop below
    ahead = max(1, RESULT_SLOTS - 1)
    out["t_wall0"] = time.time()
    host = [0.0, 0.0]                        # host seconds in push and poll calls
    ev0.record(cur)
    for k in range(steps):
        h0 = time.perf_counter()
        push(T)
        h1 = time.perf_counter()
        T += 1
        if k >= ahead:
            poll()
        host[0] += h1 - h0
        host[1] += time.perf_counter() - h1
    for _ in range(min(ahead, steps)):     # the frames still unpolled
        poll()
    ev1.record(cur)
    torch.cuda.synchronize()
    out["t_wall1"] = time.time()
    s.set_profiling(False)
    out["elapsed"] = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dist, dev)
    out["host_ms"] = {"push": 1e3 * host[0] / steps, "poll": 1e3 * host[1] / steps}
    kt = s.kernel_times(reset=True)
    out["per_push"] = {n: kt[n][0] / max(kt[n][1], 1) for n in kt}
    out["ncand"] = float(np.mean(polled[-steps:]))
    if e2e_steps:
        # end to end through the C ABI with host buffers: H2D of the frame, D2H of the
        # candidates, as a user streams frames: push frame T, then poll the oldest
        # frame once result_slots - 1 frames are in flight (the upload of T overlaps
        # the search of T - 1); latency is push call -> poll return of the same frame
        lat, e2e_cands, t_push = [], [], {}
        inflight = max(1, RESULT_SLOTS - 1)

        def poll_host():
            Tp, c, n, _ = s.poll(timeout_ms=600000, copy=False)
            e2e_cands.append(n)
            lat.append(time.perf_counter() - t_push.pop(Tp))

        torch.cuda.synchronize()
        t_e0 = time.perf_counter()
        for k in range(e2e_steps):
            t_push[T] = time.perf_counter()
            s.push_host(pool_pin[T % pool_n], T)
            T += 1
            if len(t_push) >= inflight + 1:
                poll_host()
        while t_push:
            poll_host()
        out["e2e_s"] = max_over_ranks(time.perf_counter() - t_e0, dist, dev)
        out["lat"], out["e2e_cands"] = lat, e2e_cands
        out["t_wall1e"] = time.time()
        # the host link alone: pinned frame -> device, CUDA events, 10 copies
        dst = torch.empty_like(pool_dev[0])
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(cur):
            dst.copy_(pool_pin[0], non_blocking=True)
            c0.record(cur)
            for _ in range(10):
                dst.copy_(pool_pin[0], non_blocking=True)
            c1.record(cur)
        torch.cuda.synchronize()
        out["h2d_gbs"] = 10 * dst.numel() * dst.element_size() / (c0.elapsed_time(c1) / 1e3) / 1e9
    s.close()
    return out


def path_roofline(spec, dtype, delays, ms_per_step, hbm_peak, peak_src, traffic=None):
    nb = algorithmic_bytes(spec, delays, dtype)
    ach = nb["path"] / (ms_per_step / 1e3) / 1e9
    return {"kernel": "whole push (ingest, shift-sum, filter, detect; the step)", "bound": "hbm",
            "achieved": ach, "peak": hbm_peak, "unit": "GB/s", "frac": ach / hbm_peak, "peak_source": peak_src,
            "traffic": traffic, "algorithmic_bytes_per_step": nb["path"],
            "note": "algorithmic bytes: sum over subbands of the distinct delay planes read once "
                    f"({nb['U']} planes) + ingest of the frame; CUDA-event time of the whole step"}


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
    clocks = Clocks(local)
    clocks.start()                     # before the ring fill, so the short timed region has samples
    spec = workload_spec(args.dtype)
    m = measure(lpf, torch, dev, spec, args.dtype, args.steps, args.warmup, args.pool, 1 + rank, qc=args.qc,
                e2e_steps=args.e2e_steps, dist=dist, suppress_steady=args.suppress_steady)
    f16 = None
    if not args.no_fp16 and args.dtype == "fp32" and not args.qc:
        f16 = measure(lpf, torch, dev, workload_spec("fp16"), "fp16", args.steps, args.warmup, args.pool,
                      1 + rank, dist=dist)
    clocks.stop()
    serving = None
    if rank == 0 and ws == 1 and args.serve_seconds > 0:
        serving = serve_mix(lpf, seconds=args.serve_seconds, cadence=1.0, jitter=0.05)
    if rank != 0:
        return
    info, delays, per_push = m["info"], m["delays"], m["per_push"]
    elapsed = m["elapsed"]
    pix_dm = spec.H * spec.W * spec.n_dm
    value = pix_dm * args.steps * ws / elapsed
    ms_step = 1e3 * elapsed / args.steps
    e2e_value = pix_dm * args.e2e_steps * ws / m["e2e_s"] if args.e2e_steps else None
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
    # the committed captures: per storage type for the shift-sum, FP32 and FP16 for the filter
    fkey = "k_filter_res" if args.dtype == "fp32" else "k_filter_res_" + args.dtype
    HW = spec.H * spec.W
    nd = info["n_distinct"]
    nb = algorithmic_bytes(spec, delays, args.dtype)
    # the shift-sum: its algorithmic bytes are the ring reads only (the D - C images it
    # writes are an intermediate of this design, not work the method requires)
    dd_ms = per_push["dedisperse"]
    dd_ach = nb["ring_reads"] / (dd_ms / 1e3) / 1e9
    roof_dd = {"kernel": "k_dedisperse (shift-sum)", "bound": "hbm", "achieved": dd_ach, "peak": hbm_peak,
               "unit": "GB/s", "frac": dd_ach / hbm_peak, "peak_source": peak_src,
               "traffic": traffic.get("k_dedisperse_" + args.dtype),
               "algorithmic_bytes_per_launch": nb["ring_reads"], "avg_launch_ms": dd_ms, "launches_per_step": 1}
    f_ms = per_push["filter_detect"]
    f_ops = FILTER_OPS_PER_PIXEL_TRIAL * HW * nd
    f_ach = f_ops / (f_ms / 1e3) / 1e12
    roof_f = {"kernel": "k_filter_res<15> (box spread, S/N, threshold, stats)", "bound": "alu",
              "achieved": f_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": f_ach / alu_peak,
              "peak_source": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz",
              "traffic": traffic.get(fkey),
              "algorithmic_flop_per_launch": f_ops, "avg_launch_ms": f_ms, "launches_per_step": 1}
    # the filter is bound by instruction issue: executed warp instructions per launch
    # (ncu) over the event-timed launch, against 4 schedulers per SM at the clock
    f_inst = kernel_traffic("warp_inst_per_launch").get(fkey)
    issue_peak = sms * 4 * sm_mhz * 1e6 / 1e12
    roof_f_issue = {"kernel": "k_filter_res<15> (instruction issue)", "bound": "issue",
                    "achieved": f_inst / (f_ms / 1e3) / 1e12 if f_inst else None, "peak": issue_peak,
                    "unit": "T warp-instructions/s",
                    "frac": f_inst / (f_ms / 1e3) / 1e12 / issue_peak if f_inst else None,
                    "peak_source": f"{sms} SMs x 4 schedulers x {sm_mhz:.0f} MHz",
                    "warp_instructions_per_launch": f_inst, "avg_launch_ms": f_ms}
    step_traffic = None
    tr_keys = ["k_dedisperse_" + args.dtype, fkey]
    if all(traffic.get(k) for k in tr_keys):
        # DRAM bytes of the main-stream kernels that move the bulk (ncu, one launch each)
        step_traffic = sum(traffic[k] for k in tr_keys)
    roof = path_roofline(spec, args.dtype, delays, ms_step, hbm_peak, peak_src, step_traffic)
    if step_traffic:
        roof["traffic_note"] = "ncu DRAM bytes of k_dedisperse + k_filter_res per push"
    rooflines = [roof, roof_dd, roof_f, roof_f_issue]
    if args.qc:
        # quality control + ingest (k_qc_scan, k_qc_decide, k_residual, k_ingest_qc): the
        # QC passes read the frame and the running mean and m2 twice and write them once
        b = 4 if args.dtype == "fp32" else 2
        qc_bytes = spec.F * HW * (12 + 20 + b)
        qc_ms = per_push["ingest"] + per_push.get("ring_write", 0.0)
        rooflines.append({"kernel": "quality control + ingest (k_qc_scan, k_qc_decide, k_ingest_qc, k_residual)",
                          "bound": "hbm", "achieved": qc_bytes / (qc_ms / 1e3) / 1e9, "peak": hbm_peak,
                          "unit": "GB/s", "frac": qc_bytes / (qc_ms / 1e3) / 1e9 / hbm_peak,
                          "peak_source": peak_src, "traffic": None, "algorithmic_bytes_per_launch": qc_bytes,
                          "avg_launch_ms": qc_ms, "launches_per_step": 1})
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_NAME[args.dtype],
        "data": "synthetic (seeded AARTFAAC-shaped stream: noise, 3-sigma cosine gradient, "
                "500 Gaussian-PSF sources, 20 dispersed pulses)",
        "config": {"workload": WORKLOAD, "H": spec.H, "W": spec.W, "subbands": spec.F,
                   "dm_trials": spec.n_dm, "depth": spec.depth, "box": 2 * spec.box_r + 1,
                   "storage": args.dtype, "arithmetic": "f32 (delay table f64, statistics f64)",
                   "distinct_delay_rows": nd, "quality_control": bool(args.qc),
                   "suppress_steady": args.suppress_steady,
                   "l2": "inputs larger than L2 (ring %.2f GB)" % (info["ring_bytes"] / 1e9),
                   "parallelism": f"{ws} independent stream(s), one per GPU"},
        "gpu_launches": int(args.steps * launches_per_push(spec, args.qc, args.suppress_steady)),
        "roofline": roof,
        "rooflines": rooflines,
        "kernel_ms_per_step": per_push,
        "candidates_per_step": m["ncand"],
        "host_ms_per_step": m["host_ms"],
        "clocks": clocks.summary(m["t_wall0"], m["t_wall1"]),
    }
    if e2e_value is not None:
        line["e2e"] = {"value": e2e_value, "unit": METRIC,
                       "h2d_bytes_per_step": spec.F * spec.H * spec.W * 4,
                       "d2h_bytes_per_step": int(np.mean(m["e2e_cands"]) * 24 + spec.n_dm * 16),
                       "h2d_link_gbs": m["h2d_gbs"],
                       "note": "frames are uploaded while earlier ones are searched: a step takes the "
                               "longer of the search and the upload over the host link"}
        line["latency_ms"] = {"p50": 1e3 * float(np.percentile(m["lat"], 50)),
                              "p99": 1e3 * float(np.percentile(m["lat"], 99)),
                              "what": f"push_frame_host -> poll of the same frame, up to {RESULT_SLOTS} "
                                      "frames in flight"}
    if f16 is not None:
        sp16 = workload_spec("fp16")
        tr16 = ["k_dedisperse_fp16", "k_filter_res_fp16"]
        traffic16 = sum(traffic[k] for k in tr16) if all(traffic.get(k) for k in tr16) else None
        ms16 = 1e3 * f16["elapsed"] / args.steps
        line["fp16"] = {"storage": "fp16", "ms_per_step": ms16, "value": pix_dm * args.steps * ws / f16["elapsed"],
                        "speedup_vs_fp32": ms_step / ms16,
                        "roofline": path_roofline(sp16, "fp16", f16["delays"], ms16, hbm_peak, peak_src,
                                                  traffic16),
                        "kernel_ms_per_step": f16["per_push"], "candidates_per_step": f16["ncand"],
                        "host_ms_per_step": f16["host_ms"],
                        "clocks": clocks.summary(f16["t_wall0"], f16["t_wall1"])}
    if serving is not None:
        line["serving"] = serving
    if ws == 1:
        line["cnn"] = cnn_throughput(lpf, torch)
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(spec, delays)
    print(json.dumps(line), flush=True)


def cnn_throughput(lpf, torch, n=10000, F=32, Tw=64, steps=20, warmup=3):
    """The parameter-inference network on n F x Tw spectra already on the device
    (synthetic noise, fixed random weights): spectra per second, CUDA-event timed
    on the network's stream."""
    st = torch.cuda.Stream()
    x = torch.randn((n, F, Tw), device="cuda", dtype=torch.float32)
    out = torch.empty((n, 5), device="cuda", dtype=torch.float32)
    with lpf.Cnn(F, Tw, synth.cnn_params(3), max_batch=n, cuda_stream=st) as net:
        torch.cuda.synchronize()
        for _ in range(warmup):
            net.forward(x, out=out, sync=False)
        net.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(steps):
            net.forward(x, out=out, sync=False)
        e1.record(st)
        net.sync()
        ms = e0.elapsed_time(e1) / steps
    flops = n * 2 * (F * Tw * 9 * 16 + (F // 2) * (Tw // 2) * 144 * 32 + (F // 4) * (Tw // 4) * 288 * 64)
    return {"workload": f"{n} dynamic spectra of {F} x {Tw} (conv 1->16, 16->32, 32->64, head 64->5)",
            "ms_per_batch": ms, "spectra_per_s": n / (ms / 1e3), "tflops": flops / (ms / 1e3) / 1e12,
            "flop_per_batch": flops}


def launches_per_push(spec, qc, suppress_steady=0):
    """Kernels of one push: residuals, counter reset, shift-sum, ring write, filter,
    3x3 pass, 4 ordering kernels (count, scan, scatter, sort + format), statistics
    (+ 2 with quality control, + 2 with steady-source suppression: run-length
    update and drop; the zero-delay marks are set by the kernels that find the
    candidates, after a memset of the lane's bit map)."""
    return 11 + (2 if qc else 0) + (2 if suppress_steady else 0)


# ---------------------------------------------------------------------------
def serve_mix(lpf, seconds, cadence, jitter, seed=7):
    """The four-stream FP16 serving mix replayed through the C++ serving loop: the
    2048^2/16/501 and 1024^2/16/251 streams and a 512^2/8/128 stream for the whole
    replay; a second 512^2 stream for its first half, closed there, and a third
    opened in its place for the second half (four live streams throughout).  Frame
    T of a stream is submitted at (T + k/4) * cadence +- jitter (uniform, seeded).
    Reports submit -> fetch latency (the fetching thread's wall clock) and the
    aggregate pixel * DM-trials/s served."""
    specs = synth.spec_serving_mix()
    late = synth.StreamSpec(**{**specs[3].__dict__, "name": "mix-512c"})
    n = max(2, int(round(seconds / cadence)))
    half = n // 2
    # (spec, first frame slot, frames): the slot is the cadence tick of its frame 0
    plan = [(specs[0], 0, n), (specs[1], 0, n), (specs[2], 0, n), (specs[3], 0, half), (late, half, n - half)]
    pools = []
    for i, (sp, _, _) in enumerate(plan):
        st = synth.SyntheticStream(sp, seed=60 + i)
        pools.append([st.frame(t) for t in range(4)])
    budget = 80 << 30
    rng = np.random.default_rng(seed)
    lat = {i: [] for i in range(len(plan))}
    submit_t = {}
    lock = threading.Lock()
    with lpf.Server(budget, max_streams=8) as srv:
        ids = [None] * len(plan)

        def drain(i, count):
            while ids[i] is None:
                time.sleep(0.001)
            for _ in range(count):
                T, c, nf, _ = srv.fetch(ids[i], timeout_ms=600000)
                t = time.perf_counter()
                with lock:
                    lat[i].append(1e3 * (t - submit_t.pop((i, T))))
        events = []
        for i, (sp, first, cnt) in enumerate(plan):
            for T in range(cnt):
                events.append(((first + T + i / 4.0) * cadence + rng.uniform(-jitter, jitter), i, T))
        events.sort()
        threads = [threading.Thread(target=drain, args=(i, cnt)) for i, (_, _, cnt) in enumerate(plan)]
        for th in threads:
            th.start()
        t0 = time.perf_counter()
        for due, i, T in events:
            sp, first, cnt = plan[i]
            if ids[i] is None:
                ids[i] = srv.open_stream(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, kappa=sp.kappa,
                                         box_r=sp.box_r, dtype=sp.dtype)
            wait = t0 + max(due, 0.0) - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            while True:
                with lock:
                    submit_t[(i, T)] = time.perf_counter()
                if srv.submit(ids[i], pools[i][T % 4], T) != lpf.LPF_E_BUSY:
                    break
                time.sleep(0.0005)
            if T == cnt - 1 and cnt < n:
                srv.close_stream(ids[i])          # stream leaves mid-replay
        for th in threads:
            th.join()
        wall = time.perf_counter() - t0
        st_all = srv.stats()
    all_lat = np.concatenate([np.asarray(v) for v in lat.values()])
    pixdm = sum(sp.H * sp.W * sp.n_dm * cnt for sp, _, cnt in plan)
    return {"workload": "serving-mix-4-streams-fp16 (2048^2/16/501, 1024^2/16/251, 512^2/8/128, "
                        "512^2/8/128 closed at half time and replaced by a third)",
            "seconds": seconds, "cadence_s": cadence, "jitter_s": jitter, "frames": int(len(all_lat)),
            "p50_ms": float(np.percentile(all_lat, 50)), "p99_ms": float(np.percentile(all_lat, 99)),
            "max_ms": float(all_lat.max()),
            "per_stream_p99_ms": {plan[i][0].name: float(np.percentile(v, 99)) for i, v in lat.items() if v},
            "pixel_dm_per_s": pixdm / wall, "latency": "submit -> fetch return (host wall clock)",
            "hbm_budget_bytes": budget, "peak_used_bytes": st_all["used_bytes"]}


def run_serving(args):
    """The serving mix of the default line at full length (config: 10 minutes)."""
    import paper_2103_15418_b300 as lpf
    res = serve_mix(lpf, seconds=args.seconds, cadence=args.cadence, jitter=args.jitter)
    res["metric"] = METRIC
    print(json.dumps(res), flush=True)


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


def run_stress(args):
    """Stress workload: 2048^2 px, 32 subbands (57.6-63.85 MHz), 1001 DM trials, FP16
    ring of depth 114 (the DM 500 sweep spans 113 frames).  Each step pushes a frame,
    polls the oldest unpolled one, gathers the 32 x 64 FP32 dynamic spectra of its
    candidates and runs the parameter-inference network on them; frames per second
    against the 1 s cadence is the real-time factor.
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
    cnn_out = torch.empty((16384, 5), dtype=torch.float32, device="cuda")
    net = lpf.Cnn(spec.F, Tw, synth.cnn_params(3), max_batch=16384, cuda_stream=cur)

    def poll_and_gather():
        Tp, c, n, _ = s.poll(timeout_ms=600000)
        g = 0
        if len(c) and Tp >= Tw - 1:         # once Tw frames exist
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            e[0].record(cur)
            c = c[: gbuf.shape[0]]
            s.dynspec(c, Tw, out=gbuf[: len(c)], sync=False)   # [n, 32, 64] FP32 on the search stream
            net.forward(gbuf[: len(c)], out=cnn_out[: len(c)], sync=False)   # mu, L of every candidate
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
    for _ in range(min(ahead, args.steps)):     # the frames still unpolled
        poll_and_gather()
    ev1.record(cur)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    kt = s.kernel_times(reset=True)
    s.close()
    per_push = {n: kt[n][0] / max(kt[n][1], 1) for n in kt}
    per_push["dynspec_gather_and_cnn"] = float(np.mean([a.elapsed_time(b) for a, b in gev])) if gev else 0.0
    net.close()
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
