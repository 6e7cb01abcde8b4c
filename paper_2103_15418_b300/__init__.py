"""Python binding of liblpf, the B300 image-plane dispersed-transient search.

Argument marshalling only: every step of the search runs in the CUDA kernels of
liblpf.so (built in-tree by build.py for sm_103a).  PyTorch is used for device
memory and CUDA streams.  There is no CPU fallback: if the library cannot be
loaded, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, Structure, c_char_p, c_double, c_float, c_int, c_int32, c_int64,
                    c_size_t, c_void_p)
from typing import Dict, Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblpf.so")

LPF_OK = 0
LPF_E_ARG, LPF_E_DEPTH, LPF_E_ORDER, LPF_E_OOM, LPF_E_BUDGET = -1, -2, -3, -4, -5
LPF_E_TRUNCATED, LPF_E_STALE, LPF_E_TIMEOUT, LPF_E_CUDA = -6, -7, -8, -9
LPF_E_BUSY, LPF_E_NODATA, LPF_E_CAPACITY = -10, -11, -12
LPF_STATIC_DYNSPEC_MAX = 65536      # records accepted by lpf_extract_dynspec_static
DTYPES = {"fp32": 0, "fp16": 1, "bf16": 2}

# Every exported symbol declared in include/lpf.h (checked by the CPU tests).
EXPORTS = [
    "lpf_default_params", "lpf_stream_open", "lpf_push_frame", "lpf_push_frame_host",
    "lpf_poll_candidates", "lpf_extract_dynspec", "lpf_get_delay_table", "lpf_get_stats",
    "lpf_stream_info", "lpf_stream_sync", "lpf_stream_close", "lpf_strerror", "lpf_get_qc",
    "lpf_set_profiling", "lpf_get_kernel_times", "lpf_extract_dynspec_static",
    "lpf_stream_footprint", "lpf_server_open", "lpf_server_open_stream", "lpf_server_submit",
    "lpf_server_fetch", "lpf_server_close_stream", "lpf_server_stream_state", "lpf_server_stats",
    "lpf_server_close", "lpf_cnn_param_count", "lpf_cnn_open", "lpf_cnn_forward", "lpf_cnn_sync",
    "lpf_cnn_close",
]
SERVE_PENDING, SERVE_ACTIVE, SERVE_CLOSED = 0, 1, 3
MODES = {"dispersed": 0, "subband": 1}
KERNELS = {"box": 0, "gauss": 1}


class Params(Structure):
    _fields_ = [("cadence_s", c_double), ("kappa", c_float), ("box_r", c_int), ("lmax_r", c_int),
                ("dtype", c_int), ("cand_cap", c_int), ("dyn_box_r", c_int),
                ("result_slots", c_int), ("cuda_stream", c_void_p), ("filter_impl", c_int),
                ("qc", c_int), ("qc_z", c_float), ("qc_zeta", c_float), ("qc_min_frames", c_int),
                ("mode", c_int), ("clip_iters", c_int), ("kernel", c_int), ("gauss_sigma", c_float),
                ("suppress_steady", c_int)]


class Candidate(Structure):
    _fields_ = [("t0", c_int64), ("dm_idx", c_int32), ("y", c_int32), ("x", c_int32),
                ("snr", c_float)]


class ServeStats(Structure):
    _fields_ = [("frames", c_int64), ("p50_ms", c_double), ("p99_ms", c_double), ("max_ms", c_double),
                ("pixel_dm_per_s", c_double), ("budget_bytes", c_size_t), ("used_bytes", c_size_t)]


class StreamInfo(Structure):
    _fields_ = [("H", c_int), ("W", c_int), ("F", c_int), ("n_dm", c_int), ("depth", c_int),
                ("dtype", c_int), ("n_distinct", c_int), ("max_delay", c_int),
                ("ring_bytes", c_size_t), ("device_bytes", c_size_t),
                ("frames_pushed", c_int64), ("last_T", c_int64)]


CANDIDATE_DTYPE = np.dtype([("t0", "<i8"), ("dm_idx", "<i4"), ("y", "<i4"), ("x", "<i4"),
                            ("snr", "<f4")])
assert CANDIDATE_DTYPE.itemsize == ctypes.sizeof(Candidate) == 24

_lib = None


class LpfError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib.lpf_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{what}: {msg} ({code})" if what else f"{msg} ({code})")


def _host_records(n: int):
    """A reusable host array of n candidate records and the object owning its memory,
    page-locked where CUDA can pin it (the poll's device-to-host copy is then one
    DMA, not a staged copy)."""
    try:
        import torch
        t = torch.empty(n * CANDIDATE_DTYPE.itemsize, dtype=torch.uint8, pin_memory=True)
        return t.numpy().view(CANDIDATE_DTYPE), t
    except Exception:
        return np.zeros(n, dtype=CANDIDATE_DTYPE), None


def load(path: Optional[str] = None):
    """Load liblpf.so (building it first if it is missing) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        from . import build as _build
        _build.build()
    lib = ctypes.CDLL(path)
    lib.lpf_default_params.argtypes = [POINTER(Params)]
    lib.lpf_default_params.restype = None
    lib.lpf_stream_open.argtypes = [POINTER(c_void_p), c_int, c_int, c_int, POINTER(c_double), c_int,
                                    POINTER(c_double), c_int, POINTER(Params)]
    lib.lpf_push_frame.argtypes = [c_void_p, c_void_p, c_int64]
    lib.lpf_push_frame_host.argtypes = [c_void_p, c_void_p, c_int64]
    lib.lpf_poll_candidates.argtypes = [c_void_p, c_void_p, c_int, POINTER(c_int), POINTER(c_int64), c_int]
    lib.lpf_extract_dynspec.argtypes = [c_void_p, c_void_p, c_int, c_int, c_void_p]
    lib.lpf_get_delay_table.argtypes = [c_void_p, c_void_p]
    lib.lpf_get_stats.argtypes = [c_void_p, c_void_p]
    lib.lpf_get_qc.argtypes = [c_void_p, POINTER(c_int64), POINTER(ctypes.c_uint32), c_void_p]
    lib.lpf_stream_info.argtypes = [c_void_p, POINTER(StreamInfo)]
    lib.lpf_stream_sync.argtypes = [c_void_p]
    lib.lpf_stream_close.argtypes = [c_void_p]
    lib.lpf_strerror.argtypes = [c_int]
    lib.lpf_strerror.restype = c_char_p
    lib.lpf_set_profiling.argtypes = [c_void_p, c_int]
    lib.lpf_get_kernel_times.argtypes = [c_void_p, POINTER(c_char_p), POINTER(c_double),
                                         POINTER(c_int64), c_int, c_int]
    lib.lpf_stream_footprint.argtypes = [c_int, c_int, c_int, POINTER(c_double), c_int, POINTER(c_double),
                                         c_int, POINTER(Params), POINTER(c_size_t)]
    lib.lpf_server_open.argtypes = [POINTER(c_void_p), c_size_t, c_int]
    lib.lpf_server_open_stream.argtypes = [c_void_p, c_int, c_int, c_int, POINTER(c_double), c_int,
                                           POINTER(c_double), c_int, POINTER(Params), POINTER(c_int)]
    lib.lpf_server_submit.argtypes = [c_void_p, c_int, c_void_p, c_int64]
    lib.lpf_server_fetch.argtypes = [c_void_p, c_int, c_void_p, c_int, POINTER(c_int), POINTER(c_int64),
                                     POINTER(c_double), c_int]
    lib.lpf_server_close_stream.argtypes = [c_void_p, c_int]
    lib.lpf_server_stream_state.argtypes = [c_void_p, c_int, POINTER(c_int)]
    lib.lpf_server_stats.argtypes = [c_void_p, c_int, POINTER(ServeStats)]
    lib.lpf_server_close.argtypes = [c_void_p]
    lib.lpf_cnn_param_count.argtypes = []
    lib.lpf_cnn_param_count.restype = c_size_t
    lib.lpf_cnn_open.argtypes = [POINTER(c_void_p), c_int, c_int, c_void_p, c_size_t, c_int, c_void_p]
    lib.lpf_cnn_forward.argtypes = [c_void_p, c_void_p, c_int, c_void_p]
    lib.lpf_cnn_sync.argtypes = [c_void_p]
    lib.lpf_cnn_close.argtypes = [c_void_p]
    _lib = lib
    return lib


def _host_frame_ptr(frame, n: int) -> int:
    """Address of a host frame of n FP32 values in C order (numpy array or CPU
    tensor).  The library reads exactly 4 n bytes from it, so anything else (a
    CUDA tensor, another dtype, a strided view, another size) is refused here."""
    if hasattr(frame, "data_ptr"):
        if frame.is_cuda:
            raise ValueError("push_host takes a host frame; use push for a CUDA tensor")
        if str(frame.dtype) != "torch.float32" or not frame.is_contiguous() or frame.numel() != n:
            raise ValueError(f"frame must be a contiguous float32 tensor of {n} values")
        return frame.data_ptr()
    a = frame
    if not isinstance(a, np.ndarray) or a.dtype != np.float32 or not a.flags["C_CONTIGUOUS"] or a.size != n:
        raise ValueError(f"frame must be a C-contiguous float32 array of {n} values")
    return a.ctypes.data


def _out_ptr(out, shape) -> int:
    """Address of a caller-supplied output: a contiguous FP32 CUDA tensor of
    exactly this shape (the gather writes prod(shape) values through it)."""
    if not getattr(out, "is_cuda", False) or str(out.dtype) != "torch.float32" or not out.is_contiguous():
        raise ValueError("out must be a contiguous float32 CUDA tensor")
    if tuple(out.shape) != tuple(shape):
        raise ValueError(f"out has shape {tuple(out.shape)}, expected {tuple(shape)}")
    return out.data_ptr()


def _check(rc: int, what: str):
    if rc != LPF_OK:
        raise LpfError(rc, what)


def make_params(*, cadence_s: float = 1.0, kappa: float = 6.0, box_r: int = 15, dtype: str = "fp32",
                cand_cap: int = 1 << 20, dyn_box_r: int = 0, result_slots: int = 2,
                filter_impl: str = "auto", qc: bool = False, qc_z: float = 5.0, qc_zeta: float = 20.0,
                qc_min_frames: int = 128, mode: str = "dispersed", lmax_r: int = 1,
                clip_iters: int = 1, kernel: str = "box", gauss_sigma: float = 0.0,
                suppress_steady: int = 0) -> "Params":
    p = default_params()
    p.cadence_s, p.kappa, p.box_r = cadence_s, kappa, box_r
    p.dtype, p.cand_cap, p.dyn_box_r, p.result_slots = DTYPES[dtype], cand_cap, dyn_box_r, result_slots
    p.filter_impl = {"auto": 0, "tiled": 1, "streaming": 2}[filter_impl]
    p.qc, p.qc_z, p.qc_zeta, p.qc_min_frames = int(bool(qc)), qc_z, qc_zeta, qc_min_frames
    p.mode, p.lmax_r, p.clip_iters = MODES[mode], lmax_r, clip_iters
    p.kernel, p.gauss_sigma = KERNELS[kernel], gauss_sigma
    p.suppress_steady = int(suppress_steady)
    return p


def footprint(H: int, W: int, freqs_mhz, dm_grid, depth: int, **kw) -> int:
    """Device bytes a stream with these arguments allocates (host-side plan, no GPU)."""
    f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
    d = np.zeros(0) if dm_grid is None else np.ascontiguousarray(dm_grid, dtype=np.float64)
    p = make_params(**kw)
    out = c_size_t(0)
    _check(load().lpf_stream_footprint(int(H), int(W), len(f), f.ctypes.data_as(POINTER(c_double)), len(d),
                                       d.ctypes.data_as(POINTER(c_double)) if len(d) else None, int(depth),
                                       ctypes.byref(p),
                                       ctypes.byref(out)), "lpf_stream_footprint")
    return int(out.value)


def default_params() -> Params:
    p = Params()
    load().lpf_default_params(ctypes.byref(p))
    return p


class Stream:
    """One image stream: ring buffer, delay table and search state on one GPU."""

    def __init__(self, H: int, W: int, freqs_mhz, dm_grid, depth: int, *, cadence_s: float = 1.0,
                 kappa: float = 6.0, box_r: int = 15, dtype: str = "fp32", cand_cap: int = 1 << 20,
                 dyn_box_r: int = 0, result_slots: int = 2, cuda_stream=None,
                 filter_impl: str = "auto", qc: bool = False, qc_z: float = 5.0, qc_zeta: float = 20.0,
                 qc_min_frames: int = 128, mode: str = "dispersed", lmax_r: int = 1, clip_iters: int = 1,
                 kernel: str = "box", gauss_sigma: float = 0.0, suppress_steady: int = 0):
        """mode "subband": the per-subband detector (dm_grid ignored, may be None; a
        candidate's dm_idx is its band, t0 its frame; lmax_r 3 gives the paper's 7x7
        maximum filter; kernel "gauss" with gauss_sigma s: the Gaussian background
        kernel on the (2 box_r + 1)^2 window).  suppress_steady K > 0: drop the
        candidates of dispersed trials at pixels that were zero-delay candidates in
        the K most recent pushes (lpf.h)."""
        lib = load()
        self.H, self.W = int(H), int(W)
        self.freqs = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
        band = mode == "subband"
        self.dms = np.zeros(0) if band else np.ascontiguousarray(dm_grid, dtype=np.float64)
        self.F, self.depth = len(self.freqs), int(depth)
        self.n_dm = self.F if band else len(self.dms)
        p = make_params(cadence_s=cadence_s, kappa=kappa, box_r=box_r, dtype=dtype, cand_cap=cand_cap,
                        dyn_box_r=dyn_box_r, result_slots=result_slots, filter_impl=filter_impl, qc=qc,
                        qc_z=qc_z, qc_zeta=qc_zeta, qc_min_frames=qc_min_frames, mode=mode, lmax_r=lmax_r,
                        clip_iters=clip_iters, kernel=kernel, gauss_sigma=gauss_sigma,
                        suppress_steady=suppress_steady)
        if cuda_stream is not None:
            p.cuda_stream = int(getattr(cuda_stream, "cuda_stream", cuda_stream))
        self.params = p
        self._cap = int(cand_cap)
        h = c_void_p()
        _check(lib.lpf_stream_open(ctypes.byref(h), self.H, self.W, self.F,
                                   self.freqs.ctypes.data_as(POINTER(c_double)), len(self.dms),
                                   self.dms.ctypes.data_as(POINTER(c_double)) if len(self.dms) else None,
                                   self.depth, ctypes.byref(p)), "lpf_stream_open")
        self._h = h
        self._out, self._out_owner = _host_records(self._cap)

    # ---------------------------------------------------------------- pushes
    def push(self, frame, T: int) -> None:
        """frame: CUDA float32 tensor [F, H, W], contiguous, on this stream's device."""
        if not (frame.is_cuda and frame.dtype.__str__() == "torch.float32" and frame.is_contiguous()):
            raise ValueError("frame must be a contiguous float32 CUDA tensor")
        if tuple(frame.shape) != (self.F, self.H, self.W):
            raise ValueError(f"frame shape {tuple(frame.shape)} != {(self.F, self.H, self.W)}")
        _check(load().lpf_push_frame(self._h, c_void_p(frame.data_ptr()), int(T)), "lpf_push_frame")

    def push_host(self, frame, T: int) -> None:
        """frame: host float32 array/tensor [F, H, W], C order (pinned for asynchronous copies)."""
        ptr = _host_frame_ptr(frame, self.F * self.H * self.W)
        _check(load().lpf_push_frame_host(self._h, c_void_p(ptr), int(T)), "lpf_push_frame_host")

    def poll(self, cap: Optional[int] = None, timeout_ms: int = -1, copy: bool = True):
        """Candidates of the oldest unpolled frame: (T, records, n_found, truncated).
        copy=False returns a view of the stream's page-locked record buffer instead
        of a copy; it is overwritten by the next poll."""
        cap = self._cap if cap is None else int(cap)
        buf = self._out if cap <= self._out.size else np.zeros(cap, dtype=CANDIDATE_DTYPE)
        n = c_int(0)
        T = c_int64(-1)
        rc = load().lpf_poll_candidates(self._h, c_void_p(buf.ctypes.data), cap, ctypes.byref(n),
                                        ctypes.byref(T), int(timeout_ms))
        if rc not in (LPF_OK, LPF_E_TRUNCATED):
            raise LpfError(rc, "lpf_poll_candidates")
        k = min(n.value, cap, self._cap)
        return T.value, (buf[:k].copy() if copy else buf[:k]), n.value, rc == LPF_E_TRUNCATED

    def dynspec(self, cands, Tw: int, out=None, sync: bool = True):
        """FP32 CUDA tensor [n, F, Tw] of the candidates' dynamic spectra (last polled frame).
        The gather is enqueued on the stream's CUDA stream; sync=True waits for the
        stream, so the tensor may be read from any torch stream.  sync=False leaves it
        to the caller (work that follows on the CUDA stream given at construction is
        ordered after the gather)."""
        import torch
        c = np.ascontiguousarray(cands, dtype=CANDIDATE_DTYPE)
        n = len(c)
        if out is None:
            out = torch.empty((n, self.F, Tw), dtype=torch.float32, device="cuda")
        optr = _out_ptr(out, (n, self.F, int(Tw))) if n else 0
        _check(load().lpf_extract_dynspec(self._h, c_void_p(c.ctypes.data) if n else None, n, int(Tw),
                                          c_void_p(optr) if n else None),
               "lpf_extract_dynspec")
        if sync:
            self.sync()
        return out

    # ---------------------------------------------------------------- queries
    def delay_table(self) -> np.ndarray:
        out = np.zeros((self.n_dm, self.F), dtype=np.int32)
        _check(load().lpf_get_delay_table(self._h, c_void_p(out.ctypes.data)), "lpf_get_delay_table")
        return out

    def stats(self) -> np.ndarray:
        out = np.zeros((self.n_dm, 2), dtype=np.float64)
        _check(load().lpf_get_stats(self._h, c_void_p(out.ctypes.data)), "lpf_get_stats")
        return out

    def qc(self):
        """Quality control of the last polled frame: (T, discarded [F] bool, z [F])."""
        T = c_int64(-1)
        m = ctypes.c_uint32(0)
        z = np.zeros(self.F, dtype=np.float32)
        _check(load().lpf_get_qc(self._h, ctypes.byref(T), ctypes.byref(m), c_void_p(z.ctypes.data)),
               "lpf_get_qc")
        disc = np.array([(m.value >> f) & 1 for f in range(self.F)], dtype=bool)
        return T.value, disc, z

    def info(self) -> Dict[str, int]:
        i = StreamInfo()
        _check(load().lpf_stream_info(self._h, ctypes.byref(i)), "lpf_stream_info")
        return {k: getattr(i, k) for k, _ in StreamInfo._fields_}

    def sync(self) -> None:
        _check(load().lpf_stream_sync(self._h), "lpf_stream_sync")

    def set_profiling(self, on: bool) -> None:
        _check(load().lpf_set_profiling(self._h, 1 if on else 0), "lpf_set_profiling")

    def kernel_times(self, reset: bool = False) -> Dict[str, Tuple[float, int]]:
        n = 16
        names = (c_char_p * n)()
        ms = (c_double * n)()
        cnt = (c_int64 * n)()
        k = load().lpf_get_kernel_times(self._h, names, ms, cnt, n, 1 if reset else 0)
        if k < 0:
            raise LpfError(k, "lpf_get_kernel_times")
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(k)}

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().lpf_stream_close(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop: concurrent streams on one GPU under an HBM budget (C++ worker thread)."""

    def __init__(self, hbm_budget_bytes: int, max_streams: int = 16):
        h = c_void_p()
        _check(load().lpf_server_open(ctypes.byref(h), int(hbm_budget_bytes), int(max_streams)),
               "lpf_server_open")
        self._h = h
        self._meta = {}

    def open_stream(self, H: int, W: int, freqs_mhz, dm_grid, depth: int, **kw) -> int:
        f = np.ascontiguousarray(freqs_mhz, dtype=np.float64)
        d = np.ascontiguousarray(dm_grid, dtype=np.float64)
        p = make_params(**kw)
        sid = c_int(-1)
        _check(load().lpf_server_open_stream(self._h, int(H), int(W), len(f),
                                             f.ctypes.data_as(POINTER(c_double)), len(d),
                                             d.ctypes.data_as(POINTER(c_double)), int(depth),
                                             ctypes.byref(p), ctypes.byref(sid)), "lpf_server_open_stream")
        self._meta[sid.value] = (len(f), int(H), int(W), int(p.cand_cap))
        return sid.value

    def submit(self, sid: int, frame: np.ndarray, T: int) -> int:
        """Returns LPF_OK or LPF_E_BUSY (retry after a fetch); raises on other errors."""
        fr = np.ascontiguousarray(frame, dtype=np.float32)
        meta = self._meta.get(int(sid))
        if meta is not None and fr.size != meta[0] * meta[1] * meta[2]:
            # the library copies F H W values from the frame
            raise ValueError(f"frame has {fr.size} values, the stream takes {meta[0] * meta[1] * meta[2]}")
        rc = load().lpf_server_submit(self._h, int(sid), c_void_p(fr.ctypes.data), int(T))
        if rc not in (LPF_OK, LPF_E_BUSY):
            raise LpfError(rc, "lpf_server_submit")
        return rc

    def fetch(self, sid: int, timeout_ms: int = -1):
        """(T, candidates, n_found, latency_ms) of the stream's next finished frame."""
        cap = self._meta[sid][3]
        buf = np.zeros(cap, dtype=CANDIDATE_DTYPE)
        n = c_int(0)
        T = c_int64(-1)
        lat = c_double(0.0)
        rc = load().lpf_server_fetch(self._h, int(sid), c_void_p(buf.ctypes.data), cap, ctypes.byref(n),
                                     ctypes.byref(T), ctypes.byref(lat), int(timeout_ms))
        if rc not in (LPF_OK, LPF_E_TRUNCATED):
            raise LpfError(rc, "lpf_server_fetch")
        return T.value, buf[:min(n.value, cap)].copy(), n.value, lat.value

    def close_stream(self, sid: int) -> None:
        _check(load().lpf_server_close_stream(self._h, int(sid)), "lpf_server_close_stream")

    def state(self, sid: int) -> int:
        st = c_int(-1)
        _check(load().lpf_server_stream_state(self._h, int(sid), ctypes.byref(st)), "lpf_server_stream_state")
        return st.value

    def stats(self, sid: int = -1) -> Dict[str, float]:
        o = ServeStats()
        _check(load().lpf_server_stats(self._h, int(sid), ctypes.byref(o)), "lpf_server_stats")
        return {k: getattr(o, k) for k, _ in ServeStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().lpf_server_close(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Cnn:
    """The parameter-inference network on F x Tw dynamic spectra (Sec. 2.3), with
    the caller's weights (float32 vector of lpf_cnn_param_count() values)."""

    def __init__(self, F: int, Tw: int, params, max_batch: int, cuda_stream=None):
        lib = load()
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        if p.size != lib.lpf_cnn_param_count():
            raise ValueError(f"{p.size} parameters, the network takes {lib.lpf_cnn_param_count()}")
        h = c_void_p()
        st = int(getattr(cuda_stream, "cuda_stream", cuda_stream)) if cuda_stream is not None else None
        _check(lib.lpf_cnn_open(ctypes.byref(h), int(F), int(Tw), c_void_p(p.ctypes.data), p.size, int(max_batch),
                                c_void_p(st) if st else None), "lpf_cnn_open")
        self._h, self.F, self.Tw, self.max_batch = h, int(F), int(Tw), int(max_batch)

    def forward(self, x, out=None, sync: bool = True):
        """x: CUDA float32 [n, F, Tw] (contiguous) -> CUDA float32 [n, 5] =
        (mu0, mu1, L00, L10, L11)."""
        import torch
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
            raise ValueError("x must be a contiguous float32 CUDA tensor")
        n = int(x.shape[0])
        if tuple(x.shape) != (n, self.F, self.Tw):
            raise ValueError(f"x shape {tuple(x.shape)} != (n, {self.F}, {self.Tw})")
        if out is None:
            out = torch.empty((n, 5), dtype=torch.float32, device=x.device)
        optr = _out_ptr(out, (n, 5)) if n else 0
        _check(load().lpf_cnn_forward(self._h, c_void_p(x.data_ptr()) if n else None, n,
                                      c_void_p(optr) if n else None), "lpf_cnn_forward")
        if sync:
            self.sync()
        return out

    def sync(self) -> None:
        _check(load().lpf_cnn_sync(self._h), "lpf_cnn_sync")

    def close(self) -> None:
        if getattr(self, "_h", None):
            load().lpf_cnn_close(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
