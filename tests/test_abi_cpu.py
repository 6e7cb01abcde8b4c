"""The C-ABI library builds, loads and exports every symbol include/lpf.h declares.

No compute call is made here (no GPU on this host); only argument validation
that returns before any CUDA call is exercised.
"""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2103_15418_b300 as lpf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lpf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lpf_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = lpf.load()
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lpf.EXPORTS)


def test_struct_layouts():
    assert ctypes.sizeof(lpf.Candidate) == 24
    assert lpf.CANDIDATE_DTYPE.itemsize == 24
    p = lpf.default_params()
    assert (p.cadence_s, p.kappa, p.box_r, p.lmax_r, p.dtype) == (1.0, 6.0, 15, 1, 0)
    assert p.cand_cap == 1 << 20 and p.result_slots == 2 and not p.cuda_stream
    # the fields after the pointer read back the library's defaults: same layout
    assert (p.filter_impl, p.qc, p.qc_z, p.qc_zeta, p.qc_min_frames, p.mode, p.clip_iters) == \
        (0, 0, 5.0, 20.0, 128, 0, 1)
    assert (p.kernel, p.gauss_sigma) == (0, 0.0)
    # the last field: the library's defaults overwrite a sentinel at the binding's
    # offset of it, and the struct sizes agree
    q = lpf.Params()
    q.suppress_steady = 77
    lpf.load().lpf_default_params(ctypes.byref(q))
    assert q.suppress_steady == 0
    assert lpf.Params.suppress_steady.offset + 4 <= ctypes.sizeof(lpf.Params)


def test_strerror_names_every_code():
    lib = lpf.load()
    for code in range(0, -12, -1):
        assert lib.lpf_strerror(code).decode() not in ("", "unknown error")
    assert lib.lpf_strerror(-99).decode() == "unknown error"


def test_argument_validation_before_any_cuda_call():
    f = np.array([60.0, 61.0])
    dm = np.array([0.0, 10.0])
    bad = [
        dict(H=0, W=8, freqs_mhz=f, dm_grid=dm, depth=8),
        dict(H=8, W=8, freqs_mhz=np.array([60.0, -1.0]), dm_grid=dm, depth=8),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=np.array([-1.0]), depth=8),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, box_r=17),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, box_r=0),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, cadence_s=0.0),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, result_slots=0),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, qc=True, qc_z=0.0),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, qc=True, qc_zeta=-1.0),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, qc=True, qc_min_frames=1),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, lmax_r=3),              # 3x3 only for DM trials
        dict(H=8, W=8, freqs_mhz=f, dm_grid=None, depth=2, mode="subband", lmax_r=4),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=None, depth=2, mode="subband", box_r=5),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=None, depth=2, mode="subband", filter_impl="tiled"),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, clip_iters=3, filter_impl="streaming"),  # direct form
        dict(H=8, W=8, freqs_mhz=f, dm_grid=None, depth=2, mode="subband", clip_iters=17),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=dm, depth=8, kernel="gauss", gauss_sigma=2.0),  # subband only
        dict(H=8, W=8, freqs_mhz=f, dm_grid=None, depth=2, mode="subband", kernel="gauss"),  # s = 0
        dict(H=8, W=8, freqs_mhz=f, dm_grid=None, depth=2, mode="subband", kernel="gauss",
             gauss_sigma=float("inf")),
        dict(H=8, W=8, freqs_mhz=f, dm_grid=None, depth=2, mode="subband", kernel="gauss",
             gauss_sigma=2.0, box_r=17),
    ]
    for kw in bad:
        with pytest.raises(lpf.LpfError) as e:
            lpf.Stream(**kw)
        assert e.value.code == lpf.LPF_E_ARG, kw
    # depth shorter than the largest delay + 1 (DM 400 over 60-61 MHz is ~30 s)
    with pytest.raises(lpf.LpfError) as e:
        lpf.Stream(8, 8, f, np.array([0.0, 400.0]), 4)
    assert e.value.code == lpf.LPF_E_DEPTH


def test_null_handles_are_rejected():
    lib = lpf.load()
    assert lib.lpf_get_qc(None, None, None, None) == lpf.LPF_E_ARG
    assert lib.lpf_push_frame(None, None, 0) == lpf.LPF_E_ARG
    assert lib.lpf_poll_candidates(None, None, 0, None, None, 0) == lpf.LPF_E_ARG
    assert lib.lpf_stream_close(None) == lpf.LPF_OK


def test_footprint_is_planned_without_a_gpu():
    import synth
    sp = synth.spec_aartfaac()
    fp32 = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth)
    fp16 = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, dtype="fp16")
    plane = sp.F * sp.H * sp.W * 4                 # one FP32 frame
    # residual path (box 31): raw and residual rings of depth + 2 slots (the raw-ring
    # write follows the shift-sum), two sets of the 205 images of D - C and two
    # crossing lists (12 bytes for 1/32 of all pixels of the 205 delay rows; the
    # filter of a push runs beside the next push's shift-sum), staging frames and
    # candidate buffers
    rings = 2 * (sp.depth + 2) * plane
    imgs = 2 * 205 * sp.H * sp.W * 4
    xlists = 2 * 12 * (205 * sp.H * sp.W // 32)
    assert rings + imgs + xlists < fp32 < rings + imgs + xlists + 400 * 2 ** 20
    assert fp32 - fp16 == (sp.depth + 2) * plane
    deeper = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth + 10)
    assert deeper - fp32 == 2 * 10 * plane
    tiled = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, filter_impl="tiled")
    # the tiled path: the raw ring of depth slots and one set of images, no residual
    # ring or crossing list; partials: strips vs tiles
    extra = (sp.depth + 2) * plane + 2 * plane + 205 * sp.H * sp.W * 4 + xlists
    assert abs(fp32 - tiled - extra) < 4 * 2 ** 20
    with pytest.raises(lpf.LpfError) as e:
        lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, 40)
    assert e.value.code == lpf.LPF_E_DEPTH


def test_stress_config_depth_96_is_rejected():
    """2048^2 x 32 subbands over 57.6-63.85 MHz, DM up to 500: the sweep needs 114 frames."""
    import synth
    sp = synth.spec_stress(depth=96)
    with pytest.raises(lpf.LpfError) as e:
        lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, dtype="fp16")
    assert e.value.code == lpf.LPF_E_DEPTH
    fp = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, 114, dtype="fp16")
    # 2 x 31.1 GB rings (raw, residual; 116 slots) + 2 x 14.2 GB images of D - C
    # + 2 x 1.3 GB crossing lists
    assert 90e9 < fp < 96e9


def test_quality_control_footprint():
    """Quality control adds the running mean and m2 planes ([F][P] FP32 each) and a
    few hundred bytes of scratch per stream."""
    import synth
    sp = synth.spec_aartfaac(H=256, W=256)
    off = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth)
    on = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, qc=True)
    planes = 2 * sp.F * sp.H * sp.W * 4
    assert planes < on - off < planes + 64 * 1024


def test_subband_detector_footprint():
    """Per-subband detector: F rows of images (one per band), no delay table, any
    depth >= 1, dm_grid not needed."""
    import synth
    sp = synth.spec_aartfaac(H=256, W=256)
    fp = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, None, 2, mode="subband", lmax_r=3)
    rings = 2 * (2 + 2) * sp.F * sp.H * sp.W * 4    # raw and residual rings, depth 2 + 2 spare slots
    imgs = 2 * sp.F * sp.H * sp.W * 4               # band planes, one set per lane
    # plus the 1M-record candidate, crossing and result buffers and two staging frames
    assert rings + imgs < fp < rings + imgs + 160 * 2 ** 20


def test_clipping_footprint():
    """The clipping path (iterations, or the Gaussian kernel) adds a flag plane and
    five FP32 planes per band and drops what the box path needs beside them: the
    residual ring (depth 2 + 2 spare slots, FP32), the two spare raw-ring slots,
    the second set of band planes and the two crossing lists (max(cand_cap,
    F H W / 32) keys and S/N values each)."""
    import synth
    sp = synth.spec_aartfaac(H=256, W=256)
    one = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, None, 2, mode="subband", lmax_r=3)
    many = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, None, 2, mode="subband", lmax_r=3, clip_iters=4)
    gauss = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, None, 2, mode="subband", lmax_r=3, kernel="gauss",
                          gauss_sigma=4.0, box_r=9)
    px = sp.F * sp.H * sp.W
    xcap = max(1 << 20, px // 32)
    delta = px * 21 - (2 + 4) * px * 4 - px * 4 - 2 * xcap * 12
    # (+ the kernel factors and the statistics partials of the other block layout)
    assert delta <= many - one < delta + 65536
    assert delta <= gauss - one < delta + 65536


def test_dispersed_clipping_footprint():
    """Clipping in the dispersed search runs on the direct-form path: the tiled
    path's buffers plus a flag plane and five FP32 planes per distinct delay row."""
    import synth
    from oracle import lpf_oracle as O
    sp = synth.spec_aartfaac(H=256, W=256)
    tiled = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, filter_impl="tiled")
    clip = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, clip_iters=3)
    rows = len({tuple(r) for r in O.delay_table(sp.freqs_mhz, sp.dm_grid, sp.cadence_s).tolist()})
    delta = rows * sp.H * sp.W * 21
    assert delta <= clip - tiled < delta + 65536


def test_binding_refuses_buffers_the_library_would_overrun():
    """push_host reads exactly F H W FP32 values and dynspec writes exactly n F Tw:
    buffers of another dtype, layout or size are refused before any library call."""
    n = 2 * 3 * 4
    ok = np.zeros((2, 3, 4), np.float32)
    assert lpf._host_frame_ptr(ok, n) == ok.ctypes.data
    for bad in (np.zeros((2, 3, 4), np.float64), np.zeros((2, 3, 4), np.float16),
                np.zeros((2, 3, 8), np.float32)[:, :, ::2], np.zeros((2, 3, 5), np.float32), [0.0] * n):
        with pytest.raises(ValueError):
            lpf._host_frame_ptr(bad, n)
    import torch
    t = torch.zeros((2, 3, 4))
    assert lpf._host_frame_ptr(t, n) == t.data_ptr()
    for bad in (t.half(), t.double(), t.transpose(0, 2), torch.zeros(n + 1)):
        with pytest.raises(ValueError):
            lpf._host_frame_ptr(bad, n)

    class FakeCuda:                          # shape / dtype / layout of a CUDA tensor, no device
        is_cuda = True

        def __init__(self, shape, dtype="torch.float32", contiguous=True):
            self.shape, self.dtype, self._c = shape, dtype, contiguous

        def is_contiguous(self):
            return self._c

        def data_ptr(self):
            return 4096

    assert lpf._out_ptr(FakeCuda((5, 16, 12)), (5, 16, 12)) == 4096
    for bad in (FakeCuda((4, 16, 12)), FakeCuda((5, 16, 12), "torch.float16"),
                FakeCuda((5, 16, 12), contiguous=False), torch.zeros((5, 16, 12))):
        with pytest.raises(ValueError):
            lpf._out_ptr(bad, (5, 16, 12))


def test_cnn_arguments_are_checked_before_any_cuda_call():
    """F and Tw multiples of 4 with (F/4)(Tw/4) a power of two <= 128, the parameter
    count and the batch limit are refused with LPF_E_ARG on a machine without a GPU."""
    import synth
    p = synth.cnn_params(1)
    assert lpf.load().lpf_cnn_param_count() == p.size == 23621
    for F, Tw, mb in [(12, 64, 4), (32, 66, 4), (8, 16, 0), (64, 64, 4), (2, 16, 4)]:
        with pytest.raises(lpf.LpfError) as e:
            lpf.Cnn(F, Tw, p, max_batch=mb)
        assert e.value.code == lpf.LPF_E_ARG, (F, Tw, mb)
    with pytest.raises(ValueError):
        lpf.Cnn(8, 16, p[:-1], max_batch=4)


def test_steady_suppression_arguments_and_footprint():
    """suppress_steady: 0..255, dispersed search only; its state is one bit per
    pixel of the 2^(bx + by) key space for each of the two push lanes and one byte
    per pixel, planned without a GPU."""
    import synth
    lib = lpf
    spec = synth.spec_tiny()
    fp = lambda **kw: lib.footprint(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth,
                                    box_r=spec.box_r, **kw)
    npix = 1 << (2 * int(np.ceil(np.log2(spec.W))))          # 64 x 64: 6 + 6 key bits
    assert spec.H == spec.W == 64
    assert fp(suppress_steady=3) - fp() == 2 * (npix // 8) + npix
    assert fp(suppress_steady=255) == fp(suppress_steady=1)
    for bad in (-1, 256):
        with pytest.raises(lib.LpfError):
            fp(suppress_steady=bad)
    with pytest.raises(lib.LpfError):
        lib.footprint(spec.H, spec.W, spec.freqs_mhz, None, 1, box_r=7, mode="subband", suppress_steady=2)
