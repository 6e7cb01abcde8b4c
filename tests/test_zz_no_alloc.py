"""lpf_extract_dynspec_static, the gather that allocates no device memory.

Some callers cannot let a library call allocate device memory: a real-time loop
with a frame deadline (cudaMalloc can stall the device), a server that admits
streams against a fixed HBM budget, or a plug-in whose host owns all device
memory.  lpf_extract_dynspec may grow its candidate buffer with cudaMalloc;
lpf_extract_dynspec_static stages the candidates in a fixed array compiled
into the library instead.  This test calls it through the C ABI and checks it
against lpf_extract_dynspec on two calls in a row (the second smaller than the
first, so nothing left in the shared array from the first call may show), with
the exact equality the other gather tests use, plus its errors: capacity, an
out-of-image pixel, and an oversized request before the first poll.
The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _static_gather(lib):
    fn = lib.load().lpf_extract_dynspec_static
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    return fn


@pytest.mark.parametrize("dtype,box", [("fp32", 0), ("fp16", 1), ("bf16", 0)])
def test_static_gather_matches_allocating_gather(lib, dtype, box):
    spec = synth.spec_tiny(kappa=4.0)
    st = synth.SyntheticStream(spec, seed=21)
    fn = _static_gather(lib)
    Tw = 12
    big = np.zeros(lib.LPF_STATIC_DYNSPEC_MAX + 1, dtype=lib.CANDIDATE_DTYPE)
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                    box_r=spec.box_r, dtype=dtype) as s0:
        # before the first poll an oversized request fails as the allocating gather
        # would (no frame polled), ahead of the capacity check
        out = torch.empty((len(big), spec.F, 1), device="cuda")
        assert fn(s0._h, big.ctypes.data, len(big), 1, out.data_ptr()) == lib.LPF_E_NODATA
        del out
    with lib.Stream(spec.H, spec.W, spec.freqs_mhz, spec.dm_grid, spec.depth, kappa=spec.kappa,
                    box_r=spec.box_r, dtype=dtype, dyn_box_r=box) as s:
        for T in range(20):
            s.push(torch.from_numpy(st.frame(T)).cuda(), T)
            _, cands, n, _ = s.poll(timeout_ms=60000)
        assert len(cands) > 4
        edges = np.zeros(4, dtype=lib.CANDIDATE_DTYPE)
        edges["y"] = [0, spec.H - 1, 0, spec.H - 1]
        edges["x"] = [0, spec.W - 1, spec.W - 1, 0]
        first = np.ascontiguousarray(np.concatenate([cands, edges]))
        second = np.ascontiguousarray(first[::-1][: len(first) // 2])
        for c in (first, second):                      # two calls in a row
            ref = s.dynspec(c, Tw)
            torch.cuda.synchronize()
            out = torch.full_like(ref, float("nan"))
            rc = fn(s._h, c.ctypes.data, len(c), Tw, out.data_ptr())
            assert rc == lib.LPF_OK, rc
            torch.cuda.synchronize()
            assert torch.equal(out, ref)
        # more records than the fixed array holds: rejected before any copy
        out = torch.empty((len(big), spec.F, 1), device="cuda")
        assert fn(s._h, big.ctypes.data, len(big), 1, out.data_ptr()) == lib.LPF_E_CAPACITY
        # an out-of-image pixel is an argument error, as for the allocating gather
        bad = first[:1].copy()
        bad["y"] = spec.H
        assert fn(s._h, bad.ctypes.data, 1, Tw, out.data_ptr()) == lib.LPF_E_ARG
