"""The C ABI from plain C: tests/c/abi_plain_c.c includes include/lpf.h as C99
(no C++), links liblpf.so and calls the entry points that need no GPU; its
results must equal the same calls made through the Python binding."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_2103_15418_b300 as lpf
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_header_compiles_as_c99_and_calls_agree():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib = lpf.load()
    libdir = os.path.dirname(lpf.LIB_PATH)
    out_dir = os.path.join(ROOT, "tests", "c", "_build")          # git-ignored
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "abi_plain_c")
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "c", "abi_plain_c.c"),
                    "-L", libdir, "-l:liblpf.so", "-Wl,-rpath," + libdir, "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.split()
    sp = synth.spec_aartfaac()
    want = lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth)
    assert np.allclose(np.asarray(sp.freqs_mhz), [(57.6 if i < 8 else 61.2) + ((i % 8) + 0.5) * 0.1953125
                                                  for i in range(16)])
    assert int(out[0]) == lpf.LPF_OK and int(out[1]) == want
    assert int(out[2]) == lpf.LPF_OK and int(out[3]) == want          # NULL params = defaults
    assert int(out[4]) == lpf.LPF_E_DEPTH and int(out[5]) == lpf.LPF_E_ARG
    assert (int(out[6]), int(out[7]), float(out[8])) == (15, 1 << 20, 6.0)
    assert out[9] == "named" and lib.lpf_strerror(lpf.LPF_E_DEPTH)
    # the last field of lpf_params set from C: the same plan as through the binding
    assert int(out[10]) == lpf.LPF_OK
    assert int(out[11]) == lpf.footprint(sp.H, sp.W, sp.freqs_mhz, sp.dm_grid, sp.depth, suppress_steady=8) > want
    assert int(out[12]) == ctypes.sizeof(lpf.Params)
