"""The two-lane double-float operations (csrc/df2.cuh, packed FP32 instructions) against the
scalar ones (csrc/df.cuh), bit for bit, lane by lane, on a million pseudo-random lane pairs:
every operation the direction and adjoint passes use, the WENO5 offset of the direction pass
and its squared smoothness indicators.  The division's last step takes its error term from the
exact product (df2.cuh); its reference is written out in that form in tests/cuda/df2_check.cu.
The check is built here from its own source into a temporary library; nothing of it is in
libns3d.so."""
import ctypes
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
NAMES = ["add_fast", "sub", "mul_u", "mul", "sqr_u", "mul_f_u", "add_pos_u", "add_ordered_u", "add_ordered",
         "twice", "two_prod", "div", "weno_offset", "indicator_B1", "indicator_B2", "indicator_B3"]


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2211_16718_gb300 import build as B
    out = str(tmp_path_factory.mktemp("df2") / "libdf2check.so")
    cmd = [B.nvcc()] + B.ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I", B.INCLUDE, "-I",
                                 B.CSRC, os.path.join(HERE, "cuda", "df2_check.cu"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    lib.df2_check.restype = ctypes.c_int
    lib.df2_check.argtypes = [ctypes.c_int, ctypes.c_ulonglong, ctypes.POINTER(ctypes.c_int)]
    lib.df2_check_nops.restype = ctypes.c_int
    assert lib.df2_check_nops() == len(NAMES)
    return lib


@pytest.mark.gpu
@pytest.mark.parametrize("seed", [1, 20261204])
def test_two_lane_double_float_equals_scalar_bitwise(checker, seed):
    bad = (ctypes.c_int * len(NAMES))()
    assert checker.df2_check(1 << 20, seed, bad) == 0
    mismatches = {n: bad[i] for i, n in enumerate(NAMES) if bad[i]}
    assert not mismatches, mismatches
