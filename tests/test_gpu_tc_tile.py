"""One tensor-core tile through the library's tcgen05 primitives (csrc/tc.cuh),
compiled into a small harness (tests/harness/tc_tile.cu) and checked against a
float64 host GEMM: D (128 x N) = A (128 x K) B^T.

Bounds: with inputs already representable in TF32 every product is exact in
FP32 and only the FP32 accumulation rounds, so |D - D_ref| <= K 2^-24 sum|a||b|
(taken as 4e-6 sum|a||b| for K <= 32); with the three-term split of FP32 inputs
the dropped lo*lo term and the TF32 reading of lo add about 2^-21 per product
(bound 2e-6 sum|a||b|), while one plain TF32 product of the same FP32 inputs is
off by up to 2^-10 per operand."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path_factory.mktemp("tc") / "libtc_tile.so")
    src = os.path.join(ROOT, "tests", "harness", "tc_tile.cu")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                        "-gencode", "arch=compute_103a,code=sm_103a", src, "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    fp = ctypes.POINTER(ctypes.c_float)
    lib.tc_tile.argtypes = [fp, fp, fp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.tc_tile.restype = ctypes.c_int
    return lib


def _run(H, A, B, mode):
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    N, K = B.shape
    D = np.zeros((128, N), dtype=np.float32)
    p = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))  # noqa: E731
    rc = H.tc_tile(p(A), p(B), p(D), N, K, mode)
    assert rc == 0, f"harness status {rc}"
    return D.astype(np.float64)


def _tf32(a):
    """Round to nearest TF32 (10 explicit mantissa bits), ties away from zero."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


def _err(D, A, B):
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    return float(np.max(np.abs(D - ref) / scale))


@pytest.mark.parametrize("N,K,mode", [(64, 32, 0), (128, 32, 0), (16, 8, 0), (64, 32, 1), (128, 16, 1)],
                         ids=["ts_n64", "ts_n128", "ts_n16_k8", "ss_n64", "ss_n128_k16"])
def test_tile_exact_tf32_inputs(H, N, K, mode):
    rng = np.random.default_rng(N + K + mode)
    A = _tf32(rng.standard_normal((128, K)))
    B = _tf32(rng.standard_normal((N, K)))
    D = _run(H, A, B, mode)
    assert _err(D, A, B) <= 4e-6


def test_tile_three_term_split_reaches_fp32(H):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((128, 32)).astype(np.float32)
    B = rng.standard_normal((64, 32)).astype(np.float32)
    e_split = _err(_run(H, A, B, 2), A, B)
    e_plain = _err(_run(H, A, B, 0), A, B)
    assert e_split <= 2e-6, e_split
    assert e_plain >= 20 * e_split, (e_plain, e_split)
