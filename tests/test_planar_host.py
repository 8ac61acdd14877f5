"""CPU checks of the library's two-dimensional operator functions (csrc/planar.cuh,
the code the GPU kernels run), compiled for the host by a small test harness:
Hankel functions against SciPy, kernel remainders and whole Galerkin matrices
against the oracle (oracle.planar).  No GPU is used."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy.special import hankel2

import workloads as W
from oracle import planar as PL

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def H(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("planar") / "libplanar_host.so")
    src = os.path.join(ROOT, "tests", "harness", "planar_host.cu")
    r = subprocess.run([nvcc, "-O2", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC", "-shared",
                        "-gencode", "arch=compute_103a,code=sm_103a", src, "-o", out], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    dp = ctypes.POINTER(ctypes.c_double)
    lib.h2_hankel01.argtypes = [ctypes.c_double, ctypes.c_double, dp]
    lib.h2_green_rem.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    lib.h2_dgreen_rem.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
    lib.h2_operators.argtypes = [dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp, dp]
    lib.h2_hankel01_asym_f.argtypes = [ctypes.c_double, ctypes.c_double, dp]
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def test_hankel_functions_match_scipy(H):
    """Relative error of H0^(2), H1^(2) across the series / asymptotic switch at |z| = 12,
    for real arguments and lossy ones (arg z down to -0.3 rad); the bound 2e-9 follows
    from the series' cancellation (largest term / result times e^{2|Im z|}) and the
    asymptotic remainder near the switch."""
    out = np.zeros(4)
    worst = 0.0
    for mag in np.concatenate([np.geomspace(1e-3, 11.99, 40), np.geomspace(12.0, 3000.0, 40)]):
        for ang in (0.0, -0.05, -0.15, -0.3):
            z = mag * np.exp(1j * ang)
            H.h2_hankel01(z.real, z.imag, _p(out))
            ref = np.array([hankel2(0, z), hankel2(1, z)])
            if not np.all(np.abs(ref) > 1e-280):        # underflows far into the lower half-plane
                continue
            got = np.array([out[0] + 1j * out[1], out[2] + 1j * out[3]])
            worst = max(worst, float(np.max(np.abs(got - ref) / np.abs(ref))))
    assert worst < 2e-9, worst


def test_kernel_remainders_match_oracle(H):
    out = np.zeros(2)
    for k in (3.0 + 0j, 2.0 - 0.6j, 50.0 - 1.0j):
        for R in (0.0, 1e-6, 0.01, 0.3, 0.49, 0.6, 2.0, 7.0):
            H.h2_green_rem(k.real, k.imag, R, _p(out))
            ref = PL.green_rem(k, np.array([R]))[0]
            assert abs(out[0] + 1j * out[1] - ref) <= 1e-9 * max(1.0, abs(ref)), (k, R)
            if R > 0:
                H.h2_dgreen_rem(k.real, k.imag, R, _p(out))
                ref = PL.dgreen_rem(k, np.array([R]))[0]
                assert abs(out[0] + 1j * out[1] - ref) <= 1e-9 * max(1.0, abs(ref)), (k, R)


@pytest.mark.parametrize("curve,k", [("circle", 3.0 + 0j), ("ellipse", 4.0 - 0.7j), ("airfoil", 6.0 + 0j)])
def test_galerkin_matrices_match_oracle(H, curve, k):
    verts = {"circle": W.circle_polygon(40), "ellipse": W.ellipse_polygon(56, 1.5, 2 * np.pi),
             "airfoil": W.airfoil_polygon(64)}[curve]
    n = len(verts)
    S = np.zeros((n, n, 2))
    D = np.zeros((n, n, 2))
    N = np.zeros((n, n, 2))
    v = np.ascontiguousarray(verts)
    H.h2_operators(_p(v), n, k.real, k.imag, 0, _p(S), _p(D), _p(N))
    Sr, Dr, _, Nr, _ = PL.operators(PL.Polygon(verts), k)
    for got, ref in ((S, Sr), (D, Dr), (N, Nr)):
        g = got[..., 0] + 1j * got[..., 1]
        assert np.abs(g - ref).max() <= 1e-9 * np.abs(ref).max()


def test_fp32_hankel_expansion_matches_scipy(H):
    """FP32 Hankel expansion for |z| >= 8 (its smallest term is below FP32 rounding
    there): relative error <= 2e-6 against SciPy, real and lossy arguments up to
    |z| = 3000 (the phase comes from FP64, so large |z| loses nothing)."""
    out = np.zeros(4)
    worst = 0.0
    for mag in np.geomspace(8.0, 3000.0, 60):
        for ang in (0.0, -0.05, -0.15):
            z = mag * np.exp(1j * ang)
            ref = np.array([hankel2(0, z), hankel2(1, z)])
            if not np.all(np.abs(ref) > 1e-30):
                continue
            H.h2_hankel01_asym_f(z.real, z.imag, _p(out))
            got = np.array([out[0] + 1j * out[1], out[2] + 1j * out[3]])
            worst = max(worst, float(np.max(np.abs(got - ref) / np.abs(ref))))
    assert worst < 2e-6, worst


@pytest.mark.parametrize("n,k", [(288, 16.0 + 0j), (576, 32.0 - 0.4j)])
def test_fp32_form_matches_oracle(H, n, k):
    """The FP32 form (well-separated pairs with |k R| >= 8 in FP32) on the N = 18 k0
    ellipse: S within 2e-6 of its largest entry, D within 3e-6, N within 2e-6
    (measured 1e-7, 1.3e-6 and 3.5e-7)."""
    verts = W.ellipse_polygon(n, 1.5, 2 * np.pi)
    S = np.zeros((n, n, 2))
    D = np.zeros((n, n, 2))
    N = np.zeros((n, n, 2))
    v = np.ascontiguousarray(verts)
    H.h2_operators(_p(v), n, k.real, k.imag, 1, _p(S), _p(D), _p(N))
    Sr, Dr, _, Nr, _ = PL.operators(PL.Polygon(verts), k)
    for got, ref, bound in ((S, Sr, 2e-6), (D, Dr, 3e-6), (N, Nr, 2e-6)):
        g = got[..., 0] + 1j * got[..., 1]
        err = np.abs(g - ref).max() / np.abs(ref).max()
        print(n, k, err)
        assert err <= bound, err
