"""GPU parity of the paper's two-dimensional fast direct solver (Sec. III) with the
oracle (`oracle/planar.py`): the batched FFT (numpy), the Calderon-preconditioned
CFIE C_p of Eq. 16 and its right-hand-side maps, the circulant counterpart solved
by FFT, the randomized skeleton of Eq. 17 and the Woodbury solve of Eq. 18.

Tolerances: FFT 1e-12 relative (FP64, length up to 2048); C_p, L_e, L_h 1e-8 of
their largest entry (the GPU operators S, D, N equal the oracle's to 1e-9); the
skeleton: |A - U V^T|_2 <= tol |A|_2 and the rank within one block of the oracle's
on the same test vectors; Woodbury against the oracle's dense solve of C_p to
10 tol (the bound of the oracle's own test)."""
import numpy as np
import pytest

import workloads as W
from oracle import planar as PL

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_15644_gb300.build import build

    build()
    import paper_2310_15644_gb300.bem as mod

    return mod


def _stream():
    return torch.cuda.current_stream().cuda_stream


@pytest.mark.parametrize("n,batch", [(5, 3), (18, 1), (144, 4), (1152, 2), (2048, 1)])
def test_fft_equals_numpy(B, n, batch):
    X = W.complex_normal(n, seed=n, nrhs=batch)  # (n, batch)
    # column-major storage: vector b at b * n, stride 1
    xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(DEV)
    B.bem_fft(None, xd.data_ptr(), n, 1, batch, n, False, _stream())
    F = xd.cpu().numpy().T
    assert np.abs(F - np.fft.fft(X, axis=0)).max() <= 1e-12 * np.abs(F).max() * np.sqrt(n)
    B.bem_fft(None, xd.data_ptr(), n, 1, batch, n, True, _stream())
    assert np.abs(xd.cpu().numpy().T - X).max() <= 1e-12 * np.abs(X).max() * np.sqrt(n)
    # strided: the rows of a row-major n x batch array
    yd = torch.from_numpy(np.ascontiguousarray(X)).to(DEV)
    B.bem_fft(None, yd.data_ptr(), n, batch, batch, 1, False, _stream())
    assert np.abs(yd.cpu().numpy() - np.fft.fft(X, axis=0)).max() <= 1e-12 * np.abs(F).max() * np.sqrt(n)


@pytest.fixture(scope="module")
def ellipse8():
    k0 = 8.0
    n = int(round(18 * k0))
    verts = W.ellipse_polygon(n, 1.5, 2 * np.pi)
    poly = PL.Polygon(verts)
    Cp, Le, Lh = PL.calderon_cfie(poly, k0)
    circ = PL.circular_counterpart(poly)
    a = PL.curvature_radius(poly)
    Cc, _, _ = PL.calderon_cfie(circ, k0, a=a)
    return k0, n, verts, circ.verts, a, Cp, Le, Lh, Cc


def gpu_calderon(B, verts, k0, a=0.0):
    n = len(verts)
    mats = [torch.empty((n, n), dtype=torch.complex128, device=DEV) for _ in range(3)]
    B.bem_planar_calderon(None, verts, k0, mats[0].data_ptr(), mats[1].data_ptr(), mats[2].data_ptr(), a, _stream())
    return mats


def test_calderon_equals_oracle(B, ellipse8):
    k0, n, verts, cverts, a, Cp, Le, Lh, Cc = ellipse8
    g = gpu_calderon(B, verts, k0)
    for got, want in zip(g, (Cp, Le, Lh)):
        got = got.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-8 * np.abs(want).max()
    gc = gpu_calderon(B, cverts, k0, a)[0].cpu().numpy()
    assert np.abs(gc - Cc).max() <= 1e-8 * np.abs(Cc).max()


def test_circulant_solve_equals_oracle(B, ellipse8):
    k0, n, verts, cverts, a, Cp, Le, Lh, Cc = ellipse8
    gc = gpu_calderon(B, cverts, k0, a)[0]
    cc0 = gc[:, 0].contiguous()
    b = W.complex_normal(n, seed=3, nrhs=2)
    bd = torch.from_numpy(np.ascontiguousarray(b.T)).to(DEV)
    xd = torch.empty_like(bd)
    B.bem_planar_woodbury_solve(None, cc0.data_ptr(), n, 0, 0, 0, bd.data_ptr(), xd.data_ptr(), 2, _stream())
    want = PL.circulant_solve(Cc, b)
    assert np.abs(xd.cpu().numpy().T - want).max() <= 1e-9 * np.abs(want).max()


@pytest.mark.parametrize("tol", [1e-3, 1e-8])
def test_skeleton_and_woodbury_equal_oracle(B, ellipse8, tol):
    k0, n, verts, cverts, a, Cp, Le, Lh, Cc = ellipse8
    cp = gpu_calderon(B, verts, k0)[0]
    cc = gpu_calderon(B, cverts, k0, a)[0]
    A = (cp - cc).contiguous()
    omega = W.complex_normal(n, seed=7, nrhs=n)  # as the oracle's test: (n, n) test vectors
    od = torch.from_numpy(np.ascontiguousarray(omega.T)).to(DEV)  # column-major
    U = torch.zeros((n, n), dtype=torch.complex128, device=DEV)    # n columns of n (column-major)
    Vt = torch.zeros((n, n), dtype=torch.complex128, device=DEV)
    r = B.bem_planar_skeleton(None, A.data_ptr(), n, od.data_ptr(), n, tol, 8, U.data_ptr(), Vt.data_ptr(), _stream())
    Uh = U.cpu().numpy()[:r].T            # (n, r)
    Vth = Vt.cpu().numpy()[:r]            # (r, n)
    Ah = Cp - Cc
    assert np.linalg.norm(Ah - Uh @ Vth, 2) <= max(tol, 1e-13) * np.linalg.norm(Ah, 2) * 1.01
    Uo, Vto = PL.skeleton(Cp, Cc, omega, tol)
    assert abs(r - Uo.shape[1]) <= 8, (r, Uo.shape[1])
    # Woodbury solve against the oracle's dense solve of C_p
    b = W.complex_normal(n, seed=8)
    xd_ = np.linalg.solve(Cp, b)
    bd = torch.from_numpy(b).to(DEV)
    xd = torch.empty_like(bd)
    cc0 = cc[:, 0].contiguous()
    B.bem_planar_woodbury_solve(None, cc0.data_ptr(), n, U.data_ptr(), Vt.data_ptr(), r, bd.data_ptr(),
                                xd.data_ptr(), 1, _stream())
    xw = xd.cpu().numpy()
    assert np.linalg.norm(xw - xd_) <= max(10 * tol, 1e-11) * np.linalg.norm(xd_)
    if tol == 1e-3:
        assert r < n // 2


def test_fp32_operators_woodbury_within_tolerance(B):
    """The whole pipeline with the FP32 form of the operators on the N = 18 k0 ellipse
    (k0 = 16): the Woodbury solution at tol 1e-4 agrees with the oracle's dense solve
    of C_p to 10 tol, the FP32 form's 1e-6 error being far below the tolerance."""
    k0 = 16.0
    n = int(round(18 * k0))
    verts = W.ellipse_polygon(n, 1.5, 2 * np.pi)
    poly = PL.Polygon(verts)
    Cp, _, _ = PL.calderon_cfie(poly, k0)
    circ = PL.circular_counterpart(poly)
    a = PL.curvature_radius(poly)
    cp = torch.empty((n, n), dtype=torch.complex128, device=DEV)
    cc = torch.empty_like(cp)
    B.bem_planar_calderon(None, verts, k0, cp.data_ptr(), 0, 0, 0.0, _stream(), fp32=True)
    B.bem_planar_calderon(None, circ.verts, k0, cc.data_ptr(), 0, 0, a, _stream(), fp32=True)
    assert np.abs(cp.cpu().numpy() - Cp).max() <= 1e-5 * np.abs(Cp).max()
    A = (cp - cc).contiguous()
    omega = torch.from_numpy(np.ascontiguousarray(W.complex_normal(n, seed=7, nrhs=n).T)).to(DEV)
    U = torch.zeros((n, n), dtype=torch.complex128, device=DEV)
    Vt = torch.zeros_like(U)
    tol = 1e-4
    r = B.bem_planar_skeleton(None, A.data_ptr(), n, omega.data_ptr(), n, tol, 8, U.data_ptr(), Vt.data_ptr(),
                              _stream())
    b = W.complex_normal(n, seed=8)
    bd = torch.from_numpy(b).to(DEV)
    xd = torch.empty_like(bd)
    cc0 = cc[:, 0].contiguous()
    B.bem_planar_woodbury_solve(None, cc0.data_ptr(), n, U.data_ptr(), Vt.data_ptr(), r, bd.data_ptr(),
                                xd.data_ptr(), 1, _stream())
    xo = np.linalg.solve(Cp, b)
    assert np.linalg.norm(xd.cpu().numpy() - xo) <= 10 * tol * np.linalg.norm(xo)
