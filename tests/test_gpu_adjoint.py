"""GPU tests of the adjoint product Z^H, the adjoint solve and the gradient of the
absorbed power with respect to excitation weights.

Tolerances: the adjoint product against the oracle's dense conj(Z)^T as the
forward product tests (2e-5 complex64 at ACA 1e-6, 1e-8 complex128 at ACA 1e-10);
the adjoint identity <Z x, y> = <x, Z^H y> on the compressed operator itself to the
arithmetic's rounding (1e-5 complex64, 1e-12 complex128) -- Z^H is the exact
adjoint of the stored operator, not of a symmetrised one; weight gradients
against the oracle's dense Hermitian form to 1e-6 (complex128, dense) and against
central finite differences of the library's own P(w) to 1e-3.
"""
import numpy as np
import pytest

import workloads as W
from oracle import excitation as E
from oracle import gradient as G
from oracle import operators as O
from oracle import rwg as R

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


def make(B, v, t, k0, eps, prec, aca_tol, leaf=32, eta=2.0, **kw):
    opt = B.bem_default_options()
    opt.precision = prec
    opt.leaf_size = leaf
    opt.eta = eta
    opt.aca_tol = aca_tol
    for k, val in kw.items():
        setattr(opt, k, val)
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, k0, eps)
    B.bem_assemble(h, _stream())
    return h


def apply(B, h, X, dtype, adjoint):
    ct = torch.complex64 if dtype == B.BEM_C64 else torch.complex128
    xd = torch.from_numpy(np.ascontiguousarray(X.T)).to(DEV, ct)
    yd = torch.empty_like(xd)
    f = B.bem_matvec_adjoint if adjoint else B.bem_matvec
    f(h, xd.data_ptr(), yd.data_ptr(), X.shape[1], dtype, _stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy().astype(np.complex128).T


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def sphere3():
    v, t = W.icosphere(3)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, 10.0, 3.2 - 1.9j)
    return v, t, g, Z


@pytest.mark.parametrize("dtype,aca_tol,tol", [(0, 1e-6, 2e-5), (1, 1e-10, 1e-8)], ids=["c64", "c128"])
def test_adjoint_product_equals_oracle(B, sphere3, dtype, aca_tol, tol):
    v, t, g, Z = sphere3
    h = make(B, v, t, 10.0, 3.2 - 1.9j, 1 if dtype == 0 else 2, aca_tol)
    try:
        X = W.complex_normal(2 * g.ne, seed=31, nrhs=3)
        if dtype == 0:
            X = X.astype(np.complex64).astype(np.complex128)
        Y = apply(B, h, X, dtype, True)
        assert rel(Y, Z.conj().T @ X) <= tol
        assert np.array_equal(Y, apply(B, h, X, dtype, True)), "adjoint product is not deterministic"
    finally:
        B.bem_destroy(h)


CASES = [("sphere", lambda: W.icosphere(3), 10.0), ("box", lambda: W.box_mesh(1.0, 0.8, 0.4, 10, 8, 4), 6.0)]


@pytest.mark.parametrize("dtype,tol", [(0, 1e-5), (1, 1e-12)], ids=["c64", "c128"])
@pytest.mark.parametrize("name,mesh,k0", CASES, ids=[c[0] for c in CASES])
def test_adjoint_identity_on_compressed_operator(B, name, mesh, k0, dtype, tol):
    """<Z x, y> = <x, Z^H y> for the stored (compressed, not exactly symmetric)
    operator; 13 right-hand sides (chunks 8 + 4 + 1) against one at a time."""
    v, t = mesh()
    h = make(B, v, t, k0, 3.2 - 1.9j, 1 if dtype == 0 else 2, 1e-4, leaf=16)
    try:
        st = B.bem_stats_get(h)
        assert sum(st["factor_entries"]) > 0
        n = 2 * st["ne"]
        X = W.complex_normal(n, seed=41, nrhs=13)
        Yv = W.complex_normal(n, seed=42, nrhs=13)
        if dtype == 0:
            X = X.astype(np.complex64).astype(np.complex128)
            Yv = Yv.astype(np.complex64).astype(np.complex128)
        ZX = apply(B, h, X, dtype, False)
        ZHY = apply(B, h, Yv, dtype, True)
        lhs = np.einsum("ir,ir->r", Yv.conj(), ZX)
        rhs = np.einsum("ir,ir->r", ZHY.conj(), X)
        assert np.abs(lhs - rhs).max() <= tol * np.abs(lhs).max()
        single = np.stack([apply(B, h, Yv[:, r:r + 1], dtype, True)[:, 0] for r in range(13)], axis=1)
        assert np.abs(ZHY - single).max() <= (1e-6 if dtype == 0 else 1e-14) * np.abs(single).max()
    finally:
        B.bem_destroy(h)


def test_adjoint_solve_equals_dense(B, sphere3):
    v, t, g, Z = sphere3
    gvec = W.complex_normal(2 * g.ne, seed=51)
    lam_ref = np.linalg.solve(Z.conj().T, gvec)
    h = make(B, v, t, 10.0, 3.2 - 1.9j, 3, 1e-6, tol=1e-6, refine_tol=1e-10, maxit=3000)
    try:
        gd = torch.from_numpy(gvec).to(DEV)
        ld = torch.zeros_like(gd)
        it, relres, status = B.bem_solve_adjoint(h, gd.data_ptr(), ld.data_ptr(), 1, _stream())
        assert relres[0] <= 1e-10
        assert rel(ld.cpu().numpy(), lam_ref) <= 1e-4
    finally:
        B.bem_destroy(h)


@pytest.fixture(scope="module")
def sphere2_weights():
    v, t = W.icosphere(2)
    g = R.build(v, t)
    Z = O.pmchwt_matrix(g, 2.0, 3.2 - 1.9j)
    khat, e0 = W.plane_wave_batch(6, seed=5)
    Bm = np.stack([E.rhs_planewave(g, 2.0, khat[i], e0[i]) for i in range(6)], axis=1)
    w = W.complex_normal(6, seed=6) / np.sqrt(6.0)
    return v, t, g, Z, khat, e0, Bm, w


def _bm_device(B, h, khat, e0):
    n = B.bem_num_unknowns(h)
    bm = torch.empty((len(khat), n), dtype=torch.complex128, device=DEV)
    B.bem_rhs_planewave(h, khat, e0, bm.data_ptr(), B.BEM_C128, _stream())
    return bm


def test_weight_gradient_equals_oracle_and_fd(B, sphere2_weights):
    v, t, g, Z, khat, e0, Bm, w = sphere2_weights
    p_ref, g_ref = G.absorbed_and_weight_gradient(g, Z, Bm, w)
    h = make(B, v, t, 2.0, 3.2 - 1.9j, 2, 1e-6, eta=0.0, tol=1e-8, refine_tol=1e-12, maxit=2000)
    try:
        bm = _bm_device(B, h, khat, e0)
        p, grad, it = B.bem_grad_weights(h, bm.data_ptr(), w, stream=_stream())
        assert abs(p - p_ref) <= 1e-6 * abs(p_ref)
        assert np.abs(grad - g_ref).max() <= 1e-6 * np.abs(g_ref).max()
        # central differences of the library's own P(w)
        step = 1e-6
        fd = np.zeros(len(w), dtype=np.complex128)
        for i in range(len(w)):
            e = np.zeros(len(w))
            e[i] = step
            pr = [B.bem_grad_weights(h, bm.data_ptr(), w + d, stream=_stream())[0] for d in (e, -e, 1j * e, -1j * e)]
            fd[i] = (pr[0] - pr[1]) / (2 * step) + 1j * (pr[2] - pr[3]) / (2 * step)
        assert np.abs(2 * grad - fd).max() <= 1e-3 * np.abs(fd).max()
    finally:
        B.bem_destroy(h)


def test_autograd_function_compressed_complex64(B, sphere2_weights):
    """torch.autograd through the compressed complex64 operator with FP64
    refinement: w.grad against the oracle's dense gradient (ACA 1e-6 and FP32
    entries: 1e-4)."""
    from paper_2310_15644_gb300.autograd import absorbed_power

    v, t, g, Z, khat, e0, Bm, w = sphere2_weights
    p_ref, g_ref = G.absorbed_and_weight_gradient(g, Z, Bm, w)
    h = make(B, v, t, 2.0, 3.2 - 1.9j, 1, 1e-6, leaf=16, tol=1e-4, refine_tol=1e-10, maxit=2000)
    try:
        bm = _bm_device(B, h, khat, e0)
        wt = torch.tensor(w, dtype=torch.complex128, requires_grad=True)
        p = absorbed_power(wt, h, bm)
        p.backward()
        assert abs(p.item() - p_ref) <= 1e-4 * abs(p_ref)
        got = wt.grad.numpy()
        assert np.abs(got - 2 * g_ref).max() <= 1e-4 * np.abs(2 * g_ref).max()
    finally:
        B.bem_destroy(h)


@pytest.fixture(scope="module")
def sphere2_eps():
    v, t = W.icosphere(2)
    g = R.build(v, t)
    b = E.rhs_planewave(g, 2.0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    ref = G.absorbed_eps_gradient(g, 2.0, 3.2 - 1.9j, b)
    return v, t, g, b, ref


def _p_and_eps_grad(B, h, b):
    bd = torch.from_numpy(np.ascontiguousarray(b[None, :])).to(DEV)
    n = bd.shape[1]
    x = torch.empty(n, dtype=torch.complex128, device=DEV)
    lam = torch.empty_like(x)
    p, _, _ = B.bem_grad_weights(h, bd.data_ptr(), np.array([1.0 + 0j]), x.data_ptr(), lam.data_ptr(), _stream())
    return p, B.bem_grad_eps(h, x.data_ptr(), lam.data_ptr(), _stream())


def test_eps_gradient_dense_complex128(B, sphere2_eps):
    """dP/d eps_r by the adjoint solve and the dG/dk pass against central
    differences of the oracle's dense solution (1e-5; operator entries agree to
    1e-11) and against central differences of the library's own P (1e-3)."""
    v, t, g, b, ref = sphere2_eps
    kw = dict(eta=0.0, tol=1e-10, refine_tol=1e-13, maxit=3000)
    h = make(B, v, t, 2.0, 3.2 - 1.9j, 2, 1e-6, **kw)
    try:
        p0, d = _p_and_eps_grad(B, h, b)
        assert np.abs(d - ref).max() <= 1e-5 * np.abs(ref).max(), (d, ref)
        step = 1e-5
        fd = []
        for de in (step, 1j * step):
            pp = []
            for sgn in (1, -1):
                B.bem_set_media(h, 2.0, 3.2 - 1.9j + sgn * de)
                B.bem_assemble(h, _stream())
                pp.append(_p_and_eps_grad(B, h, b)[0])
            fd.append((pp[0] - pp[1]) / (2 * step))
        assert np.abs(d - np.array(fd)).max() <= 1e-3 * np.abs(d).max(), (d, fd)
    finally:
        B.bem_destroy(h)


def test_eps_gradient_compressed_complex64_autograd(B, sphere2_eps):
    """Through torch.autograd with the compressed complex64 operator (FP64
    refinement): eps.grad against the oracle's dense gradient to 1e-3."""
    from paper_2310_15644_gb300.autograd import absorbed_power

    v, t, g, b, ref = sphere2_eps
    h = make(B, v, t, 2.0, 3.2 - 1.9j, 1, 1e-6, leaf=16, tol=1e-4, refine_tol=1e-10, maxit=3000)
    try:
        bm = torch.from_numpy(np.ascontiguousarray(b[None, :])).to(DEV)
        w = torch.tensor([1.0 + 0j], dtype=torch.complex128, requires_grad=True)
        eps = torch.tensor([3.2, -1.9], dtype=torch.float64, requires_grad=True)
        p = absorbed_power(w, h, bm, eps=eps, k0=2.0)
        p.backward()
        got = eps.grad.numpy()
        assert np.abs(got - ref).max() <= 1e-3 * np.abs(ref).max(), (got, ref)
    finally:
        B.bem_destroy(h)
