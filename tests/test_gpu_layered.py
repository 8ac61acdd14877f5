"""GPU parity of layered bodies (several closed surfaces between homogeneous
regions) through the C interface, against the oracle's region-by-region PMCHWT
system (oracle.multiregion).

Small cases, dense oracle:
  * coated sphere: outer icosphere of 320 triangles and radius 1 (shell eps
    3.2 - 1.9j), inner icosphere of 80 triangles and radius 0.5 (core eps
    2.5 - 1.2j), k0 = 2; 600 edges, 1,200 unknowns;
  * two spheres side by side in free space (80 and 320 triangles), coupled
    through the exterior region.
Leaf 16, so that every region's partition has far blocks (stored as ACA
factors, or densely where the rank passes break-even).  Tolerances are those of
one body: compressed products 2e-5 (complex64, ACA 1e-6), 1e-3 (complex64, ACA
1e-4) and 1e-8 (complex128, ACA 1e-10); refined solves 1e-8; powers 1e-8
relative.

Full size: the coated sphere of the gradient workload (5,120 + 1,280
triangles, radii 1 and 0.5, k0 = 6; 19,200 unknowns), leaf 64, eta 2: sampled
rows of the product against the oracle's rows computed one by one, and the
solve against the stored dense oracle solution (tests/golden/make_coated_sphere.py)
and the coated-sphere series.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import multiregion as MR
from oracle import power as P
from oracle import rwg as R

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
K0 = 2.0
EPS3 = [1.0, 3.2 - 1.9j, 2.5 - 1.2j]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "coated_sphere_oracle.npz")


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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def coated(level_outer=2, level_inner=1, radius_inner=0.5):
    return W.coated_sphere(level_outer, 1.0, level_inner, radius_inner)


def side_by_side():
    a = W.icosphere(1, 0.6, (-1.0, 0.0, 0.0))
    b = W.icosphere(2, 0.5, (1.0, 0.2, 0.0))
    v, t, s = MR.union_mesh([a, b])
    return v, t, np.where(s[:, None] == 0, np.array([0, 1]), np.array([0, 2]))


def make(B, v, t, regions, k0=K0, eps=EPS3, prec=3, leaf=16, eta=2.0, aca_tol=1e-6, **kw):
    opt = B.bem_default_options()
    opt.precision = prec
    opt.leaf_size = leaf
    opt.eta = eta
    opt.aca_tol = aca_tol
    for k, val in kw.items():
        setattr(opt, k, val)
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_regions(h, k0, eps, regions)
    B.bem_assemble(h, _stream())
    return h


def apply(B, h, X, dtype, adjoint=False):
    """Columns of X through bem_matvec (or its adjoint); X is (2ne,) or (2ne, nrhs)."""
    ct = torch.complex64 if dtype == B.BEM_C64 else torch.complex128
    Xc = X if X.ndim == 2 else X[:, None]
    xd = torch.from_numpy(np.ascontiguousarray(Xc.T)).to(DEV, ct)
    yd = torch.empty_like(xd)
    f = B.bem_matvec_adjoint if adjoint else B.bem_matvec
    f(h, xd.data_ptr(), yd.data_ptr(), Xc.shape[1], dtype, _stream())
    torch.cuda.synchronize()
    Y = yd.cpu().numpy().astype(np.complex128).T
    return Y if X.ndim == 2 else Y[:, 0]


@pytest.fixture(scope="module")
def small():
    out = {}
    for name, mesh in (("coated", coated), ("side_by_side", side_by_side)):
        v, t, regions = mesh()
        g = R.build(v, t)
        out[name] = (v, t, regions, g, MR.pmchwt_regions(g, regions, K0, EPS3))
    return out


@pytest.mark.parametrize("case", ["coated", "side_by_side"])
@pytest.mark.parametrize("dtype,aca_tol,tol", [(0, 1e-6, 2e-5), (0, 1e-4, 1e-3), (1, 1e-10, 1e-8)],
                         ids=["c64", "c64_aca1e-4", "c128"])
def test_layered_product_equals_oracle(B, small, case, dtype, aca_tol, tol):
    v, t, regions, g, Z = small[case]
    h = make(B, v, t, regions, prec=1 if dtype == 0 else 2, aca_tol=aca_tol)
    try:
        st = B.bem_stats_get(h)
        assert st["ne"] == g.ne and st["n_far"] > 0
        X = W.complex_normal(2 * g.ne, seed=1, nrhs=3)
        if dtype == 0:
            X = X.astype(np.complex64).astype(np.complex128)
        x = X[:, 0]
        assert rel(apply(B, h, x, dtype), Z @ x) <= tol
        assert rel(apply(B, h, X, dtype), Z @ X) <= tol
        assert rel(apply(B, h, x, dtype, adjoint=True), Z.conj().T @ x) <= tol
    finally:
        B.bem_destroy(h)


def test_layered_rhs_equals_oracle(B, small):
    v, t, regions, g, Z = small["coated"]
    kh, e0 = W.plane_wave_batch(2, seed=3)
    ref = MR.rhs_planewave(g, regions, K0, kh, e0)
    h = make(B, v, t, regions, prec=2, aca_tol=1e-10)
    try:
        bd = torch.zeros(2, 2 * g.ne, dtype=torch.complex128, device=DEV)
        B.bem_rhs_planewave(h, kh, e0, bd.data_ptr(), B.BEM_C128, _stream())
        torch.cuda.synchronize()
        got = bd.cpu().numpy().T
        assert rel(got, ref) <= 1e-12
        assert np.all(got[MR.exterior_mask(g, regions) == 0] == 0)
    finally:
        B.bem_destroy(h)


def test_layered_solve_and_powers_match_dense_lu(B, small):
    v, t, regions, g, Z = small["coated"]
    b = MR.rhs_planewave(g, regions, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    xr = np.linalg.solve(Z, b)
    h = make(B, v, t, regions, prec=3, eta=0.0, refine_tol=1e-11)
    try:
        bd = torch.from_numpy(b).to(DEV)
        xd = torch.zeros_like(bd)
        it, relres, _ = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        x = xd.cpu().numpy()
        assert relres[0] <= 1e-11
        ne_o = 30 * 16
        for sl in (slice(0, ne_o), slice(ne_o, g.ne), slice(g.ne, g.ne + ne_o), slice(g.ne + ne_o, 2 * g.ne)):
            assert rel(x[sl], xr[sl]) <= 1e-8
        xe = MR.exterior_currents(g, regions, xr)
        pa, pe, ps = B.bem_power(h, xd.data_ptr(), bd.data_ptr(), 1, _stream())
        assert abs(pa[0] - P.absorbed(g, xe)) <= 1e-8 * abs(pa[0])
        assert abs(pe[0] - P.extinguished(g, xe, b)) <= 1e-8 * abs(pe[0])
        assert abs(ps[0] - P.scattered(g, K0, xe)) <= 1e-8 * abs(ps[0])
        dens = torch.empty(g.nt, dtype=torch.float64, device=DEV)
        B.bem_power_density(h, xd.data_ptr(), dens.data_ptr(), _stream())
        torch.cuda.synchronize()
        assert rel(dens.cpu().numpy(), P.absorbed_density(g, xe)) <= 1e-8
        # adjoint solve: Z^H lambda = g
        gv = W.complex_normal(2 * g.ne, seed=8)
        lr = np.linalg.solve(Z.conj().T, gv)
        gd = torch.from_numpy(gv).to(DEV)
        ld = torch.zeros_like(gd)
        B.bem_solve_adjoint(h, gd.data_ptr(), ld.data_ptr(), 1, _stream())
        assert rel(ld.cpu().numpy(), lr) <= 1e-8
    finally:
        B.bem_destroy(h)


def test_layered_mixed_precision_solve_meets_1e4(B, small):
    v, t, regions, g, Z = small["coated"]
    b = MR.rhs_planewave(g, regions, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    xr = np.linalg.solve(Z, b)
    h = make(B, v, t, regions, prec=1, aca_tol=1e-5, tol=1e-6)
    try:
        bd = torch.from_numpy(b).to(DEV)
        xd = torch.zeros_like(bd)
        B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        x = xd.cpu().numpy()
        assert rel(x[:g.ne], xr[:g.ne]) <= 1e-4
        assert rel(x[g.ne:], xr[g.ne:]) <= 1e-4
    finally:
        B.bem_destroy(h)


def test_layered_weight_gradient_equals_oracle(B, small):
    v, t, regions, g, Z = small["coated"]
    kh, e0 = W.plane_wave_batch(4, seed=2)
    Bm = MR.rhs_planewave(g, regions, K0, kh, e0)
    w = W.complex_normal(4, seed=6)
    p_ref, g_ref = MR.absorbed_and_weight_gradient(g, regions, Z, Bm, w)
    h = make(B, v, t, regions, prec=3, eta=0.0, refine_tol=1e-11)
    try:
        bmd = torch.from_numpy(np.ascontiguousarray(Bm.T)).to(DEV)
        p, grad, it = B.bem_grad_weights(h, bmd.data_ptr(), w)
        assert abs(p - p_ref) <= 1e-8 * abs(p_ref)
        assert rel(np.asarray(grad), g_ref) <= 1e-7
    finally:
        B.bem_destroy(h)


def test_layered_eps_gradient_equals_oracle(B, small):
    """dP/d eps of the coating and of the core by the adjoint solve and each
    region's dG/dk pass, against central differences of the oracle's dense layered
    solution (1e-5, as for one body: the operator entries agree to 1e-11)."""
    v, t, regions, g, Z = small["coated"]
    b = MR.rhs_planewave(g, regions, K0, [0.0, 0.0, 1.0], [1.0, 0.0, 0.0])
    ref = np.concatenate([MR.absorbed_eps_gradient(g, regions, K0, EPS3, r, b) for r in (1, 2)])
    h = make(B, v, t, regions, prec=2, eta=0.0, tol=1e-10, refine_tol=1e-13, maxit=3000)
    try:
        assert B.bem_num_regions(h) == 3
        bd = torch.from_numpy(np.ascontiguousarray(b[None, :])).to(DEV)
        x = torch.empty(2 * g.ne, dtype=torch.complex128, device=DEV)
        lam = torch.empty_like(x)
        B.bem_grad_weights(h, bd.data_ptr(), np.array([1.0 + 0j]), x.data_ptr(), lam.data_ptr(), _stream())
        d = B.bem_grad_eps(h, x.data_ptr(), lam.data_ptr(), _stream())
        assert d.shape == (4,)
        for r in range(2):
            assert np.abs(d[2 * r:2 * r + 2] - ref[2 * r:2 * r + 2]).max() <= 1e-5 * np.abs(ref[2 * r:2 * r + 2]).max()
    finally:
        B.bem_destroy(h)


def test_layered_context_refuses_single_body_calls(B, small):
    v, t, regions, g, Z = small["coated"]
    h = make(B, v, t, regions, prec=1)
    try:
        for call in (lambda: B.bem_partition(h),
                     lambda: B.bem_autotune(h, B.BEM_C64)):
            with pytest.raises(B.BemError) as ei:
                call()
            assert ei.value.status == B.BEM_ESTATE
        # kernel timing covers the three regions' products
        x = torch.zeros(2 * g.ne, dtype=torch.complex64, device=DEV)
        y = torch.empty_like(x)
        B.bem_profile_begin(h)
        B.bem_matvec(h, x.data_ptr(), y.data_ptr(), 1, B.BEM_C64, _stream())
        ms, launches = B.bem_profile_end(h)
        assert list(launches) == [3, 3, 3]
    finally:
        B.bem_destroy(h)


@pytest.fixture(scope="module")
def full():
    v, t, regions = coated(4, 3)
    return v, t, regions, R.build(v, t)


def test_coated_sphere_full_size_sampled_rows(B, full):
    """19,200 unknowns, k0 a = 6, leaf 64, eta 2, ACA 1e-4: the product in the
    configuration the benchmark times, on sampled rows computed one by one by
    the oracle (no dense matrix)."""
    v, t, regions, g = full
    h = make(B, v, t, regions, k0=6.0, prec=1, leaf=64, aca_tol=1e-4)
    try:
        assert B.bem_stats_get(h)["n_far_factored"] > 0
        x = W.complex_normal(2 * g.ne, seed=0).astype(np.complex64).astype(np.complex128)
        y = apply(B, h, x, B.BEM_C64)
        rows = np.random.default_rng(12).choice(2 * g.ne, 12, replace=False)
        ref = MR.pmchwt_regions_rows_apply(g, regions, 6.0, EPS3, x, rows)
        scale = np.sqrt(np.mean(np.abs(y) ** 2))
        assert np.abs(y[rows] - ref).max() / scale <= 2e-3
    finally:
        B.bem_destroy(h)


def test_coated_sphere_full_size_solve(B, full):
    """Mixed-precision solve (complex64 operator, ACA 1e-5, GMRES 1e-6) against the
    stored FP64 dense solution, and the powers against it and the coated-sphere series."""
    v, t, regions, g = full
    ref = np.load(GOLDEN)
    h = make(B, v, t, regions, k0=6.0, prec=1, leaf=64, aca_tol=1e-5, tol=1e-6, maxit=4000)
    try:
        b = MR.rhs_planewave(g, regions, 6.0, ref["khat"], ref["e0"])
        bd = torch.from_numpy(b).to(DEV)
        xd = torch.zeros_like(bd)
        B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 1, _stream())
        x = xd.cpu().numpy()
        xr = ref["x"]
        assert rel(x[:g.ne], xr[:g.ne]) <= 1e-3
        assert rel(x[g.ne:], xr[g.ne:]) <= 1e-3
        pa, pe, ps = B.bem_power(h, xd.data_ptr(), bd.data_ptr(), 1, _stream())
        for got, want in ((pa[0], ref["p_abs"]), (pe[0], ref["p_ext"]), (ps[0], ref["p_sca"])):
            assert abs(got - float(want)) <= 1e-3 * abs(float(want))
        # the discretisation error of the dense solution bounds the distance to the series
        a2 = np.pi
        for got, want, series in ((pe[0], ref["p_ext"], ref["mie"][0]), (pa[0], ref["p_abs"], ref["mie"][1]),
                                  (ps[0], ref["p_sca"], ref["mie"][2])):
            d_oracle = abs(float(want) / a2 - series) / series
            assert abs(got / a2 - series) / series <= d_oracle + 2e-3
    finally:
        B.bem_destroy(h)
