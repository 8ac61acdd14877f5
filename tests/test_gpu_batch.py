"""GPU tests of the multi-mesh graph batch (bem_batch_*) and the schedule
autotuner (bem_autotune).

The batch replays the very kernels of bem_matvec, so its products must equal the
individual calls bit for bit, on every launch.  The autotuner only changes how a
leaf's work is split among CTAs (the partial sums are grouped differently), so
products before and after agree to FP32 rounding (1e-6 relative) and stay
deterministic.
"""
import numpy as np
import pytest

import workloads as W

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


def make(B, v, t, k0, eps, prec=1):
    opt = B.bem_default_options()
    opt.precision = prec
    opt.leaf_size = 32
    opt.eta = 2.0
    opt.aca_tol = 1e-4
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, k0, eps)
    B.bem_assemble(h, _stream())
    return h


MESHES = [(lambda: W.icosphere(3), 6.0, 3.2 - 1.9j), (lambda: W.geodesic_sphere(9, 1.5), 3.0, 2.5 - 1.2j),
          (lambda: W.box_mesh(1.0, 0.8, 0.4, 10, 8, 4), 5.0, 4.0 - 2.0j)]


@pytest.mark.parametrize("prec,dtype,ct", [(1, 0, torch.complex64), (2, 1, torch.complex128)], ids=["c64", "c128"])
def test_graph_batch_equals_individual_products(B, prec, dtype, ct):
    hs, xs, ys, nr = [], [], [], []
    try:
        for i, (mesh, k0, eps) in enumerate(MESHES):
            v, t = mesh()
            h = make(B, v, t, k0, eps, prec)
            hs.append(h)
            n = B.bem_num_unknowns(h)
            r = 1 + 4 * i  # 1, 5, 9 right-hand sides
            X = W.complex_normal(n, seed=60 + i, nrhs=r)
            xs.append(torch.from_numpy(np.ascontiguousarray(X.T)).to(DEV, ct))
            ys.append(torch.empty_like(xs[-1]))
            nr.append(r)
        ref = []
        for h, x, r in zip(hs, xs, nr):
            y = torch.empty_like(x)
            B.bem_matvec(h, x.data_ptr(), y.data_ptr(), r, dtype, _stream())
            ref.append(y)
        batch = B.bem_batch_create(hs, [x.data_ptr() for x in xs], [y.data_ptr() for y in ys], nr, dtype, _stream())
        try:
            for _ in range(2):
                for y in ys:
                    y.zero_()
                B.bem_batch_launch(batch, _stream())
                torch.cuda.synchronize()
                for y, yr in zip(ys, ref):
                    assert torch.equal(y, yr)
        finally:
            B.bem_batch_destroy(batch)
    finally:
        for h in hs:
            B.bem_destroy(h)


def test_batch_rejects_a_context_twice(B):
    v, t = W.icosphere(2)
    h = make(B, v, t, 2.0, 3.2 - 1.9j)
    try:
        n = B.bem_num_unknowns(h)
        x = torch.zeros(n, dtype=torch.complex64, device=DEV)
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        with pytest.raises(B.BemError):
            B.bem_batch_create([h, h], [x.data_ptr()] * 2, [y1.data_ptr(), y2.data_ptr()], [1, 1], 0, _stream())
    finally:
        B.bem_destroy(h)


def test_autotune_keeps_the_product(B):
    v, t = W.icosphere(4)
    h = make(B, v, t, 10.0, 3.2 - 1.9j)
    try:
        n = B.bem_num_unknowns(h)
        x = torch.from_numpy(W.complex_normal(n, seed=70)).to(DEV, torch.complex64)
        y0 = torch.empty_like(x)
        B.bem_matvec(h, x.data_ptr(), y0.data_ptr(), 1, 0, _stream())
        chosen, ms = B.bem_autotune(h, 0, _stream())
        assert chosen % 152 == 0 and 4 * 152 <= chosen <= 96 * 152 and ms > 0
        y1, y2 = torch.empty_like(x), torch.empty_like(x)
        B.bem_matvec(h, x.data_ptr(), y1.data_ptr(), 1, 0, _stream())
        B.bem_matvec(h, x.data_ptr(), y2.data_ptr(), 1, 0, _stream())
        torch.cuda.synchronize()
        assert torch.equal(y1, y2)
        d = (y1 - y0).abs().max().item() / y0.abs().max().item()
        assert d <= 1e-6, d
        # the adjoint schedule is rebuilt with the new target
        z = torch.empty_like(x)
        B.bem_matvec_adjoint(h, x.data_ptr(), z.data_ptr(), 1, 0, _stream())
        torch.cuda.synchronize()
        lhs = torch.vdot(x, y1).item()
        rhs = torch.vdot(z, x).item()
        assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    finally:
        B.bem_destroy(h)


def test_profile_counts_operator_passes(B):
    """Kernel timing with 13 right-hand sides: three operator passes (8 + 4 + 1),
    so three launches of each kernel per product."""
    v, t = W.icosphere(3)
    h = make(B, v, t, 6.0, 3.2 - 1.9j)
    try:
        n = B.bem_num_unknowns(h)
        X = torch.zeros((13, n), dtype=torch.complex64, device=DEV)
        Y = torch.empty_like(X)
        B.bem_profile_begin(h)
        for _ in range(2):
            B.bem_matvec(h, X.data_ptr(), Y.data_ptr(), 13, 0, _stream())
        ms, cnt = B.bem_profile_end(h)
        assert list(cnt) == [6, 6, 6] and all(m > 0 for m in ms)
    finally:
        B.bem_destroy(h)
