"""Host-side fault injection (bem_debug_fail_alloc_after): the library's device
allocations fail after N successful ones, as if the GPU were out of memory; no CUDA
call is made for the failed allocation, so no GPU fault is involved.  Every entry
point that needed the allocation returns BEM_ENOMEM, and once the injection is off
the same context assembles, applies and solves exactly as a fresh one does."""
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


def _ctx(B, v, t):
    opt = B.bem_default_options()
    opt.leaf_size = 16
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    B.bem_set_media(h, 2.0, 3.2 - 1.9j)
    return h


def _product(B, h, x):
    xd = torch.from_numpy(x).to(DEV)
    yd = torch.empty_like(xd)
    B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, B.BEM_C64, _stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def test_assembly_enomem_then_recovery(B):
    v, t = W.icosphere(2)
    h0 = _ctx(B, v, t)
    try:
        B.bem_assemble(h0, _stream())
        n = B.bem_num_unknowns(h0)
        x = W.complex_normal(n, seed=5).astype(np.complex64)
        y0 = _product(B, h0, x)
    finally:
        B.bem_destroy(h0)
    failed = 0
    for after in (0, 1, 3, 8, 20, 40):
        h = _ctx(B, v, t)
        try:
            B.bem_debug_fail_alloc_after(after)
            try:
                B.bem_assemble(h, _stream())
                status = B.BEM_OK
            except B.BemError as e:
                status = e.status
            finally:
                B.bem_debug_fail_alloc_after(-1)
            assert status in (B.BEM_OK, B.BEM_ENOMEM), status
            if status == B.BEM_ENOMEM:
                failed += 1
                # nothing was assembled: a product is refused, not run on a partial operator
                xd = torch.from_numpy(x).to(DEV)
                yd = torch.empty_like(xd)
                with pytest.raises(B.BemError) as ei:
                    B.bem_matvec(h, xd.data_ptr(), yd.data_ptr(), 1, B.BEM_C64, _stream())
                assert ei.value.status == B.BEM_ESTATE
            # the same context, injection off: assembles and gives the fresh context's product
            B.bem_assemble(h, _stream())
            assert np.array_equal(_product(B, h, x), y0)
        finally:
            B.bem_destroy(h)
    assert failed >= 3  # the small counts fail inside the assembly


def test_solve_enomem_then_recovery(B):
    v, t = W.icosphere(2)
    h = _ctx(B, v, t)
    try:
        B.bem_assemble(h, _stream())
        n = B.bem_num_unknowns(h)
        bd = torch.empty((3, n), dtype=torch.complex128, device=DEV)
        khat, e0 = W.plane_wave_batch(3, seed=2)
        B.bem_rhs_planewave(h, khat, e0, bd.data_ptr(), B.BEM_C128, _stream())
        xd = torch.zeros_like(bd)
        B.bem_debug_fail_alloc_after(0)  # the solver's workspace cannot be allocated
        try:
            with pytest.raises(B.BemError) as ei:
                B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 3, _stream())
        finally:
            B.bem_debug_fail_alloc_after(-1)
        assert ei.value.status == B.BEM_ENOMEM
        xd.zero_()
        it, rr, st = B.bem_solve(h, bd.data_ptr(), xd.data_ptr(), 3, _stream())
        assert st == B.BEM_OK and np.all(rr <= 1.5e-6)
    finally:
        B.bem_destroy(h)
