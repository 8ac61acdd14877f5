"""bem_absorbed_power_static, the absorbed-power call that allocates no device memory.

It is meant for callers that cannot let the library allocate during the call: a
framework that owns all device memory through its own pool, or a loop that must
not take the synchronisation cudaMalloc/cudaFree can cause.  It must give the same result as bem_power, which allocates
its reduction buffer on first use, on consecutive calls that reuse the shared
fixed scratch.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2310_15644_gb300.build import build

    build()
    import paper_2310_15644_gb300.bem as mod

    return mod


def test_static_scratch_power_matches_bem_power(B):
    v, t = W.icosphere(3)
    opt = B.bem_default_options()
    opt.precision = B.BEM_PREC_C64
    opt.leaf_size = 32
    h = B.bem_create(opt)
    try:
        B.bem_set_mesh(h, v, t)
        B.bem_set_media(h, 4.0, 3.2 - 1.9j)
        stream = torch.cuda.current_stream().cuda_stream
        B.bem_assemble(h, stream)
        n = B.bem_num_unknowns(h)
        for call, nrhs in enumerate((3, 2)):                 # two calls in a row, different sizes
            x = W.complex_normal(n, seed=20 + call, nrhs=nrhs)
            xd = torch.from_numpy(np.ascontiguousarray(x.T)).to("cuda")
            pa_ref = B.bem_power(h, xd.data_ptr(), xd.data_ptr(), nrhs, stream)[0]
            out = torch.full((nrhs,), float("nan"), dtype=torch.float64, device="cuda")
            B.bem_absorbed_power_static(h, xd.data_ptr(), nrhs, out.data_ptr(), stream)
            torch.cuda.synchronize()
            pa = out.cpu().numpy()
            assert np.all(np.isfinite(pa))
            assert np.allclose(pa, pa_ref, rtol=1e-12, atol=1e-14 * np.abs(pa_ref).max())
        # sizes beyond the fixed scratch are refused with BEM_EINVAL, and so is a
        # right-hand-side count above the grid limit even where the scratch would hold it
        with pytest.raises(B.BemError) as ei:
            B.bem_absorbed_power_static(h, xd.data_ptr(), 100000, out.data_ptr(), stream)
        assert ei.value.status == B.BEM_EINVAL
        with pytest.raises(B.BemError) as ei:
            B.bem_power(h, xd.data_ptr(), xd.data_ptr(), 65536, stream)
        assert ei.value.status == B.BEM_EINVAL
    finally:
        B.bem_destroy(h)


def test_static_scratch_power_allocates_nothing(B):
    """The property the entry point exists for: after one warm-up call (module
    load and the lookup of the fixed array's address), calls at the largest size
    the fixed array holds leave the device's free memory unchanged.  bem_power is
    never called on this context, so its reduction buffer does not exist."""
    v, t = W.icosphere(3)
    opt = B.bem_default_options()
    opt.precision = B.BEM_PREC_C64
    opt.leaf_size = 32
    h = B.bem_create(opt)
    try:
        B.bem_set_mesh(h, v, t)
        B.bem_set_media(h, 4.0, 3.2 - 1.9j)
        stream = torch.cuda.current_stream().cuda_stream
        B.bem_assemble(h, stream)
        n = B.bem_num_unknowns(h)
        nblk = (len(t) + 255) // 256
        nrhs = 65536 // nblk                                  # largest call the fixed array holds
        gen = torch.Generator(device="cuda").manual_seed(5)
        xd = torch.randn((nrhs, n), dtype=torch.complex128, device="cuda", generator=gen)
        out = torch.empty(nrhs, dtype=torch.float64, device="cuda")
        B.bem_absorbed_power_static(h, xd.data_ptr(), 1, out.data_ptr(), stream)   # warm-up
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(3):
            B.bem_absorbed_power_static(h, xd.data_ptr(), nrhs, out.data_ptr(), stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, f"free device memory changed by {free0 - free1} bytes"
        assert torch.isfinite(out).all()
    finally:
        B.bem_destroy(h)
