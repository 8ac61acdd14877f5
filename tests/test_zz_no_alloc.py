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
        # sizes beyond the fixed scratch are refused with BEM_EINVAL
        with pytest.raises(B.BemError) as ei:
            B.bem_absorbed_power_static(h, xd.data_ptr(), 100000, out.data_ptr(), stream)
        assert ei.value.status == B.BEM_EINVAL
    finally:
        B.bem_destroy(h)
