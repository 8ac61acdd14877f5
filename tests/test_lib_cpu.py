"""CPU checks of the C library: it loads, exports every declared entry point, and
its host-side logic (argument checks, mesh -> RWG table, Debye helper) agrees
with the oracle.  No compute call reaches the GPU here."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import workloads as W
from oracle import debye, rwg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2310_15644_gb300.build import build

    build()
    import paper_2310_15644_gb300.bem as mod

    return mod


def _declared():
    src = open(os.path.join(ROOT, "include", "bem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bem_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(B):
    declared = _declared()
    assert declared, "no declarations parsed"
    assert sorted(B.EXPORTS) == declared
    lib = ctypes.CDLL(B.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (bem_[a-z0-9_]+)$", out, flags=re.M))
    assert set(declared) <= exported


def test_rwg_table_matches_oracle(B):
    for v, t in (W.icosphere(2), W.box_mesh(1.0, 0.7, 0.3, 5, 4, 2)):
        h = B.bem_create()
        try:
            B.bem_set_mesh(h, v, t)
            e = B.bem_edges(h)
            g = rwg.build(v, t)
            assert np.array_equal(e[:, :2], g.edges)
            assert np.array_equal(e[:, 2], g.tplus)
            assert np.array_equal(e[:, 3], g.tminus)
            assert B.bem_num_unknowns(h) == 2 * g.ne
        finally:
            B.bem_destroy(h)


def test_invalid_inputs_rejected_before_any_launch(B):
    v, t = W.icosphere(1)
    h = B.bem_create()
    try:
        with pytest.raises(B.BemError) as ei:
            B.bem_set_mesh(h, v, t[1:])
        assert ei.value.status == B.BEM_EINVAL
        bad = t.copy()
        bad[0] = bad[0][[0, 2, 1]]
        with pytest.raises(B.BemError):
            B.bem_set_mesh(h, v, bad)
        vz = v.copy()
        vz[t[0, 2]] = 0.5 * (vz[t[0, 0]] + vz[t[0, 1]])
        with pytest.raises(B.BemError):
            B.bem_set_mesh(h, vz, t)
        B.bem_set_mesh(h, v, t)
        with pytest.raises(B.BemError) as ei:
            B.bem_set_media(h, 2.0, 3.2 + 1.9j)       # gain medium under e^{+jwt}
        assert ei.value.status == B.BEM_EINVAL
        with pytest.raises(B.BemError):
            B.bem_set_media(h, -1.0, 3.0)
        # product before assembly
        with pytest.raises(B.BemError) as ei:
            B.bem_matvec(h, 0, 0, 1, B.BEM_C64)
        assert ei.value.status == B.BEM_ESTATE
        with pytest.raises(B.BemError) as ei:
            B.bem_assemble(h)                            # media not set yet
        assert ei.value.status == B.BEM_ESTATE
    finally:
        B.bem_destroy(h)
    opt = B.bem_default_options()
    opt.leaf_size = 65
    with pytest.raises(B.BemError):
        B.bem_create(opt)


def test_debye_helper_matches_oracle(B):
    for f in (0.0, 1e9, 1e11, 1e12, 3e12):
        assert abs(B.bem_debye_eps(f) - debye.eps_r(f)) < 1e-12 * abs(debye.eps_r(f))
    p = [4.0, 50.0, 5.0, 8e-12, 0.1e-12]
    assert abs(B.bem_debye_eps(1e12, p) - debye.eps_r(1e12, *p)) < 1e-12 * 10


def test_struct_layout_matches_header(B, tmp_path):
    """The ctypes mirrors of bem_options and bem_stats have the C layout of bem.h."""
    structs = {"bem_options": B.bem_options, "bem_stats": B.bem_stats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "bem.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line in filter(None, out):
        sname, what, val = line.split()
        cls = structs[sname]
        got = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert got == int(val), (sname, what, got, val)


def test_new_entry_points_check_state_and_arguments(B):
    """Adjoint, gradient, autotuning and batch calls refuse a context that is not
    assembled, and bad options, before touching the GPU."""
    v, t = W.icosphere(1)
    h = B.bem_create()
    try:
        B.bem_set_mesh(h, v, t)
        for call in (lambda: B.bem_matvec_adjoint(h, 0, 0, 1, B.BEM_C64),
                     lambda: B.bem_solve_adjoint(h, 0, 0, 1),
                     lambda: B.bem_grad_eps(h, 0, 0),
                     lambda: B.bem_grad_weights(h, 0, [1.0]),
                     lambda: B.bem_autotune(h, B.BEM_C64),
                     lambda: B.bem_absorbed_power_gradient(h, 0, 0, 1)):
            with pytest.raises(B.BemError) as ei:
                call()
            assert ei.value.status == B.BEM_ESTATE
        with pytest.raises(B.BemError) as ei:
            B.bem_batch_create([h], [0], [0], [1], B.BEM_C64)
        assert ei.value.status == B.BEM_EINVAL
    finally:
        B.bem_destroy(h)
    opt = B.bem_default_options()
    assert opt.solver == B.BEM_SOLVER_GMRES
    for field, value in (("solver", 4), ("solver", -1), ("precision", 8)):
        o = B.bem_default_options()
        setattr(o, field, value)
        with pytest.raises(B.BemError):
            B.bem_create(o)


def _layered_mesh(level_outer=2, level_inner=1, radius_inner=0.5):
    from oracle import multiregion as MR

    (vo, to), (vi, ti) = W.concentric_spheres(level_outer, 1.0, level_inner, radius_inner)
    v, t, s = MR.union_mesh([(vo, to), (vi, ti)])
    regions = np.where(s[:, None] == 0, np.array([0, 1]), np.array([1, 2]))
    return v, t, regions


def test_layered_boundaries_match_oracle(B):
    """bem_set_regions (host only): each region's boundary edges and signs are the
    oracle's, for a coated sphere and for two spheres side by side in free space."""
    from oracle import multiregion as MR

    cases = [_layered_mesh()]
    (va, ta), (vb, tb) = W.icosphere(1, 0.6, (-1.0, 0.0, 0.0)), W.icosphere(2, 0.5, (1.0, 0.2, 0.0))
    v2, t2, s2 = MR.union_mesh([(va, ta), (vb, tb)])
    cases.append((v2, t2, np.where(s2[:, None] == 0, np.array([0, 1]), np.array([0, 2]))))
    for v, t, regions in cases:
        g = rwg.build(v, t)
        h = B.bem_create()
        try:
            B.bem_set_mesh(h, v, t)
            assert B.bem_num_regions(h) == -1
            B.bem_set_regions(h, 2.0, [1.0, 3.2 - 1.9j, 2.5 - 1.2j], regions)
            assert B.bem_num_regions(h) == 3
            for r in range(3):
                edges, sign = B.bem_region_boundary(h, r)
                _, e_o, s_o = MR.region_boundary(g, regions, r)
                assert np.array_equal(edges, e_o), r
                assert np.array_equal(sign.astype(np.float64), s_o), r
            # bem_set_media returns to one body; a new mesh drops the regions and the media
            B.bem_set_media(h, 2.0, 3.2 - 1.9j)
            assert B.bem_num_regions(h) == 2
            B.bem_set_regions(h, 2.0, [1.0, 3.2 - 1.9j, 2.5 - 1.2j], regions)
            B.bem_set_mesh(h, v, t)
            assert B.bem_num_regions(h) == -1
            with pytest.raises(B.BemError) as ei:
                B.bem_region_boundary(h, 0)
            assert ei.value.status == B.BEM_ESTATE
        finally:
            B.bem_destroy(h)


def test_layered_regions_rejected_when_inconsistent(B):
    v, t, regions = _layered_mesh(1, 0)
    eps = [1.0, 3.2 - 1.9j, 2.5 - 1.2j]
    h = B.bem_create()
    try:
        with pytest.raises(B.BemError) as ei:       # no mesh yet
            B.bem_set_regions(h, 2.0, eps, regions)
        assert ei.value.status == B.BEM_ESTATE
        B.bem_set_mesh(h, v, t)
        bad = []
        r = regions.copy(); r[:, :] = r[:, ::-1]; bad.append(r)          # exterior normals point inward
        r = regions.copy(); r[0] = [1, 1]; bad.append(r)                  # same region on both sides
        r = regions.copy(); r[0] = [0, 5]; bad.append(r)                  # region index out of range
        r = regions.copy(); r[0] = [0, 2]; bad.append(r)                  # an edge between two region pairs
        for r in bad:
            with pytest.raises(B.BemError) as ei:
                B.bem_set_regions(h, 2.0, eps, r)
            assert ei.value.status == B.BEM_EINVAL
        B.bem_set_media(h, 2.0, 3.2 - 1.9j)
        with pytest.raises(B.BemError):                                   # region 3 has no boundary
            B.bem_set_regions(h, 2.0, eps + [2.0], regions)
        assert B.bem_num_regions(h) == 2                                  # the media set before are kept
        with pytest.raises(B.BemError):                                   # gain medium
            B.bem_set_regions(h, 2.0, [1.0, 3.2 + 1.0j, 2.5], regions)
        with pytest.raises(B.BemError):
            B.bem_set_regions(h, -1.0, eps, regions)
        # a valid call, then the calls that a layered context refuses before any launch
        B.bem_set_regions(h, 2.0, eps, regions)
        for call in (lambda: B.bem_matvec(h, 0, 0, 1, B.BEM_C64),
                     lambda: B.bem_solve(h, 0, 0, 1)):
            with pytest.raises(B.BemError) as ei:
                call()
            assert ei.value.status == B.BEM_ESTATE
    finally:
        B.bem_destroy(h)


def test_autograd_refuses_eps_on_a_layered_context(B):
    torch = pytest.importorskip("torch")
    from paper_2310_15644_gb300.autograd import absorbed_power

    v, t, regions = _layered_mesh(1, 0)
    h = B.bem_create()
    try:
        B.bem_set_mesh(h, v, t)
        B.bem_set_regions(h, 2.0, [1.0, 3.2 - 1.9j, 2.5 - 1.2j], regions)
        w = torch.ones(1, dtype=torch.complex128)
        eps = torch.tensor([3.2, -1.9], dtype=torch.float64)
        bm = torch.zeros(1, 2, dtype=torch.complex128)
        with pytest.raises(ValueError, match="single-body"):
            absorbed_power(w, h, bm, eps=eps, k0=2.0)
    finally:
        B.bem_destroy(h)


def test_planar_operators_reject_bad_input_before_any_launch(B):
    sq = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    for verts, k in ((sq[:2], 1.0), (sq[::-1].copy(), 1.0), (sq, 1.0 + 0.1j), (sq, -1.0),
                     (np.array([[0.0, 0.0], [0.0, 0.0], [1.0, 1.0]]), 1.0)):
        with pytest.raises(B.BemError) as ei:
            B.bem_planar_operators(None, verts, k, 0, 0, 0)
        assert ei.value.status == B.BEM_EINVAL


def _precond_ctx(B, v, t):
    opt = B.bem_default_options()
    opt.preconditioner = B.BEM_PRECOND_CALDERON
    h = B.bem_create(opt)
    B.bem_set_mesh(h, v, t)
    return h


def _dense(rows, cols, ptr, col, val):
    A = np.zeros((rows, cols))
    for r in range(rows):
        A[r, col[ptr[r]:ptr[r + 1]]] += val[ptr[r]:ptr[r + 1]]
    return A


@pytest.mark.parametrize("mesh", ["ico2", "box"])
def test_calderon_matrices_match_oracle(B, mesh):
    """The library's Buffa-Christiansen coefficients C and mixed Gram matrix G (host,
    FP64, built from the closed-form fluxes and a three-point rule) against the
    oracle's (least-norm solves, seven-point rule) on a sphere and on a box whose
    vertices have 4 to 8 neighbours."""
    from oracle import calderon as CA

    v, t = W.icosphere(2) if mesh == "ico2" else W.box_mesh(1.0, 0.7, 0.3, 4, 3, 2)
    ref = CA.refine(rwg.build(v, t))
    h = _precond_ctx(B, v, t)
    try:
        C = _dense(*B.bem_precond_matrix(h, 0))
        G = _dense(*B.bem_precond_matrix(h, 1))
    finally:
        B.bem_destroy(h)
    assert C.shape == ref.C.shape
    assert np.abs(C - ref.C).max() <= 1e-12 * np.abs(ref.C).max()
    Go = CA.mixed_gram(ref)
    assert np.abs(G - Go).max() <= 1e-12 * np.abs(Go).max()


def test_calderon_matrix_argument_checks(B):
    v, t = W.icosphere(1)
    h = B.bem_create()
    try:
        B.bem_set_mesh(h, v, t)
        with pytest.raises(B.BemError):
            B.bem_precond_matrix(h, 0)  # created without the preconditioner
    finally:
        B.bem_destroy(h)
    h = _precond_ctx(B, v, t)
    try:
        with pytest.raises(B.BemError):
            B.bem_precond_matrix(h, 2)
    finally:
        B.bem_destroy(h)
