"""Thin ctypes binding of libbem (include/bem.h): argument marshalling only.

Every function here forwards to the C entry point of the same name; device
buffers are passed as raw pointers (``tensor.data_ptr()``) and streams as
``torch.cuda.Stream.cuda_stream``.  There is no fallback: if the shared library
is missing or fails to load, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbem.so")

BEM_OK, BEM_EINVAL, BEM_ENOMEM, BEM_ECUDA, BEM_ENOCONV, BEM_ETIMEOUT, BEM_ESTATE = range(7)
BEM_PREC_C64, BEM_PREC_C128, BEM_PREC_BF16F = 1, 2, 4
BEM_C64, BEM_C128, BEM_C64_BF16F, BEM_C64_TC = 0, 1, 2, 3
BEM_SOLVER_GMRES, BEM_SOLVER_CGS, BEM_SOLVER_BICGSTAB, BEM_SOLVER_CGNR = 0, 1, 2, 3
BEM_PRECOND_NONE, BEM_PRECOND_CALDERON = 0, 1
STATUS_NAMES = {0: "BEM_OK", 1: "BEM_EINVAL", 2: "BEM_ENOMEM", 3: "BEM_ECUDA", 4: "BEM_ENOCONV",
                5: "BEM_ETIMEOUT", 6: "BEM_ESTATE"}

# Every entry point declared in include/bem.h (checked by the test-suite).
EXPORTS = [
    "bem_default_options", "bem_create", "bem_destroy", "bem_last_error", "bem_set_mesh", "bem_set_media",
    "bem_debye_eps", "bem_assemble", "bem_num_edges", "bem_num_unknowns", "bem_edges", "bem_stats_get",
    "bem_partition", "bem_eval_entries", "bem_matvec", "bem_rhs_planewave", "bem_solve", "bem_power",
    "bem_power_density", "bem_profile_begin", "bem_profile_end", "bem_absorbed_power_static",
    "bem_matvec_adjoint", "bem_solve_adjoint", "bem_absorbed_power_gradient", "bem_grad_weights", "bem_grad_eps",
    "bem_autotune", "bem_batch_create", "bem_batch_launch", "bem_batch_destroy", "bem_set_regions",
    "bem_region_boundary", "bem_num_regions", "bem_planar_operators", "bem_measure_fma_peak",
    "bem_debug_fail_alloc_after", "bem_planar_calderon", "bem_fft", "bem_planar_skeleton",
    "bem_planar_woodbury_solve", "bem_precond_apply", "bem_precond_matrix",
]
KERNEL_NAMES = ["k_gather", "k_vhx", "k_rows"]   # BEM_KERNEL_GATHER, _VHX, _ROWS


class bem_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int), ("leaf_size", ctypes.c_int), ("eta", ctypes.c_double),
        ("aca_tol", ctypes.c_double), ("aca_max_rank", ctypes.c_int), ("gmres_restart", ctypes.c_int),
        ("maxit", ctypes.c_int), ("tol", ctypes.c_double), ("refine_tol", ctypes.c_double),
        ("refine_maxit", ctypes.c_int), ("solver", ctypes.c_int), ("aca_recompress", ctypes.c_int),
        ("preconditioner", ctypes.c_int), ("precond_aca_tol", ctypes.c_double), ("precond_near_only", ctypes.c_int),
    ]


# parts of bem_assemble, in the order of BEM_PHASE_* in bem.h
PHASE_NAMES = ("tree", "singular", "aca", "near", "plan")


class bem_stats(ctypes.Structure):
    _fields_ = [
        ("ne", ctypes.c_int64), ("nt", ctypes.c_int64), ("n_clusters", ctypes.c_int64),
        ("n_leaves", ctypes.c_int64), ("n_near", ctypes.c_int64), ("n_far", ctypes.c_int64),
        ("n_far_dense", ctypes.c_int64), ("n_far_split", ctypes.c_int64), ("n_far_factored", ctypes.c_int64),
        ("near_entries", ctypes.c_int64), ("factor_entries", ctypes.c_int64 * 3), ("max_rank", ctypes.c_int64),
        ("singular_pairs", ctypes.c_int64), ("matvec_bytes_c64", ctypes.c_int64),
        ("matvec_bytes_c128", ctypes.c_int64), ("kernel_bytes_c64", ctypes.c_int64 * 3),
        ("kernel_bytes_c128", ctypes.c_int64 * 3),
        ("matvec_bytes_bf16f", ctypes.c_int64), ("kernel_bytes_bf16f", ctypes.c_int64 * 3),
        ("matvec_bytes_tc", ctypes.c_int64), ("kernel_bytes_tc", ctypes.c_int64 * 3), ("t_rows", ctypes.c_int64),
        ("assemble_ms", ctypes.c_double),
        ("assemble_phase_ms", ctypes.c_double * 5),
        ("tc_passes", ctypes.c_int64),
        ("precond_fine_ne", ctypes.c_int64), ("precond_gram_nnz", ctypes.c_int64),
        ("precond_gram_steps", ctypes.c_int64), ("precond_bytes_c64", ctypes.c_int64),
        ("precond_gram_interval", ctypes.c_double * 2), ("precond_assemble_ms", ctypes.c_double),
    ]


class bem_c128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class BemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbem.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i32p, i64p, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)
    ctx = ctypes.c_void_p
    sig = {
        "bem_default_options": (None, [ctypes.POINTER(bem_options)]),
        "bem_create": (ctypes.c_int, [ctypes.POINTER(bem_options), ctypes.POINTER(ctx)]),
        "bem_destroy": (None, [ctx]),
        "bem_last_error": (ctypes.c_char_p, [ctx]),
        "bem_set_mesh": (ctypes.c_int, [ctx, dp, ctypes.c_int64, i32p, ctypes.c_int64]),
        "bem_set_media": (ctypes.c_int, [ctx, ctypes.c_double, bem_c128, bem_c128]),
        "bem_set_regions": (ctypes.c_int, [ctx, ctypes.c_double, ctypes.c_int, ctypes.POINTER(bem_c128),
                                           ctypes.POINTER(bem_c128), i32p]),
        "bem_region_boundary": (ctypes.c_int, [ctx, ctypes.c_int, i64p, i32p, ctypes.POINTER(ctypes.c_int8)]),
        "bem_num_regions": (ctypes.c_int, [ctx]),
        "bem_planar_operators": (ctypes.c_int, [ctx, dp, ctypes.c_int, bem_c128, ctypes.c_int, vp, vp, vp, vp]),
        "bem_debye_eps": (ctypes.c_int, [ctypes.c_double, dp, ctypes.POINTER(bem_c128)]),
        "bem_assemble": (ctypes.c_int, [ctx, vp]),
        "bem_num_edges": (ctypes.c_int64, [ctx]),
        "bem_num_unknowns": (ctypes.c_int64, [ctx]),
        "bem_edges": (ctypes.c_int, [ctx, i32p]),
        "bem_stats_get": (ctypes.c_int, [ctx, ctypes.POINTER(bem_stats)]),
        "bem_partition": (ctypes.c_int, [ctx, i64p, i32p, i32p]),
        "bem_eval_entries": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int64, vp, ctypes.c_int, vp]),
        "bem_matvec": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
        "bem_matvec_adjoint": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
        "bem_solve_adjoint": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int), dp]),
        "bem_absorbed_power_gradient": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int, vp]),
        "bem_grad_eps": (ctypes.c_int, [ctx, vp, vp, dp, vp]),
        "bem_autotune": (ctypes.c_int, [ctx, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int), dp]),
        "bem_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                            ctypes.POINTER(ctypes.c_int), ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "bem_batch_launch": (ctypes.c_int, [vp, vp]),
        "bem_batch_destroy": (None, [vp]),
        "bem_grad_weights": (ctypes.c_int, [ctx, vp, ctypes.c_int, ctypes.POINTER(bem_c128), dp,
                                            ctypes.POINTER(bem_c128), vp, vp, vp, ctypes.POINTER(ctypes.c_int)]),
        "bem_rhs_planewave": (ctypes.c_int, [ctx, dp, ctypes.POINTER(bem_c128), ctypes.c_int, vp, ctypes.c_int, vp]),
        "bem_solve": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_int), dp]),
        "bem_power": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int, dp, dp, dp, vp]),
        "bem_power_density": (ctypes.c_int, [ctx, vp, vp, vp]),
        "bem_profile_begin": (ctypes.c_int, [ctx]),
        "bem_profile_end": (ctypes.c_int, [ctx, dp, i64p]),
        "bem_absorbed_power_static": (ctypes.c_int, [ctx, vp, ctypes.c_int, vp, vp]),
        "bem_measure_fma_peak": (ctypes.c_int, [ctypes.c_int, vp, dp]),
        "bem_planar_calderon": (ctypes.c_int, [ctx, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                               vp, vp, vp, vp]),
        "bem_fft": (ctypes.c_int, [ctx, vp, ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_longlong,
                                   ctypes.c_int, vp]),
        "bem_planar_skeleton": (ctypes.c_int, [ctx, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                               vp, vp, ctypes.POINTER(ctypes.c_int), vp]),
        "bem_planar_woodbury_solve": (ctypes.c_int, [ctx, vp, ctypes.c_int, vp, vp, ctypes.c_int, vp, vp,
                                                     ctypes.c_int, vp]),
        "bem_debug_fail_alloc_after": (None, [ctypes.c_longlong]),
        "bem_precond_apply": (ctypes.c_int, [ctx, vp, vp, ctypes.c_int, ctypes.c_int, vp]),
        "bem_precond_matrix": (ctypes.c_int, [ctx, ctypes.c_int, i64p, i64p, i64p, i32p, i32p, dp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


lib = _load()


def _np_ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _check(ctx, st):
    if st != BEM_OK:
        msg = lib.bem_last_error(ctx) if ctx else b""
        raise BemError(st, (msg or b"").decode())


# ---- one-to-one wrappers (same names as the C entry points) ---------------------------------

def bem_default_options() -> bem_options:
    o = bem_options()
    lib.bem_default_options(ctypes.byref(o))
    return o


def bem_create(opt: bem_options | None = None):
    h = ctypes.c_void_p()
    st = lib.bem_create(ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    _check(None, st)
    return h


def bem_destroy(ctx) -> None:
    lib.bem_destroy(ctx)


def bem_last_error(ctx) -> str:
    return (lib.bem_last_error(ctx) or b"").decode()


def bem_set_mesh(ctx, verts, tris) -> None:
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tris, dtype=np.int32)
    _check(ctx, lib.bem_set_mesh(ctx, _np_ptr(v, ctypes.c_double), len(v), _np_ptr(t, ctypes.c_int32), len(t)))


def bem_set_media(ctx, k0: float, eps_r: complex, mu_r: complex = 1.0) -> None:
    e, m = complex(eps_r), complex(mu_r)
    _check(ctx, lib.bem_set_media(ctx, float(k0), bem_c128(e.real, e.imag), bem_c128(m.real, m.imag)))


def bem_set_regions(ctx, k0: float, eps_r, tri_regions, mu_r=None) -> None:
    """Layered body: eps_r / mu_r per region (entry 0, the exterior, ignored),
    tri_regions (nt, 2) = (region on the normal side, region behind) per triangle."""
    n = len(eps_r)
    mu_r = [1.0] * n if mu_r is None else mu_r
    if len(mu_r) != n:
        raise ValueError("eps_r and mu_r need one value per region")
    eps = (bem_c128 * n)(*[bem_c128(complex(e).real, complex(e).imag) for e in eps_r])
    mu = (bem_c128 * n)(*[bem_c128(complex(m).real, complex(m).imag) for m in mu_r])
    tr = np.ascontiguousarray(tri_regions, dtype=np.int32)
    _check(ctx, lib.bem_set_regions(ctx, float(k0), n, eps, mu, _np_ptr(tr, ctypes.c_int32)))


def bem_region_boundary(ctx, r: int):
    """(edges, sign) of region r's boundary: the context's edge indices and +1 / -1."""
    n = ctypes.c_int64()
    _check(ctx, lib.bem_region_boundary(ctx, int(r), ctypes.byref(n), None, None))
    edges = np.zeros(n.value, dtype=np.int32)
    sign = np.zeros(n.value, dtype=np.int8)
    _check(ctx, lib.bem_region_boundary(ctx, int(r), ctypes.byref(n), _np_ptr(edges, ctypes.c_int32),
                                        _np_ptr(sign, ctypes.c_int8)))
    return edges, sign


def bem_planar_operators(ctx, verts, k: complex, s_ptr: int, d_ptr: int, n_ptr: int, stream: int = 0,
                         fp32: bool = False) -> None:
    """Dense 2-D Galerkin S, D, N (device complex128 n x n, row-major) of a closed polygon."""
    v = np.ascontiguousarray(verts, dtype=np.float64)
    kk = complex(k)
    _check(ctx, lib.bem_planar_operators(ctx, _np_ptr(v, ctypes.c_double), len(v), bem_c128(kk.real, kk.imag),
                                    1 if fp32 else 0, ctypes.c_void_p(s_ptr or None), ctypes.c_void_p(d_ptr or None),
                                    ctypes.c_void_p(n_ptr or None), ctypes.c_void_p(stream)))


def bem_debye_eps(freq_hz: float, params=None) -> complex:
    out = bem_c128()
    p = None if params is None else _np_ptr(np.ascontiguousarray(params, dtype=np.float64), ctypes.c_double)
    _check(None, lib.bem_debye_eps(float(freq_hz), p, ctypes.byref(out)))
    return complex(out.re, out.im)


def bem_assemble(ctx, stream: int = 0) -> None:
    _check(ctx, lib.bem_assemble(ctx, ctypes.c_void_p(stream)))


def bem_num_edges(ctx) -> int:
    return int(lib.bem_num_edges(ctx))


def bem_num_unknowns(ctx) -> int:
    return int(lib.bem_num_unknowns(ctx))


def bem_edges(ctx) -> np.ndarray:
    ne = bem_num_edges(ctx)
    out = np.zeros((ne, 4), dtype=np.int32)
    _check(ctx, lib.bem_edges(ctx, _np_ptr(out, ctypes.c_int32)))
    return out


def bem_stats_get(ctx) -> dict:
    s = bem_stats()
    _check(ctx, lib.bem_stats_get(ctx, ctypes.byref(s)))
    d = {name: getattr(s, name) for name, _ in bem_stats._fields_}
    for k in ("factor_entries", "kernel_bytes_c64", "kernel_bytes_c128", "kernel_bytes_bf16f", "kernel_bytes_tc",
              "precond_gram_interval"):
        d[k] = list(getattr(s, k))
    d["assemble_phase_ms"] = dict(zip(PHASE_NAMES, s.assemble_phase_ms))
    return d


def bem_partition(ctx):
    s = bem_stats_get(ctx)
    perm = np.zeros(s["ne"], dtype=np.int64)
    near = np.zeros((s["n_near"], 4), dtype=np.int32)
    far = np.zeros((s["n_far"], 4), dtype=np.int32)
    _check(ctx, lib.bem_partition(ctx, _np_ptr(perm, ctypes.c_int64), _np_ptr(near, ctypes.c_int32),
                                  _np_ptr(far, ctypes.c_int32)))
    return perm, near, far


def bem_eval_entries(ctx, rows_ptr: int, cols_ptr: int, count: int, out_ptr: int, dtype: int, stream: int = 0) -> None:
    _check(ctx, lib.bem_eval_entries(ctx, ctypes.c_void_p(rows_ptr), ctypes.c_void_p(cols_ptr), int(count),
                                     ctypes.c_void_p(out_ptr), int(dtype), ctypes.c_void_p(stream)))


def bem_precond_apply(ctx, x_ptr: int, y_ptr: int, nrhs: int, dtype: int, stream: int = 0) -> None:
    """y = P x with the Calderon preconditioner (device pointers, 2ne x nrhs)."""
    _check(ctx, lib.bem_precond_apply(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), int(nrhs), int(dtype),
                                      ctypes.c_void_p(stream)))


def bem_precond_matrix(ctx, which: int):
    """(rows, cols, ptr, col, val) of the preconditioner's matrix `which` (0: C, 1: G), host arrays."""
    rows, cols, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(ctx, lib.bem_precond_matrix(ctx, int(which), ctypes.byref(rows), ctypes.byref(cols), ctypes.byref(nnz),
                                       None, None, None))
    ptr = np.empty(rows.value + 1, np.int32)
    col = np.empty(nnz.value, np.int32)
    val = np.empty(nnz.value, np.float64)
    _check(ctx, lib.bem_precond_matrix(ctx, int(which), None, None, None,
                                       ptr.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       col.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       val.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return rows.value, cols.value, ptr, col, val


def bem_matvec(ctx, x_ptr: int, y_ptr: int, nrhs: int, dtype: int, stream: int = 0) -> None:
    _check(ctx, lib.bem_matvec(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), int(nrhs), int(dtype),
                               ctypes.c_void_p(stream)))


def bem_matvec_adjoint(ctx, x_ptr: int, y_ptr: int, nrhs: int, dtype: int, stream: int = 0) -> None:
    _check(ctx, lib.bem_matvec_adjoint(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), int(nrhs), int(dtype),
                                       ctypes.c_void_p(stream)))


def bem_rhs_planewave(ctx, khat, e0, b_ptr: int, dtype: int, stream: int = 0) -> None:
    kh = np.ascontiguousarray(np.atleast_2d(khat), dtype=np.float64)
    e = np.ascontiguousarray(np.atleast_2d(e0), dtype=np.complex128)
    _check(ctx, lib.bem_rhs_planewave(ctx, _np_ptr(kh, ctypes.c_double), e.ctypes.data_as(ctypes.POINTER(bem_c128)),
                                      len(kh), ctypes.c_void_p(b_ptr), int(dtype), ctypes.c_void_p(stream)))


def bem_solve(ctx, b_ptr: int, x_ptr: int, nrhs: int, stream: int = 0, raise_on_noconv: bool = True):
    """Returns (iterations, relative residual per right-hand side, status)."""
    it = ctypes.c_int(0)
    rel = np.zeros(nrhs, dtype=np.float64)
    st = lib.bem_solve(ctx, ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr), int(nrhs), ctypes.c_void_p(stream),
                       ctypes.byref(it), _np_ptr(rel, ctypes.c_double))
    if st != BEM_OK and not (st == BEM_ENOCONV and not raise_on_noconv):
        _check(ctx, st)
    return it.value, rel, st


def bem_solve_adjoint(ctx, g_ptr: int, lam_ptr: int, nrhs: int, stream: int = 0, raise_on_noconv: bool = True):
    """Solve Z^H lambda = g.  Returns (iterations, relative residual per right-hand side, status)."""
    it = ctypes.c_int(0)
    rel = np.zeros(nrhs, dtype=np.float64)
    st = lib.bem_solve_adjoint(ctx, ctypes.c_void_p(g_ptr), ctypes.c_void_p(lam_ptr), int(nrhs),
                               ctypes.c_void_p(stream), ctypes.byref(it), _np_ptr(rel, ctypes.c_double))
    if st != BEM_OK and not (st == BEM_ENOCONV and not raise_on_noconv):
        _check(ctx, st)
    return it.value, rel, st


def bem_planar_calderon(ctx, verts, k0: float, cp_ptr: int, le_ptr: int = 0, lh_ptr: int = 0, a: float = 0.0,
                        stream: int = 0, fp32: bool = False) -> None:
    v = np.ascontiguousarray(verts, dtype=np.float64)
    _check(ctx, lib.bem_planar_calderon(ctx, _np_ptr(v, ctypes.c_double), int(v.shape[0]), float(k0), float(a),
                                        1 if fp32 else 0, ctypes.c_void_p(cp_ptr), ctypes.c_void_p(le_ptr or None),
                                        ctypes.c_void_p(lh_ptr or None), ctypes.c_void_p(stream)))


def bem_fft(ctx, x_ptr: int, n: int, stride: int = 1, batch: int = 1, batch_stride: int | None = None,
            inverse: bool = False, stream: int = 0) -> None:
    bs = n * stride if batch_stride is None else batch_stride
    _check(ctx, lib.bem_fft(ctx, ctypes.c_void_p(x_ptr), int(n), int(stride), int(batch), int(bs), 1 if inverse else 0,
                            ctypes.c_void_p(stream)))


def bem_planar_skeleton(ctx, a_ptr: int, n: int, omega_ptr: int, p: int, tol: float, block: int, u_ptr: int,
                        vt_ptr: int = 0, stream: int = 0) -> int:
    r = ctypes.c_int(0)
    _check(ctx, lib.bem_planar_skeleton(ctx, ctypes.c_void_p(a_ptr), int(n), ctypes.c_void_p(omega_ptr), int(p),
                                        float(tol), int(block), ctypes.c_void_p(u_ptr), ctypes.c_void_p(vt_ptr or None),
                                        ctypes.byref(r), ctypes.c_void_p(stream)))
    return r.value


def bem_planar_woodbury_solve(ctx, cc0_ptr: int, n: int, u_ptr: int, vt_ptr: int, r: int, b_ptr: int, x_ptr: int,
                              nrhs: int = 1, stream: int = 0) -> None:
    _check(ctx, lib.bem_planar_woodbury_solve(ctx, ctypes.c_void_p(cc0_ptr), int(n), ctypes.c_void_p(u_ptr or None),
                                              ctypes.c_void_p(vt_ptr or None), int(r), ctypes.c_void_p(b_ptr),
                                              ctypes.c_void_p(x_ptr), int(nrhs), ctypes.c_void_p(stream)))


def bem_measure_fma_peak(fp64: bool, stream: int = 0) -> float:
    """FMA throughput of the current device in TFLOP/s (FP64 if fp64 else FP32)."""
    t = ctypes.c_double(0.0)
    st = lib.bem_measure_fma_peak(1 if fp64 else 0, ctypes.c_void_p(stream), ctypes.byref(t))
    if st != BEM_OK:
        raise BemError(st, "bem_measure_fma_peak failed")
    return t.value


def bem_debug_fail_alloc_after(after: int) -> None:
    """Test hook: the library's device allocations fail after `after` more (negative: off)."""
    lib.bem_debug_fail_alloc_after(int(after))


def bem_absorbed_power_gradient(ctx, x_ptr: int, g_ptr: int, nrhs: int, stream: int = 0) -> None:
    _check(ctx, lib.bem_absorbed_power_gradient(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(g_ptr), int(nrhs),
                                                ctypes.c_void_p(stream)))


def bem_grad_weights(ctx, bm_ptr: int, w, x_ptr: int = 0, lam_ptr: int = 0, stream: int = 0):
    """Returns (P_abs, dP/d conj(w) as a complex128 array, inner iterations)."""
    w = np.ascontiguousarray(w, dtype=np.complex128)
    nw = len(w)
    grad = np.zeros(nw, dtype=np.complex128)
    p = ctypes.c_double(0.0)
    it = ctypes.c_int(0)
    _check(ctx, lib.bem_grad_weights(ctx, ctypes.c_void_p(bm_ptr), nw, w.ctypes.data_as(ctypes.POINTER(bem_c128)),
                                     ctypes.byref(p), grad.ctypes.data_as(ctypes.POINTER(bem_c128)),
                                     ctypes.c_void_p(x_ptr or None), ctypes.c_void_p(lam_ptr or None),
                                     ctypes.c_void_p(stream), ctypes.byref(it)))
    return p.value, grad, it.value


def bem_grad_eps(ctx, x_ptr: int, lam_ptr: int, stream: int = 0):
    """(dP/d Re eps_r, dP/d Im eps_r) from the forward and adjoint solutions; for a
    layered context the pairs of regions 1, 2, ... one after another."""
    out = np.zeros(2 * max(1, bem_num_regions(ctx) - 1), dtype=np.float64)
    _check(ctx, lib.bem_grad_eps(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(lam_ptr), _np_ptr(out, ctypes.c_double),
                                 ctypes.c_void_p(stream)))
    return out


def bem_num_regions(ctx) -> int:
    return int(lib.bem_num_regions(ctx))


def bem_autotune(ctx, dtype: int, stream: int = 0):
    """Returns (slots chosen, ms per product)."""
    ch = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(ctx, lib.bem_autotune(ctx, int(dtype), ctypes.c_void_p(stream), ctypes.byref(ch), ctypes.byref(ms)))
    return ch.value, ms.value


def bem_batch_create(ctxs, x_ptrs, y_ptrs, nrhs, dtype: int, stream: int = 0):
    n = len(ctxs)
    arr = lambda vals: (ctypes.c_void_p * n)(*[ctypes.c_void_p(int(v.value) if hasattr(v, "value") else int(v))  # noqa: E731
                                                for v in vals])
    out = ctypes.c_void_p()
    st = lib.bem_batch_create(arr(ctxs), n, arr(x_ptrs), arr(y_ptrs), (ctypes.c_int * n)(*[int(r) for r in nrhs]),
                              int(dtype), ctypes.c_void_p(stream), ctypes.byref(out))
    _check(ctxs[0], st)
    return out


def bem_batch_launch(batch, stream: int = 0) -> None:
    st = lib.bem_batch_launch(batch, ctypes.c_void_p(stream))
    if st != BEM_OK:
        raise BemError(st, "bem_batch_launch failed")


def bem_batch_destroy(batch) -> None:
    lib.bem_batch_destroy(batch)


def bem_power(ctx, x_ptr: int, b_ptr: int, nrhs: int, stream: int = 0, scattered: bool = True):
    """(P_abs, P_ext, P_sca) per right-hand side; scattered=False skips the far-field
    integral of P_sca (returned as NaN)."""
    pa = np.zeros(nrhs)
    pe = np.zeros(nrhs)
    ps = np.zeros(nrhs) if scattered else np.full(nrhs, np.nan)
    _check(ctx, lib.bem_power(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(b_ptr), int(nrhs),
                              _np_ptr(pa, ctypes.c_double), _np_ptr(pe, ctypes.c_double),
                              _np_ptr(ps, ctypes.c_double) if scattered else None, ctypes.c_void_p(stream)))
    return pa, pe, ps


def bem_power_density(ctx, x_ptr: int, per_tri_ptr: int, stream: int = 0) -> None:
    _check(ctx, lib.bem_power_density(ctx, ctypes.c_void_p(x_ptr), ctypes.c_void_p(per_tri_ptr),
                                      ctypes.c_void_p(stream)))


def bem_profile_begin(ctx) -> None:
    _check(ctx, lib.bem_profile_begin(ctx))


def bem_profile_end(ctx):
    """Returns (ms_sum[3], launches[3]) per kernel of the product."""
    ms = np.zeros(3)
    cnt = np.zeros(3, dtype=np.int64)
    _check(ctx, lib.bem_profile_end(ctx, _np_ptr(ms, ctypes.c_double), _np_ptr(cnt, ctypes.c_int64)))
    return ms, cnt


def bem_absorbed_power_static(ctx, x_ptr: int, nrhs: int, p_abs_ptr: int, stream: int = 0) -> None:
    """Absorbed power into device memory (p_abs_ptr: nrhs doubles) without any device allocation."""
    _check(ctx, lib.bem_absorbed_power_static(ctx, ctypes.c_void_p(x_ptr), int(nrhs), ctypes.c_void_p(p_abs_ptr),
                                              ctypes.c_void_p(stream)))
