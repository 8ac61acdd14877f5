"""Calderon preconditioning of PMCHWT with Buffa-Christiansen functions (oracle,
test infrastructure: only the tests, the smoke check and the benchmark's CPU leg
use it).

Sec. III preconditions the 2-D CFIE with the Calderon identity: the
hypersingular operator is composed with the single layer through the inverse
Gram matrix G^-1, so that the product is the identity plus a compact operator
and the iteration count no longer grows with the discretisation density.  The
3-D PMCHWT operator Z (``operators.pmchwt_matrix``) has the same structure:
its square is bounded with a bounded inverse on smooth surfaces, while Z alone
has a condition number growing like h^-2.  Composing Z with itself needs a
second, dual discretisation in which the rotated field n x E is a current:
the Buffa-Christiansen (BC) functions on the barycentric refinement, which are
div-conforming like RWG functions and pair with n x RWG through a
well-conditioned mixed Gram matrix.

Definitions written out here (the readings are stated where the construction
has a choice):

  * Barycentric refinement: every coarse triangle (a, b, c) is cut into six
    triangles by its centroid g and its edge midpoints, (v, m(v, next), g) and
    (v, g, m(prev, v)) for each corner v, all keeping the outward orientation.
    Fine vertices are numbered coarse vertices, then edge midpoints (coarse
    edge order), then centroids (coarse triangle order).
  * R: the coarse RWG function f_m written in the fine RWG basis.  It is
    exactly representable; its coefficient on fine edge k is the normal
    component of f_m across that edge in the fine RWG's direction (T+ to T-).
  * C: the BC function g_e of coarse edge e in the fine RWG basis.  With
    (a, b) the order in which T+ of e traverses the edge, g_e carries the
    flux l_e from the dual cell of a into that of b, l_e / 2 through each of
    the two fine edges joining the midpoint of e to the centroids of its
    triangles, and nothing through the rest of the cells' boundaries.  The
    dual cell of a coarse vertex is the union of the fine triangles touching
    it.  Inside a cell of N fine triangles every fine triangle takes the same
    charge l_e / N (reading: equal charge per triangle, the count-based
    weights of the classical construction), and among the fluxes on the
    radial fine edges of the cell that satisfy this the one of least
    Euclidean norm is taken (reading; it is the one symmetric about the line
    from the vertex to the midpoint of e, with radial fluxes l_e (1/2 - i/N),
    i = 1 .. N-1, counted around the vertex from that line, and 0 on it).
  * Mixed Gram matrix G[m, e] = int (n x f_m) . g_e dS (real).
  * BC-tested PMCHWT: Z_BC = Cb^T Z_fine Cb with Cb = diag(C, C) and Z_fine
    the PMCHWT matrix of the fine mesh.
  * Preconditioner: P = -Gb^-T Z_BC Gb^-1 with Gb = diag(G, G).  Z x is a
    vector of RWG-tested fields; Gb^-1 turns it into the BC expansion of the
    rotated fields, Z_BC applies the operator to that current and tests it
    with BC functions, and -Gb^-T turns the result into RWG coefficients
    again (the identity <f, E> = <n x f, n x E> for tangential E fixes the
    transposes and the sign; the sign is immaterial for Krylov methods).
    Reading: no exchange of the J and M blocks.  With the impedances scaled
    out of Z (unknowns [eta0 J ; M]) both diagonal blocks of Z are of the
    same order already; exchanging them, the other choice, gave larger
    condition numbers and more GMRES iterations on the test spheres.  The
    library applies P on the right (Z P y = b, x = P y).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import operators as O
from . import quadrature as Q
from . import rwg as R


@dataclass
class Refinement:
    coarse: R.RWG
    fine: R.RWG
    parent: np.ndarray   # (6 nt,) coarse triangle of each fine triangle
    R: np.ndarray        # (ne_f, ne_c) coarse RWG functions in the fine RWG basis
    C: np.ndarray        # (ne_f, ne_c) BC functions in the fine RWG basis


def barycentric_refine(coarse: R.RWG):
    """Fine vertices (nv + ne + nt, 3), fine triangles (6 nt, 3) and parents."""
    nv, ne, nt = len(coarse.verts), coarse.ne, coarse.nt
    cen = coarse.verts[coarse.tris].mean(axis=1)
    fv = np.vstack([coarse.verts, coarse.midpoints(), cen])
    ft, parent = [], []
    for t in range(nt):
        g = nv + ne + t
        for i in range(3):
            v = int(coarse.tris[t, i])
            m_next = nv + int(coarse.tri_edge[t, (i + 2) % 3])  # edge (v, next) is opposite corner i+2
            m_prev = nv + int(coarse.tri_edge[t, (i + 1) % 3])  # edge (prev, v) is opposite corner i+1
            ft.append((v, m_next, g))
            ft.append((v, g, m_prev))
            parent += [t, t]
    return fv, np.array(ft, dtype=np.int64), np.array(parent, dtype=np.int64)


def _edge_normal(fine: R.RWG, k: int):
    """Unit in-plane normal of fine edge k pointing out of its T+ (into T-) and its midpoint."""
    a, b = fine.verts[fine.edges[k, 0]], fine.verts[fine.edges[k, 1]]
    mid = 0.5 * (a + b)
    e = b - a
    d = mid - fine.verts[fine.pplus[k]]
    nu = d - (d @ e) / (e @ e) * e
    return nu / np.linalg.norm(nu), mid


def rwg_in_fine(coarse: R.RWG, fine: R.RWG, parent):
    """R: coefficient of fine RWG k in coarse RWG m = normal component of f_m across k."""
    Rm = np.zeros((fine.ne, coarse.ne))
    for k in range(fine.ne):
        nu, mid = _edge_normal(fine, k)
        T = int(parent[fine.tplus[k]])
        for slot in range(3):
            m = int(coarse.tri_edge[T, slot])
            Rm[k, m] = R.eval_basis(coarse, m, T, mid) @ nu
    return Rm


def _fine_edge_lookup(fine: R.RWG):
    return {(int(a), int(b)): k for k, (a, b) in enumerate(fine.edges)}


def bc_in_fine(coarse: R.RWG, fine: R.RWG):
    """C: the BC function of every coarse edge in the fine RWG basis (module docstring)."""
    nv, ne = len(coarse.verts), coarse.ne
    look = _fine_edge_lookup(fine)
    cell = {}
    for tau in range(fine.nt):  # every fine triangle starts at the coarse vertex of its cell
        cell.setdefault(int(fine.tris[tau, 0]), []).append(tau)
    Cm = np.zeros((fine.ne, ne))
    for e in range(ne):
        tri = [int(x) for x in coarse.tris[coarse.tplus[e]]]
        ends = {int(coarse.edges[e, 0]), int(coarse.edges[e, 1])}
        a = b = None
        for i in range(3):
            if {tri[i], tri[(i + 1) % 3]} == ends:
                a, b = tri[i], tri[(i + 1) % 3]
        le = coarse.length[e]
        col = np.zeros(fine.ne)
        m = nv + e
        for t in (coarse.tplus[e], coarse.tminus[e]):
            c = nv + ne + int(t)
            k = look[(min(m, c), max(m, c))]
            sgn = 1.0 if a in fine.tris[fine.tplus[k]] else -1.0
            assert b in fine.tris[fine.tminus[k] if sgn > 0 else fine.tplus[k]]
            col[k] = sgn * 0.5 * le / fine.length[k]
        for v, q in ((a, le), (b, -le)):
            taus = cell[v]
            radial = sorted({int(fine.tri_edge[tau, s]) for tau in taus for s in range(3)
                             if v in fine.edges[fine.tri_edge[tau, s]]})
            ridx = {k: j for j, k in enumerate(radial)}
            A = np.zeros((len(taus), len(radial)))
            rhs = np.full(len(taus), q / len(taus))
            for r, tau in enumerate(taus):
                for s in range(3):
                    k = int(fine.tri_edge[tau, s])
                    sg = float(fine.tri_sign[tau, s])
                    if k in ridx:
                        A[r, ridx[k]] += sg
                    else:
                        rhs[r] -= sg * col[k] * fine.length[k]
            flux = np.linalg.lstsq(A, rhs, rcond=None)[0]  # least-norm radial fluxes
            col[radial] = flux / fine.length[radial]
        Cm[:, e] = col
    return Cm


def refine(coarse: R.RWG) -> Refinement:
    fv, ft, parent = barycentric_refine(coarse)
    fine = R.build(fv, ft)
    return Refinement(coarse, fine, parent, rwg_in_fine(coarse, fine, parent), bc_in_fine(coarse, fine))


def fine_basis_on_triangle(fine: R.RWG, tau: int, pts):
    """Values (3, q, 3) of the three fine RWG functions of triangle tau at points (q, 3)
    and their edge numbers."""
    vals, ks = [], []
    for s in range(3):
        k = int(fine.tri_edge[tau, s])
        p = fine.verts[fine.tris[tau, s]]  # the corner opposite edge s is its free vertex
        vals.append(fine.tri_sign[tau, s] * fine.length[k] / (2.0 * fine.area[tau]) * (pts - p))
        ks.append(k)
    return np.array(vals), ks


def fine_rotated_gram(fine: R.RWG):
    """Gf[k, l] = int (n x phi_k) . phi_l dS over the fine mesh, 7-point rule (exact:
    the integrand is quadratic)."""
    bary, w = Q.rule7()
    Gf = np.zeros((fine.ne, fine.ne))
    for tau in range(fine.nt):
        pts = bary @ fine.verts[fine.tris[tau]]
        vals, ks = fine_basis_on_triangle(fine, tau, pts)
        rot = np.cross(fine.normal[tau], vals)
        for i in range(3):
            for j in range(3):
                Gf[ks[i], ks[j]] += fine.area[tau] * np.sum(w * np.sum(rot[i] * vals[j], axis=1))
    return Gf


def mixed_gram(ref: Refinement):
    """G[m, e] = int (n x f_m) . g_e dS."""
    return ref.R.T @ fine_rotated_gram(ref.fine) @ ref.C


def pmchwt_bc(ref: Refinement, k0: float, eps_r: complex, mu_r: complex = 1.0):
    """Z_BC = Cb^T Z_fine Cb: the PMCHWT matrix with BC test and trial functions."""
    Zf = O.pmchwt_matrix(ref.fine, k0, eps_r, mu_r)
    z = np.zeros_like(ref.C)
    Cb = np.block([[ref.C, z], [z, ref.C]])
    return Cb.T @ Zf @ Cb


def preconditioner(G, Zbc):
    """P = -Gb^-T Z_BC Gb^-1 (dense)."""
    z = np.zeros_like(G)
    Gb = np.block([[G, z], [z, G]])
    return -np.linalg.solve(Gb.T, Zbc @ np.linalg.inv(Gb))
