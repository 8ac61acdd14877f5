"""Bodies made of several homogeneous regions (oracle, test infrastructure).

The PMCHWT system of a single penetrable body (Eq. 7, second and third rows;
the blocks P11..P22 after Eq. 8) couples the exterior and the interior of one
closed boundary.  A layered body, such as a coated sphere, has several closed
surfaces, each separating two regions.  Writing the tangential continuity of E
and H on every surface, with the field of each region radiated by the currents
on that region's own boundary, gives the system region by region:

  * surface s separates the region its normals point into, out(s), from the
    region behind it, in(s); its unknowns are x_s = [eta0 J_s ; M_s] with
    J = n x H and M = E x n taken on the out(s) side;
  * region r sees the currents of every surface on its boundary with the sign
    sigma(s, r) = +1 if r = out(s) and -1 if r = in(s);
  * region r contributes its single-medium operator
        Z_r = [[ eta_r T^_{k_r} ,  K_{k_r}          ],
               [ -K_{k_r}       ,  T^_{k_r} / eta_r ]],
    k_r = k0 sqrt(eps_r mu_r), eta_r = sqrt(mu_r / eps_r) (relative to eta0),
    evaluated between the surfaces of its boundary;
  * Z = sum_r Q_r^T Z_r Q_r, with Q_r selecting the unknowns of region r's
    boundary and multiplying them by sigma(s, r);
  * the incident field lives in region 0 only, so the right-hand side is the
    single-body one on the surfaces that bound region 0 (their normals must
    point into region 0) and zero elsewhere.

For one surface between region 0 and region 1 this is exactly the single-body
matrix of ``operators.pmchwt_matrix``.  The powers that leave region 0 (the
absorbed, extinguished and scattered powers of the whole body) depend only on
the currents of region 0's boundary (``exterior_currents``).
"""
from __future__ import annotations

import numpy as np

from . import excitation, operators
from .rwg import RWG, build


def union_mesh(meshes):
    """Concatenate closed meshes [(verts, tris), ...] into one mesh.

    Returns (verts, tris, tri_surface): the vertices of mesh i follow those of
    meshes 0..i-1, so the edges of mesh i follow those of the earlier meshes in
    the lexicographic edge order, and tri_surface[t] is the index of the mesh
    triangle t comes from.
    """
    vs, ts, ss = [], [], []
    off = 0
    for i, (v, t) in enumerate(meshes):
        v = np.asarray(v, dtype=np.float64)
        t = np.asarray(t, dtype=np.int64)
        vs.append(v)
        ts.append(t + off)
        ss.append(np.full(len(t), i, dtype=np.int64))
        off += len(v)
    return np.concatenate(vs), np.concatenate(ts), np.concatenate(ss)


def region_boundary(rwg: RWG, tri_regions, r: int):
    """Boundary of region r: its sub-mesh, the union edges it holds and their signs.

    Returns (sub_rwg, edges, sigma): sub_rwg is the RWG table of the triangles
    that touch region r (in increasing union order, vertices renumbered in
    increasing union order), edges[i] the union edge of sub edge i and
    sigma[i] = +1 if region r is on the normal side of that edge's surface.
    """
    tri_regions = np.asarray(tri_regions, dtype=np.int64)
    tsel = np.nonzero((tri_regions[:, 0] == r) | (tri_regions[:, 1] == r))[0]
    if len(tsel) == 0:
        raise ValueError(f"region {r} has no boundary")
    vsel = np.unique(rwg.tris[tsel].ravel())
    newid = np.full(len(rwg.verts), -1, dtype=np.int64)
    newid[vsel] = np.arange(len(vsel))
    sub = build(rwg.verts[vsel], newid[rwg.tris[tsel]])
    # union edge of each sub edge, by its (global) vertex pair
    lookup = {(int(a), int(b)): e for e, (a, b) in enumerate(rwg.edges)}
    edges = np.array([lookup[(int(vsel[a]), int(vsel[b]))] for a, b in sub.edges], dtype=np.int64)
    # every edge lies on one surface: both its triangles carry the same region pair
    tp, tm = rwg.tplus[edges], rwg.tminus[edges]
    if np.any(tri_regions[tp] != tri_regions[tm]):
        raise ValueError("the two triangles of an edge bound different regions")
    sigma = np.where(tri_regions[tp, 0] == r, 1.0, -1.0)
    return sub, edges, sigma


def single_medium_matrix(rwg: RWG, k, eta_r):
    """Z_r = [[eta_r T^_k, K_k], [-K_k, T^_k / eta_r]] on one region's boundary."""
    T, K = operators.assemble_TK(rwg, k)
    return np.block([[eta_r * T, K], [-K, T / eta_r]])


def region_media(k0: float, eps_r, mu_r=None):
    """(k_r, eta_r) per region; region 0 is free space whatever eps_r[0] says."""
    n = len(eps_r)
    mu_r = [1.0] * n if mu_r is None else mu_r
    out = [(complex(k0), 1.0 + 0.0j)]
    for r in range(1, n):
        out.append(operators.media(k0, eps_r[r], mu_r[r]))
    return out


def pmchwt_regions(rwg: RWG, tri_regions, k0: float, eps_r, mu_r=None):
    """Dense multi-region PMCHWT matrix (2 ne x 2 ne) on the union mesh's [J ; M] order."""
    ne = rwg.ne
    Z = np.zeros((2 * ne, 2 * ne), dtype=np.complex128)
    for r, (k, eta_r) in enumerate(region_media(k0, eps_r, mu_r)):
        sub, edges, sigma = region_boundary(rwg, tri_regions, r)
        Zr = single_medium_matrix(sub, k, eta_r)
        idx = np.concatenate([edges, ne + edges])
        sg = np.concatenate([sigma, sigma])
        Z[np.ix_(idx, idx)] += sg[:, None] * Zr * sg[None, :]
    return Z


def exterior_mask(rwg: RWG, tri_regions):
    """1 on the unknowns of edges bounding region 0, else 0 (length 2 ne).

    Raises if a surface bounding region 0 has its normals pointing away from it.
    """
    tri_regions = np.asarray(tri_regions, dtype=np.int64)
    sub, edges, sigma = region_boundary(rwg, tri_regions, 0)
    if np.any(sigma < 0):
        raise ValueError("normals of the exterior boundary must point into region 0")
    m = np.zeros(rwg.ne)
    m[edges] = 1.0
    return np.concatenate([m, m])


def rhs_planewave(rwg: RWG, tri_regions, k0: float, khat, e0):
    """Right-hand side of a plane wave incident in region 0."""
    b = excitation.rhs_planewave(rwg, k0, khat, e0)
    m = exterior_mask(rwg, tri_regions)
    return b * (m if np.ndim(b) == 1 else m[:, None])


def exterior_currents(rwg: RWG, tri_regions, x):
    """The currents of region 0's boundary (other surfaces zeroed)."""
    m = exterior_mask(rwg, tri_regions)
    return x * (m if np.ndim(x) == 1 else m[:, None])


def pmchwt_regions_rows_apply(rwg: RWG, tri_regions, k0: float, eps_r, x, rows, mu_r=None):
    """Entries ``rows`` (indices into the 2 ne unknowns) of Z @ x, Z never stored.

    Each region whose boundary holds a row's edge contributes sigma times the
    row of its single-medium operator (``operators.operator_rows`` on the
    region's boundary mesh) applied to that boundary's signed currents.
    """
    ne = rwg.ne
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros(len(rows), dtype=np.complex128)
    for r, (k, eta_r) in enumerate(region_media(k0, eps_r, mu_r)):
        sub, edges, sigma = region_boundary(rwg, tri_regions, r)
        where = {int(e): i for i, e in enumerate(edges)}
        hit = [(j, where[int(row % ne)]) for j, row in enumerate(rows) if int(row % ne) in where]
        if not hit:
            continue
        T, K = operators.operator_rows(sub, k, [i for _, i in hit])
        xJ = sigma * x[edges]
        xM = sigma * x[ne + edges]
        for n, (j, i) in enumerate(hit):
            if rows[j] < ne:
                v = eta_r * (T[n] @ xJ) + K[n] @ xM
            else:
                v = -(K[n] @ xJ) + (T[n] @ xM) / eta_r
            out[j] += sigma[i] * v
    return out


def absorbed_and_weight_gradient(rwg: RWG, tri_regions, Z, Bm, w):
    """(P(w), dP/d conj(w)) of the power absorbed by a layered body, b = Bm w.

    P = xe^H H xe with xe the currents of region 0's boundary (the power that
    leaves region 0), x = Z^-1 b: a Hermitian form w^H Q w in the weights,
    Q = (E Z^-1 Bm)^H H (E Z^-1 Bm), E the mask of ``exterior_mask``; its
    gradient with respect to conj(w) is Q w (dense LU, no adjoint system).
    """
    from . import gradient

    Y = np.linalg.solve(Z, Bm) * exterior_mask(rwg, tri_regions)[:, None]
    Q = Y.conj().T @ (gradient.hermitian_form(rwg) @ Y)
    w = np.asarray(w, dtype=np.complex128)
    return float(np.real(np.vdot(w, Q @ w))), Q @ w


def absorbed_eps_gradient(rwg: RWG, tri_regions, k0: float, eps_r, region: int, b, h: float = 1e-6):
    """(dP/d Re eps, dP/d Im eps) of the region's permittivity, P = Re(xeJ^H X xeM)
    the power absorbed by the layered body (region 0's boundary currents), by
    central differences of the dense LU solution (b does not depend on eps)."""
    from . import power

    def p_of(e):
        eps = list(eps_r)
        eps[region] = e
        Z = pmchwt_regions(rwg, tri_regions, k0, eps)
        return power.absorbed(rwg, exterior_currents(rwg, tri_regions, np.linalg.solve(Z, b)))

    e0 = complex(eps_r[region])
    d_re = (p_of(e0 + h) - p_of(e0 - h)) / (2 * h)
    d_im = (p_of(e0 + 1j * h) - p_of(e0 - 1j * h)) / (2 * h)
    return np.array([d_re, d_im])
