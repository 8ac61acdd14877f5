"""Dense Galerkin operators and the PMCHWT matrix (oracle, test infrastructure).

Operators (Sec. II, Eqs. 1-4, lifted to 3-D; e^{+j w t}, G_k = e^{-jkR}/(4 pi R)):

  T^_k[m,n] = jk  int int f_m.f_n G_k  -  (j/k) int int (div f_m)(div' f_n) G_k
              (the single-layer operator of Eq. 1 acting on a surface current:
               vector-potential plus scalar-potential parts; T_k = eta_k T^_k
               is the tested electric field of an electric current up to sign)
  K_k[m,n]  = p.v. int int f_m . (grad G_k(r - r') x f_n(r'))
              (the double-layer operators of Eqs. 2-3 acting on a surface current)

PMCHWT (Eq. 7, rows 2-3, and P11..P22 after Eq. 8) in the 3-D form used by the
library, with unknowns x = [eta0 J ; M] and right-hand side b = [e ; eta0 h]:

  Z = [[ T^_0 + eta_r T^_1 ,  K_0 + K_1        ],
       [ -(K_0 + K_1)      ,  T^_0 + T^_1/eta_r ]],   eta_r = eta_1/eta_0

which is the paper's block pattern (P11 a k0/k1 sum of single layers, P12 = a
sum of double layers, P21 = minus that sum, P22 a sum of the dual single
layers) with the impedances scaled out.  It follows from tangential continuity
of E and H with J = n x H and M = E x n.

Quadrature: 7-point rule on test and source triangles.  A triangle pair is
"singular" when the two triangles share a vertex or their centroids are closer
than NEAR_FACTOR times the larger longest-edge; for those pairs the terms
1/(4 pi R) - k^2 R/(8 pi) of G and grad(1/(4 pi R)) - k^2 grad R/(8 pi) of
grad G are integrated over the source triangle in closed form (see
``potentials``) and the smooth remainder by the 7-point rule.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import potentials, quadrature
from .rwg import RWG

NEAR_FACTOR = 2.0
FOUR_PI = 4.0 * math.pi
SERIES_KR = 1.0      # |k| R below which the smooth remainders use their Taylor series
SERIES_TERMS = 30


def _geometry(rwg: RWG):
    tv = rwg.verts[rwg.tris]                        # (nt,3,3)
    bary, w = quadrature.rule7()
    pts = np.einsum("qk,tkd->tqd", bary, tv)        # (nt,7,3)
    wts = rwg.area[:, None] * w[None, :]            # (nt,7)
    cen = tv.mean(axis=1)
    el = np.stack([np.linalg.norm(tv[:, (i + 1) % 3] - tv[:, (i + 2) % 3], axis=1) for i in range(3)], axis=1)
    diam = el.max(axis=1)
    coef = rwg.tri_sign * rwg.length[rwg.tri_edge]  # s_i l_i per local basis (nt,3)
    return tv, pts, wts, cen, diam, coef


def green(k, R):
    """G_k(R) = e^{-jkR}/(4 pi R)."""
    return np.exp(-1j * k * R) / (FOUR_PI * R)


def green_g(k, R):
    """g_k(R) with grad G_k(r-r') = g_k(R) (r - r')."""
    return -(1.0 + 1j * k * R) * np.exp(-1j * k * R) / (FOUR_PI * R ** 3)


def smooth_G(k, R):
    """G_k - 1/(4 pi R) + k^2 R/(8 pi), finite at R = 0."""
    R = np.asarray(R, dtype=np.float64)
    x = np.abs(k) * R
    out = np.empty(R.shape, dtype=np.complex128)
    small = x < SERIES_KR
    # series: (1/4pi) [ -jk + sum_{n>=3} (-jk)^n R^{n-1}/n! ]
    Rs = R[small]
    acc = np.full(Rs.shape, -1j * k, dtype=np.complex128)
    for n in range(3, SERIES_TERMS):
        acc = acc + (-1j * k) ** n * Rs ** (n - 1) / math.factorial(n)
    out[small] = acc / FOUR_PI
    Rl = R[~small]
    out[~small] = (np.exp(-1j * k * Rl) - 1.0) / (FOUR_PI * Rl) + k * k * Rl / (8.0 * math.pi)
    return out


def smooth_g(k, R):
    """g_k + 1/(4 pi R^3) + k^2/(8 pi R), finite at R = 0."""
    R = np.asarray(R, dtype=np.float64)
    x = np.abs(k) * R
    out = np.empty(R.shape, dtype=np.complex128)
    small = x < SERIES_KR
    Rs = R[small]
    acc = np.zeros(Rs.shape, dtype=np.complex128)
    for n in range(3, SERIES_TERMS):
        acc = acc + (n - 1) * (-1j * k) ** n * Rs ** (n - 3) / math.factorial(n)
    out[small] = acc / FOUR_PI
    Rl = R[~small]
    out[~small] = (1.0 - (1.0 + 1j * k * Rl) * np.exp(-1j * k * Rl) + 0.5 * (k * Rl) ** 2) / (FOUR_PI * Rl ** 3)
    return out


def singular_mask(rwg: RWG, a_idx, b_idx, cen, diam):
    """True where the triangle pair (a,b) gets singularity extraction."""
    ta = rwg.tris[a_idx]
    tb = rwg.tris[b_idx]
    share = np.zeros(np.broadcast(a_idx, b_idx).shape, dtype=bool)
    for i in range(3):
        for j in range(3):
            share |= ta[..., i] == tb[..., j]
    d = np.linalg.norm(cen[a_idx] - cen[b_idx], axis=-1)
    return share | (d < NEAR_FACTOR * np.maximum(diam[a_idx], diam[b_idx]))


def _local_regular(k, pa, wa, va, pb, wb, vb, mask):
    """Regular 7x7 quadrature of the local integrals for test triangles a vs source triangles b.

    pa (A,7,3), wa (A,7), va (A,3,3); pb, wb, vb likewise for B source triangles.
    Returns Iff (A,B,3,3), I0 (A,B), Ik (A,B,3,3); pairs with mask True are zeroed.

    The sums over the 49 point pairs are taken through point moments, using
        (r - v_i).(r' - v_j) = r.r' - r.v_j - v_i.r' + v_i.v_j
        (r - v_i).((r - r') x (r' - v_j)) = (v_i - v_j).((r' - v_j) x (r - v_i))
        (r' - v_j) x (r - v_i) = r' x r - r' x v_i - v_j x r + v_j x v_i,
    so that only sums of G, G r, G r', G r.r' (and of g, g r, g r', g r' x r)
    over the point pairs are needed.
    """
    d = pa[:, None, :, None, :] - pb[None, :, None, :, :]          # (A,B,7,7,3)
    R = np.sqrt(np.einsum("abpqd,abpqd->abpq", d, d))
    with np.errstate(divide="ignore", invalid="ignore"):
        W = wa[:, None, :, None] * wb[None, :, None, :]
        WG = np.where(mask[:, :, None, None], 0.0, W * green(k, R))
        Wg = np.where(mask[:, :, None, None], 0.0, W * green_g(k, R))
    def moments(F):
        m0 = F.sum(axis=(2, 3))                                      # sum F
        mr = np.einsum("abp,apd->abd", F.sum(axis=3), pa)           # sum F r
        Fs = np.einsum("abpq,bqd->abpd", F, pb)                     # sum_q F r'   (A,B,7p,3)
        ms = Fs.sum(axis=2)                                         # sum F r'
        return m0, mr, ms, Fs

    G0, Gr, Gs, WGs = moments(WG)
    Grr = np.einsum("abpd,apd->ab", WGs, pa)                        # sum G r.r'
    vdot = lambda x, y: np.sum(x * y, axis=-1)
    # Iff[i,j] = Grr - Gr.v_j - v_i.Gs + (v_i.v_j) G0
    Iff = (Grr[:, :, None, None]
           - vdot(Gr[:, :, None, None, :], vb[None, :, None, :, :])
           - vdot(va[:, None, :, None, :], Gs[:, :, None, None, :])
           + vdot(va[:, None, :, None, :], vb[None, :, None, :, :]) * G0[:, :, None, None])
    g0, gr, gs, Wgs = moments(Wg)
    gx = np.cross(Wgs, pa[:, None, :, :]).sum(axis=2)               # sum g r' x r
    vi = va[:, None, :, None, :]                                    # (A,1,i,1,3)
    vj = vb[None, :, None, :, :]                                    # (1,B,1,j,3)
    inner = (gx[:, :, None, None, :]
             - np.cross(gs[:, :, None, None, :], vi)
             - np.cross(vj, gr[:, :, None, None, :])
             + np.cross(vj, vi) * g0[:, :, None, None, None])
    Ik = vdot(vi - vj, inner)
    return Iff, G0, Ik


def _local_singular(k, pa, wa, va, pb, wb, vb, nb, same):
    """Local integrals with singularity extraction for P triangle pairs.

    pa (P,NO,3), wa (P,NO) outer points and weights on the test triangle (the
    7-point rule in the operators; tests pass refined outer rules); pb (P,7,3),
    wb (P,7) the source rule; va, vb (P,3,3); nb (P,3) source normals;
    same (P,) True where the two triangles coincide.
    """
    P, NO = pa.shape[0], pa.shape[1]                                # NO outer points (7 by default)
    d = pa[:, :, None, :] - pb[:, None, :, :]                       # (P,NO,7,3) r_p - r'_q
    R = np.sqrt(np.einsum("pabd,pabd->pab", d, d))
    Gs = smooth_G(k, R) * wb[:, None, :]
    gs = smooth_g(k, R) * wb[:, None, :]
    V = pb[:, :, None, :] - vb[:, None, :, :]                       # (P,7q,j,3)
    rr = pa.reshape(-1, 3)
    tv = np.repeat(vb, NO, axis=0)
    nn = np.repeat(nb, NO, axis=0)
    inpl = np.repeat(same, NO)
    ana = potentials.triangle_integrals(rr, tv, nn, inplane=inpl)
    S_m1 = ana["S_m1"].reshape(P, NO)
    S_1 = ana["S_1"].reshape(P, NO)
    V_m1 = ana["V_m1"].reshape(P, NO, 3)
    V_1 = ana["V_1"].reshape(P, NO, 3)
    G_m3 = ana["G_m3"].reshape(P, NO, 3)
    G_1 = ana["G_1"].reshape(P, NO, 3)
    rho = ana["rho"].reshape(P, NO, 3)
    k2 = k * k
    # F_j(r_p) = int_b (r' - v_j) G dS'
    rho_v = rho[:, :, None, :] - vb[:, None, :, :]                  # (P,7p,j,3)
    F = np.einsum("apq,aqjd->apjd", Gs, V)
    F = F + (V_m1[:, :, None, :] + rho_v * S_m1[:, :, None, None]) / FOUR_PI
    F = F - k2 * (V_1[:, :, None, :] + rho_v * S_1[:, :, None, None]) / (8.0 * math.pi)
    Phi = Gs.sum(axis=2) + S_m1 / FOUR_PI - k2 * S_1 / (8.0 * math.pi)  # (P,7p)
    # H_j(r_p) = int_b grad G(r_p - r') x (r' - v_j) dS'
    # sum_q gs (r_p - r'_q) x (r'_q - v_j) = r_p x (S1 - v_j S0) + S1 x v_j,
    # with S0 = sum_q gs and S1 = sum_q gs r'_q
    S0 = gs.sum(axis=2)                                             # (P,NO)
    S1 = np.einsum("apq,aqd->apd", gs, pb)                          # (P,NO,3)
    H = (np.cross(pa[:, :, None, :], S1[:, :, None, :] - vb[:, None, :, :] * S0[:, :, None, None])
         + np.cross(S1[:, :, None, :], vb[:, None, :, :]))
    gvec = G_m3 / FOUR_PI - k2 * G_1 / (8.0 * math.pi)              # (P,7p,3)
    rp_v = pa[:, :, None, :] - vb[:, None, :, :]                    # r_p - v_j  (P,7p,j,3)
    H = H + np.cross(gvec[:, :, None, :], rp_v)
    U = pa[:, :, None, :] - va[:, None, :, :]                       # (P,7p,i,3)
    Iff = np.einsum("ap,apid,apjd->aij", wa, U, F)
    I0 = np.einsum("ap,ap->a", wa, Phi)
    Ik = np.einsum("ap,apid,apjd->aij", wa, U, H)
    return Iff, I0, Ik


def _combine(k, Iff, I0, Ik, ca, cb, Aa, Ab):
    """Local 3x3 matrices of T^_k and K_k from the local integrals."""
    cc = ca[..., :, None] * cb[..., None, :]
    AA = (Aa * Ab)[..., None, None]
    That = cc * (1j * k * Iff / (4.0 * AA) - 1j * I0[..., None, None] / (k * AA))
    Kl = cc * Ik / (4.0 * AA)
    return That, Kl


class _Scatter:
    """Collects local contributions (row, col, value) and sums them into a dense matrix once."""

    def __init__(self, n):
        self.n = n
        self.lin, self.val = [], []

    def add(self, rows, cols, vals):
        self.lin.append((rows * self.n + cols).ravel())
        self.val.append(np.asarray(vals).ravel())

    def dense(self):
        lin = np.concatenate(self.lin)
        val = np.concatenate(self.val)
        size = self.n * self.n
        Z = np.bincount(lin, weights=val.real, minlength=size) + 1j * np.bincount(lin, weights=val.imag, minlength=size)
        return Z.reshape(self.n, self.n)


def assemble_TK(rwg: RWG, k: complex, chunk: int = 8, threads: int | None = None):
    """Dense T^_k and K_k (ne x ne, complex128) on the RWG basis.

    Test-triangle chunks are independent; they are spread over a thread pool
    (numpy releases the interpreter lock inside its array loops).  The result
    does not depend on the number of threads: contributions are summed in a
    fixed order by one bincount at the end.
    """
    k = complex(k)
    tv, pts, wts, cen, diam, coef = _geometry(rwg)
    nt, ne = rwg.nt, rwg.ne
    allb = np.arange(nt)

    def regular_chunk(a0):
        a = np.arange(a0, min(nt, a0 + chunk))
        mask = singular_mask(rwg, a[:, None], allb[None, :], cen, diam)
        Iff, I0, Ik = _local_regular(k, pts[a], wts[a], tv[a], pts, wts, tv, mask)
        Tl, Kl = _combine(k, Iff, I0, Ik, coef[a][:, None, :], coef[None, :, :], rwg.area[a][:, None], rwg.area[None, :])
        Tl[mask] = 0.0
        Kl[mask] = 0.0
        rows = np.broadcast_to(rwg.tri_edge[a][:, None, :, None], Tl.shape)
        cols = np.broadcast_to(rwg.tri_edge[None, :, None, :], Tl.shape)
        ia, ib = np.nonzero(mask)
        return rows, cols, Tl, Kl, np.stack([a[ia], ib], axis=1)

    def singular_chunk(sp):
        pa, pb = sp[:, 0], sp[:, 1]
        Iff, I0, Ik = _local_singular(k, pts[pa], wts[pa], tv[pa], pts[pb], wts[pb], tv[pb], rwg.normal[pb], pa == pb)
        Tl, Kl = _combine(k, Iff, I0, Ik, coef[pa], coef[pb], rwg.area[pa], rwg.area[pb])
        rows = np.broadcast_to(rwg.tri_edge[pa][:, :, None], Tl.shape)
        cols = np.broadcast_to(rwg.tri_edge[pb][:, None, :], Tl.shape)
        return rows, cols, Tl, Kl

    if threads is None:
        threads = min(8, os.cpu_count() or 1)
    T = _Scatter(ne)
    K = _Scatter(ne)
    with ThreadPoolExecutor(max_workers=threads) as ex:
        reg = list(ex.map(regular_chunk, range(0, nt, chunk)))
        sp = np.concatenate([r[4] for r in reg], axis=0)
        for rows, cols, Tl, Kl, _ in reg:
            T.add(rows, cols, Tl)
            K.add(rows, cols, Kl)
        del reg
        for rows, cols, Tl, Kl in ex.map(singular_chunk, [sp[i:i + 2048] for i in range(0, len(sp), 2048)]):
            T.add(rows, cols, Tl)
            K.add(rows, cols, Kl)
    return T.dense(), K.dense()


def media(k0: float, eps_r: complex, mu_r: complex = 1.0):
    """Interior wavenumber and relative impedance (principal square roots).

    k1 = k0 sqrt(eps_r mu_r) (Im k1 <= 0 for a lossy medium under e^{+j w t}),
    eta_r = eta1/eta0 = sqrt(mu_r/eps_r).
    """
    k1 = k0 * np.sqrt(complex(eps_r) * complex(mu_r))
    eta_r = np.sqrt(complex(mu_r) / complex(eps_r))
    return complex(k1), complex(eta_r)


def pmchwt_blocks(rwg: RWG, k0: float, eps_r: complex, mu_r: complex = 1.0):
    """The three distinct PMCHWT blocks A, B, C (each ne x ne)."""
    k1, eta_r = media(k0, eps_r, mu_r)
    T0, K0 = assemble_TK(rwg, k0)
    T1, K1 = assemble_TK(rwg, k1)
    A = T0 + eta_r * T1
    B = K0 + K1
    C = T0 + T1 / eta_r
    return A, B, C


def pmchwt_matrix(rwg: RWG, k0: float, eps_r: complex, mu_r: complex = 1.0):
    """Full 2ne x 2ne normalised PMCHWT matrix [[A, B], [-B, C]]."""
    A, B, C = pmchwt_blocks(rwg, k0, eps_r, mu_r)
    return np.block([[A, B], [-B, C]])


def operator_rows(rwg: RWG, k: complex, rows):
    """Rows ``rows`` of T^_k and K_k evaluated on the fly (no dense matrix kept).

    Each RWG row needs its two support triangles against every source
    triangle; the full row is returned as arrays (len(rows), ne).
    """
    k = complex(k)
    rows = np.asarray(rows, dtype=np.int64)
    tv, pts, wts, cen, diam, coef = _geometry(rwg)
    nt, ne = rwg.nt, rwg.ne
    Tr = np.zeros((len(rows), ne), dtype=np.complex128)
    Kr = np.zeros((len(rows), ne), dtype=np.complex128)
    allb = np.arange(nt)
    for ir, m in enumerate(rows):
        for tri in (rwg.tplus[m], rwg.tminus[m]):
            li = int(np.nonzero(rwg.tri_edge[tri] == m)[0][0])
            a = np.array([tri])
            for b0 in range(0, nt, 4096):
                b = allb[b0:b0 + 4096]
                mask = singular_mask(rwg, a[:, None], b[None, :], cen, diam)
                Iff, I0, Ik = _local_regular(k, pts[a], wts[a], tv[a], pts[b], wts[b], tv[b], mask)
                Tl, Kl = _combine(k, Iff, I0, Ik, coef[a][:, None, :], coef[b][None, :, :], rwg.area[a][:, None], rwg.area[b][None, :])
                Tl = np.where(mask[:, :, None, None], 0.0, Tl)[0, :, li, :]
                Kl = np.where(mask[:, :, None, None], 0.0, Kl)[0, :, li, :]
                np.add.at(Tr[ir], rwg.tri_edge[b].ravel(), Tl.ravel())
                np.add.at(Kr[ir], rwg.tri_edge[b].ravel(), Kl.ravel())
                sb = b[mask[0]]
                if len(sb):
                    pa = np.full(len(sb), tri)
                    Iff, I0, Ik = _local_singular(k, pts[pa], wts[pa], tv[pa], pts[sb], wts[sb], tv[sb], rwg.normal[sb], pa == sb)
                    Tl, Kl = _combine(k, Iff, I0, Ik, coef[pa], coef[sb], rwg.area[pa], rwg.area[sb])
                    np.add.at(Tr[ir], rwg.tri_edge[sb].ravel(), Tl[:, li, :].ravel())
                    np.add.at(Kr[ir], rwg.tri_edge[sb].ravel(), Kl[:, li, :].ravel())
    return Tr, Kr


def pmchwt_rows_apply(rwg: RWG, k0: float, eps_r: complex, x, rows, mu_r: complex = 1.0):
    """Entries ``rows`` (indices into the 2ne unknowns) of Z @ x, Z never stored
    (x a vector, or a matrix of several right-hand sides as columns)."""
    ne = rwg.ne
    rows = np.asarray(rows, dtype=np.int64)
    k1, eta_r = media(k0, eps_r, mu_r)
    edge_rows = rows % ne
    T0, K0 = operator_rows(rwg, k0, edge_rows)
    T1, K1 = operator_rows(rwg, k1, edge_rows)
    xJ, xM = x[:ne], x[ne:]
    out = np.empty((len(rows),) + np.shape(x)[1:], dtype=np.complex128)
    for i, r in enumerate(rows):
        B = K0[i] + K1[i]
        if r < ne:
            out[i] = (T0[i] + eta_r * T1[i]) @ xJ + B @ xM
        else:
            out[i] = -B @ xJ + (T0[i] + T1[i] / eta_r) @ xM
    return out
