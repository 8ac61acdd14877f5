"""The paper's two-dimensional TM pipeline (oracle, test infrastructure).

Setting (Sec. II): fields invariant along z, a closed boundary curve Gamma with
outward normal n, the free-space kernel G_k(R) = -(j/4) H0^(2)(k R) (Eq. 5) and
the single-layer, double-layer, adjoint double-layer and hypersingular
operators S, D, D*, N of Eqs. 1-4.  Discretisation (Sec. III, Eq. 8): Galerkin
testing with piecewise-linear hat functions lambda_i on a polygon whose
vertices lie on Gamma; (O)_ij = (lambda_i, O lambda_j) for each operator and
the Gram matrix (G)_ij = (lambda_i, lambda_j).

Matrices built from them:
  * the penetrable body's TM PMCHWT blocks P11, P12, P21, P22 (Eqs. 12-15),
    here scaled by eta0 (unknowns [eta0 j_z ; m_t], right-hand side
    [e_z ; eta0 h_t]);
  * the metal boundary's CFIE C = S + G/2 + D* (Eq. 11);
  * its Calderon-stabilised form C_p = N~ G^-1 S + (G/2 - D*~) G^-1 (G/2 + D*)
    (Eq. 16), ~ marking the complexified wavenumber k~ = k0 - 0.4j k0^(1/3) a^(-2/3);
  * the circular counterpart C_p,c: C_p built on the regular polygon of equal
    perimeter and vertex count, which is circulant;
  * the skeleton C_p - C_p,c ~ U V^T (Eq. 17) by an adaptive randomized range
    finder, and C_p^-1 by the Woodbury identity (Eq. 18) with FFT solves of the
    circulant part.

Quadrature.  Segment pairs are integrated with Gauss-Legendre rules on both
segments after splitting off the static parts of the kernels,
    G_k(R) = -ln(R)/(2 pi) + Gr_k(R),
    d_n' G_k = [1/(2 pi R^2) + Ar_k(R)] ((r - r').n'),
whose integrals over a straight source segment against a linear function are
written in closed form; the remainders Gr_k (continuous) and Ar_k (a logarithmic
singularity multiplied by (r - r').n' = O(R)) go to the product rule.  On a
segment paired with itself the logarithm is integrated over both segments in
closed form and D vanishes ((r - r').n' = 0 on a straight segment); on two
segments sharing a vertex the outer rule is graded toward that vertex
(u = s^2).  N follows from S by the identity, valid on a closed curve,
    (lambda_i, N lambda_j) = int int G [lambda_i' lambda_j' - k^2 (n.n') lambda_i lambda_j],
with N = -d_n D as in Eq. 4 (' the derivative along the curve), and D* = D^T
(exchange of test and source in the Galerkin pairing).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import hankel2

EULER = 0.5772156649015329
TWO_PI = 2.0 * math.pi
SERIES_X = 1.0        # |k R| below which the remainders use their power series
SERIES_TERMS = 24
N_OUTER = 10
N_INNER = 10
# closed-form double integrals over the unit segment: int int ln|u - w| phi_p(u) phi_q(w),
# phi_0 = 1 - u, phi_1 = u
_K_SELF = np.array([[-7.0 / 16.0, -5.0 / 16.0], [-5.0 / 16.0, -7.0 / 16.0]])


# ---------------------------------------------------------------------------
# kernels
# ---------------------------------------------------------------------------
def green(k, R):
    """G_k(R) = -(j/4) H0^(2)(k R) (Eq. 5)."""
    return -0.25j * hankel2(0, k * R)


def _harmonic(m):
    return sum(1.0 / i for i in range(1, m + 1))


def green_rem(k, R):
    """Gr_k(R) = G_k(R) + ln(R) / (2 pi): continuous, Gr_k(0) = -j/4 - (ln(k/2) + gamma)/(2 pi).

    Small |k R|: J0 and Y0 from their power series,
        Y0(x) = (2/pi) [(ln(x/2) + gamma) J0(x) + sum_{m>=1} (-1)^(m+1) H_m (x^2/4)^m / (m!)^2],
    so that the logarithm cancels exactly instead of numerically.
    """
    k = complex(k)
    R = np.asarray(R, dtype=np.float64)
    out = np.empty(R.shape, dtype=np.complex128)
    x = k * R
    small = np.abs(x) < SERIES_X
    big = ~small
    if np.any(big):
        out[big] = green(k, R[big]) + np.log(R[big]) / TWO_PI
    if np.any(small):
        Rs = R[small]
        q = (k * Rs / 2.0) ** 2
        J0 = np.zeros_like(q)
        S = np.zeros_like(q)
        term = np.ones_like(q)
        for m in range(SERIES_TERMS):
            if m > 0:
                term = term * (-q) / (m * m)
                S = S - _harmonic(m) * term      # (-1)^(m+1) H_m q^m/(m!)^2 = -H_m * term
            J0 = J0 + term
        with np.errstate(divide="ignore", invalid="ignore"):
            lnR = np.where(Rs > 0, np.log(np.where(Rs > 0, Rs, 1.0)), 0.0)
        out[small] = -0.25j * J0 - ((np.log(k / 2.0) + EULER) * J0 + lnR * (J0 - 1.0) + S) / TWO_PI
    return out


def dgreen_coef(k, R):
    """A_k(R) with d_n' G_k(r - r') = A_k(R) ((r - r').n'):  A_k = -(j k / (4 R)) H1^(2)(k R)."""
    return -0.25j * k * hankel2(1, k * R) / R


def dgreen_rem(k, R):
    """Ar_k(R) = A_k(R) - 1/(2 pi R^2) for R > 0.

    Small |k R|: with T_m = (-1)^m (x/2)^(2m) / (m! (m+1)!), J1(x) = (x/2) sum T_m and
    Y1(x) = (2/pi)(ln(x/2) + gamma) J1(x) - 2/(pi x) - (1/pi) sum (H_m + H_(m+1)) (x/2)^(2m+1)/(m!(m+1)!),
        Ar = -(j k^2/8) sum T_m - (k^2/(4 pi)) (ln(x/2) + gamma) sum T_m + (k^2/(8 pi)) sum (H_m + H_(m+1)) T_m.
    """
    k = complex(k)
    R = np.asarray(R, dtype=np.float64)
    out = np.empty(R.shape, dtype=np.complex128)
    x = k * R
    small = np.abs(x) < SERIES_X
    big = ~small
    if np.any(big):
        out[big] = dgreen_coef(k, R[big]) - 1.0 / (TWO_PI * R[big] ** 2)
    if np.any(small):
        xs = x[small]
        q = (xs / 2.0) ** 2
        sT = np.zeros_like(q)
        sH = np.zeros_like(q)
        term = np.ones_like(q)                   # T_0 = 1
        for m in range(SERIES_TERMS):
            if m > 0:
                term = term * (-q) / (m * (m + 1))
            sT = sT + term
            sH = sH + (_harmonic(m) + _harmonic(m + 1)) * term
        out[small] = (-0.125j * k * k * sT - (k * k / (4.0 * math.pi)) * (np.log(xs / 2.0) + EULER) * sT
                      + (k * k / (8.0 * math.pi)) * sH)
    return out


# ---------------------------------------------------------------------------
# geometry
# ---------------------------------------------------------------------------
class Polygon:
    """Closed polygon, vertices counter-clockwise; segment e runs from vertex e to e + 1."""

    def __init__(self, verts):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.n = len(self.verts)
        if self.n < 3:
            raise ValueError("a closed polygon needs at least 3 vertices")
        d = np.roll(self.verts, -1, axis=0) - self.verts
        self.length = np.hypot(d[:, 0], d[:, 1])
        self.tangent = d / self.length[:, None]
        self.normal = np.stack([self.tangent[:, 1], -self.tangent[:, 0]], axis=1)   # outward for CCW
        area2 = float(np.sum(self.verts[:, 0] * np.roll(self.verts[:, 1], -1)
                             - np.roll(self.verts[:, 0], -1) * self.verts[:, 1]))
        if area2 <= 0:
            raise ValueError("vertices must run counter-clockwise")

    @property
    def perimeter(self):
        return float(self.length.sum())

    def points(self, u):
        """Points at fractions u (array) of every segment: (n, len(u), 2)."""
        return self.verts[:, None, :] + (u[None, :, None] * self.length[:, None, None]) * self.tangent[:, None, :]


def gauss01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


# ---------------------------------------------------------------------------
# closed-form integrals over a straight source segment (local coordinates of the
# target: u along the segment from its start, v along its outward normal)
# ---------------------------------------------------------------------------
def _log_moments(u, v, L):
    """(int_0^L ln R dt, int_0^L t ln R dt), R = |(u - t, v)|."""
    def F0(s):
        Q = s * s + v * v
        with np.errstate(divide="ignore", invalid="ignore"):
            lnr = np.where(Q > 0, 0.5 * np.log(np.where(Q > 0, Q, 1.0)), 0.0)
            at = np.where(np.abs(v) > 0, v * np.arctan(s / np.where(np.abs(v) > 0, v, 1.0)), 0.0)
        return s * lnr - s + at, Q, lnr

    def F1(Q, lnr, s):
        return 0.5 * Q * lnr - 0.25 * s * s

    s1, s0 = L - u, -u
    f1, Q1, l1 = F0(s1)
    f0, Q0, l0 = F0(s0)
    m0 = f1 - f0
    m1 = (F1(Q1, l1, s1) + u * f1) - (F1(Q0, l0, s0) + u * f0)
    return m0, m1


def _angle_moments(u, v, L):
    """(int_0^L v / R^2 dt, int_0^L t v / R^2 dt); both 0 when v = 0."""
    nz = np.abs(v) > 0
    vs = np.where(nz, v, 1.0)

    def prim(s):
        Q = s * s + v * v
        with np.errstate(divide="ignore", invalid="ignore"):
            a = np.arctan(s / vs)
            lq = np.where(Q > 0, np.log(np.where(Q > 0, Q, 1.0)), 0.0)
        return a, 0.5 * v * lq + u * a

    a1, b1 = prim(L - u)
    a0, b0 = prim(-u)
    return np.where(nz, a1 - a0, 0.0), np.where(nz, b1 - b0, 0.0)


# ---------------------------------------------------------------------------
# local 2 x 2 integrals of every segment pair and assembly
# ---------------------------------------------------------------------------
def _pair_integrals(poly: Polygon, k, a_idx, b_idx, ua, wa):
    """S and D local matrices (P, 2, 2) for test segments a_idx against source segments
    b_idx (arrays of P pairs, no pair a == b), outer points ua (P, NO) with weights wa
    (P, NO) as fractions of the test segment."""
    k = complex(k)
    La, Lb = poly.length[a_idx], poly.length[b_idx]
    ta, tb, nb = poly.tangent[a_idx], poly.tangent[b_idx], poly.normal[b_idx]
    P0a, P0b = poly.verts[a_idx], poly.verts[b_idx]
    r = P0a[:, None, :] + (ua * La[:, None])[..., None] * ta[:, None, :]          # (P, NO, 2) outer points
    rel = r - P0b[:, None, :]
    u = np.einsum("pod,pd->po", rel, tb)
    v = np.einsum("pod,pd->po", rel, nb)
    Lb2 = Lb[:, None]
    # static parts, inner integrals in closed form against phi_0 = 1 - t/L, phi_1 = t/L
    m0, m1 = _log_moments(u, v, Lb2)
    logq = np.stack([m0 - m1 / Lb2, m1 / Lb2], axis=-1)                           # (P, NO, 2)
    e0, e1 = _angle_moments(u, v, Lb2)
    angq = np.stack([e0 - e1 / Lb2, e1 / Lb2], axis=-1)
    # remainders by the inner product rule
    xi, wi = gauss01(N_INNER)
    rp = P0b[:, None, :] + (xi[None, :] * Lb2)[..., None] * tb[:, None, :]        # (P, NI, 2)
    d = r[:, :, None, :] - rp[:, None, :, :]                                       # (P, NO, NI, 2)
    R = np.sqrt(np.einsum("poid,poid->poi", d, d))
    vv = np.einsum("poid,pd->poi", d, nb)
    phi_in = np.stack([1.0 - xi, xi], axis=-1)                                     # (NI, 2)
    Wi = (wi[None, :] * Lb2)[:, None, :]                                           # (P, 1, NI)
    gr = green_rem(k, R) * Wi
    ar = dgreen_rem(k, R) * vv * Wi
    Sq = -logq / TWO_PI + np.einsum("poi,iq->poq", gr, phi_in)                     # int_b G phi_q
    Dq = angq / TWO_PI + np.einsum("poi,iq->poq", ar, phi_in)                      # int_b d_n'G phi_q
    phi_out = np.stack([1.0 - ua, ua], axis=-1)                                    # (P, NO, 2)
    Wo = wa * La[:, None]
    S = np.einsum("po,pox,poq->pxq", Wo, phi_out, Sq)
    D = np.einsum("po,pox,poq->pxq", Wo, phi_out, Dq)
    return S, D


def _self_integrals(poly: Polygon, k):
    """S local matrices (n, 2, 2) of every segment with itself (D vanishes there)."""
    k = complex(k)
    L = poly.length
    xg, wg = gauss01(N_INNER)
    phi = np.stack([1.0 - xg, xg], axis=-1)
    # closed-form logarithm: int int ln|t - t'| phi_p phi_q = L^2 (ln L / 4 + K_pq)
    logpart = (L * L)[:, None, None] * (np.log(L)[:, None, None] / 4.0 + _K_SELF[None])
    R = np.abs(xg[:, None] - xg[None, :])[None] * L[:, None, None]                 # (n, NG, NG)
    gr = green_rem(k, R)
    W = (wg[:, None] * wg[None, :])[None] * (L * L)[:, None, None]
    rem = np.einsum("nij,ip,jq->npq", gr * W, phi, phi)
    return -logpart / TWO_PI + rem


def _graded(n, at_end):
    """Gauss-Legendre rule on [0, 1] graded toward 0 (or toward 1 if at_end) by u = s^2."""
    s, w = gauss01(n)
    u, wu = s * s, 2.0 * s * w
    return (1.0 - u[::-1], wu[::-1]) if at_end else (u, wu)


def operators(poly: Polygon, k, chunk: int = 64):
    """Galerkin matrices (S, D, Dt, N, G) of Eqs. 1-4 and the Gram matrix, n x n complex128."""
    k = complex(k)
    n = poly.n
    Sl = np.zeros((n, n, 2, 2), dtype=np.complex128)     # local matrices [a, b, p, q]
    Dl = np.zeros((n, n, 2, 2), dtype=np.complex128)
    xo, wo = gauss01(N_OUTER)
    aa, bb = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    nxt = (aa + 1) % n
    prv = (aa - 1) % n
    regular = (bb != aa) & (bb != nxt) & (bb != prv)
    ra, rb = aa[regular], bb[regular]
    for c0 in range(0, len(ra), chunk * n):
        a_i, b_i = ra[c0:c0 + chunk * n], rb[c0:c0 + chunk * n]
        P = len(a_i)
        S, D = _pair_integrals(poly, k, a_i, b_i, np.broadcast_to(xo, (P, N_OUTER)),
                               np.broadcast_to(wo, (P, N_OUTER)))
        Sl[a_i, b_i] = S
        Dl[a_i, b_i] = D
    # neighbours: outer rule graded toward the shared vertex
    a_all = np.arange(n)
    for b_of, at_end in (((a_all + 1) % n, True), ((a_all - 1) % n, False)):
        ug, wg = _graded(2 * N_OUTER, at_end)
        S, D = _pair_integrals(poly, k, a_all, b_of, np.broadcast_to(ug, (n, len(ug))),
                               np.broadcast_to(wg, (n, len(ug))))
        Sl[a_all, b_of] = S
        Dl[a_all, b_of] = D
    Sl[a_all, a_all] = _self_integrals(poly, k)
    # assemble: local p of segment e is vertex (e + p) mod n
    def assemble(loc):
        M = np.zeros((n, n), dtype=np.complex128)
        for p in range(2):
            for q in range(2):
                np.add.at(M, ((aa + p) % n, (bb + q) % n), loc[:, :, p, q])
        return M

    Smat = assemble(Sl)
    Dmat = assemble(Dl)
    # Maue: N_ab[p, q] = sig_p sig_q / (La Lb) sum(S_ab) - k^2 (n_a . n_b) S_ab[p, q]
    sig = np.array([-1.0, 1.0])
    tot = Sl.sum(axis=(2, 3))
    nn = poly.normal @ poly.normal.T
    Nl = (sig[:, None] * sig[None, :])[None, None] * (tot / np.outer(poly.length, poly.length))[:, :, None, None] \
        - (k * k) * nn[:, :, None, None] * Sl
    Nmat = assemble(Nl)
    return Smat, Dmat, Dmat.T.copy(), Nmat, gram(poly)


def gram(poly: Polygon):
    """(lambda_i, lambda_j): L/6 [[2, 1], [1, 2]] per segment."""
    n = poly.n
    G = np.zeros((n, n))
    L = poly.length
    i = np.arange(n)
    j = (i + 1) % n
    np.add.at(G, (i, i), L / 3.0)
    np.add.at(G, (j, j), L / 3.0)
    np.add.at(G, (i, j), L / 6.0)
    np.add.at(G, (j, i), L / 6.0)
    return G


# ---------------------------------------------------------------------------
# right-hand sides (TM plane wave E_z = exp(-j k0 khat . r))
# ---------------------------------------------------------------------------
def rhs_tm(poly: Polygon, k0: float, khat):
    """(e, eta0 h) with e_i = (lambda_i, E_z^inc), h_i = (lambda_i, H_t^inc), H_t = H . t,
    t = z x n the counter-clockwise tangent; eta0 H^inc = (khat x z) E_z^inc."""
    khat = np.asarray(khat, dtype=np.float64)
    xg, wg = gauss01(N_OUTER)
    pts = poly.points(xg)                                                         # (n, NG, 2)
    E = np.exp(-1j * k0 * (pts @ khat))
    kxz = np.array([khat[1], -khat[0]])                                           # khat x z
    Ht = (poly.tangent @ kxz)[:, None] * E
    phi = np.stack([1.0 - xg, xg], axis=-1)
    W = wg[None, :] * poly.length[:, None]
    n = poly.n
    e = np.zeros(n, dtype=np.complex128)
    h = np.zeros(n, dtype=np.complex128)
    for p in range(2):
        np.add.at(e, (np.arange(n) + p) % n, np.einsum("ng,ng,g->n", W, E, phi[:, p]))
        np.add.at(h, (np.arange(n) + p) % n, np.einsum("ng,ng,g->n", W, Ht, phi[:, p]))
    return e, h


# ---------------------------------------------------------------------------
# the paper's matrices
# ---------------------------------------------------------------------------
def pmchwt_tm(poly: Polygon, k0: float, eps_r: complex, mu_r: complex = 1.0):
    """[[P11, P12], [P21, P22]] of Eqs. 12-15 scaled by eta0, acting on [eta0 j_z ; m_t].

    With j_z = (n x H)_z and m_t = E_z (n outgoing, the orientation under which the
    metal row of Eq. 7 holds as printed), the continuity of E_z and H_t gives these
    matrices with the incident fields negated on the right (``rhs_pmchwt_tm``): the
    printed rows hold for the opposite orientation of the currents."""
    k1 = k0 * np.sqrt(complex(eps_r) * complex(mu_r))
    eta_r = np.sqrt(complex(mu_r) / complex(eps_r))
    S0, D0, Dt0, N0, _ = operators(poly, k0)
    S1, D1, Dt1, N1, _ = operators(poly, k1)
    P11 = -1j * k0 * S0 - 1j * k1 * eta_r * S1
    P12 = D0 + D1
    P21 = -(Dt0 + Dt1)
    P22 = -N0 / (1j * k0) - N1 / (1j * k1 * eta_r)
    return np.block([[P11, P12], [P21, P22]])


def rhs_pmchwt_tm(poly: Polygon, k0: float, khat):
    """Right-hand side -[e_z ; eta0 h_t] of ``pmchwt_tm`` for the physical currents."""
    e, h = rhs_tm(poly, k0, khat)
    return -np.concatenate([e, h])


def cfie(poly: Polygon, k0: float):
    """C = S + G/2 + D* (Eq. 11) for the unknown eta0 j_z; right-hand side e / (j k0) + eta0 h."""
    S, D, Dt, N, G = operators(poly, k0)
    return S + 0.5 * G + Dt


def curvature_radius(poly: Polygon):
    """The radius a of k~: perimeter / (2 pi) (the radius of the equal-perimeter circle)."""
    return poly.perimeter / TWO_PI


def k_tilde(k0: float, a: float):
    """k~ = k0 - 0.4j k0^(1/3) a^(-2/3)."""
    return complex(k0) - 0.4j * k0 ** (1.0 / 3.0) * a ** (-2.0 / 3.0)


def calderon_cfie(poly: Polygon, k0: float, a: float | None = None):
    """(C_p, L_e, L_h) of Eq. 16: C_p = N~ G^-1 S + (G/2 - D*~) G^-1 (G/2 + D*), and the
    maps of the right-hand side, rhs_p = L_e (e / (j k0)) + L_h (eta0 h)."""
    a = curvature_radius(poly) if a is None else a
    kt = k_tilde(k0, a)
    S, D, Dt, N, G = operators(poly, k0)
    _, _, Dtt, Nt, _ = operators(poly, kt)
    Ginv = np.linalg.inv(G)
    Le = Nt @ Ginv
    Lh = (0.5 * G - Dtt) @ Ginv
    Cp = Le @ S + Lh @ (0.5 * G + Dt)
    return Cp, Le, Lh


def circular_counterpart(poly: Polygon):
    """The regular polygon with the same vertex count and perimeter."""
    n = poly.n
    radius = poly.perimeter / (2.0 * n * math.sin(math.pi / n))
    th = TWO_PI * np.arange(n) / n
    return Polygon(np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1))


def range_finder(A, omega, tol: float, block: int = 8):
    """Adaptive randomized range finder (Halko, Martinsson and Tropp 2011): orthonormal
    Q (n x r) with ||(I - Q Q^H) A w|| <= tol * max ||A w_first|| for the test vectors w
    drawn block by block from the columns of omega (the random numbers are an input).
    Returns Q; the skeleton is U = Q, V^T = Q^H A."""
    n = A.shape[0]
    Q = np.zeros((n, 0), dtype=np.complex128)
    ref = None
    for c0 in range(0, omega.shape[1], block):
        Y = A @ omega[:, c0:c0 + block]
        if ref is None:
            ref = float(np.linalg.norm(Y, axis=0).max())
        for _ in range(2):
            Y = Y - Q @ (Q.conj().T @ Y)
        if float(np.linalg.norm(Y, axis=0).max()) <= tol * ref:
            return Q
        q, _ = np.linalg.qr(Y)
        Q = np.concatenate([Q, q], axis=1)[:, :n]
        if Q.shape[1] >= n:             # the whole space: the skeleton is exact
            return Q
    raise RuntimeError("range finder: the test vectors ran out before the tolerance was met")


def skeleton(Cp, Cc, omega, tol: float, block: int = 8):
    """U, V^T with C_p - C_p,c ~ U V^T (Eq. 17)."""
    A = Cp - Cc
    U = range_finder(A, omega, tol, block)
    return U, U.conj().T @ A


def circulant_solve(Cc, b):
    """Cc^-1 b for a circulant Cc by the FFT of its first column."""
    lam = np.fft.fft(Cc[:, 0])
    if np.ndim(b) == 1:
        return np.fft.ifft(np.fft.fft(b) / lam)
    return np.fft.ifft(np.fft.fft(b, axis=0) / lam[:, None], axis=0)


def woodbury_solve(Cc, U, Vt, b):
    """C_p^-1 b with C_p = Cc + U Vt (Eq. 18)."""
    y = circulant_solve(Cc, b)
    CU = circulant_solve(Cc, U)
    cap = np.eye(U.shape[1]) + Vt @ CU
    return y - CU @ np.linalg.solve(cap, Vt @ y)


# ---------------------------------------------------------------------------
# closed forms on a circle of radius a (pins)
# ---------------------------------------------------------------------------
def circle_eigenvalues(k, a, m):
    """Continuous eigenvalues of S, D (= D*) and N on the circle r = a for exp(j m theta)."""
    from scipy.special import h2vp, jv, jvp

    k = complex(k)
    x = k * a
    J, Jp = jv(m, x), jvp(m, x)
    H, Hp = hankel2(m, x), h2vp(m, x)
    s = -0.5j * math.pi * a * J * H
    d = -0.25j * math.pi * x * (Jp * H + J * Hp)
    nn = 0.5j * math.pi * k * x * Jp * Hp
    return s, d, nn


def cylinder_tm_currents(k0: float, eps_r: complex, a: float, theta, nmax: int | None = None):
    """Surface fields of a dielectric cylinder of radius a under E_z = exp(-j k0 x):
    (eta0 j_z, m_t) = (eta0 H_t, E_z) at the angles theta (series, e^{+j w t})."""
    from scipy.special import h2vp, jv, jvp

    k1 = k0 * np.sqrt(complex(eps_r))
    if nmax is None:
        nmax = int(abs(k1) * a + 4 * abs(k1 * a) ** (1 / 3) + 12)
    m = np.arange(-nmax, nmax + 1)
    x0, x1 = k0 * a, k1 * a
    J0, J0p, H0, H0p = jv(m, x0), jvp(m, x0), hankel2(m, x0), h2vp(m, x0)
    J1, J1p = jv(m, x1), jvp(m, x1)
    # E_z continuous, (1/mu) d_r E_z continuous (mu_r = 1)
    det = H0 * k1 * J1p - k0 * H0p * J1
    c = (J1 * k0 * J0p - J0 * k1 * J1p) / det
    dm = (H0 * k0 * J0p - k0 * H0p * J0) / det
    phase = (-1j) ** m
    ez = np.exp(1j * np.outer(theta, m)) @ (phase * dm * J1)
    dr = np.exp(1j * np.outer(theta, m)) @ (phase * k0 * (J0p + c * H0p))
    return dr / (1j * k0), ez


def cylinder_pec_current(k0: float, a: float, theta, nmax: int | None = None):
    """eta0 j_z on a PEC cylinder of radius a under E_z = exp(-j k0 x) (series)."""
    if nmax is None:
        nmax = int(k0 * a + 4 * (k0 * a) ** (1 / 3) + 12)
    m = np.arange(-nmax, nmax + 1)
    coef = (-1j) ** m * 2.0 / (math.pi * k0 * a * hankel2(m, k0 * a))
    return np.exp(1j * np.outer(theta, m)) @ coef


# ---------------------------------------------------------------------------
# powers per unit length (TM), in the normalised units of the unknowns:
# 2 eta0 P for x = [eta0 j_z ; m_t] and a unit incident field
# ---------------------------------------------------------------------------
def absorbed(poly: Polygon, x):
    """2 eta0 P_abs = Re int m_t conj(eta0 j_z) dl = Re(xJ^H G xM): the power flowing
    into the body, -1/2 Re oint (E x H*).n dl with (E x H*).n = -E_z conj(H_t)."""
    n = poly.n
    return float(np.real(np.vdot(x[:n], gram(poly) @ x[n:])))


def extinguished(poly: Polygon, x, e, eta0_h):
    """2 eta0 P_ext = Re(xJ^H e + (eta0 h)^H xM), from the surface fields
    (P_abs + P_sca = -1/2 Re oint (E^i x H^s* + E^s x H^i*).n dl, the incident
    field's own flux through the closed curve vanishing)."""
    n = poly.n
    return float(np.real(np.vdot(x[:n], e) + np.vdot(eta0_h, x[n:])))


def far_field(poly: Polygon, k0: float, x, phi):
    """F(phi) with E_z^s ~ -(j/4) sqrt(2/(pi k0 rho)) e^{-j(k0 rho - pi/4)} F(phi):
    F = j k0 int [(rhat . n') m_t - eta0 j_z] e^{j k0 rhat . r'} dl'."""
    n = poly.n
    xg, wg = gauss01(N_OUTER)
    pts = poly.points(xg)                                                          # (n, NG, 2)
    W = wg[None, :] * poly.length[:, None]
    phi_b = np.stack([1.0 - xg, xg], axis=-1)
    idx = (np.arange(n)[:, None] + np.arange(2)[None, :]) % n                     # vertices of segment e
    J = np.einsum("gp,ep->eg", phi_b, x[:n][idx])                                  # eta0 j_z at the points
    M = np.einsum("gp,ep->eg", phi_b, x[n:][idx])
    rhat = np.stack([np.cos(phi), np.sin(phi)], axis=-1)                           # (nphi, 2)
    ph = np.exp(1j * k0 * np.einsum("fd,egd->feg", rhat, pts))
    rn = rhat @ poly.normal.T                                                      # (nphi, n)
    integrand = (rn[:, :, None] * M[None] - J[None]) * W[None]
    return 1j * k0 * np.einsum("feg,feg->f", ph, integrand)


def scattered(poly: Polygon, k0: float, x, nphi: int = 720):
    """2 eta0 P_sca = (1 / (8 pi k0)) int_0^{2 pi} |F(phi)|^2 dphi (trapezoidal rule,
    exponentially accurate for the periodic integrand)."""
    phi = 2.0 * math.pi * np.arange(nphi) / nphi
    F = far_field(poly, k0, x, phi)
    return float(np.sum(np.abs(F) ** 2) * (2.0 * math.pi / nphi) / (8.0 * math.pi * k0))


def interior_field(poly: Polygon, k0: float, eps_r: complex, x, points, mu_r: complex = 1.0):
    """E_z at points inside the body from its boundary currents: the interior
    representation E_z(r) = oint [G_1 d_n' E_z - E_z d_n' G_1] dl' (n' outgoing) with
    d_n E_z = j k1 eta1 j_z, i.e. E_z = j k1 eta_r S1[eta0 j_z] - D1[m_t], by the
    10-point rule on every segment (points away from the boundary)."""
    k1 = k0 * np.sqrt(complex(eps_r) * complex(mu_r))
    eta_r = np.sqrt(complex(mu_r) / complex(eps_r))
    n = poly.n
    xg, wg = gauss01(N_OUTER)
    pts = poly.points(xg).reshape(-1, 2)                                           # (n*NG, 2)
    W = (wg[None, :] * poly.length[:, None]).reshape(-1)
    phi_b = np.stack([1.0 - xg, xg], axis=-1)
    idx = (np.arange(n)[:, None] + np.arange(2)[None, :]) % n
    J = np.einsum("gp,ep->eg", phi_b, x[:n][idx]).reshape(-1)
    M = np.einsum("gp,ep->eg", phi_b, x[n:][idx]).reshape(-1)
    nrm = np.repeat(poly.normal, len(xg), axis=0)
    d = np.asarray(points, dtype=np.float64)[:, None, :] - pts[None, :, :]         # r - r'
    R = np.sqrt(np.einsum("pqd,pqd->pq", d, d))
    G = green(k1, R)
    dG = dgreen_coef(k1, R) * np.einsum("pqd,qd->pq", d, nrm)                      # d_n' G
    return (1j * k1 * eta_r) * (G * W[None, :]) @ J - (dG * W[None, :]) @ M


def cylinder_tm_interior(k0: float, eps_r: complex, a: float, r, theta, nmax: int | None = None):
    """E_z inside the dielectric cylinder at polar points (r, theta) (series)."""
    from scipy.special import h2vp, jv, jvp

    k1 = k0 * np.sqrt(complex(eps_r))
    if nmax is None:
        nmax = int(abs(k1) * a + 4 * abs(k1 * a) ** (1 / 3) + 12)
    m = np.arange(-nmax, nmax + 1)
    x0, x1 = k0 * a, k1 * a
    J0, J0p, H0, H0p = jv(m, x0), jvp(m, x0), hankel2(m, x0), h2vp(m, x0)
    J1, J1p = jv(m, x1), jvp(m, x1)
    det = H0 * k1 * J1p - k0 * H0p * J1
    dm = (H0 * k0 * J0p - k0 * H0p * J0) / det
    r = np.asarray(r, dtype=np.float64)
    theta = np.asarray(theta, dtype=np.float64)
    return np.sum((-1j) ** m * dm * jv(m, k1 * r[:, None]) * np.exp(1j * m * theta[:, None]), axis=1)


# ---------------------------------------------------------------------------
# TE polarisation (H_z) on the metal boundary
# ---------------------------------------------------------------------------
def rhs_te(poly: Polygon, k0: float, khat):
    """(h, dh) with h_i = (lambda_i, H_z^inc), dh_i = (lambda_i, d_n H_z^inc) for
    H_z^inc = exp(-j k0 khat . r) (unit amplitude), d_n H^inc = -j k0 (khat . n) H^inc."""
    khat = np.asarray(khat, dtype=np.float64)
    xg, wg = gauss01(N_OUTER)
    pts = poly.points(xg)
    H = np.exp(-1j * k0 * (pts @ khat))
    dH = (-1j * k0 * (poly.normal @ khat))[:, None] * H
    phi = np.stack([1.0 - xg, xg], axis=-1)
    W = wg[None, :] * poly.length[:, None]
    n = poly.n
    h = np.zeros(n, dtype=np.complex128)
    dh = np.zeros(n, dtype=np.complex128)
    for p in range(2):
        np.add.at(h, (np.arange(n) + p) % n, np.einsum("ng,ng,g->n", W, H, phi[:, p]))
        np.add.at(dh, (np.arange(n) + p) % n, np.einsum("ng,ng,g->n", W, dH, phi[:, p]))
    return h, dh


def cfie_te(poly: Polygon, k0: float):
    """TE combined field operator N/(j k0) + G/2 - D for the metal's tangential current
    j_t = (n x H).t = -H_z (n outgoing, t = z x n); right-hand side
    -(dh / (j k0) + h).  From the exterior representation
    H_z = H^inc + oint [H_z d_n'G - G d_n'H_z] with d_n H_z = 0 on the metal (E_t = 0):
    magnetic row (G/2 - D) j_t = -h, electric row N j_t = -dh (N = -d_n D)."""
    S, D, Dt, N, G = operators(poly, k0)
    return N / (1j * k0) + 0.5 * G - D


def calderon_cfie_te(poly: Polygon, k0: float, a: float | None = None):
    """(C_p, L_e, L_h) of the TE counterpart of Eq. 16: the electric row N j = -dh is
    preconditioned by S~ (S N = 1/4 - D^2) and the magnetic row (G/2 - D) j = -h by
    (G/2 + D~): C_p = S~ G^-1 N + (G/2 + D~) G^-1 (G/2 - D), right-hand side
    L_e (-dh) + L_h (-h).  The paper prints only the TM form; this is its dual."""
    a = curvature_radius(poly) if a is None else a
    kt = k_tilde(k0, a)
    S, D, Dt, N, G = operators(poly, k0)
    St, Dtl, _, _, _ = operators(poly, kt)
    Ginv = np.linalg.inv(G)
    Le = St @ Ginv
    Lh = (0.5 * G + Dtl) @ Ginv
    return Le @ N + Lh @ (0.5 * G - D), Le, Lh


def cylinder_pec_te_current(k0: float, a: float, theta, nmax: int | None = None):
    """j_t = -H_z on a PEC cylinder of radius a under H_z = exp(-j k0 x) (series):
    j_t = sum (-j)^m (2j / (pi k0 a H_m^(2)'(k0 a))) exp(j m theta)."""
    from scipy.special import h2vp

    if nmax is None:
        nmax = int(k0 * a + 4 * (k0 * a) ** (1 / 3) + 12)
    m = np.arange(-nmax, nmax + 1)
    coef = (-1j) ** m * 2j / (math.pi * k0 * a * h2vp(m, k0 * a))
    return np.exp(1j * np.outer(theta, m)) @ coef
