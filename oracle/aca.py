"""Partial-pivot adaptive cross approximation (oracle, test infrastructure).

The paper compresses the non-circulant part of its operator into a skeleton
U V^T (Eq. 17) with a randomized range finder; the library compresses each
admissible block by adaptive cross approximation into U V^H.  This is the
textbook partial-pivot form, in float64, on a block seen only through its
rows and columns:

  start at row i = 0;  repeat
    r  = B[i,:] - sum_l u_l[i] w_l            (residual row)
    j  = argmax |r_j|  (smallest index on ties); if r_j = 0 move to the next unused row
    w  = r / r_j
    u  = B[:,j] - sum_l w_l[j] u_l            (residual column)
    |S|_F^2 += |u|^2 |w|^2 + 2 Re sum_l (u_l^H u)(w_l^H w)
    stop when |u| |w| <= tol |S|_F
    i  = argmax over unused rows of |u_i|
  B ~= sum_l u_l w_l^T = U V^H with V = conj(W).

Recompression (the factors ACA returns, truncated to the rank their singular
values need): U = Q_U R_U, V = Q_V R_V (QR), R_U R_V^H = X S Y^H (SVD), keep the r
largest singular values with r the smallest rank whose discarded tail satisfies
sqrt(sum_{i > r} s_i^2) <= tol sqrt(sum_i s_i^2); U' = Q_U X_r S_r, V' = Q_V Y_r.
"""
from __future__ import annotations

import numpy as np


def aca(row, col, m: int, n: int, tol: float, rmax: int | None = None):
    """Return (U (m,r), V (n,r)) with B ~= U @ V.conj().T."""
    if rmax is None:
        rmax = min(m, n)
    us, ws = [], []
    used = np.zeros(m, dtype=bool)
    i = 0
    norm2 = 0.0
    while len(us) < rmax:
        used[i] = True
        r = np.array(row(i), dtype=np.complex128)
        for u_l, w_l in zip(us, ws):
            r -= u_l[i] * w_l
        j = int(np.argmax(np.abs(r)))
        if np.abs(r[j]) == 0.0:
            free = np.nonzero(~used)[0]
            if len(free) == 0:
                break
            i = int(free[0])
            continue
        w = r / r[j]
        u = np.array(col(j), dtype=np.complex128)
        for u_l, w_l in zip(us, ws):
            u -= w_l[j] * u_l
        nu, nw = np.linalg.norm(u), np.linalg.norm(w)
        cross = sum(np.vdot(u_l, u) * np.vdot(w_l, w) for u_l, w_l in zip(us, ws))
        norm2 += (nu * nw) ** 2 + 2.0 * float(np.real(cross))
        us.append(u)
        ws.append(w)
        if nu * nw <= tol * np.sqrt(max(norm2, 0.0)):
            break
        cand = np.abs(u)
        cand[used] = -1.0
        i = int(np.argmax(cand))
        if cand[i] < 0.0:
            break
    if not us:
        return np.zeros((m, 0), np.complex128), np.zeros((n, 0), np.complex128)
    U = np.stack(us, axis=1)
    V = np.conj(np.stack(ws, axis=1))
    return U, V


def aca_dense(B: np.ndarray, tol: float, rmax: int | None = None):
    """ACA of an explicitly stored block (for tests)."""
    return aca(lambda i: B[i, :], lambda j: B[:, j], B.shape[0], B.shape[1], tol, rmax)


def recompress(U: np.ndarray, V: np.ndarray, tol: float):
    """Return (U', V') with U' V'^H the best approximation of U V^H whose discarded
    singular values hold at most a fraction tol of its Frobenius norm."""
    k = U.shape[1]
    if k == 0:
        return U, V
    Qu, Ru = np.linalg.qr(U)
    Qv, Rv = np.linalg.qr(V)
    X, s, Yh = np.linalg.svd(Ru @ Rv.conj().T)
    total = float(np.sum(s ** 2))
    if total == 0.0:
        return U[:, :0], V[:, :0]
    r = k
    tail = 0.0
    while r > 1 and tail + s[r - 1] ** 2 <= tol * tol * total:
        r -= 1
        tail += s[r] ** 2
    return Qu @ (X[:, :r] * s[:r]), Qv @ Yh[:r].conj().T
