"""Write skin_2d_oracle.npz: the FP64 dense oracle solution of the paper's 2-D skin
sample (Sec. IV): an ellipse of perimeter 5.85 mm (aspect ratio 1.5, not stated
in the paper), double-Debye skin permittivity (Eq. 6) at 1 THz, a TM plane wave
travelling at the angle -pi/5; TM PMCHWT (Eqs. 12-15) with hat functions on a
polygon of 18 vertices per wavelength in the skin.

Stored: the coefficients x = [eta0 j_z ; m_t], the normalised powers per unit
length 2 eta0 P_abs, P_ext, P_sca and the parameters.  Only oracle/ is called; a
few minutes on 8 cores.

    python tests/golden/make_skin_2d.py
"""
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import debye, planar  # noqa: E402

FREQ = 1e12
C0 = 299792458.0
PERIMETER = 5.85e-3
ASPECT = 1.5
ANGLE = -math.pi / 5
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "skin_2d_oracle.npz")


def setup():
    k0 = 2.0 * math.pi * FREQ / C0
    eps = debye.eps_r(FREQ)
    lam1 = 2.0 * math.pi / (k0 * abs(np.sqrt(eps)))
    n = int(math.ceil(18 * PERIMETER / lam1))
    verts = W.ellipse_polygon(n, ASPECT, PERIMETER)
    khat = np.array([math.cos(ANGLE), math.sin(ANGLE)])
    return k0, eps, verts, khat


def main():
    t0 = time.time()
    k0, eps, verts, khat = setup()
    poly = planar.Polygon(verts)
    Z = planar.pmchwt_tm(poly, k0, eps)
    b = planar.rhs_pmchwt_tm(poly, k0, khat)
    x = np.linalg.solve(Z, b)
    e, h = planar.rhs_tm(poly, k0, khat)
    pa, pe, ps = planar.absorbed(poly, x), planar.extinguished(poly, x, e, h), planar.scattered(poly, k0, x)
    np.savez_compressed(OUT, x=x, p_abs=pa, p_ext=pe, p_sca=ps, k0=k0, eps_r=eps, n=len(verts),
                        perimeter=PERIMETER, aspect=ASPECT, angle=ANGLE)
    print(f"n={len(verts)} eps={eps:.6f} {time.time() - t0:.0f}s  2eta0 P abs/ext/sca = {pa:.6e} {pe:.6e} {ps:.6e}"
          f"  balance {(pe - pa - ps) / pe:.2e}")


if __name__ == "__main__":
    main()
