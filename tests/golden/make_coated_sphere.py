"""Write coated_sphere_oracle.npz: the FP64 dense oracle solution of the coated
(two-layer) lossy sphere -- outer icosphere of 5,120 triangles and radius 1 (shell
eps_r = 3.2 - 1.9j), inner icosphere of 1,280 triangles and radius 0.5 (core
eps_r = 2.5 - 1.2j), k0 = 6, 19,200 unknowns -- under a plane wave E0 = x,
khat = +z.

Stored: the coefficients x = [eta0 J; M] of the LU solve (both surfaces, the
outer one first), the absorbed, extinguished and scattered powers of the whole
body (2 eta0 P, i.e. efficiency times pi a^2) and the coated-sphere series'
efficiencies for the same body.  Only oracle/ is called; the run takes tens of
minutes and about 20 GB of memory.

    python tests/golden/make_coated_sphere.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import mie, multiregion, power, rwg  # noqa: E402

K0 = 6.0
EPS_SHELL = 3.2 - 1.9j
EPS_CORE = 2.5 - 1.2j
LEVELS = (4, 3)
RADII = (1.0, 0.5)
KHAT = (0.0, 0.0, 1.0)
E0 = (1.0, 0.0, 0.0)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "coated_sphere_oracle.npz")


def mesh():
    """Both surfaces in one mesh and per-triangle (region on the normal side, region behind)."""
    return W.coated_sphere(LEVELS[0], RADII[0], LEVELS[1], RADII[1])


def main():
    t0 = time.time()
    v, t, regions = mesh()
    g = rwg.build(v, t)
    Z = multiregion.pmchwt_regions(g, regions, K0, [1.0, EPS_SHELL, EPS_CORE])
    t1 = time.time()
    b = multiregion.rhs_planewave(g, regions, K0, KHAT, E0)
    x = np.linalg.solve(Z, b)
    del Z
    t2 = time.time()
    xe = multiregion.exterior_currents(g, regions, x)
    p_abs = power.absorbed(g, xe)
    p_ext = power.extinguished(g, xe, b)
    p_sca = power.scattered(g, K0, xe)
    q = mie.coated_efficiencies_eps(K0, RADII[1], RADII[0], EPS_CORE, EPS_SHELL)
    np.savez_compressed(OUT, x=x, p_abs=p_abs, p_ext=p_ext, p_sca=p_sca, k0=K0,
                        eps=np.array([1.0, EPS_SHELL, EPS_CORE]), levels=np.array(LEVELS), radii=np.array(RADII),
                        khat=np.array(KHAT), e0=np.array(E0),
                        mie=np.array([q["ext"], q["abs"], q["sca"]]))
    a2 = np.pi * RADII[0] ** 2
    print(f"ne={g.ne} nt={len(t)} assemble {t1 - t0:.0f}s solve {t2 - t1:.0f}s "
          f"Q ext/abs/sca = {p_ext / a2:.6f} {p_abs / a2:.6f} {p_sca / a2:.6f}  "
          f"series {q['ext']:.6f} {q['abs']:.6f} {q['sca']:.6f}")


if __name__ == "__main__":
    main()
