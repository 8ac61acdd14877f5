"""Write slab_eighth_oracle.npz: the FP64 dense oracle solution of the 1/8-scale
lossy slab (closed box 1.25 x 1.25 x 1 free-space wavelengths, 26 x 26 x 21 face
divisions, 7,072 triangles, 21,216 unknowns, eps_r = 3.2 - 1.9j, k0 = 2 pi) under a
plane wave E0 = x, khat = -z (normal incidence on the top face).

Stored: the coefficients x = [eta0 J; M] of the LU solve, the per-triangle
absorbed power density and the total absorbed and extinguished powers.  Only
oracle/ is called; the run takes several minutes and about 30 GB of memory.

    python tests/golden/make_slab_eighth.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import excitation, operators, power, rwg  # noqa: E402

K0 = 2.0 * np.pi
EPS = 3.2 - 1.9j
KHAT = (0.0, 0.0, -1.0)
E0 = (1.0, 0.0, 0.0)
DIMS = (1.25, 1.25, 1.0, 26, 26, 21)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "slab_eighth_oracle.npz")


def main():
    t0 = time.time()
    v, t = W.box_mesh(*DIMS)
    g = rwg.build(v, t)
    Z = operators.pmchwt_matrix(g, K0, EPS)
    t1 = time.time()
    b = excitation.rhs_planewave(g, K0, KHAT, E0)
    x = np.linalg.solve(Z, b)
    t2 = time.time()
    dens = power.absorbed_density(g, x)
    p_abs = power.absorbed(g, x)
    p_ext = power.extinguished(g, x, b)
    np.savez_compressed(OUT, x=x, density=dens, p_abs=p_abs, p_ext=p_ext, k0=K0, eps_r=EPS,
                        khat=np.array(KHAT), e0=np.array(E0), dims=np.array(DIMS))
    print(f"ne={g.ne} nt={len(t)} assemble {t1 - t0:.0f}s solve {t2 - t1:.0f}s p_abs={p_abs:.9g} p_ext={p_ext:.9g}")


if __name__ == "__main__":
    main()
