"""Write ellipse_rank_study.json: epsilon-ranks of the non-circulant part
C_p - C_p,c of the Calderon-stabilised CFIE (Eq. 16) on the ellipse of the
paper's rank study (aspect ratio 1.5, perimeter 2 pi, 18 unknowns per wavelength:
N = 18 k0), from the singular values of the dense oracle matrices, for
k0 = 4 ... 64 and tolerances 1e-2, 1e-3, 1e-4 (relative to the largest singular
value), for the TM form of Eq. 16 ("ranks") and its TE dual ("ranks_te").  Only
oracle/ is called; about half an hour on 8 cores.

    python tests/golden/make_rank_study.py
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import planar  # noqa: E402

K0S = (4.0, 8.0, 16.0, 32.0, 64.0)
TOLS = (1e-2, 1e-3, 1e-4)
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "ellipse_rank_study.json")


def main():
    rows = []
    for k0 in K0S:
        t0 = time.time()
        n = int(round(18 * k0))
        poly = planar.Polygon(W.ellipse_polygon(n, 1.5, 2.0 * math.pi))
        circ = planar.circular_counterpart(poly)
        a = planar.curvature_radius(poly)
        row = {"k0": k0, "n": n}
        for key, form in (("ranks", planar.calderon_cfie), ("ranks_te", planar.calderon_cfie_te)):
            Cp, _, _ = form(poly, k0)
            Cc, _, _ = form(circ, k0, a=a)
            sv = np.linalg.svd(Cp - Cc, compute_uv=False)
            row[key] = {f"{t:g}": int(np.sum(sv > t * sv[0])) for t in TOLS}
        row["seconds"] = round(time.time() - t0, 1)
        rows.append(row)
        print(rows[-1], flush=True)
    with open(OUT, "w") as f:
        json.dump({"curve": "ellipse aspect 1.5 perimeter 2pi, N = 18 k0",
                   "operator": "C_p - C_p,c (Calderon CFIE minus its equal-perimeter circular counterpart); "
                               "ranks: TM (Eq. 16), ranks_te: its TE dual",
                   "rows": rows}, f, indent=1)


if __name__ == "__main__":
    main()
