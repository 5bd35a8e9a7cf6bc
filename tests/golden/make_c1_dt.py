"""Writes tests/golden/c1_dt.json: the ERK4 stability limit of the academic
512-triangle workload (k = 1), computed from the oracle alone.

dt_max is the largest dt for which every eigenvalue lambda of
-M^-1 (K_T - K_TF K_F^-1 K_FT) satisfies |R(dt lambda)| <= 1 with R the ERK4
stability polynomial sum_{j<=4} z^j/j! (Eq. ERK, classical tableau).  The
workload's time step is 0.9 dt_max ("CFL-limited dt").  The paper's Table 3
CFL* for triangles refers to its own simplicial meshes and does not carry
over to this right-triangle grid (it would be unstable here).
Run: python tests/golden/make_c1_dt.py
"""
import json
import math
import os
import sys

import numpy as np
import scipy.linalg as sl

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import assemble as A  # noqa: E402
from oracle import mesh as M  # noqa: E402


def stability_limit(S, s=4):
    KT, KTF, KFT, KF, Mm = (x.toarray() for x in (S.KT, S.KTF, S.KFT, S.KF, S.M))
    ev = sl.eigvals(-np.linalg.solve(Mm, KT - KTF @ np.linalg.solve(KF, KFT)))
    lo, hi = 0.0, 10.0 / np.abs(ev).max()
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        z = mid * ev
        R = sum(z ** j / math.factorial(j) for j in range(s + 1))
        lo, hi = (mid, hi) if np.abs(R).max() <= 1 + 1e-12 else (lo, mid)
    return lo, float(ev.real.max()), float(np.abs(ev).max())


def main():
    w = synth.academic_c1()
    md = w["mesh"]
    m = M.build_mesh(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
    S = A.System(m, w["k"], *w["media"])
    dtmax, remax, rho = stability_limit(S)
    out = {"dt_max": dtmax, "dt": 0.9 * dtmax, "cfl_of_dt_max": dtmax * w["c_max"] / w["h"],
           "max_real_eig": remax, "spectral_radius": rho,
           "source": "tests/golden/make_c1_dt.py (oracle eigenvalues, ERK4 stability polynomial)"}
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_dt.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
