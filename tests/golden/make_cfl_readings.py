"""Writes tests/golden/cfl_readings.json: the ERK4 stability limit of the
oracle's operator on the paper's CFL test (Sec. 5.1: fluid (0,1)^2 with
rho = kappa = 1, solid (-1,0)x(0,1) with rho = 1, c_P = sqrt 3, c_S = 1;
eta_f = 0.8, eta_s = 1.5; k = 1; squares and right triangles with h = 1/8),
under the readings the paper leaves open, next to Table 2/3's CFL*
(0.282 squares, 0.265 triangles):

* tau^s = eta_s rho c^s with c^s = c_P (our reading) or c_S;
* h in c# dt / h as the edge length (our reading) or the cell diameter;
* CFL* from the eigenvalue limit (largest dt with |R(dt lambda)| <= 1 for
  every eigenvalue lambda of -M^-1 K_cond, R the ERK4 polynomial), and from
  Algorithm 1 (eps = 5 %, delta = 1 %, T_f = 1) started from random data and
  from the paper's own initial data, the sinusoid of Eq. non_poly_sol with
  omega = 5 at t = 0.

Everything is computed by the oracle alone.
Run: python tests/golden/make_cfl_readings.py
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
from oracle import cfl as CF  # noqa: E402
from oracle import erk as E  # noqa: E402
from oracle import mesh as M  # noqa: E402
from tests import exact  # noqa: E402

C_SHARP = math.sqrt(3.0)
H = 1.0 / 8


def cfl_mesh(kind):
    if kind == "squares":
        md = synth.quad_grid(16, 8, -1.0, 1.0, 0.0, 1.0)
    else:
        md = synth.tri_grid(16, 8, -1.0, 1.0, 0.0, 1.0)
    md.cell_domain = np.where(md.centroids_approx()[:, 0] < 0, 1, 0).astype(np.uint8)
    return md


def system(md, stab_speed, k=1):
    nc = md.n_cells
    sol = md.cell_domain == 1
    m = M.build_mesh(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
    return A.System(m, k, np.ones(nc), np.where(sol, 1.0, 0.0), np.where(sol, 1.0, 0.0), np.ones(nc),
                    eta_f=0.8, eta_s=1.5, stab_speed=stab_speed)


def eigen_limit(S, s=4):
    KT, KTF, KFT, KF, Mm = (x.toarray() for x in (S.KT, S.KTF, S.KFT, S.KF, S.M))
    ev = sl.eigvals(-np.linalg.solve(Mm, KT - KTF @ np.linalg.solve(KF, KFT)))
    lo, hi = 0.0, 10.0 / np.abs(ev).max()
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        z = mid * ev
        R = sum(z ** j / math.factorial(j) for j in range(s + 1))
        lo, hi = (mid, hi) if np.abs(R).max() <= 1 + 1e-12 else (lo, mid)
    return lo


def algorithm1_cfl(S, U0, dt_eig, T_f=1.0):
    st = E.Stepper(S)
    N0 = int(math.ceil(T_f / (0.7 * dt_eig)))   # start well inside the stable range
    n_stable, n_unstable = CF.algorithm1(st, U0, T_f, N0, max_trials=400)
    return {"n_stable": n_stable, "n_unstable": n_unstable,
            "cfl_edge": None if n_stable is None else C_SHARP * T_f / n_stable / H}


def main():
    out = {"setting": "Sec. 5.1 CFL test, k = 1, ERK4, eta_f = 0.8, eta_s = 1.5, h = 1/8 (edge), c# = sqrt 3",
           "table": {"squares": 0.282, "triangles": 0.265}, "cases": {}}
    ic = exact.Sinusoid(w=5.0, th=math.sqrt(2.0), lam=1.0, mu=1.0)
    for kind in ("squares", "triangles"):
        md = cfl_mesh(kind)
        for speed in ("cp", "cs"):
            S = system(md, speed)
            dt = eigen_limit(S)
            case = {"eigen_dt": dt, "eigen_cfl_edge": C_SHARP * dt / H, "eigen_cfl_diameter": C_SHARP * dt / (H * math.sqrt(2.0))}
            if True:   # Algorithm 1 from random data and from the paper's initial data
                case["algorithm1_random_ic"] = algorithm1_cfl(S, synth.random_state(S.nT, 8), dt)
                case["algorithm1_sinusoid_ic"] = algorithm1_cfl(S, S.project(ic.fields(0.0), order=6), dt)
            out["cases"]["%s_tau_s_%s" % (kind, speed)] = case
            print(kind, speed, case, flush=True)
    # the dependence on k (Table 2: CFL* 0.282 / 0.138 / 0.087 for k = 1 / 2 / 3, ratios 1 / 0.49 / 0.31),
    # eigenvalue limits on squares, h = 1/4 (k = 2, 3 hold more unknowns per cell)
    out["table_k"] = {"1": 0.282, "2": 0.138, "3": 0.087}
    out["squares_by_k"] = {}
    md = synth.quad_grid(8, 4, -1.0, 1.0, 0.0, 1.0)
    md.cell_domain = np.where(md.centroids_approx()[:, 0] < 0, 1, 0).astype(np.uint8)
    for speed in ("cp", "cs"):
        row = {}
        for k in (1, 2, 3):
            dt = eigen_limit(system(md, speed, k))
            row[str(k)] = {"eigen_cfl_edge": C_SHARP * dt / 0.25, "eigen_cfl_diameter": C_SHARP * dt / (0.25 * math.sqrt(2.0))}
        for k in ("2", "3"):
            row[k]["ratio_to_k1"] = row[k]["eigen_cfl_edge"] / row["1"]["eigen_cfl_edge"]
        out["squares_by_k"]["tau_s_" + speed] = row
        print(speed, row, flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "cfl_readings.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
