"""Empirical CFL bracketing, Algorithm 1 of Sec. 5.1.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For a final time T_f and a number of steps N (dt = T_f / N), run the scheme
from U0 without sources and watch the discrete energy E^n (Sec. 5.1).  The
run is unstable at the first step n where the relative energy increase
exceeds eps, measured against E^0 or against E^{n-1}.  After a stable run, N
decreases by delta N (rounded down, at least 1) and the run restarts, until
the first unstable run.  The result brackets the stability limit between
the last stable and the first unstable N.

Reading: "relative energy increase" is the signed increase (E^n - E^0)/E^0
and (E^n - E^{n-1})/E^{n-1}.  The absolute value printed in the listing would
flag the scheme's own dissipation as instability.
"""
from __future__ import annotations

import math

from .diagnostics import energy


def run_is_stable(stepper, U0, T_f, N, scheme="erk4", eps=0.05):
    dt = T_f / N
    U = U0.copy()
    E0 = energy(stepper.sys, U)
    Eprev = E0
    for n in range(N):
        U = stepper.step(U, n * dt, dt, scheme)
        E = energy(stepper.sys, U)
        if not math.isfinite(E) or (E - E0) / E0 > eps or (E - Eprev) / Eprev > eps:
            return False
        Eprev = E
    return True


def algorithm1(stepper, U0, T_f, N0, scheme="erk4", eps=0.05, delta=0.01, max_trials=500):
    """Returns (N_last_stable, N_first_unstable); N_last_stable is None if N0 itself is unstable."""
    N = N0
    last = None
    for _ in range(max_trials):
        if not run_is_stable(stepper, U0, T_f, N, scheme, eps):
            return last, N
        last = N
        N = N - max(1, int(math.floor(delta * N)))
        if N < 1:
            break
    return last, None
