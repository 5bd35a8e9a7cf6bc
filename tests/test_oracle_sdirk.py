"""Pins of the oracle's SDIRK stepping (Sec. 4.1, Eq. SDIRK, Eq. cp_dirk)
against what the mathematics fixes: Butcher's order conditions, A-stability
of the stability function, the equivalence of the full stage system with the
condensed ODE, the observed convergence order against the exact
semi-discrete solution exp(-t M^-1 K_cond) U0, and energy decay far beyond
the explicit stability limit."""
import numpy as np
import pytest
import scipy.linalg as sla

import synth
from oracle import diagnostics as D
from oracle import sdirk as SD
from tests.libutil import oracle_system, rel


def order_defects(name):
    """Residuals of the order conditions (Butcher) up to order 4."""
    A, b, c = SD.tableau(name)
    one = np.ones(len(b))
    Ac = A @ c
    return {
        1: [b @ one - 1.0],
        2: [b @ c - 0.5],
        3: [b @ c ** 2 - 1.0 / 3.0, b @ Ac - 1.0 / 6.0],
        4: [b @ c ** 3 - 0.25, b @ (c * Ac) - 1.0 / 8.0, b @ (A @ c ** 2) - 1.0 / 12.0, b @ (A @ Ac) - 1.0 / 24.0],
        "rows": list(A @ one - c),
    }


@pytest.mark.parametrize("name,order", [("sdirk1", 2), ("sdirk2", 2), ("sdirk23", 3), ("sdirk34", 4)])
def test_tableau_order(name, order):
    d = order_defects(name)
    assert max(abs(x) for x in d["rows"]) < 1e-14
    A, _, _ = SD.tableau(name)
    assert np.allclose(np.diag(A), A[0, 0]) and np.allclose(np.triu(A, 1), 0.0)
    for p in range(1, order + 1):
        assert max(abs(x) for x in d[p]) < 1e-14, (name, p, d[p])
    if order < 4:
        assert max(abs(x) for x in d[order + 1]) > 1e-3      # exactly that order


@pytest.mark.parametrize("name", ["sdirk1", "sdirk2", "sdirk23", "sdirk34"])
def test_a_stability(name):
    """|R(z)| <= 1 on the imaginary axis and the negative real axis, with
    R(z) = 1 + z b^T (I - z A)^-1 1 (the method applied to y' = z y)."""
    A, b, _ = SD.tableau(name)
    one = np.ones(len(b))

    def R(z):
        return 1.0 + z * (b @ np.linalg.solve(np.eye(len(b)) - z * A, one))
    for y in np.concatenate([np.linspace(-200, 200, 4001), [1e4, -1e4]]):
        assert abs(R(1j * y)) <= 1.0 + 1e-12
    for x in np.logspace(-3, 4, 200):
        assert abs(R(-x)) <= 1.0 + 1e-12


def small_case():
    md = synth.hybrid_grid(4, 4, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    media = synth.layered_media(md)
    return md, media


def test_full_system_equals_condensed_ode():
    md, media = small_case()
    S = oracle_system(md, 2, media)
    b, _ = S.point_load(0.37, 0.21, direction=(0.6, 0.8))
    st = SD.Stepper(S, lambda t: synth.ricker(t, 10.0) * b)
    U0 = synth.random_state(S.nT, 3)
    for name in ("sdirk2", "sdirk34"):
        full = st.step(U0, 0.02, 0.01, name, 3)
        cond = st.step_condensed(U0, 0.02, 0.01, name, 3)
        assert rel(full, cond) < 1e-12


@pytest.mark.parametrize("name,order", [("sdirk1", 2), ("sdirk2", 2), ("sdirk23", 3), ("sdirk34", 4)])
def test_convergence_order_against_matrix_exponential(name, order):
    md = synth.quad_grid(3, 3, 0.0, 1.0, 0.0, 1.0, 0.5)
    S = oracle_system(md, 1, synth.layered_media(md))
    st = SD.Stepper(S)
    KF = S.KF.toarray()
    Kc = S.KT.toarray() - S.KTF.toarray() @ np.linalg.solve(KF, S.KFT.toarray())
    Jm = -np.linalg.solve(S.M.toarray(), Kc)
    U0 = synth.random_state(S.nT, 11)
    T = 0.04
    exact = sla.expm(T * Jm) @ U0
    errs = [np.linalg.norm(st.step(U0, 0.0, T / N, name, N) - exact) for N in (32, 64)]
    rate = np.log2(errs[0] / errs[1])
    print(name, "errors", errs, "observed order %.2f" % rate)
    assert abs(rate - order) < 0.15


def test_energy_decays_far_beyond_explicit_limit():
    """At dt = 20 x the ERK4 stability limit of the same operator the
    SDIRK(3,4) energy (Sec. 5.1) does not grow."""
    md = synth.quad_grid(4, 4, 0.0, 1.0, 0.0, 1.0, 0.5)
    S = oracle_system(md, 2, synth.layered_media(md))
    KF = S.KF.toarray()
    Kc = S.KT.toarray() - S.KTF.toarray() @ np.linalg.solve(KF, S.KFT.toarray())
    lam = np.linalg.eigvals(-np.linalg.solve(S.M.toarray(), Kc))
    dt_erk = 2.785 / np.max(np.abs(lam))        # ERK4 reaches about 2.79 on the imaginary axis
    st = SD.Stepper(S)
    U = synth.random_state(S.nT, 5)
    E = [D.energy(S, U)]
    for _ in range(10):
        U = st.step(U, 0.0, 20 * dt_erk, "sdirk34")
        E.append(D.energy(S, U))
    assert np.all(np.diff(E) <= 1e-12 * E[0])
