"""Implicit SDIRK stepping on the GPU (hho_sdirk_step: matrix-free GMRES on
the stage systems, the ERK stage kernel as the operator) against the
oracle's full non-condensed stage solves (Eq. cp_dirk, sparse LU): relative
L2 <= 1e-12 after several steps far beyond the explicit stability limit."""
import numpy as np
import pytest

import synth
from oracle import sdirk as SD
from tests.libutil import ensure_built, oracle_system, rel
from tests.test_gpu_parity import random_media

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NAMES = {1: "sdirk1", 2: "sdirk2", 3: "sdirk34", 23: "sdirk23"}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, solver
    return hho, solver


def explicit_limit(S):
    """ERK4 step limit of the semi-discrete operator (largest |eigenvalue|)."""
    Kc = S.KT.toarray() - S.KTF.toarray() @ np.linalg.solve(S.KF.toarray(), S.KFT.toarray())
    lam = np.linalg.eigvals(-np.linalg.solve(S.M.toarray(), Kc))
    return 2.785 / np.max(np.abs(lam))


@pytest.mark.parametrize("s", [3, 2, 23, 1])
def test_sdirk_with_source_matches_oracle(lib, s):
    hho, solver = lib
    md = synth.hybrid_grid(5, 5, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    media = synth.layered_media(md)
    S = oracle_system(md, 2, media)
    b, _ = S.point_load(0.37, 0.21, direction=(0.6, 0.8))
    st = SD.Stepper(S, lambda t: synth.ricker(t, 10.0) * b)
    U0 = synth.random_state(S.nT, 3)
    dt = 8.0 * explicit_limit(S)
    ref = st.step(U0, 0.02, dt, NAMES[s], 4)
    P = solver.Problem(md, media, 2)
    P.set_sources([(0.37, 0.21)], [(0.6, 0.8)], 10.0)
    x = P.to_device(U0)
    its = P.sdirk_step(x, s, 0.02, dt, 4, tol=1e-14, restart=40, max_iter=4000)
    err = rel(P.to_canonical(x), ref)
    print("SDIRK s=%d dt = 8 x explicit limit: rel err %.3e, %d GMRES applications (%.1f per stage)"
          % (s, err, its, its / (4.0 * (2 if s == 23 else s))))
    assert err <= 1e-12


@pytest.mark.parametrize("k", [1, 2, 3])
def test_sdirk34_random_media_matches_oracle(lib, k):
    hho, solver = lib
    md = synth.quad_grid(5, 5, 0.0, 1.0, 0.0, 1.0, 0.45)
    media = random_media(md, 9)
    S = oracle_system(md, k, media)
    st = SD.Stepper(S)
    U0 = synth.random_state(S.nT, 4)
    dt = 5.0 * explicit_limit(S)
    ref = st.step(U0, 0.0, dt, "sdirk34", 3)
    P = solver.Problem(md, media, k)
    x = P.to_device(U0)
    its = P.sdirk_step(x, 3, 0.0, dt, 3, tol=1e-14, restart=40, max_iter=4000)
    err = rel(P.to_canonical(x), ref)
    print("SDIRK(3,4) k=%d: rel err %.3e, %d GMRES applications" % (k, err, its))
    assert err <= 1e-12


def test_sdirk_energy_decays_on_bilayer(lib):
    """128 x 64 bilayer (random-field solid under water), k = 2, SDIRK(3,4)
    at 4 x the ERK4 square CFL limit: the discrete energy does not grow."""
    hho, solver = lib
    w = synth.bilayer_c2(nx=128, ny=64, k=2)
    P = solver.Problem(w["mesh"], w["media"], 2)
    n = P.layout.n_canonical
    x = P.to_device(synth.random_state(n, 8))
    dt = 4.0 * hho.hho_cfl_dt(P.ops, 0.122, 1.0)
    E = [P.energy(x)]
    total = 0
    for _ in range(5):
        total += P.sdirk_step(x, 3, 0.0, dt, 1, tol=1e-10, restart=40, max_iter=4000)
        E.append(P.energy(x))
    print("bilayer 128x64 SDIRK(3,4): energies", ["%.6e" % e for e in E], "GMRES applications", total)
    assert np.all(np.diff(E) <= 1e-12 * E[0])


@pytest.mark.parametrize("k", [1, 2])
def test_block_jacobi_preconditioner(lib, k):
    """Block-Jacobi right preconditioning (the cell blocks of Eq. sc2) on a
    quad/triangle mesh with an interface (more than two colours): the same
    solution as the unpreconditioned solve and the oracle, with fewer
    operator applications.  (k = 3, with 50 x 50 solid blocks, runs
    preconditioned in test_sdirk34_random_media_matches_oracle; unpreconditioned
    GMRES(40) does not reach this tolerance there within 8000 applications.)"""
    hho, solver = lib
    md = synth.hybrid_grid(6, 6, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    media = random_media(md, 11)
    S = oracle_system(md, k, media)
    st = SD.Stepper(S)
    U0 = synth.random_state(S.nT, 6)
    dt = 8.0 * explicit_limit(S)
    ref = st.step(U0, 0.0, dt, "sdirk34", 2)
    out = {}
    for kind in (0, 1):
        P = solver.Problem(md, media, k)
        hho.hho_sdirk_set_preconditioner(P.ops, kind)
        x = P.to_device(U0)
        its = P.sdirk_step(x, 3, 0.0, dt, 2, tol=1e-14, restart=40, max_iter=8000)
        out[kind] = (rel(P.to_canonical(x), ref), its)
        P.close()
    print("k=%d SDIRK(3,4) at 8 x the explicit limit: no preconditioner err %.2e, %d applications; "
          "block Jacobi err %.2e, %d applications" % (k, out[0][0], out[0][1], out[1][0], out[1][1]))
    assert out[0][0] <= 1e-12 and out[1][0] <= 1e-12
    assert out[1][1] < out[0][1]


def test_preconditioner_kind_is_checked(lib):
    hho, solver = lib
    md = synth.quad_grid(2, 2, 0.0, 1.0, 0.0, 1.0, 0.5)
    P = solver.Problem(md, synth.layered_media(md), 1)
    with pytest.raises(Exception):
        hho.hho_sdirk_set_preconditioner(P.ops, 2)
    P.close()
