"""Algorithm 1 of Sec. 5.1 (empirical CFL bracketing) run through the GPU stage,
against the oracle's run of the same algorithm and against Table 2."""
import numpy as np
import pytest

import synth
from oracle import cfl as CF
from oracle import erk as E
from tests.libutil import ensure_built, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, solver
    return hho, solver


def cfl_case(nx=6):
    """The paper's CFL test medium (rho = kappa = 1, c_P^s = sqrt 3, c_S = 1), squares."""
    md = synth.quad_grid(nx, nx // 2, -1.0, 1.0, 0.0, 1.0)
    md.cell_domain = np.where(md.centroids_approx()[:, 0] < 0, 1, 0).astype(np.uint8)
    nc = md.n_cells
    sol = md.cell_domain == 1
    media = (np.ones(nc), np.where(sol, 1.0, 0.0), np.where(sol, 1.0, 0.0), np.ones(nc))
    return md, media


def gpu_bracket(hho, P, U0, T_f, N0, s=4):
    tab = hho.hho_tableau_erk(s)
    x0 = P.to_device(U0)
    x = P.empty_state()
    work = torch.empty(hho.hho_work_size(P.ops, tab), dtype=torch.float64, device=P.dev)
    return hho.hho_cfl_bracket(P.ops, tab, x0.data_ptr(), T_f, N0, 0.05, 0.01, 500, x.data_ptr(), work.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)


def test_gpu_algorithm1_matches_oracle(lib):
    hho, solver = lib
    md, media = cfl_case()
    S = oracle_system(md, 1, media)
    st = E.Stepper(S)
    U0 = synth.random_state(S.nT, 8)
    T_f, N0 = 1.0, 450
    ref = CF.algorithm1(st, U0, T_f, N0)
    P = solver.Problem(md, media, 1)
    got = gpu_bracket(hho, P, U0, T_f, N0)
    print("oracle", ref, "gpu", got)
    assert tuple(got) == tuple(ref)


def test_gpu_algorithm1_stage_ratios_table2(lib):
    """Table 2: CFL* ratios wrt s (ERK2 : ERK3 : ERK4 = 1 : 1.23-1.25 : 1.38-1.39)
    from Algorithm 1 run on the GPU with random initial data."""
    hho, solver = lib
    md, media = cfl_case(8)
    P = solver.Problem(md, media, 1)
    U0 = synth.random_state(P.layout.n_canonical, 9)
    T_f = 1.0
    dts = []
    for s, N0 in ((2, 900), (3, 700), (4, 600)):
        n_stable, n_unstable = gpu_bracket(hho, P, U0, T_f, N0, s)
        assert n_stable > 0 and n_unstable > 0
        dts.append(T_f / n_stable)
    r3, r4 = dts[1] / dts[0], dts[2] / dts[0]
    print("ratios", r3, r4)
    assert abs(r3 - 1.23) < 0.05 and abs(r4 - 1.38) < 0.05


def test_gpu_algorithm1_rejects_zero_initial_energy(lib):
    """Algorithm 1's test is relative to E^0, so a zero state has no answer:
    the call fails with HHO_EINVAL instead of counting every trial stable."""
    hho, solver = lib
    md, media = cfl_case()
    P = solver.Problem(md, media, 1)
    U0 = np.zeros(P.layout.n_canonical)
    with pytest.raises(hho.HHOError) as e:
        gpu_bracket(hho, P, U0, 1.0, 100)
    assert e.value.code == hho.HHO_EINVAL
    assert "initial energy" in str(e.value)
