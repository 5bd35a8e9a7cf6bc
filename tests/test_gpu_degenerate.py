"""Degenerate meshes against the oracle, in both arithmetics: one domain only
(no interface; the device's fluid or solid block is empty), two cells (one
of each domain: every face on the boundary or the interface), a single
cell, and a zero-step call."""
import numpy as np
import pytest

import synth
from oracle import erk as E
from tests.libutil import ensure_built, oracle_system, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, solver
    return hho, solver


def meshes():
    return [
        ("fluid_only", synth.quad_grid(5, 3, 0.0, 1.0, 0.0, 1.0, y_interface=-1.0)),
        ("solid_only", synth.quad_grid(3, 5, 0.0, 1.0, 0.0, 1.0, y_interface=2.0)),
        ("two_quads", synth.quad_grid(1, 2, 0.0, 1.0, 0.0, 1.0, 0.5)),
        ("two_triangles", synth.tri_grid(1, 1)),
        ("one_quad", synth.quad_grid(1, 1, 0.0, 1.0, 0.0, 1.0, y_interface=-1.0)),
    ]


@pytest.mark.parametrize("arith", ["f64", "f32x2"])
@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("name,md", meshes())
def test_degenerate_mesh_parity(lib, name, md, k, arith):
    """The rate operator and three ERK4 steps against the oracle."""
    hho, solver = lib
    media = synth.layered_media(md)
    S = oracle_system(md, k, media)
    st = E.Stepper(S)
    U = synth.random_state(S.nT, 11 + k)
    P = solver.Problem(md, media, k)
    P.set_arithmetic(hho.HHO_F64 if arith == "f64" else hho.HHO_F32X2)
    e_rate = rel(P.to_canonical(P.apply(P.to_device(U))), st.rate(U, 0.0))
    dt = 0.005 / k
    x = P.to_device(U)
    P.step(x, 4, 0.0, dt, 3)
    e_step = rel(P.to_canonical(x), st.step(U, 0.0, dt, "erk4", 3))
    print(name, k, arith, "rate %.2e steps %.2e" % (e_rate, e_step))
    assert e_rate <= TOL and e_step <= TOL
    P.close()


def test_zero_steps_leave_the_state_unchanged(lib):
    hho, solver = lib
    md = synth.hybrid_grid(4, 4, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    P = solver.Problem(md, synth.layered_media(md), 2)
    U = synth.random_state(P.layout.n_canonical, 5)
    for arith in (hho.HHO_F64, hho.HHO_F32X2):
        P.set_arithmetic(arith)
        x = P.to_device(U)
        P.step(x, 4, 0.0, 0.001, 0)
        assert np.array_equal(P.to_canonical(x), U)
    P.close()
