"""The paper's Ricker initial-condition workloads (Sec. 5.2, Eq. ricker_ic):
the L2 projection of the pulse (hho_project_field) against the oracle's
projection, short ERK4 runs from it with the three sensors against the
oracle (FP64 and double-float), and the paper-size runs to T_f with the
discrete energy (Sec. 5.1) checked to be non-increasing."""
import numpy as np
import pytest

import synth
from oracle import diagnostics as D
from oracle import erk as E
from tests.libutil import ensure_built, oracle_system, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFL_SQUARES_ERK4 = {1: 0.233, 2: 0.122, 3: 0.082}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, solver
    return hho, solver


def pulse_fields(pulse):
    xc, yc, theta, lam = pulse

    def fields(x, y, dom):
        if dom == 1:
            return np.zeros((5, len(x)))
        g = theta * np.exp(-np.pi ** 2 * ((x - xc) ** 2 + (y - yc) ** 2) / lam ** 2)
        return np.stack([g * (x - xc), g * (y - yc), np.zeros_like(x)])
    return fields


def workloads():
    return [("academic", synth.ricker_academic(16, 2)), ("academic_k3", synth.ricker_academic(12, 3)),
            ("granite", synth.granite_water(0.1, 2))]


@pytest.mark.parametrize("name,w", workloads())
def test_projection_matches_oracle(lib, name, w):
    hho, solver = lib
    md, media, k = w["mesh"], w["media"], w["k"]
    S = oracle_system(md, k, media)
    ref = S.project(pulse_fields(w["pulse"]), order=24)
    P = solver.Problem(md, media, k)
    got = hho.hho_project_field(P.ops, hho.HHO_FIELD_RICKER, w["pulse"])
    err = rel(got, ref)
    print(name, "projection rel err %.3e, |U0| %.3e" % (err, np.linalg.norm(ref)))
    assert np.linalg.norm(ref) > 0
    assert err <= 1e-12


@pytest.mark.parametrize("arith", ["f64", "f32x2"])
@pytest.mark.parametrize("name,w", workloads())
def test_short_run_with_sensors(lib, name, w, arith):
    """40 ERK4 steps from the projected pulse at 0.9 x the square CFL limit,
    sensors S^f, S^s, S^i recorded after every step (in-kernel records)."""
    hho, solver = lib
    md, media, k = w["mesh"], w["media"], w["k"]
    S = oracle_system(md, k, media)
    st = E.Stepper(S)
    U0 = S.project(pulse_fields(w["pulse"]), order=24)
    dt = 0.9 * CFL_SQUARES_ERK4[k] * w["h"] / w["c_max"]
    nsteps = 40
    U = U0.copy()
    tr_ref = []
    for n in range(nsteps):
        U = st.step(U, n * dt, dt, "erk4")
        tr_ref.append(D.sensors(st, U, w["sensors"]))
    tr_ref = np.array(tr_ref)
    P = solver.Problem(md, media, k)
    P.set_arithmetic(hho.HHO_F64 if arith == "f64" else hho.HHO_F32X2)
    P.set_receivers(w["sensors"])
    x = P.to_device(hho.hho_project_field(P.ops, hho.HHO_FIELD_RICKER, w["pulse"]))
    tab = hho.hho_tableau_erk(4)
    seis = torch.zeros((nsteps, len(w["sensors"]), 5), dtype=torch.float64, device=P.dev)
    hho.hho_erk_step_record(P.ops, tab, 0.0, dt, nsteps, x.data_ptr(), P.work(tab).data_ptr(), seis.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    e_state = rel(P.to_canonical(x), U)
    e_tr = rel(seis.cpu().numpy()[:, :, :3], tr_ref[:, :, :3])
    print(name, arith, "state rel err %.3e sensors rel err %.3e" % (e_state, e_tr))
    assert e_state <= 1e-12
    assert e_tr <= 1e-12


@pytest.mark.parametrize("name,w", [("academic 64x64", synth.ricker_academic(64, 2)),
                                    ("granite-water 25 m", synth.granite_water(0.025, 2))])
def test_paper_size_run_to_final_time(lib, name, w):
    """The full runs of Sec. 5.2 (k = 2, ERK4, CFL-limited dt, no source):
    every step's sensors finite, the discrete energy non-increasing at every
    tenth of the run (the stabilisation only dissipates) and still positive."""
    hho, solver = lib
    md, media, k = w["mesh"], w["media"], w["k"]
    P = solver.Problem(md, media, k)
    P.set_arithmetic(hho.HHO_F32X2)
    P.set_receivers(w["sensors"])
    x = P.to_device(hho.hho_project_field(P.ops, hho.HHO_FIELD_RICKER, w["pulse"]))
    dt = 0.9 * CFL_SQUARES_ERK4[k] * w["h"] / w["c_max"]
    nsteps = int(np.ceil(w["T_f"] / dt))
    dt = w["T_f"] / nsteps
    tab = hho.hho_tableau_erk(4)
    chunk = (nsteps + 9) // 10
    seis = torch.zeros((chunk, len(w["sensors"]), 5), dtype=torch.float64, device=P.dev)
    energies = [P.energy(x)]
    done = 0
    while done < nsteps:
        m = min(chunk, nsteps - done)
        hho.hho_erk_step_record(P.ops, tab, done * dt, dt, m, x.data_ptr(), P.work(tab).data_ptr(), seis.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
        assert bool(torch.isfinite(seis[:m]).all())
        done += m
        energies.append(P.energy(x))
    e = np.array(energies)
    print(name, "%d steps, energy E(T_f)/E(0) = %.4f" % (nsteps, e[-1] / e[0]))
    assert np.all(np.diff(e) <= 1e-12 * e[0])
    assert e[-1] > 0
