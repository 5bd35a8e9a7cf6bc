"""The double-float arithmetic (HHO_F32X2: every value a pair of FP32 numbers,
error-free transforms on the FP32 pipes) against the FP64 oracle, at the
FP64 bar: relative L2 <= 1e-12, for the rate operator on every mesh family,
ERK(2,3,4) steps, the academic full run with receivers, the full-size
bilayer (sampled), and batched shots."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import diagnostics as D
from oracle import erk as E
from tests.libutil import ROOT, ensure_built, oracle_system, rel
from tests.test_gpu_parity import _edge_neighbours, _patch, cases, media_for

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


def problem(lib, md, media, k):
    hho, solver = lib
    P = solver.Problem(md, media, k)
    P.set_arithmetic(hho.HHO_F32X2)
    return P


@pytest.mark.parametrize("name,md,k,seed", cases())
def test_rate_operator_f32x2(lib, name, md, k, seed):
    media = media_for(md, seed)
    S = oracle_system(md, k, media)
    U = synth.random_state(S.nT, 100 + k)
    ref = E.Stepper(S).rate(U, 0.0)
    P = problem(lib, md, media, k)
    err = rel(P.to_canonical(P.apply(P.to_device(U))), ref)
    print(name, "f32x2 rate rel err %.3e" % err)
    assert err <= TOL


@pytest.mark.parametrize("s", [2, 3, 4])
@pytest.mark.parametrize("name,md,k,seed", [cases()[1], cases()[3], cases()[4], cases()[7]])
def test_erk_steps_f32x2(lib, name, md, k, seed, s):
    media = media_for(md, seed)
    S = oracle_system(md, k, media)
    U = synth.random_state(S.nT, 7)
    dt = 0.02 / (k * k) * (0.4 if name == "basin_k2" else 1.0)
    ref = E.Stepper(S).step(U, 0.0, dt, "erk%d" % s, 5)
    P = problem(lib, md, media, k)
    x = P.to_device(U)
    P.step(x, s, 0.0, dt, 5)
    err = rel(P.to_canonical(x), ref)
    print(name, s, "f32x2 erk rel err %.3e" % err)
    assert err <= TOL


def test_academic_c1_full_run_f32x2(lib):
    """512 triangles, k = 1, ERK4, 200 CFL-limited steps, Ricker point force,
    8 interface receivers recorded every step (one call, in-kernel records)."""
    hho, _ = lib
    w = synth.academic_c1()
    md, media, k = w["mesh"], w["media"], w["k"]
    dt = json.load(open(os.path.join(ROOT, "tests/golden/c1_dt.json")))["dt"]
    S = oracle_system(md, k, media)
    b, _ = S.point_load(*w["source"], direction=(0.0, 1.0))
    f0 = w["f0"]
    st = E.Stepper(S, lambda t: synth.ricker(t, f0) * b)
    P = problem(lib, md, media, k)
    P.set_sources([w["source"]], [(0.0, 1.0)], f0)
    P.set_receivers(w["receivers"])
    U = np.zeros(S.nT)
    tr_ref = []
    for n in range(w["nsteps"]):
        U = st.step(U, n * dt, dt, "erk4")
        tr_ref.append(D.sensors(st, U, w["receivers"]))
    tr_ref = np.array(tr_ref)
    x = P.to_device(np.zeros(S.nT))
    tab = hho.hho_tableau_erk(4)
    seis = torch.zeros((w["nsteps"], len(w["receivers"]), 5), dtype=torch.float64, device=P.dev)
    hho.hho_erk_step_record(P.ops, tab, 0.0, dt, w["nsteps"], x.data_ptr(), P.work(tab).data_ptr(), seis.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    e_state = rel(P.to_canonical(x), U)
    e_tr = rel(seis.cpu().numpy()[:, :, :3], tr_ref[:, :, :3])
    print("C1 f32x2 state rel err %.3e receiver rel err %.3e" % (e_state, e_tr))
    assert np.linalg.norm(U) > 0
    assert e_state <= TOL
    assert e_tr <= TOL


@pytest.mark.parametrize("k", [2, 3])
def test_full_size_bilayer_sampled_f32x2(lib, k):
    """The 1024 x 512 bilayer at full size in the benchmark's launch
    configuration: one ERK4 step of a seeded random state, checked on 24
    sample cells against the oracle on each sample's 4-ring patch."""
    w = synth.bilayer_c2(k=k)
    md, media = w["mesh"], w["media"]
    P = problem(lib, md, media, k)
    n = (k + 1) * (k + 2) // 2
    sizes = np.where(md.cell_domain == 0, 3 * n, 5 * n)
    off = np.concatenate([[0], np.cumsum(sizes)])
    U = synth.random_state(int(off[-1]), 21)
    x = P.to_device(U)
    dt = 0.9 * 0.1 * (1.0 / 512) / 3.6 / k
    P.step(x, 4, 0.0, dt, 1)
    got = P.to_canonical(x)
    nbr = _edge_neighbours(md)
    rng = np.random.default_rng(5)
    iface = [c for c in range(md.n_cells) if any(md.cell_domain[o] != md.cell_domain[c] for o in nbr[c])]
    samples = list(rng.choice(md.n_cells, 20, replace=False)) + list(rng.choice(iface, 4, replace=False))
    worst = 0.0
    for c in samples:
        cells, sub = _patch(md, nbr, int(c), 4)
        sub_media = tuple(np.asarray(a)[cells] for a in media)
        S = oracle_system(sub, k, sub_media)
        Us = np.concatenate([U[off[o]:off[o + 1]] for o in cells])
        ref_all = E.Stepper(S).step(Us, 0.0, dt, "erk4", 1)
        i = cells.index(int(c))
        worst = max(worst, rel(got[off[c]:off[c + 1]], ref_all[S.cell_off[i]:S.cell_off[i + 1]]))
    print("full-size f32x2 k=%d worst sampled rel err %.3e" % (k, worst))
    assert worst <= TOL


@pytest.mark.parametrize("name,md,k", [
    ("hybrid_k3", synth.hybrid_grid(6, 6, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5), 3),
    ("basin_k2", synth.basin_c5(nx=40, ny=10)["mesh"], 2),
])
def test_batched_f32x2_matches_oracle_per_shot(lib, name, md, k):
    hho, solver = lib
    media = synth.layered_media(md)
    S = oracle_system(md, k, media)
    P = solver.Problem(md, media, k)
    shots = 3
    pts = [(0.21, 0.13), (0.55, 0.31), (0.8, 0.41)]
    dirs = [(0.0, 1.0), (1.0, 0.0), (0.6, 0.8)]
    P.set_shot_sources(pts, dirs, 10.0)
    U0 = np.stack([synth.random_state(S.nT, 40 + i) for i in range(shots)])
    x = P.batch_to_device(U0, precision=hho.HHO_F32X2)
    _, work = P.batch_buffers(4, shots, precision=hho.HHO_F32X2)
    dt = 0.01 / k * (0.4 if name == "basin_k2" else 1.0)
    P.batch_step(x, work, shots, 4, 0.05, dt, 4, precision=hho.HHO_F32X2)
    got = P.batch_to_canonical(x, shots, precision=hho.HHO_F32X2)
    for i in range(shots):
        b, _ = S.point_load(*pts[i], direction=dirs[i])
        st = E.Stepper(S, lambda t, b=b: synth.ricker(t, 10.0) * b)
        ref = st.step(U0[i], 0.05, dt, "erk4", 4)
        err = rel(got[i], ref)
        print(name, "f32x2 shot", i, "rel err %.3e" % err)
        assert err <= TOL
