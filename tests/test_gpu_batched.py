"""Batched shots (S right-hand sides on one mesh, one launch per stage for all
shots) in FP64 and FP32, against the CPU oracle run shot by shot."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import diagnostics as D
from oracle import erk as E
from tests.libutil import ROOT, ensure_built, oracle_system, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, solver
    return hho, solver


@pytest.mark.parametrize("name,md,k", [
    ("quad_k2", synth.quad_grid(6, 5, 0.0, 1.2, 0.0, 1.0, 0.5), 2),
    ("hybrid_k3", synth.hybrid_grid(6, 6, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5), 3),
    ("hanging_k1", synth.hanging_node_patch(6, 6, refine_rows=(2, 3)), 1),
    ("basin_k2", synth.basin_c5(nx=40, ny=10)["mesh"], 2),
])
def test_batched_f64_matches_oracle_per_shot(lib, name, md, k):
    """Each of 3 shots (own random state, own point force) after 4 ERK4 steps
    equals the oracle's single run of that shot: rel L2 <= 1e-12."""
    hho, solver = lib
    media = synth.layered_media(md)
    S = oracle_system(md, k, media)
    P = solver.Problem(md, media, k)
    shots = 3
    pts = [(0.21, 0.13), (0.55, 0.31), (0.8, 0.41)]
    dirs = [(0.0, 1.0), (1.0, 0.0), (0.6, 0.8)]
    P.set_shot_sources(pts, dirs, 10.0)
    U0 = np.stack([synth.random_state(S.nT, 40 + i) for i in range(shots)])
    x = P.batch_to_device(U0)
    _, work = P.batch_buffers(4, shots)
    dt = 0.01 / k * (0.4 if name == "basin_k2" else 1.0)
    P.batch_step(x, work, shots, 4, 0.05, dt, 4)
    got = P.batch_to_canonical(x, shots)
    for i in range(shots):
        b, _ = S.point_load(*pts[i], direction=dirs[i])
        st = E.Stepper(S, lambda t, b=b: synth.ricker(t, 10.0) * b)
        ref = st.step(U0[i], 0.05, dt, "erk4", 4)
        err = rel(got[i], ref)
        print(name, "shot", i, "rel err", err)
        assert err <= 1e-12


def test_batched_single_shot_equals_single_path(lib):
    hho, solver = lib
    md = synth.tri_grid(8, 8)
    media = synth.layered_media(md)
    P = solver.Problem(md, media, 2)
    U = synth.random_state(P.layout.n_canonical, 3)
    x1 = P.to_device(U)
    P.step(x1, 4, 0.0, 0.002, 5)
    xb = P.batch_to_device(U[None, :])
    _, work = P.batch_buffers(4, 1)
    P.batch_step(xb, work, 1, 4, 0.0, 0.002, 5)
    assert np.array_equal(P.batch_to_canonical(xb, 1)[0], P.to_canonical(x1))


@pytest.mark.parametrize("k,nsteps", [(1, 200), (3, 60)])
def test_batched_f32_seismograms(lib, k, nsteps):
    """FP32 batched shots against the FP64 oracle: 4 shots (Ricker point forces
    at seeded solid points) on the academic bilayer, receivers on the
    interface recorded every step; relative l2 error of every trace <= 1e-5."""
    hho, solver = lib
    w = synth.academic_c1()
    md, media = w["mesh"], w["media"]
    dt = json.load(open(os.path.join(ROOT, "tests/golden/c1_dt.json")))["dt"] / (k * k)
    S = oracle_system(md, k, media)
    P = solver.Problem(md, media, k)
    shots = 4
    pts = [synth.seeded_point(50 + i, 0.0, 1.0, 0.0, 0.5) for i in range(shots)]
    dirs = [(0.0, 1.0)] * shots
    P.set_shot_sources(pts, dirs, 10.0)
    P.set_receivers(w["receivers"])
    x = P.batch_to_device(np.zeros((shots, S.nT)), precision=hho.HHO_F32)
    _, work = P.batch_buffers(4, shots, hho.HHO_F32)
    seis = torch.zeros((nsteps, shots, len(w["receivers"]), 5), dtype=torch.float32, device=P.dev)
    P.batch_step(x, work, shots, 4, 0.0, dt, nsteps, precision=hho.HHO_F32, seismogram=seis)
    seis = seis.double().cpu().numpy()
    worst = 0.0
    for i in range(shots):
        b, _ = S.point_load(*pts[i], direction=dirs[i])
        st = E.Stepper(S, lambda t, b=b: synth.ricker(t, 10.0) * b)
        U = np.zeros(S.nT)
        ref = []
        for n in range(nsteps):
            U = st.step(U, n * dt, dt, "erk4")
            ref.append(D.sensors(st, U, w["receivers"]))
        ref = np.array(ref)[:, :, :3]
        e = rel(seis[:, i, :, :3], ref)
        worst = max(worst, e)
    print("k=%d FP32 worst seismogram rel err %.3e" % (k, worst))
    assert worst <= 1e-5
