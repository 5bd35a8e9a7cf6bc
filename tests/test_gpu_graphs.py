"""Graph-replayed ERK steps (hho_set_launch_mode: one captured step per
distinct set of kernel arguments, stage times and Ricker wavelets from a
device clock) against stream launches and the oracle."""
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


def test_academic_c1_full_run_graph_mode(lib):
    """The 200-step academic run (k = 1, ERK4, Ricker source, 8 interface
    receivers recorded in every replayed step) against the oracle."""
    hho, solver = lib
    w = synth.academic_c1()
    md, media, k = w["mesh"], w["media"], w["k"]
    dt = json.load(open(os.path.join(ROOT, "tests/golden/c1_dt.json")))["dt"]
    S = oracle_system(md, k, media)
    b, _ = S.point_load(*w["source"], direction=(0.0, 1.0))
    st = E.Stepper(S, lambda t: synth.ricker(t, w["f0"]) * b)
    U = np.zeros(S.nT)
    tr_ref = []
    for n in range(w["nsteps"]):
        U = st.step(U, n * dt, dt, "erk4")
        tr_ref.append(D.sensors(st, U, w["receivers"]))
    tr_ref = np.array(tr_ref)
    P = solver.Problem(md, media, k)
    P.set_launch_mode(hho.HHO_LAUNCH_GRAPH)
    P.set_sources([w["source"]], [(0.0, 1.0)], w["f0"])
    P.set_receivers(w["receivers"])
    x = P.to_device(np.zeros(S.nT))
    tab = hho.hho_tableau_erk(4)
    seis = torch.zeros((w["nsteps"], len(w["receivers"]), 5), dtype=torch.float64, device=P.dev)
    hho.hho_erk_step_record(P.ops, tab, 0.0, dt, w["nsteps"], x.data_ptr(), P.work(tab).data_ptr(), seis.data_ptr(),
                            torch.cuda.current_stream().cuda_stream)
    e_state = rel(P.to_canonical(x), U)
    e_tr = rel(seis.cpu().numpy()[:, :, :3], tr_ref[:, :, :3])
    print("C1 graph mode: state rel err %.3e receivers rel err %.3e" % (e_state, e_tr))
    assert e_state <= 1e-12 and e_tr <= 1e-12


@pytest.mark.parametrize("s", [3, 4])
@pytest.mark.parametrize("arith", ["f64", "f32x2"])
def test_graph_equals_stream(lib, s, arith):
    """Same run, graph replay vs stream launches, in two calls each (the
    second call starts from the first's end at a later time, so the clock's
    start time and the trace buffers' parity change): state and every
    recorded trace agree to 1e-14."""
    hho, solver = lib
    md = synth.hybrid_grid(8, 8, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    media = synth.layered_media(md)
    rec = synth.receivers_on_line(6, 0.0, 1.0, 0.5)
    out = {}
    for mode in (hho.HHO_LAUNCH_STREAM, hho.HHO_LAUNCH_GRAPH):
        P = solver.Problem(md, media, 2)
        P.set_arithmetic(hho.HHO_F64 if arith == "f64" else hho.HHO_F32X2)
        P.set_launch_mode(mode)
        P.set_sources([(0.37, 0.21)], [(0.6, 0.8)], 10.0)
        P.set_receivers(rec)
        x = P.to_device(synth.random_state(P.layout.n_canonical, 5))
        tab = hho.hho_tableau_erk(s)
        dt = 0.002
        seis = []
        for t0, n in ((0.01, 9), (0.01 + 9 * dt, 12)):
            sz = torch.zeros((n, len(rec), 5), dtype=torch.float64, device=P.dev)
            hho.hho_erk_step_record(P.ops, tab, t0, dt, n, x.data_ptr(), P.work(tab).data_ptr(), sz.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
            seis.append(sz.cpu().numpy())
        out[mode] = (P.to_canonical(x), np.concatenate(seis))
        P.close()
    e_state = rel(out[hho.HHO_LAUNCH_GRAPH][0], out[hho.HHO_LAUNCH_STREAM][0])
    e_tr = rel(out[hho.HHO_LAUNCH_GRAPH][1], out[hho.HHO_LAUNCH_STREAM][1])
    print("ERK%d %s graph vs stream: state %.3e traces %.3e" % (s, arith, e_state, e_tr))
    assert e_state <= 1e-14 and e_tr <= 1e-14


def test_batched_graph_equals_stream(lib):
    """Batched FP32 shots (one source per shot), graph vs stream, with the
    step buffers changed between calls (a fresh state and work pair)."""
    hho, solver = lib
    md = synth.hybrid_grid(8, 8, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    media = synth.layered_media(md)
    pts = [(0.21, 0.13), (0.55, 0.31), (0.8, 0.41)]
    out = {}
    for mode in (hho.HHO_LAUNCH_STREAM, hho.HHO_LAUNCH_GRAPH):
        P = solver.Problem(md, media, 2)
        P.set_launch_mode(mode)
        P.set_shot_sources(pts, [(0.0, 1.0)] * 3, 10.0)
        res = []
        for seed in (1, 2):
            U0 = np.stack([synth.random_state(P.layout.n_canonical, 10 * seed + i) for i in range(3)])
            x = P.batch_to_device(U0, precision=hho.HHO_F32)
            _, work = P.batch_buffers(4, 3, precision=hho.HHO_F32)
            P.batch_step(x, work, 3, 4, 0.0, 0.002, 10, precision=hho.HHO_F32)
            res.append(P.batch_to_canonical(x, 3, precision=hho.HHO_F32))
        out[mode] = np.concatenate(res)
        P.close()
    err = rel(out[hho.HHO_LAUNCH_GRAPH], out[hho.HHO_LAUNCH_STREAM])
    print("batched FP32 graph vs stream: %.3e" % err)
    assert err <= 1e-6
