"""The adjoint workload at full size: 256 x 256 quads, k = 2, two-layer
medium, true model with a +10 % Gaussian v_S anomaly, smooth background as
the current model, 8 shots, 128 receivers, 800 ERK4 steps, checkpoints every
50 steps, L2 receiver misfit.  The GPU gradient (the stabilisation weights
following the materials, as in the forward model) is checked against
central differences of the GPU misfit on 20 seeded random directions."""
import time

import numpy as np
import pytest

import synth
from tests.libutil import ROOT, ensure_built

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho
    return hho


def test_c4_misfit_gradient_vs_central_differences(lib):
    hho = lib
    w = synth.adjoint_c4()
    md = w["mesh"]
    nc = md.n_cells
    k, nsteps, ckpt = w["k"], 800, 50
    stream = torch.cuda.current_stream().cuda_stream
    tab = hho.hho_tableau_erk(4)

    def build(media):
        mesh = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
        ops = hho.hho_operators_build(mesh, k, *media)
        hho.hho_mesh_destroy(mesh)
        hho.hho_receivers_set(ops, w["receivers"])
        return ops

    def shot(ops, s):
        hho.hho_sources_set(ops, [w["sources"][s]], [(0.0, 1.0)], [w["f0"]], [1.0 / w["f0"]], [1.0])

    probe = build(w["background"])
    dt = hho.hho_cfl_dt(probe, 0.122, 0.9)
    lay = hho.hho_state_layout(probe)
    hho.hho_ops_destroy(probe)
    x = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")

    def traces(ops):
        x.zero_()
        wk = torch.empty(hho.hho_work_size(ops, tab), dtype=torch.float64, device="cuda")
        seis = torch.zeros((nsteps, len(w["receivers"]), 5), dtype=torch.float64, device="cuda")
        hho.hho_erk_step_record(ops, tab, 0.0, dt, nsteps, x.data_ptr(), wk.data_ptr(), seis.data_ptr(), stream)
        return seis

    shots = len(w["sources"])
    observed = []
    ops = build(w["true"])
    for s in range(shots):
        shot(ops, s)
        observed.append(traces(ops).clone())
    hho.hho_ops_destroy(ops)

    def misfit(media):
        J = 0.0
        ops = build(media)
        for s in range(shots):
            shot(ops, s)
            J += 0.5 * float(((traces(ops) - observed[s]) ** 2).sum())
        hho.hho_ops_destroy(ops)
        return J

    grad = np.zeros((nc, 4))
    zero0 = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
    ops = build(w["background"])
    nw = hho.hho_adjoint_work_size(ops, tab, nsteps, ckpt)
    wk = torch.empty(nw, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t_adj = 0.0
    for s in range(shots):
        shot(ops, s)
        resid = (traces(ops) - observed[s]).contiguous()
        torch.cuda.synchronize()
        t = time.perf_counter()
        g, _ = hho.hho_adjoint_vjp(ops, tab, 0.0, dt, nsteps, ckpt, zero0.data_ptr(), resid.data_ptr(),
                                   wk.data_ptr(), nw, nc, n_src=1, stream=stream)
        t_adj += time.perf_counter() - t
        grad += g
    hho.hho_ops_destroy(ops)
    rho, lam, mu, kap = w["background"]
    J0 = misfit(w["background"])
    assert J0 > 0
    rng = np.random.default_rng(20)
    scale = np.stack([rho, kap, lam, mu], axis=1)
    worst = 0.0
    for trial in range(20):
        d = rng.standard_normal((nc, 4)) * scale * 0.01
        eps = 1e-4
        fd = (misfit((rho + eps * d[:, 0], lam + eps * d[:, 2], mu + eps * d[:, 3], kap + eps * d[:, 1])) -
              misfit((rho - eps * d[:, 0], lam - eps * d[:, 2], mu - eps * d[:, 3], kap - eps * d[:, 1]))) / (2 * eps)
        an = float(np.sum(grad * d))
        err = abs(fd - an) / abs(fd)
        print("direction %2d: adjoint %.9e  central difference %.9e  rel err %.2e" % (trial, an, fd, err))
        worst = max(worst, err)
    print("C4 misfit %.6e, adjoint %.2f s for %d shots, worst rel err %.3e over 20 directions"
          % (J0, t_adj, shots, worst))
    assert worst <= 1e-6
