"""Discrete adjoint on the GPU (hho_adjoint_vjp) against the oracle's dense
reverse mode and against central differences of the GPU forward traces.
The stabilisation weights follow the materials (Sec. 3.3) unless they are
given explicitly (hho_operators_build_tau), which freezes them."""
import numpy as np
import pytest

import synth
from oracle import adjoint as ADJ
from oracle import erk as E
from tests.libutil import ensure_built, oracle_system

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PTS = [(0.31, 0.2), (0.77, 0.41), (0.18, 0.5), (0.62, 0.5), (0.4, 0.8), (0.9, 0.66)]
SRC = (0.55, 0.3)
F0 = 6.0


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, solver
    return hho, solver


def media(md, seed):
    rng = np.random.default_rng(seed)
    nc = md.n_cells
    sol = md.cell_domain == 1
    rho = 1 + rng.random(nc)
    lam = np.where(sol, 3 + rng.random(nc), 0.0)
    mu = np.where(sol, 2 + rng.random(nc), 0.0)
    kap = np.where(sol, 0.0, 1 + rng.random(nc))
    return rho, lam, mu, kap


def gpu_problem(hho, md, k, med, tau=None):
    mesh = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
    ops = hho.hho_operators_build_tau(mesh, k, *med, tau)
    hho.hho_mesh_destroy(mesh)
    hho.hho_sources_set(ops, [SRC], [(0.0, 1.0)], [F0], [1.0 / F0], [1.0])
    hho.hho_receivers_set(ops, PTS)
    return ops


def gpu_traces(hho, ops, U0, dt, nsteps, s=4):
    tab = hho.hho_tableau_erk(s)
    lay = hho.hho_state_layout(ops)
    c = torch.as_tensor(U0).cuda()
    x = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
    hho.hho_state_pack(ops, c.data_ptr(), x.data_ptr())
    work = torch.empty(hho.hho_work_size(ops, tab), dtype=torch.float64, device="cuda")
    seis = torch.zeros((nsteps, len(PTS), 5), dtype=torch.float64, device="cuda")
    hho.hho_erk_step_record(ops, tab, 0.0, dt, nsteps, x.data_ptr(), work.data_ptr(), seis.data_ptr())
    return seis.cpu().numpy()


def gpu_vjp(hho, ops, U0, dt, nsteps, G, nc, s=4, ckpt=5, with_tau=False):
    tab = hho.hho_tableau_erk(s)
    lay = hho.hho_state_layout(ops)
    c = torch.as_tensor(U0).cuda()
    x0 = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
    hho.hho_state_pack(ops, c.data_ptr(), x0.data_ptr())
    nw = hho.hho_adjoint_work_size(ops, tab, nsteps, ckpt)
    work = torch.empty(nw, dtype=torch.float64, device="cuda")
    g = torch.as_tensor(G.reshape(nsteps, len(PTS), 5)).cuda().contiguous()
    return hho.hho_adjoint_vjp(ops, tab, 0.0, dt, nsteps, ckpt, x0.data_ptr(), g.data_ptr(), work.data_ptr(), nw,
                               nc, n_src=1, with_tau=with_tau)


@pytest.mark.parametrize("k,s,frozen", [(1, 4, False), (2, 3, False), (2, 4, True)])
def test_adjoint_matches_oracle(lib, k, s, frozen):
    """Material gradients dL/d(rho, kappa, lambda, mu), wavelet gradients
    dL/dw(t_i) and (tau following the materials) dL/dtau of L = <G, traces>
    agree with the oracle's dense reverse mode; cell and interface receivers."""
    hho, solver = lib
    md = synth.quad_grid(6, 6)
    med = media(md, 1)
    Sy = oracle_system(md, k, med)
    if frozen:
        Sy = oracle_system(md, k, med, tau_override=Sy.tau)
    st = E.Stepper(Sy)
    load, _ = Sy.point_load(*SRC, direction=(0.0, 1.0))
    dense = ADJ.DenseAdjoint(st, PTS, load, lambda t: synth.ricker(t, F0))
    nsteps, dt = 17, 0.004
    rng = np.random.default_rng(7)
    U0 = synth.random_state(Sy.nT, 5)
    G = rng.standard_normal((nsteps, len(PTS) * 5))
    tr_ref, _ = dense.run(U0, 0.0, dt, nsteps, "erk%d" % s)
    ops = gpu_problem(hho, md, k, med, Sy.tau if frozen else None)
    try:
        tr = gpu_traces(hho, ops, U0, dt, nsteps, s)
        assert np.linalg.norm(tr.reshape(nsteps, -1) - tr_ref) <= 1e-12 * np.linalg.norm(tr_ref)
        g_ref, w_ref, t_ref = dense.vjp(U0, 0.0, dt, nsteps, G, "erk%d" % s, with_tau=True)
        g, w, gt = gpu_vjp(hho, ops, U0, dt, nsteps, G, md.n_cells, s, with_tau=True)
    finally:
        hho.hho_ops_destroy(ops)
    eg = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
    ew = np.linalg.norm(w[:, :, 0] - w_ref) / np.linalg.norm(w_ref)
    et = np.linalg.norm(gt - t_ref) / np.linalg.norm(t_ref)
    print("k=%d ERK%d frozen=%s gradient rel err %.3e wavelet %.3e dL/dtau %.3e" % (k, s, frozen, eg, ew, et))
    assert eg <= 1e-10 and ew <= 1e-10 and et <= 1e-10


@pytest.mark.parametrize("frozen", [False, True])
def test_adjoint_matches_finite_differences(lib, frozen):
    """<grad, delta> against central differences of L = <G, traces> computed
    with the GPU forward on 6 seeded random material directions, relative
    error <= 1e-6.  Unfrozen: every forward rebuilds tau from the materials;
    frozen: tau fixed at the base model (hho_operators_build_tau)."""
    hho, solver = lib
    md = synth.quad_grid(8, 8)
    med = media(md, 2)
    nc = md.n_cells
    nsteps, dt = 30, 0.003
    rng = np.random.default_rng(11)
    base = gpu_problem(hho, md, 2, med)
    tau = hho.hho_ops_tau(base, nc)
    if frozen:
        hho.hho_ops_destroy(base)
        base = gpu_problem(hho, md, 2, med, tau)
    lay = hho.hho_state_layout(base)
    U0 = synth.random_state(lay.n_canonical, 3)
    G = rng.standard_normal((nsteps, len(PTS) * 5))
    g, _ = gpu_vjp(hho, base, U0, dt, nsteps, G, nc, 4, ckpt=7)
    hho.hho_ops_destroy(base)
    rho, lam, mu, kap = med
    worst = 0.0
    for trial in range(6):
        d = rng.standard_normal((nc, 4)) * np.stack([rho, kap, lam, mu], axis=1) * 0.05
        eps = 1e-5

        def L(sign):
            ops = gpu_problem(hho, md, 2, (rho + sign * eps * d[:, 0], lam + sign * eps * d[:, 2],
                                           mu + sign * eps * d[:, 3], kap + sign * eps * d[:, 1]),
                              tau if frozen else None)
            try:
                tr = gpu_traces(hho, ops, U0, dt, nsteps)
            finally:
                hho.hho_ops_destroy(ops)
            return float(np.sum(tr.reshape(nsteps, -1) * G))
        fd = (L(1) - L(-1)) / (2 * eps)
        an = float(np.sum(g * d))
        worst = max(worst, abs(fd - an) / abs(fd))
    print("adjoint (frozen=%s) vs central differences, worst rel err %.3e" % (frozen, worst))
    assert worst <= 1e-6


def test_sampled_ricker_sources_step_like_ricker_sources(lib):
    """hho_sources_set_samples with the library's Ricker samples
    (hho_ricker_samples) gives bit-identical traces to hho_sources_set with
    the same wavelet (stream launches: the same host-side values)."""
    hho, solver = lib
    md = synth.quad_grid(6, 6)
    med = media(md, 3)
    nsteps, dt, s = 12, 0.004, 4
    U0 = 0.1 * synth.random_state(gpu_layout_n(hho, md, med), 2)
    out = []
    for sampled in (False, True):
        ops = gpu_problem(hho, md, 2, med)
        try:
            hho.hho_set_launch_mode(ops, hho.HHO_LAUNCH_STREAM)
            if sampled:
                w = hho.hho_ricker_samples(hho.hho_tableau_erk(s), 0.0, dt, nsteps, F0, 1.0 / F0, 1.0)
                hho.hho_sources_set_samples(ops, [SRC], [(0.0, 1.0)], 0.0, dt, w[None])
            out.append(gpu_traces(hho, ops, U0, dt, nsteps, s))
        finally:
            hho.hho_ops_destroy(ops)
    assert np.array_equal(out[0], out[1])
    assert np.abs(out[0]).max() > 0


def gpu_layout_n(hho, md, med):
    ops = gpu_problem(hho, md, 2, med)
    n = hho.hho_state_layout(ops).n_canonical
    hho.hho_ops_destroy(ops)
    return n


def test_autograd_traces_misfit(lib):
    """torch.autograd.Function: L = 1/2 |traces - observed|^2; backward gives
    dL/d(rho, lambda, mu, kappa) and dL/dw per step and stage of the source
    time function through the GPU adjoint, with tau following the materials;
    checked against central differences of the same forward in a random
    direction of materials and wavelet."""
    hho, solver = lib
    from paper_2505_15771_gb300.autograd import TraceModel, Traces
    md = synth.quad_grid(6, 6)
    rho, lam, mu, kap = media(md, 4)
    nsteps, dt = 20, 0.004
    model = TraceModel(md, 1, SRC, (0.0, 1.0), PTS, dt, nsteps, stages=4, checkpoint_every=6)
    U0 = 0.1 * synth.random_state(hho_layout_k1(hho, md, (rho, lam, mu, kap)), 9)
    rng = np.random.default_rng(5)
    obs = torch.as_tensor(rng.standard_normal((nsteps, len(PTS), 5))).cuda()
    T = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in (rho, lam, mu, kap)]
    w0 = model.ricker(F0)
    wav = w0.clone().requires_grad_(True)
    tr = Traces.apply(T[0], T[1], T[2], T[3], wav, model, U0)
    loss = 0.5 * ((tr - obs) ** 2).sum()
    loss.backward()
    assert wav.grad.shape == (nsteps, 4)
    d = rng.standard_normal((md.n_cells, 4)) * np.stack([rho, lam, mu, kap], axis=1) * 0.05
    dw = rng.standard_normal((nsteps, 4)) * 0.3
    an = sum(float(np.sum(T[j].grad.numpy() * d[:, j])) for j in range(4)) + float(np.sum(wav.grad.numpy() * dw))
    eps = 1e-6
    obs_np = obs.cpu().numpy()

    def L(sign):
        ops = model.build(rho + sign * eps * d[:, 0], lam + sign * eps * d[:, 1], mu + sign * eps * d[:, 2],
                          kap + sign * eps * d[:, 3], w0.numpy() + sign * eps * dw)
        try:
            t = gpu_traces(hho, ops, U0, dt, nsteps)
        finally:
            hho.hho_ops_destroy(ops)
        return 0.5 * float(np.sum((t - obs_np) ** 2))
    fd = (L(1) - L(-1)) / (2 * eps)
    print("autograd vs central differences: %.12e %.12e" % (an, fd))
    assert abs(fd - an) <= 1e-6 * abs(fd)


def hho_layout_k1(hho, md, med):
    mesh = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
    ops = hho.hho_operators_build_tau(mesh, 1, *med, None)
    hho.hho_mesh_destroy(mesh)
    n = hho.hho_state_layout(ops).n_canonical
    hho.hho_ops_destroy(ops)
    return n


def test_fp32_adjoint_against_fp64(lib):
    """The FP32 reverse mode (FP32 stage kernels, FP64 gradient sums) against
    the FP64 one on the same problem, tau following the materials: material,
    wavelet and tau gradients within 1e-3 relative (FP32 rounding over 30
    steps), with cell and interface receivers."""
    hho, solver = lib
    md = synth.quad_grid(8, 8)
    med = media(md, 6)
    nc = md.n_cells
    nsteps, dt, ckpt = 30, 0.003, 7
    tab = hho.hho_tableau_erk(4)
    ops = gpu_problem(hho, md, 2, med)
    try:
        lay = hho.hho_state_layout(ops)
        U0 = synth.random_state(lay.n_canonical, 12)
        G = np.random.default_rng(13).standard_normal((nsteps, len(PTS), 5))
        g64, w64, t64 = gpu_vjp(hho, ops, U0, dt, nsteps, G, nc, 4, ckpt=ckpt, with_tau=True)
        c = torch.as_tensor(U0).cuda()
        x64 = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
        hho.hho_state_pack(ops, c.data_ptr(), x64.data_ptr())
        x32 = x64.float()
        g32t = torch.as_tensor(G).float().cuda().contiguous()
        nw = hho.hho_adjoint_work_size_f32(ops, tab, nsteps, ckpt)
        work = torch.empty(nw, dtype=torch.float32, device="cuda")
        g32, w32, t32 = hho.hho_adjoint_vjp_f32(ops, tab, 0.0, dt, nsteps, ckpt, x32.data_ptr(), g32t.data_ptr(),
                                                work.data_ptr(), nw, nc, n_src=1, with_tau=True)
    finally:
        hho.hho_ops_destroy(ops)
    eg = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
    ew = np.linalg.norm(w32 - w64) / np.linalg.norm(w64)
    et = np.linalg.norm(t32 - t64) / np.linalg.norm(t64)
    print("FP32 adjoint vs FP64: materials %.2e, wavelet %.2e, tau %.2e" % (eg, ew, et))
    assert eg <= 1e-3 and ew <= 1e-3 and et <= 1e-3
