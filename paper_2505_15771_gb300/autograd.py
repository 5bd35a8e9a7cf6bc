"""torch.autograd bridge: receiver traces as a differentiable function of the
per-cell materials and the source amplitude.

forward runs the GPU ERK stage path (hho_erk_step_record); backward runs the
discrete adjoint on the GPU (hho_adjoint_vjp).  The stabilisation weights
tau are those of the forward model and are held fixed in the backward pass
(the gradient of the discrete scheme with tau frozen).  Materials are
per-cell float64 tensors (rho, lambda, mu, kappa) in input cell order.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hho


class TraceModel:
    """Mesh, degree, source, receivers and time stepping of a trace simulation."""

    def __init__(self, mesh, k, source_xy, source_dir, f0, receivers, dt, nsteps, stages=4, checkpoint_every=50,
                 t0=0.0):
        self.mesh = mesh
        self.k = k
        self.source_xy = source_xy
        self.source_dir = source_dir
        self.f0 = f0
        self.receivers = receivers
        self.dt = dt
        self.nsteps = nsteps
        self.stages = stages
        self.ckpt = checkpoint_every
        self.t0 = t0

    def build(self, rho, lam, mu, kappa, amp, tau=None):
        m = self.mesh
        handle = hho.hho_mesh_create(m.xy, m.cell_ptr, m.cell_vtx, m.cell_domain, getattr(m, "vertex_rep", None))
        try:
            ops = hho.hho_operators_build_tau(handle, self.k, rho, lam, mu, kappa, tau)
        finally:
            hho.hho_mesh_destroy(handle)
        hho.hho_sources_set(ops, [self.source_xy], [self.source_dir], [self.f0], [1.0 / self.f0], [amp])
        hho.hho_receivers_set(ops, self.receivers)
        return ops


def _state(ops, U0):
    lay = hho.hho_state_layout(ops)
    x = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
    c = torch.as_tensor(np.ascontiguousarray(U0, dtype=np.float64)).cuda()
    hho.hho_state_pack(ops, c.data_ptr(), x.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return x


class Traces(torch.autograd.Function):
    """traces = Traces.apply(rho, lam, mu, kappa, amp, model, U0): [nsteps, n_rec, 5]."""

    @staticmethod
    def forward(ctx, rho, lam, mu, kappa, amp, model, U0):
        mats = [t.detach().cpu().numpy().astype(np.float64) for t in (rho, lam, mu, kappa)]
        a = float(amp.detach().cpu().item())
        ops = model.build(*mats, a)
        try:
            nc = len(mats[0])
            tau = hho.hho_ops_tau(ops, nc)
            tab = hho.hho_tableau_erk(model.stages)
            x = _state(ops, U0)
            work = torch.empty(hho.hho_work_size(ops, tab), dtype=torch.float64, device="cuda")
            seis = torch.zeros((model.nsteps, len(model.receivers), 5), dtype=torch.float64, device="cuda")
            hho.hho_erk_step_record(ops, tab, model.t0, model.dt, model.nsteps, x.data_ptr(), work.data_ptr(),
                                    seis.data_ptr(), torch.cuda.current_stream().cuda_stream)
        finally:
            hho.hho_ops_destroy(ops)
        ctx.model = model
        ctx.mats = mats
        ctx.amp = a
        ctx.tau = tau
        ctx.U0 = U0
        return seis

    @staticmethod
    def backward(ctx, grad_out):
        model = ctx.model
        ops = model.build(*ctx.mats, ctx.amp, ctx.tau)
        try:
            nc = len(ctx.mats[0])
            tab = hho.hho_tableau_erk(model.stages)
            x0 = _state(ops, ctx.U0)
            nw = hho.hho_adjoint_work_size(ops, tab, model.nsteps, model.ckpt)
            work = torch.empty(nw, dtype=torch.float64, device="cuda")
            g = grad_out.detach().to(device="cuda", dtype=torch.float64).contiguous()
            grad, gw = hho.hho_adjoint_vjp(ops, tab, model.t0, model.dt, model.nsteps, model.ckpt, x0.data_ptr(),
                                           g.data_ptr(), work.data_ptr(), nw, nc, n_src=1,
                                           stream=torch.cuda.current_stream().cuda_stream)
        finally:
            hho.hho_ops_destroy(ops)
        # the wavelet is proportional to the amplitude: dL/damp = sum dL/dw * w / amp
        _, _, c = _tableau_arrays(tab)
        ts = model.t0 + (np.arange(model.nsteps)[:, None] + c[None, :]) * model.dt
        a2 = (np.pi * model.f0 * (ts - 1.0 / model.f0)) ** 2
        w_unit = (1.0 - 2.0 * a2) * np.exp(-a2)
        g_amp = float(np.sum(gw[:, :, 0] * w_unit))
        out = [torch.as_tensor(grad[:, j].copy()) for j in (0, 2, 3, 1)]
        return out[0], out[1], out[2], out[3], torch.tensor(g_amp, dtype=torch.float64), None, None


def _tableau_arrays(tab):
    s = tab.s
    return None, None, np.array([tab.c[i] for i in range(s)])
