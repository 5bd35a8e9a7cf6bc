"""torch.autograd bridge: receiver traces as a differentiable function of the
per-cell materials and of the source time function.

forward runs the GPU ERK stage path (hho_erk_step_record); backward runs the
discrete adjoint on the GPU (hho_adjoint_vjp).  Materials are per-cell
float64 tensors (rho, lambda, mu, kappa) in input cell order.  The
stabilisation weights follow the materials (Sec. 3.3: tau^f = eta_f/(rho c_P),
tau^s = eta_s rho c^s) in both passes, so the gradient is that of the forward
model.  Passing explicit weights (``tau``) instead holds them constant: the
gradient with tau frozen.

The source time function is a [nsteps, s] tensor of its values at the stage
times t0 + (n + c_j) dt (hho_sources_set_samples); its gradient is dL/dw per
step and stage.  ``TraceModel.ricker`` gives the Ricker samples, evaluated by
the library at the same rounded times as its ERK loops.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hho


class TraceModel:
    """Mesh, degree, one point source, receivers and time stepping of a trace simulation."""

    def __init__(self, mesh, k, source_xy, source_dir, receivers, dt, nsteps, stages=4, checkpoint_every=50,
                 t0=0.0, params=None):
        self.mesh = mesh
        self.k = k
        self.source_xy = source_xy
        self.source_dir = source_dir
        self.receivers = receivers
        self.dt = dt
        self.nsteps = nsteps
        self.stages = stages
        self.ckpt = checkpoint_every
        self.t0 = t0
        self.params = params

    def tableau(self):
        return hho.hho_tableau_erk(self.stages)

    def ricker(self, f0, t0=None, amp=1.0):
        """[nsteps, s] float64 tensor of Ricker values at the stage times."""
        w = hho.hho_ricker_samples(self.tableau(), self.t0, self.dt, self.nsteps, f0, 1.0 / f0 if t0 is None else t0,
                                   amp)
        return torch.as_tensor(w)

    def build(self, rho, lam, mu, kappa, wavelet, tau=None):
        """Operators with this model's source (time function ``wavelet``, [nsteps, s]) and receivers.
        tau None: weights from the materials; an array: those constants."""
        m = self.mesh
        handle = hho.hho_mesh_create(m.xy, m.cell_ptr, m.cell_vtx, m.cell_domain, getattr(m, "vertex_rep", None))
        try:
            ops = hho.hho_operators_build_tau(handle, self.k, rho, lam, mu, kappa, tau, params=self.params)
        finally:
            hho.hho_mesh_destroy(handle)
        try:
            hho.hho_sources_set_samples(ops, [self.source_xy], [self.source_dir], self.t0, self.dt,
                                        np.asarray(wavelet, dtype=np.float64)[None])
            hho.hho_receivers_set(ops, self.receivers)
        except Exception:
            hho.hho_ops_destroy(ops)
            raise
        return ops


def _state(ops, U0):
    lay = hho.hho_state_layout(ops)
    x = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
    c = torch.as_tensor(np.ascontiguousarray(U0, dtype=np.float64)).cuda()
    hho.hho_state_pack(ops, c.data_ptr(), x.data_ptr(), torch.cuda.current_stream().cuda_stream)
    return x


class Traces(torch.autograd.Function):
    """traces = Traces.apply(rho, lam, mu, kappa, wavelet, model, U0[, tau]): [nsteps, n_rec, 5]."""

    @staticmethod
    def forward(ctx, rho, lam, mu, kappa, wavelet, model, U0, tau=None):
        mats = [t.detach().cpu().numpy().astype(np.float64) for t in (rho, lam, mu, kappa)]
        w = wavelet.detach().cpu().numpy().astype(np.float64)
        ops = model.build(*mats, w, tau)
        try:
            tab = model.tableau()
            x = _state(ops, U0)
            work = torch.empty(hho.hho_work_size(ops, tab), dtype=torch.float64, device="cuda")
            seis = torch.zeros((model.nsteps, len(model.receivers), 5), dtype=torch.float64, device="cuda")
            hho.hho_erk_step_record(ops, tab, model.t0, model.dt, model.nsteps, x.data_ptr(), work.data_ptr(),
                                    seis.data_ptr(), torch.cuda.current_stream().cuda_stream)
        finally:
            hho.hho_ops_destroy(ops)
        ctx.model = model
        ctx.mats = mats
        ctx.w = w
        ctx.tau = tau
        ctx.U0 = U0
        return seis

    @staticmethod
    def backward(ctx, grad_out):
        model = ctx.model
        ops = model.build(*ctx.mats, ctx.w, ctx.tau)
        try:
            nc = len(ctx.mats[0])
            tab = model.tableau()
            x0 = _state(ops, ctx.U0)
            nw = hho.hho_adjoint_work_size(ops, tab, model.nsteps, model.ckpt)
            work = torch.empty(nw, dtype=torch.float64, device="cuda")
            g = grad_out.detach().to(device="cuda", dtype=torch.float64).contiguous()
            grad, gw = hho.hho_adjoint_vjp(ops, tab, model.t0, model.dt, model.nsteps, model.ckpt, x0.data_ptr(),
                                           g.data_ptr(), work.data_ptr(), nw, nc, n_src=1,
                                           stream=torch.cuda.current_stream().cuda_stream)
        finally:
            hho.hho_ops_destroy(ops)
        out = [torch.as_tensor(grad[:, j].copy()) for j in (0, 2, 3, 1)]   # rho, lambda, mu, kappa
        return out[0], out[1], out[2], out[3], torch.as_tensor(gw[:, :, 0].copy()), None, None, None
