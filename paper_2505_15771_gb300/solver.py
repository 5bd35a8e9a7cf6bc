"""Convenience layer over the C ABI: torch tensors for device memory and streams.

PyTorch only allocates device buffers and provides the stream; every step of
the stage path runs in libhho's kernels (see hho.py for the raw binding).
"""
from __future__ import annotations

import numpy as np
import torch

from . import hho


def _stream(stream):
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


class Problem:
    """A mesh, its media and the stage operator of degree k on the current GPU.

    ``mesh`` is anything with xy, cell_ptr, cell_vtx, cell_domain and optional
    vertex_rep arrays; ``media`` = (rho, lambda, mu, kappa) per cell."""

    def __init__(self, mesh, media, k, params=None):
        if not torch.cuda.is_available():
            raise RuntimeError("the HHO stage operator needs a CUDA device")
        self.mesh = hho.hho_mesh_create(mesh.xy, mesh.cell_ptr, mesh.cell_vtx, mesh.cell_domain,
                                        getattr(mesh, "vertex_rep", None))
        try:
            self.ops = hho.hho_operators_build(self.mesh, k, *media, params=params)
        except Exception:
            hho.hho_mesh_destroy(self.mesh)
            raise
        self.k = k
        self.layout = hho.hho_state_layout(self.ops)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self._work = {}

    def close(self):
        if getattr(self, "ops", None):
            hho.hho_ops_destroy(self.ops)
            self.ops = None
        if getattr(self, "mesh", None):
            hho.hho_mesh_destroy(self.mesh)
            self.mesh = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- buffers -------------------------------------------------------------------
    def empty_state(self):
        return torch.zeros(self.layout.n_state, dtype=torch.float64, device=self.dev)

    def work(self, tab):
        key = tab.s if isinstance(tab, hho.Tableau) else int(tab)
        t = tab if isinstance(tab, hho.Tableau) else hho.hho_tableau_erk(int(tab))
        n = hho.hho_work_size(self.ops, t)
        if key not in self._work or self._work[key].numel() < n:
            self._work[key] = torch.empty(n, dtype=torch.float64, device=self.dev)
        return self._work[key]

    def to_device(self, canonical, stream=None):
        c = torch.as_tensor(np.ascontiguousarray(canonical, dtype=np.float64)).to(self.dev)
        st = self.empty_state()
        hho.hho_state_pack(self.ops, c.data_ptr(), st.data_ptr(), _stream(stream))
        return st

    def to_canonical(self, state, stream=None):
        c = torch.empty(self.layout.n_canonical, dtype=torch.float64, device=self.dev)
        hho.hho_state_unpack(self.ops, state.data_ptr(), c.data_ptr(), _stream(stream))
        return c.cpu().numpy()

    # ---- operations --------------------------------------------------------------------
    def set_sources(self, xy, direction, f0, t0=None, amp=None):
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        ns = xy.shape[0]
        f0 = np.broadcast_to(np.asarray(f0, dtype=np.float64), (ns,))
        t0 = 1.0 / f0 if t0 is None else np.broadcast_to(np.asarray(t0, dtype=np.float64), (ns,))
        amp = np.ones(ns) if amp is None else np.broadcast_to(np.asarray(amp, dtype=np.float64), (ns,))
        hho.hho_sources_set(self.ops, xy, direction, f0, t0, amp)

    def set_receivers(self, xy):
        self.n_rec = len(xy)
        hho.hho_receivers_set(self.ops, xy)

    def step(self, state, s, t0, dt, nsteps, stream=None):
        tab = hho.hho_tableau_erk(s)
        hho.hho_erk_step(self.ops, tab, t0, dt, nsteps, state.data_ptr(), self.work(tab).data_ptr(), _stream(stream))

    def sdirk_step(self, state, s, t0, dt, nsteps, tol=1e-12, restart=40, max_iter=2000, stream=None,
                   preconditioner=None):
        """Implicit SDIRK steps (hho_sdirk_step); returns the GMRES operator applications.
        preconditioner: None keeps the current setting, 1 block Jacobi, 0 none."""
        if preconditioner is not None:
            hho.hho_sdirk_set_preconditioner(self.ops, preconditioner)
        tab = hho.hho_tableau_sdirk(s)
        n = hho.hho_sdirk_work_size(self.ops, tab, restart)
        key = ("sdirk", s, restart)
        if key not in self._work or self._work[key].numel() < n:
            self._work[key] = torch.empty(n, dtype=torch.float64, device=self.dev)
        return hho.hho_sdirk_step(self.ops, tab, t0, dt, nsteps, tol, restart, max_iter, state.data_ptr(),
                                  self._work[key].data_ptr(), _stream(stream))

    def apply(self, state, t=0.0, stream=None):
        rate = self.empty_state()
        hho.hho_apply(self.ops, t, state.data_ptr(), rate.data_ptr(), self.work(2).data_ptr(), _stream(stream))
        return rate

    def record(self, state, out=None, stream=None):
        if out is None:
            out = torch.empty((self.n_rec, 5), dtype=torch.float64, device=self.dev)
        hho.hho_record(self.ops, state.data_ptr(), out.data_ptr(), _stream(stream))
        return out

    def energy(self, state, stream=None):
        return hho.hho_energy(self.ops, state.data_ptr(), self.work(2).data_ptr(), _stream(stream))

    # ---- batched shots ---------------------------------------------------------------
    @staticmethod
    def _elem_dtype(precision):
        # HHO_F32X2 pairs occupy 8 bytes an element: float64 tensors serve as raw storage;
        # HHO_BF16X3 keeps FP32 state (only its products run in split BF16)
        return torch.float32 if precision in (hho.HHO_F32, hho.HHO_BF16X3) else torch.float64

    def set_launch_mode(self, mode):
        """hho.HHO_LAUNCH_STREAM, HHO_LAUNCH_GRAPH or HHO_LAUNCH_AUTO for step / batch_step / run_host."""
        hho.hho_set_launch_mode(self.ops, mode)

    def set_arithmetic(self, arith):
        """hho.HHO_F64 or hho.HHO_F32X2 for step / apply / run_host."""
        hho.hho_set_arithmetic(self.ops, arith)

    def batch_buffers(self, s, n_shots, precision=hho.HHO_F64):
        tab = hho.hho_tableau_erk(s)
        ns, nw = hho.hho_batch_sizes(self.ops, tab, n_shots, precision)
        dt = self._elem_dtype(precision)
        return (torch.zeros(ns, dtype=dt, device=self.dev), torch.empty(nw, dtype=dt, device=self.dev))

    def batch_to_device(self, canonicals, precision=hho.HHO_F64, stream=None):
        """canonicals: [n_shots, n_canonical] host array -> batched device state."""
        c = torch.as_tensor(np.ascontiguousarray(canonicals, dtype=np.float64)).to(self.dev)
        S = c.shape[0]
        dt = self._elem_dtype(precision)
        st = torch.zeros(S * self.layout.n_state, dtype=dt, device=self.dev)
        hho.hho_batch_pack(self.ops, S, precision, c.data_ptr(), st.data_ptr(), _stream(stream))
        return st

    def batch_to_canonical(self, state, n_shots, precision=hho.HHO_F64, stream=None):
        c = torch.empty((n_shots, self.layout.n_canonical), dtype=torch.float64, device=self.dev)
        hho.hho_batch_unpack(self.ops, n_shots, precision, state.data_ptr(), c.data_ptr(), _stream(stream))
        return c.cpu().numpy()

    def set_shot_sources(self, xy, direction, f0, t0=None, amp=1.0):
        hho.hho_batch_sources_set(self.ops, xy, direction, f0, 1.0 / f0 if t0 is None else t0, amp)

    def batch_step(self, state, work, n_shots, s, t0, dt, nsteps, precision=hho.HHO_F64, seismogram=None,
                   stream=None):
        tab = hho.hho_tableau_erk(s)
        hho.hho_batch_erk_step(self.ops, tab, n_shots, precision, t0, dt, nsteps, state.data_ptr(), work.data_ptr(),
                               None if seismogram is None else seismogram.data_ptr(), _stream(stream))

    def run_host(self, canonical, s, t0, dt, nsteps, stream=None):
        """End to end from a host array (updated in place)."""
        tab = hho.hho_tableau_erk(s)
        hho.hho_erk_run_host(self.ops, tab, t0, dt, nsteps, canonical, _stream(stream))
        return canonical
