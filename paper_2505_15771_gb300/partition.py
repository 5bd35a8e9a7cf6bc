"""Mesh partition into subdomains with one halo exchange of face traces per ERK stage.

The stage of Eq. ex_solve couples a cell to its neighbours only through the
face solve, which needs the traces w that each neighbour publishes on the
shared face.  So a subdomain holds its owned cells plus one layer of ghost
cells (the other cells of its owned cells' faces), and before every stage
each subdomain receives, for every face between one of its owned cells and a
ghost, the traces that the ghost's owner published there.  Its owned cells
then compute exactly what they compute in the undivided mesh: the sub-mesh
keeps the parent's class matrices (hho_mesh_submesh) and a cell's stage
arithmetic does not depend on where it sits in the layout.  Ghost cells are
stepped too (their results are discarded): their outer faces are boundary
faces of the sub-mesh.

Pieces:
* ``strip_partition``: cells to parts by x-strips of equal cell count.
* ``HaloPlan``: for every part, its cells (owned + ghosts, in increasing
  parent id) and, for every other part, the (cell, local face) entries it
  sends and receives.  Both sides derive the same ordered lists from the
  parent mesh's tables, so a send buffer and the matching receive buffer
  line up entry by entry.  Host only (mesh tables, no device).
* ``Subdomain`` / ``run_partitioned``: the GPU side (sub-mesh, operators,
  trace offsets of the halo entries, gather / exchange / scatter around
  hho_erk_stage).
* ``exchange_dist``: point-to-point exchange of the packed buffers through
  torch.distributed (NCCL on GPUs, gloo on CPUs), each rank receiving into its
  own buffers; ``exchange_local`` does the same between subdomains of one
  process.
"""
from __future__ import annotations

import numpy as np

from . import hho


def strip_partition(centroid_x, n_parts):
    """Part of every cell: x-strips with about equal cell counts.  Strip
    bounds are quantiles of the cell centroids' x, so cells with the same x
    (a grid column) share a part."""
    x = np.asarray(centroid_x, dtype=np.float64)
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    bounds = np.quantile(x, np.arange(1, n_parts) / n_parts)
    return np.searchsorted(bounds, x, side="right").astype(np.int32)


class HaloPlan:
    """Cells and halo lists of every part of a partition of a mesh.

    ``tables``: hho.hho_mesh_tables of the parent mesh; ``cell_part``: part of
    every parent cell.  Per part p:
      cells[p]      parent ids of p's sub-mesh cells (owned and ghosts, increasing)
      owned[p]      bool mask over cells[p]
      send[p][q]    (parent cell, local face) entries p publishes for q, sorted
      recv[p][q]    the entries p receives from q (= send[q][p])
    """

    def __init__(self, tables, cell_part, n_parts):
        part = np.asarray(cell_part, dtype=np.int64)
        fc = np.asarray(tables["face_cells"])
        ptr = np.asarray(tables["cell_faces_ptr"])
        cf = np.asarray(tables["cell_faces"])
        nc = len(ptr) - 1
        if len(part) != nc or part.min() < 0 or part.max() >= n_parts:
            raise ValueError("cell_part must give a part in [0, n_parts) for every cell")
        self.n_parts = n_parts
        self.part = part
        # local face index of every (face, side): position of the face in the cell's list
        local = {}
        for c in range(nc):
            for j, F in enumerate(cf[ptr[c]:ptr[c + 1]]):
                local[(int(F), c)] = j
        pairs = {}
        for F in range(len(fc)):
            a, b = int(fc[F, 0]), int(fc[F, 1])
            if b < 0 or part[a] == part[b]:
                continue
            pairs.setdefault((int(part[a]), int(part[b])), []).append((a, local[(F, a)]))
            pairs.setdefault((int(part[b]), int(part[a])), []).append((b, local[(F, b)]))
        self.send = [dict() for _ in range(n_parts)]
        self.recv = [dict() for _ in range(n_parts)]
        ghosts = [set() for _ in range(n_parts)]
        for (p, q), lst in pairs.items():
            lst = sorted(set(lst))
            self.send[p][q] = lst
            self.recv[q][p] = lst
            ghosts[q].update(c for c, _ in lst)
        self.cells, self.owned = [], []
        for p in range(n_parts):
            own = np.flatnonzero(part == p)
            cells = np.union1d(own, np.fromiter(ghosts[p], dtype=np.int64, count=len(ghosts[p])))
            self.cells.append(cells)
            self.owned.append(part[cells] == p)

    def local_index(self, p):
        """Parent id -> index in p's sub-mesh (dict)."""
        return {int(c): i for i, c in enumerate(self.cells[p])}

    def offsets(self, p, entries, trace_offsets):
        """Flat trace-buffer offsets of the entries (parent cell, local face) of
        part p, in entry order: ``trace_offsets(local_cells, faces)`` gives the
        [n, 2f] offsets (-1 padded) in p's layout."""
        if not entries:
            return np.zeros(0, dtype=np.int64)
        g2l = self.local_index(p)
        cells = np.array([g2l[c] for c, _ in entries], dtype=np.int64)
        faces = np.array([j for _, j in entries], dtype=np.int32)
        o = np.asarray(trace_offsets(cells, faces))
        return o[o >= 0].astype(np.int64)


def exchange_local(send_bufs, recv_bufs):
    """Subdomains of one process: recv_bufs[p][q] <- send_bufs[q][p] (device copies)."""
    for p, row in enumerate(recv_bufs):
        for q, buf in row.items():
            buf.copy_(send_bufs[q][p])


def exchange_dist(send, recv, dist):
    """This rank's part of the exchange: send[q] goes to rank q, recv[q] is
    filled from rank q (each rank receives into its own buffers).  One batch
    of point-to-point operations, so the order of calls cannot deadlock."""
    ops = [dist.P2POp(dist.irecv, t, q) for q, t in sorted(recv.items())]
    ops += [dist.P2POp(dist.isend, t, q) for q, t in sorted(send.items())]
    if not ops:
        return
    for r in dist.batch_isend_irecv(ops):
        r.wait()


class Subdomain:
    """One part on the current GPU: sub-mesh, operators and packed halo buffers."""

    def __init__(self, parent_mesh, plan, p, k, media, params=None, tab=None):
        import torch
        self.p = p
        self.plan = plan
        cells = plan.cells[p]
        self.mesh = hho.hho_mesh_submesh(parent_mesh, cells)
        try:
            self.ops = hho.hho_operators_build(self.mesh, k, *[np.asarray(m)[cells] for m in media], params=params)
        except Exception:
            hho.hho_mesh_destroy(self.mesh)
            raise
        self.tab = tab if tab is not None else hho.hho_tableau_erk(4)
        self.layout = hho.hho_state_layout(self.ops)
        self.dev = torch.device("cuda", torch.cuda.current_device())
        self.work = torch.empty(hho.hho_work_size(self.ops, self.tab), dtype=torch.float64, device=self.dev)
        self.tr_off = [hho.hho_trace_buffer_offset(self.ops, self.tab, w) for w in (0, 1)]
        f = k + 1

        def offs(local_cells, faces):
            return hho.hho_trace_offsets(self.ops, f, local_cells, faces)

        def dev_idx(a):
            return torch.as_tensor(a, dtype=torch.int64).to(self.dev)
        self.send_idx = {q: dev_idx(plan.offsets(p, e, offs)) for q, e in plan.send[p].items()}
        self.recv_idx = {q: dev_idx(plan.offsets(p, e, offs)) for q, e in plan.recv[p].items()}
        self.send_buf = {q: torch.empty(len(i), dtype=torch.float64, device=self.dev) for q, i in self.send_idx.items()}
        self.recv_buf = {q: torch.empty(len(i), dtype=torch.float64, device=self.dev) for q, i in self.recv_idx.items()}

    def set_sources(self, xy, direction, f0, t0, amp):
        """hho_sources_set with the sources whose point lies in this sub-mesh
        (the lowest-index containing cell, as in the parent: the sub-mesh keeps
        the parent's cell order).  A source in a ghost cell only changes that
        ghost's discarded update; its owner applies it."""
        xy = np.asarray(xy, dtype=np.float64).reshape(-1, 2)
        keep = hho.hho_locate_points(self.ops, xy) >= 0
        sel = lambda a: np.asarray(a, dtype=np.float64).reshape(len(xy), -1)[keep]
        hho.hho_sources_set(self.ops, xy[keep], sel(direction), sel(f0).ravel(), sel(t0).ravel(), sel(amp).ravel())

    def trace_ptr(self, which):
        return self.work.data_ptr() + 8 * self.tr_off[which]

    def pack(self, which, stream):
        for q, idx in self.send_idx.items():
            hho.hho_halo_gather(self.trace_ptr(which), idx.data_ptr(), idx.numel(), self.send_buf[q].data_ptr(),
                                stream)

    def unpack(self, which, stream):
        for q, idx in self.recv_idx.items():
            hho.hho_halo_scatter(self.recv_buf[q].data_ptr(), idx.data_ptr(), idx.numel(), self.trace_ptr(which),
                                 stream)

    def close(self):
        if getattr(self, "ops", None):
            hho.hho_ops_destroy(self.ops)
            self.ops = None
        if getattr(self, "mesh", None):
            hho.hho_mesh_destroy(self.mesh)
            self.mesh = None


def run_partitioned(subs, states, t0, dt, nsteps, exchange, stream):
    """nsteps ERK steps of every subdomain in ``subs`` (its state in
    ``states``, device layout), exchanging the halo traces after the trace
    publication and after every stage: pack, exchange(subs), unpack.
    ``exchange`` moves the packed buffers (exchange_local over all subdomains
    of the process, or exchange_dist for one subdomain per rank)."""
    tab = subs[0].tab
    s = tab.s

    def halo(which):
        for d in subs:
            d.pack(which, stream)
        exchange(subs)
        for d in subs:
            d.unpack(which, stream)
    for d, x in zip(subs, states):
        hho.hho_erk_traces(d.ops, tab, x.data_ptr(), d.work.data_ptr(), stream)
    halo(0)
    for n in range(nsteps):
        tn = t0 + n * dt
        for j in range(s):
            for d, x in zip(subs, states):
                hho.hho_erk_stage(d.ops, tab, n, j, tn, dt, x.data_ptr(), d.work.data_ptr(), stream)
            halo((n * s + j + 1) % 2)
