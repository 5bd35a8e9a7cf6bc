"""Mesh partition and halo exchange (host logic), on the CPU.

The stage kernels need a GPU; what is checked here is everything around
them: the partition, the ghost layers, the per-pair halo lists, and the
exchange of packed trace buffers between gloo ranks (world size 2 and 4),
on emulated trace buffers whose entries carry their (cell, face, component)
so that a misrouted or missing value is seen.  The GPU test
(test_gpu_partition.py) runs the same plan through the stage kernels and
compares with the undivided mesh bit for bit."""
import os
import socket

import numpy as np
import pytest

import synth
from tests.libutil import ensure_built

torch = pytest.importorskip("torch")

MESHES = {
    "bilayer_quads": lambda: synth.quad_grid(8, 4, 0.0, 2.0, 0.0, 1.0, 0.5),
    "triangles": lambda: synth.tri_grid(6, 5),
    "hybrid": lambda: synth.hybrid_grid(6, 6, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5),
    "hanging_nodes": lambda: synth.hanging_node_patch(6, 6, refine_rows=(2, 3)),
    "periodic_strip": lambda: synth.quad_grid(6, 4, 0.0, 0.6, -0.5, 0.5, y_interface=0.0, periodic_x=True),
}
F = 3   # face polynomial size (k = 2)


def plan_for(name, n_parts):
    hho = ensure_built()
    from paper_2505_15771_gb300 import partition as PT
    md = MESHES[name]()
    mesh = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain, md.vertex_rep)
    try:
        tables = hho.hho_mesh_tables(mesh)
    finally:
        hho.hho_mesh_destroy(mesh)
    part = PT.strip_partition(md.centroids_approx()[:, 0], n_parts)
    return md, tables, PT.HaloPlan(tables, part, n_parts)


def fake_offsets(md, cells_of_part):
    """An emulated trace layout for one part: (local cell, face, component) ->
    (cell * 16 + face) * 2F + component; F components in fluid cells, 2F in
    solid ones (the layout the library's offsets have, up to the slot order)."""
    dom = md.cell_domain

    def offs(local_cells, faces):
        out = np.full((len(local_cells), 2 * F), -1, np.int64)
        for i, (c, j) in enumerate(zip(local_cells, faces)):
            m = F if dom[cells_of_part[c]] == 0 else 2 * F
            out[i, :m] = (c * 16 + j) * 2 * F + np.arange(m)
        return out
    return offs


def value(c, j, l):
    return 1000.0 * c + 10.0 * j + l


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("n_parts", [2, 3, 4])
def test_halo_plan_is_consistent(name, n_parts):
    """Every cell is owned once; a part's cells are its owned cells plus the
    ghosts its owned cells' faces reach; every face between two parts appears
    on both sides, once each way, with the same ordered lists."""
    md, tables, plan = plan_for(name, n_parts)
    nc = md.n_cells
    owned_all = np.concatenate([plan.cells[p][plan.owned[p]] for p in range(n_parts)])
    assert np.array_equal(np.sort(owned_all), np.arange(nc))
    fc = tables["face_cells"]
    cut = 0
    for F_, (a, b) in enumerate(fc):
        if b < 0:
            continue
        pa, pb = plan.part[a], plan.part[b]
        for p in (pa, pb):
            assert a in plan.cells[p] and b in plan.cells[p]
        if pa != pb:
            cut += 1
            assert any(c == a for c, _ in plan.send[pa][pb]) and any(c == b for c, _ in plan.send[pb][pa])
    for p in range(n_parts):
        for q, lst in plan.send[p].items():
            assert plan.recv[q][p] == lst
            assert all(plan.part[c] == p for c, _ in lst)
        ghosts = set(plan.cells[p][~plan.owned[p]].tolist())
        assert ghosts == {c for q in plan.recv[p] for c, _ in plan.recv[p][q]}
    assert sum(len(v) for p in range(n_parts) for v in plan.send[p].values()) == 2 * cut
    if n_parts > 1:
        assert cut > 0


def _rank_main(rank, world, port, name, result_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2505_15771_gb300 import partition as PT
        md, tables, plan = plan_for(name, world)
        cells = plan.cells[rank]
        offs = fake_offsets(md, cells)
        buf = np.full(len(cells) * 16 * 2 * F, np.nan)
        g2l = plan.local_index(rank)
        for c in cells[plan.owned[rank]]:   # owned cells publish their traces on every face
            m = F if md.cell_domain[c] == 0 else 2 * F
            for j in range(16):
                for l in range(m):
                    buf[(g2l[int(c)] * 16 + j) * 2 * F + l] = value(int(c), j, l)
        send_idx = {q: plan.offsets(rank, e, offs) for q, e in plan.send[rank].items()}
        recv_idx = {q: plan.offsets(rank, e, offs) for q, e in plan.recv[rank].items()}
        send = {q: torch.as_tensor(buf[i]) for q, i in send_idx.items()}
        recv = {q: torch.empty(len(i), dtype=torch.float64) for q, i in recv_idx.items()}
        PT.exchange_dist(send, recv, dist)
        for q, i in recv_idx.items():
            buf[i] = recv[q].numpy()
        # every ghost entry its owned neighbours read now holds the owner's value
        bad = 0
        n_checked = 0
        for q, lst in plan.recv[rank].items():
            for c, j in lst:
                m = F if md.cell_domain[c] == 0 else 2 * F
                for l in range(m):
                    n_checked += 1
                    bad += buf[(g2l[c] * 16 + j) * 2 * F + l] != value(c, j, l)
        np.save(os.path.join(result_dir, "r%d.npy" % rank), np.array([bad, n_checked, plan.owned[rank].sum()]))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,name", [(2, "bilayer_quads"), (2, "periodic_strip"), (4, "hybrid"),
                                        (4, "hanging_nodes")])
def test_halo_exchange_over_gloo_ranks(tmp_path, world, name):
    """One process per part (gloo, 127.0.0.1): each rank packs the traces its
    owned cells publish on cut faces, exchange_dist moves them point to point
    into the peers' own buffers, and every ghost entry ends up with the
    owner's value; the ranks' owned cells add up to the mesh."""
    ensure_built()
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(world, _free_port(), name, str(tmp_path)), nprocs=world, join=True)
    res = [np.load(tmp_path / ("r%d.npy" % r)) for r in range(world)]
    assert all(r[0] == 0 for r in res), res
    assert all(r[1] > 0 for r in res)
    assert sum(int(r[2]) for r in res) == MESHES[name]().n_cells
