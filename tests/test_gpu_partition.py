"""Partitioned stepping on the GPU: x-strip subdomains (owned cells + one
ghost layer, hho_mesh_submesh), one halo exchange of the published face
traces after every stage (hho_halo_gather / hho_halo_scatter around
hho_erk_stage), against hho_erk_step on the undivided mesh in stream launch
mode.  The owned cells' states must be bit-identical.

All subdomains live in this one process and GPU: their stage kernels run one
after the other and the exchange is a device copy between them, so no kernel
waits on another (the multi-process transport is exercised on CPU ranks in
test_partition_cpu.py)."""
import numpy as np
import pytest

import synth
from tests.libutil import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, partition
    return hho, partition


def canon_offsets(md, k):
    n = (k + 1) * (k + 2) // 2
    size = np.where(md.cell_domain == 0, 3 * n, 5 * n)
    return np.concatenate([[0], np.cumsum(size)]), size


CASES = [
    ("bilayer_quads", lambda: synth.quad_grid(12, 6, 0.0, 2.0, 0.0, 1.0, 0.5), 2, 4, 3),
    ("triangles_k3", lambda: synth.tri_grid(8, 6), 3, 4, 2),
    ("hybrid_erk3", lambda: synth.hybrid_grid(8, 8, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5), 2, 3, 4),
    ("hanging_nodes", lambda: synth.hanging_node_patch(8, 6, refine_rows=(2, 3)), 1, 4, 3),
    ("periodic_strip", lambda: synth.quad_grid(8, 6, 0.0, 0.8, -0.5, 0.5, y_interface=0.0, periodic_x=True), 2, 4, 2),
]


@pytest.mark.parametrize("name,make,k,s,n_parts", CASES, ids=[c[0] for c in CASES])
def test_partitioned_steps_bit_identical(lib, name, make, k, s, n_parts):
    hho, PT = lib
    md = make()
    media = synth.layered_media(md)
    rng = np.random.default_rng(17)
    nc = md.n_cells
    media = tuple(m * (1.0 + 0.1 * rng.random(nc)) for m in media)   # per-cell media
    src = (0.31, 0.27)
    tab = hho.hho_tableau_erk(s)
    nsteps, dt = 12, 0.002
    stream = torch.cuda.current_stream().cuda_stream
    parent = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain, md.vertex_rep)
    subs = []
    try:
        # the undivided mesh, stream launches
        ops = hho.hho_operators_build(parent, k, *media)
        hho.hho_set_launch_mode(ops, hho.HHO_LAUNCH_STREAM)
        hho.hho_sources_set(ops, [src], [(0.0, 1.0)], [8.0], [0.125], [1.0])
        lay = hho.hho_state_layout(ops)
        U0 = synth.random_state(lay.n_canonical, 5)
        c0 = torch.as_tensor(U0).cuda()
        x = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
        hho.hho_state_pack(ops, c0.data_ptr(), x.data_ptr(), stream)
        work = torch.empty(hho.hho_work_size(ops, tab), dtype=torch.float64, device="cuda")
        hho.hho_erk_step(ops, tab, 0.0, dt, nsteps, x.data_ptr(), work.data_ptr(), stream)
        ref = torch.empty(lay.n_canonical, dtype=torch.float64, device="cuda")
        hho.hho_state_unpack(ops, x.data_ptr(), ref.data_ptr(), stream)
        ref = ref.cpu().numpy()
        hho.hho_ops_destroy(ops)

        # the partition
        tables = hho.hho_mesh_tables(parent)
        part = PT.strip_partition(md.centroids_approx()[:, 0], n_parts)
        plan = PT.HaloPlan(tables, part, n_parts)
        off, size = canon_offsets(md, k)
        states = []
        for p in range(n_parts):
            d = PT.Subdomain(parent, plan, p, k, media, tab=tab)
            subs.append(d)
            d.set_sources([src], [(0.0, 1.0)], [8.0], [0.125], [1.0])
            cells = plan.cells[p]
            loc = np.concatenate([U0[off[c]:off[c] + size[c]] for c in cells])
            cl = torch.as_tensor(loc).cuda()
            xs = torch.zeros(d.layout.n_state, dtype=torch.float64, device="cuda")
            hho.hho_state_pack(d.ops, cl.data_ptr(), xs.data_ptr(), stream)
            states.append(xs)
        PT.run_partitioned(subs, states, 0.0, dt, nsteps,
                           lambda ss: PT.exchange_local([d.send_buf for d in ss], [d.recv_buf for d in ss]), stream)
        got = np.full_like(ref, np.nan)
        for p, d in enumerate(subs):
            cl = torch.empty(d.layout.n_canonical, dtype=torch.float64, device="cuda")
            hho.hho_state_unpack(d.ops, states[p].data_ptr(), cl.data_ptr(), stream)
            cl = cl.cpu().numpy()
            lo = np.concatenate([[0], np.cumsum(size[plan.cells[p]])])
            for i, c in enumerate(plan.cells[p]):
                if plan.owned[p][i]:
                    got[off[c]:off[c] + size[c]] = cl[lo[i]:lo[i + 1]]
    finally:
        for d in subs:
            d.close()
        hho.hho_mesh_destroy(parent)
    assert not np.isnan(got).any()
    n_halo = sum(len(v) for p in range(n_parts) for v in plan.send[p].values())
    print("%s: %d parts, %d halo entries per exchange, max |diff| %.3e"
          % (name, n_parts, n_halo, np.abs(got - ref).max()))
    assert n_halo > 0
    assert np.array_equal(got, ref)
