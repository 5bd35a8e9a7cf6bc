"""GPU parity: the CUDA stage path (through the C ABI) against the CPU oracle.

Bar: relative L2 <= 1e-12 in FP64 over all cell DOFs in the
canonical layout, and on receiver traces.  Each test states its tolerance.
"""
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

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import solver
    return solver


def random_media(md, seed):
    rng = np.random.default_rng(seed)
    nc = md.n_cells
    rho = 1.0 + rng.random(nc)
    vp = 2.5 + rng.random(nc)
    vs = 1.0 + 0.5 * rng.random(nc)
    mu = rho * vs ** 2
    lam = rho * vp ** 2 - 2 * mu
    kap = rho * (1.0 + rng.random(nc)) ** 2
    sol = md.cell_domain == 1
    return rho, np.where(sol, lam, 0.0), np.where(sol, mu, 0.0), np.where(sol, 0.0, kap)


def cases():
    return [
        ("c1_tri_k1", synth.tri_grid(16, 16), 1, None),
        ("quad_k2", synth.quad_grid(6, 5, 0.0, 1.2, 0.0, 1.0, 0.5), 2, None),
        ("tri_k3", synth.tri_grid(5, 6, 0.0, 1.0, 0.0, 1.0, 0.5), 3, None),
        ("hanging_k2", synth.hanging_node_patch(6, 6, refine_rows=(2, 3)), 2, 7),
        ("hybrid_k3", synth.hybrid_grid(6, 6, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5), 3, 8),
        ("periodic_k2", synth.quad_grid(4, 10, 0.0, 0.4, -0.5, 0.5, y_interface=0.0, periodic_x=True), 2, None),
        ("random_media_k1", synth.quad_grid(7, 7, 0.0, 1.0, 0.0, 1.0, 0.45), 1, 9),
        # the basin section at 40 x 10 coarse cells: 4x-refined squares, 7- and
        # 9-vertex hanging-node polygons, triangles along the basin floor
        ("basin_k2", synth.basin_c5(nx=40, ny=10)["mesh"], 2, "basin"),
    ]


def media_for(md, seed):
    if seed == "basin":
        return synth.basin_c5(nx=40, ny=10)["media"]
    return synth.layered_media(md) if seed is None else random_media(md, seed)


@pytest.mark.parametrize("name,md,k,seed", cases())
def test_rate_operator_parity(lib, name, md, k, seed):
    """One application of the condensed operator M^-1(F - K_cond U) (the core
    of every stage of Eq. ex_solve) on a seeded random state."""
    media = media_for(md, seed)
    S = oracle_system(md, k, media)
    st = E.Stepper(S)
    U = synth.random_state(S.nT, 100 + k)
    ref = st.rate(U, 0.0)
    P = lib.Problem(md, media, k)
    got = P.to_canonical(P.apply(P.to_device(U)))
    err = rel(got, ref)
    print(name, "rate rel err", err)
    assert err <= TOL


@pytest.mark.parametrize("s", [2, 3, 4])
@pytest.mark.parametrize("name,md,k,seed", [cases()[1], cases()[3], cases()[4], cases()[7]])
def test_erk_steps_parity(lib, name, md, k, seed, s):
    """A few ERK(s) steps (Eq. ERK_compact) at a stable dt."""
    media = media_for(md, seed)
    S = oracle_system(md, k, media)
    st = E.Stepper(S)
    U = synth.random_state(S.nT, 7)
    dt = 0.02 / (k * k) * (0.4 if name == "basin_k2" else 1.0)   # basin: h/c_max is 0.4x the unit meshes'
    ref = st.step(U, 0.0, dt, "erk%d" % s, 5)
    P = lib.Problem(md, media, k)
    x = P.to_device(U)
    P.step(x, s, 0.0, dt, 5)
    err = rel(P.to_canonical(x), ref)
    print(name, s, "erk rel err", err)
    assert err <= TOL


def test_academic_c1_full_run(lib):
    """The academic workload: 512 triangles, k = 1, ERK4, 200 CFL-limited
    steps, Ricker point force (f0 = 10, e_y) at a seeded solid point, 8
    interface receivers recorded every step.  State and traces <= 1e-12."""
    w = synth.academic_c1()
    md, media, k = w["mesh"], w["media"], w["k"]
    dt = json.load(open(os.path.join(ROOT, "tests/golden/c1_dt.json")))["dt"]
    S = oracle_system(md, k, media)
    b, _ = S.point_load(*w["source"], direction=(0.0, 1.0))
    f0 = w["f0"]
    st = E.Stepper(S, lambda t: synth.ricker(t, f0) * b)
    P = lib.Problem(md, media, k)
    P.set_sources([w["source"]], [(0.0, 1.0)], f0)
    P.set_receivers(w["receivers"])
    U = np.zeros(S.nT)
    x = P.to_device(U)
    tr_ref, tr_gpu = [], []
    for n in range(w["nsteps"]):
        U = st.step(U, n * dt, dt, "erk4")
        P.step(x, 4, n * dt, dt, 1)
        tr_ref.append(D.sensors(st, U, w["receivers"]))
        tr_gpu.append(P.record(x).cpu().numpy())
    tr_ref = np.array(tr_ref)
    tr_gpu = np.array(tr_gpu)
    e_state = rel(P.to_canonical(x), U)
    e_tr = rel(tr_gpu[:, :, :3], tr_ref[:, :, :3])
    print("C1 state rel err", e_state, "receiver rel err", e_tr, "|U|", np.linalg.norm(U))
    assert np.linalg.norm(U) > 0
    assert e_state <= TOL
    assert e_tr <= TOL


def test_energy_and_receivers_parity(lib):
    md = synth.quad_grid(8, 6, 0.0, 1.0, 0.0, 1.0, 0.5)
    media = random_media(md, 3)
    S = oracle_system(md, 2, media)
    st = E.Stepper(S)
    U = synth.random_state(S.nT, 5)
    P = lib.Problem(md, media, 2)
    x = P.to_device(U)
    assert abs(P.energy(x) - D.energy(S, U)) / D.energy(S, U) <= 1e-13
    pts = [(0.31, 0.2), (0.77, 0.41), (0.52, 0.5), (0.18, 0.5), (0.9, 0.8), (0.05, 0.66)]
    P.set_receivers(pts)
    got = P.record(x).cpu().numpy()
    ref = D.sensors(st, U, pts)
    assert rel(got, ref) <= TOL


def test_pack_roundtrip_and_host_entry_point(lib):
    md = synth.hybrid_grid(5, 5, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    media = synth.layered_media(md)
    P = lib.Problem(md, media, 2)
    U = synth.random_state(P.layout.n_canonical, 1)
    x = P.to_device(U)
    assert np.array_equal(P.to_canonical(x), U)
    P.step(x, 4, 0.0, 0.003, 3)
    h = U.copy()
    P.run_host(h, 4, 0.0, 0.003, 3)
    assert np.array_equal(h, P.to_canonical(x))


@pytest.mark.parametrize("arith", ["f64", "f32x2"])
@pytest.mark.parametrize("k", [1, 3])
def test_host_entry_point_on_pinned_buffer(lib, k, arith):
    """hho_erk_run_host on a pinned host buffer takes the mapped path (the
    pack kernels read and write the host buffer directly): bit-identical to
    packing on the device, stepping and unpacking."""
    from paper_2505_15771_gb300 import hho
    md = synth.hybrid_grid(9, 7, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    media = synth.layered_media(md)
    P = lib.Problem(md, media, k)
    P.set_arithmetic(hho.HHO_F64 if arith == "f64" else hho.HHO_F32X2)
    P.set_sources([(0.37, 0.21)], [(0.6, 0.8)], 10.0)
    U = synth.random_state(P.layout.n_canonical, 7)
    x = P.to_device(U)
    P.step(x, 4, 0.01, 0.002, 3)
    ref = P.to_canonical(x)
    h = torch.from_numpy(U.copy()).pin_memory()
    for _ in range(2):   # the second call reuses the buffers of the first
        h.copy_(torch.from_numpy(U))
        P.run_host(h.numpy(), 4, 0.01, 0.002, 3)
        assert np.array_equal(h.numpy(), ref)


def test_energy_decays_without_source(lib):
    """Sec. 5.1: no source, Dirichlet walls, dt below the stability limit
    (tests/golden/c1_dt.json): the discrete energy never increases."""
    w = synth.academic_c1()
    dt = json.load(open(os.path.join(ROOT, "tests/golden/c1_dt.json")))["dt"]
    P = lib.Problem(w["mesh"], w["media"], 1)
    x = P.to_device(synth.random_state(P.layout.n_canonical, 2))
    e0 = P.energy(x)
    for _ in range(20):
        P.step(x, 4, 0.0, dt, 10)
        e1 = P.energy(x)
        assert e1 <= e0 * (1 + 1e-13)
        e0 = e1


# ---------------------------------------------------------------- full-size sampled parity

def _edge_neighbours(md):
    edges = {}
    nbr = [[] for _ in range(md.n_cells)]
    for c in range(md.n_cells):
        vs = md.cell_vtx[md.cell_ptr[c]:md.cell_ptr[c + 1]]
        for j in range(len(vs)):
            key = tuple(sorted((int(vs[j]), int(vs[(j + 1) % len(vs)]))))
            if key in edges:
                o = edges.pop(key)
                nbr[c].append(o)
                nbr[o].append(c)
            else:
                edges[key] = c
    return nbr


def _patch(md, nbr, centre, radius):
    cells = {centre}
    front = {centre}
    for _ in range(radius):
        front = {o for c in front for o in nbr[c]} - cells
        cells |= front
    cells = sorted(cells)
    sub_vtx = []
    ptr = [0]
    for c in cells:
        vs = md.cell_vtx[md.cell_ptr[c]:md.cell_ptr[c + 1]]
        sub_vtx.extend(int(v) for v in vs)
        ptr.append(len(sub_vtx))
    used = sorted(set(sub_vtx))
    remap = {v: i for i, v in enumerate(used)}
    sub = synth.MeshData(xy=md.xy[used], cell_ptr=np.array(ptr), cell_vtx=np.array([remap[v] for v in sub_vtx]),
                         cell_domain=md.cell_domain[cells].copy())
    return cells, sub


@pytest.mark.parametrize("k,steps", [(2, 0), (3, 0), (2, 1)])
def test_full_size_bilayer_sampled(lib, k, steps):
    """The 1024 x 512 bilayer (random-field solid under water) at full size, in
    the launch configuration the benchmark times: the GPU result (rate for
    steps = 0, one ERK4 step otherwise) on all 524,288 cells, checked on 24
    seeded sample cells against the oracle run on the patch of cells each
    sample depends on (1 ring for the rate, 4 rings for one ERK4 step)."""
    w = synth.bilayer_c2(k=k)
    md, media = w["mesh"], w["media"]
    P = lib.Problem(md, media, k)
    n = (k + 1) * (k + 2) // 2
    sizes = np.where(md.cell_domain == 0, 3 * n, 5 * n)
    off = np.concatenate([[0], np.cumsum(sizes)])
    U = synth.random_state(int(off[-1]), 21)
    x = P.to_device(U)
    dt = 0.9 * 0.1 * (1.0 / 512) / 3.6 / k
    if steps == 0:
        got = P.to_canonical(P.apply(x))
    else:
        P.step(x, 4, 0.0, dt, steps)
        got = P.to_canonical(x)
    nbr = _edge_neighbours(md)
    rng = np.random.default_rng(5)
    iface = [c for c in range(md.n_cells) if any(md.cell_domain[o] != md.cell_domain[c] for o in nbr[c])]
    samples = list(rng.choice(md.n_cells, 20, replace=False)) + list(rng.choice(iface, 4, replace=False))
    radius = 1 if steps == 0 else 4
    worst = 0.0
    for c in samples:
        cells, sub = _patch(md, nbr, int(c), radius)
        sub_media = tuple(np.asarray(a)[cells] for a in media)
        S = oracle_system(sub, k, sub_media)
        st = E.Stepper(S)
        Us = np.concatenate([U[off[o]:off[o + 1]] for o in cells])
        ref_all = st.rate(Us, 0.0) if steps == 0 else st.step(Us, 0.0, dt, "erk4", steps)
        i = cells.index(int(c))
        ref = ref_all[S.cell_off[i]:S.cell_off[i + 1]]
        e = rel(got[off[c]:off[c + 1]], ref)
        worst = max(worst, e)
    print("full-size k=%d steps=%d worst sampled rel err %.3e" % (k, steps, worst))
    assert worst <= TOL
