"""CPU checks of libhho: symbols, host-side mesh tables (bit-exact against the
oracle's implementation of the same conventions), argument validation.
No compute call needs a GPU here."""
import re

import numpy as np
import pytest

import synth
from oracle import erk as E
from oracle import mesh as M
from tests.libutil import ROOT, ensure_built


@pytest.fixture(scope="module")
def hho():
    return ensure_built()


def test_library_exports_every_header_symbol(hho):
    src = open(ROOT + "/include/hho.h").read()
    declared = sorted(set(re.findall(r"\b(hho_[a-z_0-9]+)\s*\(", src)))
    assert declared, "no declarations found"
    lib = hho.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(declared) == sorted(hho.EXPORTED)


def _meshes():
    a = synth.tri_grid(16, 16)
    b = synth.quad_grid(12, 7, 0.0, 2.0, 0.0, 1.0, 0.5)
    c = synth.hybrid_grid(10, 10, 0.0, 2.0, 0.0, 1.0, 0.7, 0.5)
    d = synth.hanging_node_patch(6, 6, refine_rows=(2, 3))
    e = synth.quad_grid(5, 12, 0.0, 0.5, -1.0, 1.0, y_interface=0.0, periodic_x=True)
    f = synth.tri_grid(7, 9, 0.3, 1.7, -0.2, 0.9, y_interface=0.33)
    return [("tri", a), ("quad", b), ("hybrid", c), ("hanging", d), ("periodic", e), ("tri_offset", f)]


@pytest.mark.parametrize("name,md", _meshes())
def test_tables_bit_exact_against_oracle(hho, name, md):
    lm = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain, md.vertex_rep)
    try:
        t = hho.hho_mesh_tables(lm)
        info = hho.hho_mesh_query(lm)
    finally:
        hho.hho_mesh_destroy(lm)
    om = M.build_mesh(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain, md.vertex_rep)
    o = M.tables(om)
    for key in ("face_cells", "cell_faces_ptr", "cell_faces", "face_type", "face_colour", "cell_class"):
        assert np.array_equal(np.asarray(t[key], dtype=np.int64), np.asarray(o[key], dtype=np.int64)), key
    assert info.n_faces == om.n_faces and info.n_classes == om.cell_class.max() + 1
    assert list(info.n_faces_by_type) == [int(np.sum(om.face_type == i)) for i in range(5)]


def _expect(hho, code, fn, *args):
    with pytest.raises(hho.HHOError) as ei:
        fn(*args)
    assert ei.value.code == code, str(ei.value)


def test_mesh_errors(hho):
    xy = np.array([[0, 0], [1, 0], [1, 1], [0, 1], [2, 0], [2, 1]], dtype=float)
    # clockwise cell
    _expect(hho, hho.HHO_EMESH, hho.hho_mesh_create, xy, [0, 4], [0, 3, 2, 1], [0])
    # two vertices only
    _expect(hho, hho.HHO_EMESH, hho.hho_mesh_create, xy, [0, 2], [0, 1], [0])
    # vertex id out of range
    _expect(hho, hho.HHO_EINVAL, hho.hho_mesh_create, xy, [0, 3], [0, 1, 9], [0])
    # bad domain tag
    _expect(hho, hho.HHO_EINVAL, hho.hho_mesh_create, xy, [0, 4], [0, 1, 2, 3], [2])
    # an edge shared by three cells: (1,2) used by three triangles
    xy2 = np.array([[1, 0], [1, 1], [0, 0.5], [2, 0.5], [2, 0.6]], dtype=float)
    _expect(hho, hho.HHO_EMESH, hho.hho_mesh_create, xy2, [0, 3, 6, 9], [0, 1, 2, 1, 0, 3, 1, 0, 4], [0, 0, 0])


def test_operator_argument_errors(hho):
    md = synth.quad_grid(2, 2)
    lm = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
    rho, lam, mu, kap = synth.layered_media(md)
    try:
        _expect(hho, hho.HHO_EDEGREE, hho.hho_operators_build, lm, 0, rho, lam, mu, kap)
        _expect(hho, hho.HHO_EDEGREE, hho.hho_operators_build, lm, 4, rho, lam, mu, kap)
        bad = rho.copy(); bad[0] = -1.0
        _expect(hho, hho.HHO_EMATERIAL, hho.hho_operators_build, lm, 1, bad, lam, mu, kap)
        solid = np.where(md.cell_domain == 1)[0][0]
        badmu = mu.copy(); badmu[solid] = 0.0
        _expect(hho, hho.HHO_EMATERIAL, hho.hho_operators_build, lm, 1, rho, lam, badmu, kap)
        fluid = np.where(md.cell_domain == 0)[0][0]
        badk = kap.copy(); badk[fluid] = 0.0
        _expect(hho, hho.HHO_EMATERIAL, hho.hho_operators_build, lm, 2, rho, lam, mu, badk)
    finally:
        hho.hho_mesh_destroy(lm)


@pytest.mark.parametrize("s", [2, 3, 4])
def test_tableaux_match_oracle(hho, s):
    t = hho.hho_tableau_erk(s)
    Aext, b, c = E.tableau("erk%d" % s)
    for i in range(s):
        for j in range(s):
            assert t.a[i][j] == Aext[i, j]
        assert t.b[i] == b[i] and t.c[i] == c[i]
    _expect(hho, hho.HHO_EINVAL, hho.hho_tableau_erk, 5)


def test_tuning_tables_round_trip():
    """The tuner reads the stage_tuning.h tables the stage kernels compile
    against, and rewriting them with one entry changed touches that entry
    only."""
    from paper_2505_15771_gb300 import tune
    text = open(tune.HEADER).read()
    tables = tune.read_tables(text)
    assert tune.write_tables(text, tables) == text
    for arith in ("f64", "f32", "f2x"):
        t = tables[arith]
        assert all(len(t[f]) == 3 for f in tune.FIELDS)
        assert all(m in (2, 3, 4, 5, 6, 8, 10, 12) for m in t["min_blocks"])
        assert all(a in (0, 1) for a in t["acc_smem"])
        assert all(0 <= p < 64 for p in t["prefetch"])
        assert all(r in (0, 1) for r in t["rect_loop"])
    new = tune.with_entry(tables, "f2x", 2, {"min_blocks": 6, "acc_smem": 0, "prefetch": 48,
                                             "rect_loop": 1 - tables["f2x"]["rect_loop"][1]})
    back = tune.read_tables(tune.write_tables(text, new))
    assert back["f2x"]["min_blocks"][1] == 6 and back["f2x"]["prefetch"][1] == 48
    assert back["f2x"]["rect_loop"][1] == 1 - tables["f2x"]["rect_loop"][1]
    assert back["f64"] == tables["f64"] and back["f32"] == tables["f32"]
    assert back["f2x"]["min_blocks"][0] == tables["f2x"]["min_blocks"][0]


def test_tuner_candidate_build_is_a_complete_library(hho, tmp_path):
    """A tuner candidate (stage.cu rebuilt against a changed tuning table and
    linked with the in-tree objects) loads and exports every entry point of
    include/hho.h."""
    import ctypes
    from paper_2505_15771_gb300 import build, tune
    text = open(tune.HEADER).read()
    t = tune.with_entry(tune.read_tables(text), "f2x", 2, {"min_blocks": 6, "acc_smem": 0, "prefetch": 48})
    path = build.build_stage_variant(tune.write_tables(text, t), str(tmp_path))
    src = open(ROOT + "/include/hho.h").read()
    declared = sorted(set(re.findall(r"\b(hho_[a-z_0-9]+)\s*\(", src)))
    lib = ctypes.CDLL(path)
    for name in declared:
        assert hasattr(lib, name), name
    rl = ", ".join(map(str, t["f2x"]["rect_loop"]))
    assert "TUNED_F2X = {{8, 6, 5}, {0, 0, 0}, {0, 48, 0}, {%s}}" % rl in open(tmp_path / "csrc" / "stage_tuning.h").read()


def test_tuner_coordinate_descent_on_a_synthetic_landscape():
    """The tuner's search, with the build and the timing replaced by a
    synthetic rate surface: each candidate build sees the header with only
    the tuned entry changed, one pass reaches the optimum of a separable
    surface, and on a coupled one a second pass moves past the first pass's
    point, without timing any candidate twice."""
    from paper_2505_15771_gb300 import tune
    text = open(tune.HEADER).read()
    tables = tune.read_tables(text)
    seen = {}

    def build(header, out_dir):
        t = tune.read_tables(header)
        assert t["f64"] == tables["f64"] and t["f32"] == tables["f32"]
        e = tuple(t["f2x"][f][1] for f in tune.FIELDS)
        assert t["f2x"]["min_blocks"][0] == tables["f2x"]["min_blocks"][0]
        return e

    def separable(e, *_):
        seen[e] = seen.get(e, 0) + 1
        mb, acc, pf, rl = e
        return 100.0 - (mb - 6) ** 2 + 3.0 * acc - abs(pf - 48) / 16.0 + 0.5 * rl

    best, res, _ = tune.tune("f2x", 2, "bilayer", log=lambda *a: None, header_text=text, build_fn=build,
                             measure_fn=separable)
    assert (best["min_blocks"], best["acc_smem"], best["prefetch"], best["rect_loop"]) == (6, 1, 48, 1)
    assert all(v == 1 for v in seen.values())

    # coupled: the best block count moves from 8 to 5 once the accumulators
    # are in shared memory, which only the second pass can see
    seen.clear()

    def coupled(e, *_):
        seen[e] = seen.get(e, 0) + 1
        mb, acc, pf, rl = e
        return 50.0 - abs(mb - (5 if acc else 8)) + 4.0 * acc + (1.0 if pf == 16 else 0.0) - 0.5 * rl

    start = tune.write_tables(text, tune.with_entry(tables, "f2x", 2, {"min_blocks": 8, "acc_smem": 0,
                                                                        "prefetch": 0, "rect_loop": 1}))
    b1, _, _ = tune.tune("f2x", 2, "bilayer", log=lambda *a: None, header_text=start, build_fn=build,
                         measure_fn=coupled)
    assert (b1["min_blocks"], b1["acc_smem"], b1["prefetch"], b1["rect_loop"]) == (8, 1, 16, 0)
    seen.clear()
    b2, res, _ = tune.tune("f2x", 2, "bilayer", passes=2, log=lambda *a: None, header_text=start, build_fn=build,
                           measure_fn=coupled)
    assert (b2["min_blocks"], b2["acc_smem"], b2["prefetch"], b2["rect_loop"]) == (5, 1, 16, 0)
    assert all(v == 1 for v in seen.values()) and len(seen) == len(res)


def _ncu_csv(path, launches):
    """A minimal ncu --csv log: one row per (launch, metric)."""
    import csv
    hdr = ["ID", "Process ID", "Process Name", "Host Name", "Kernel Name", "Context", "Stream", "Block Size",
           "Grid Size", "Device", "CC", "Section Name", "Metric Name", "Metric Unit", "Metric Value"]
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(hdr)
        for i, (name, rd, wr, us) in enumerate(launches):
            for metric, unit, val in (("dram__bytes_read.sum", "Mbyte", rd), ("dram__bytes_write.sum", "Mbyte", wr),
                                      ("gpu__time_duration.sum", "usecond", us)):
                w.writerow([str(i), "1", "python", "h", name, "1", "7", "(128, 1, 1)", "(1, 1, 1)", "0", "10.3",
                            "Command line profiler metrics", metric, unit, "{:,}".format(val)])


def test_traffic_record_from_ncu_logs(tmp_path):
    """bench.py --traffic-record: per arithmetic and k, the mean DRAM bytes
    of the ERK stage launches (mode 1 only) over the captured case's cell
    DOFs, keyed by the current stage sources; bench.py scales it back."""
    import bench
    k2 = [("void <unnamed>::stage_kernel<f2x, 2, 1>(StageArgsT<T1>)", 200.0, 150.0, 130.0),
          ("void <unnamed>::stage_kernel<f2x, 2, 1>(StageArgsT<T1>)", 240.0, 160.0, 140.0),
          ("void <unnamed>::stage_kernel<f2x, 2, 0>(StageArgsT<T1>)", 999.0, 999.0, 60.0),
          ("void <unnamed>::stage_kernel<double, 2, 1>(StageArgsT<T1>)", 300.0, 170.0, 190.0)]
    k3 = [("void <unnamed>::stage_kernel<f2x, 3, 1>(StageArgsT<T1>)", 300.0, 180.0, 250.0),
          ("void <unnamed>::stage_kernel<double, 3, 1>(StageArgsT<T1>)", 320.0, 190.0, 290.0),
          ("void <unnamed>::stage_kernel<float, 3, 1>(StageArgsT<T1>)", 100.0, 50.0, 90.0),
          ("void <unnamed>::stage_kernel<double, 2, 1>(StageArgsT<T1>)", 999.0, 999.0, 90.0)]   # other k: ignored
    _ncu_csv(tmp_path / "k2.csv", k2)
    _ncu_csv(tmp_path / "k3.csv", k3)
    out = tmp_path / "traffic.json"
    rec = bench.write_traffic_record([(str(tmp_path / "k2.csv"), 48, 24, 2), (str(tmp_path / "k3.csv"), 40, 20, 3)],
                                     str(out))
    # cell DOFs counted from the meshes: half the rows of the bilayer are solid (5n), half fluid (3n)
    dofs2 = 48 * 24 * 0.5 * 8 * 6
    dofs3 = 40 * 20 * 0.5 * 8 * 10
    assert bench.bilayer_cell_dofs(48, 24, 2) == dofs2
    assert rec["stage_sources_sha256"] == bench.stage_source_sha()
    assert rec["f32x2_k2"]["dram_bytes_per_launch_mean"] == pytest.approx(375e6)   # (350 + 400) / 2 MB
    assert rec["f32x2_k2"]["dram_bytes_per_launch_per_cell_dof"] == pytest.approx(375e6 / dofs2)
    assert rec["f32x2_k2"]["kernel_time_us_mean_under_ncu"] == pytest.approx(135.0)
    assert rec["k2"]["dram_bytes_per_launch_mean"] == pytest.approx(470e6)
    assert rec["f32x2_k3"]["dram_bytes_per_launch_per_cell_dof"] == pytest.approx(480e6 / dofs3)
    assert rec["k3"]["dram_bytes_per_launch_mean"] == pytest.approx(510e6)
    assert rec["f32_k3"]["dram_bytes_per_launch_mean"] == pytest.approx(150e6)   # float is filed apart
    assert "20 stage launches" not in rec["f32x2_k2"]["captured"] and "2 stage launches" in rec["f32x2_k2"]["captured"]
    import json
    assert json.load(open(out)) == rec
