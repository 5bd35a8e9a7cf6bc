"""Benchmark: ERK stage operator of the HHO elasto-acoustic scheme on GB300.

Workload (one GPU): the 1024 x 512 quadrilateral bilayer on [0,2]x[0,1]
(random-field elastic layer under water, k = 2 by default, classical ERK4,
Ricker point force, 256 receivers recorded every step).  A "step" is one ERK
time step: every stage kernel plus the receiver recording.

Metric: cell-DOF updates per second per ERK stage =
cell DOFs x stages x steps / time.  `value` is device-timed with inputs
resident in HBM; `e2e` is the same metric through hho_erk_run_host with the
state in pinned host memory (every step reads it from and writes it back to
host memory inside the timed region).

Headline: the FP64-instruction stage path, started from a seeded random
state.  Its roofline is the FP64 pipe on this part (FP64 multiply-add rate
measured live by the probe kernel), reported as "bound": "alu" with FP64
lane-ops from the library's cost model; the HBM view (algorithmic bytes /
time against MEASURED_PEAKS.json) is reported beside it.  The double-float
path (FP64-class accuracy on the FP32 pipes, bound by HBM) is timed on the
same workload and state in `alternative`, with its own rooflines and e2e.

--impl reference times the CPU oracle (plain FP64 numpy/scipy) on a bounded
sample of the same workload on the host cores.

Multi-GPU (torchrun): independent replicas, one per GPU (the stage operator
needs a halo exchange to shard a mesh; on this pool boxes have one GPU).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell-DOF updates/s per ERK stage"
CFL_SQUARES_ERK4 = {1: 0.233, 2: 0.122, 3: 0.082}
UNIT = "cell-DOF-stage/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--k", type=int, default=2)
    ap.add_argument("--arith", default="f64", choices=["f64", "f32x2"],
                    help="arithmetic of the headline stage path: FP64 instructions (default), or double-float "
                         "pairs (FP64-class accuracy on the FP32 pipes); the other one is timed beside it")
    ap.add_argument("--stages", type=int, default=4)
    ap.add_argument("--nx", type=int, default=1024)
    ap.add_argument("--ny", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--shots", type=int, default=16, help="shots of the batched (NEXT-1) measurement")
    ap.add_argument("--batch-precision", default="f32", choices=["f32", "f64", "f32x2", "bf16x3"])
    ap.add_argument("--batch-steps", type=int, default=10)
    ap.add_argument("--batch-workload", default="c3", choices=["c3", "c5"],
                    help="c3: 1360x680 hybrid quads/triangles, k=3; c5: basin section with hanging nodes, k=2")
    ap.add_argument("--batch-nx", type=int, default=None, help="default 1360 (c3) or 2860 (c5)")
    ap.add_argument("--batch-ny", type=int, default=None, help="default 680 (c3) or 715 (c5)")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--adjoint-steps", type=int, default=800, help="steps of the adjoint (NEXT-2) measurement")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-sdirk", action="store_true")
    ap.add_argument("--traffic-record", nargs="+", metavar="CSV NX NY K", default=None,
                    help="write profiles/stage_kernel_traffic.json from ncu CSV logs (dram bytes of the stage "
                         "launches on the NX x NY bilayer at degree K), given as groups of four: CSV NX NY K; "
                         "needs no GPU")
    return ap.parse_args()


def workload_name(a):
    return ("bilayer %dx%d quads on [0,2]x[0,1], k=%d, ERK%d, random-field solid (+-20%%) under water, "
            "Ricker f0=10 point force, 256 receivers" % (a.nx, a.ny, a.k, a.stages))


# ---------------------------------------------------------------- CPU oracle sample
def oracle_sample(a, seconds=10.0, max_steps=None):
    """Times the oracle on a 64 x 32 section of the same bilayer (same media
    recipe, same k and tableau): returns (dof-stage/s, description, steps)."""
    import synth
    from oracle import assemble as A
    from oracle import erk as E
    from oracle import mesh as M
    w = synth.bilayer_c2(nx=64, ny=32, k=a.k)
    md = w["mesh"]
    m = M.build_mesh(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
    S = A.System(m, a.k, *w["media"])
    b, _ = S.point_load(*w["source"], direction=(0.0, 1.0))
    st = E.Stepper(S, lambda t: synth.ricker(t, 10.0) * b)
    U = np.zeros(S.nT)
    dt = 1e-4
    st.step(U, 0.0, dt, "erk%d" % a.stages, 1)
    t0 = time.perf_counter()
    n = 0
    while time.perf_counter() - t0 < seconds and (max_steps is None or n < max_steps):
        U = st.step(U, n * dt, dt, "erk%d" % a.stages, 1)
        n += 1
    el = time.perf_counter() - t0
    rate = S.nT * a.stages * n / el
    desc = ("oracle (global sparse LU face and mass solves, numpy/scipy FP64) on a 64x32 section of the same "
            "bilayer (2048 cells, %d cell DOFs), %d ERK%d steps in %.1f s" % (S.nT, n, a.stages, el))
    return rate, desc, n, el


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps = max(1, a.steps)
    rate, desc, n, el = oracle_sample(a, seconds=min(60.0, 0.5 * steps), max_steps=steps)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": a.gpus,
            "steps": n, "warmup": a.warmup, "ms_per_step": 1e3 * el / max(n, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(a), "sample": "64x32 section"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- GPU run
def replica_reduce(ms_local, units_local, world, dist=None, device=None):
    """Whole-job timing of independent replicas: the slowest rank's time and
    the units summed over ranks (value = units / time)."""
    if world <= 1:
        return ms_local, units_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def stage_source_sha():
    """sha256 of the stage kernel sources (stage.cu, f2x.cuh, then the tuning
    table stage_tuning.h)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("stage.cu", "f2x.cuh", "stage_tuning.h"):
        h.update(open(os.path.join(ROOT, "paper_2505_15771_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def measured_traffic(k, cell_dofs, arith="f64"):
    """DRAM bytes per stage launch from the committed ncu summary, if it was
    taken on the current stage kernel sources (same sha256), the same k and
    arithmetic; scaled from the captured case by cell DOFs.  None otherwise."""
    path = os.path.join(ROOT, "profiles", "stage_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if rec.get("stage_sources_sha256") != stage_source_sha():
        return None
    entry = rec.get(("k%d" % k) if arith == "f64" else ("%s_k%d" % (arith, k)))
    if not entry:
        return None
    return entry["dram_bytes_per_launch_per_cell_dof"] * cell_dofs


TRAFFIC_KEYS = {"double": "k%d", "f2x": "f32x2_k%d", "float": "f32_k%d"}


def bilayer_cell_dofs(nx, ny, k):
    """Cell DOFs of the nx x ny bilayer (3n per fluid cell, 5n per solid cell)."""
    import synth
    md = synth.bilayer_c2(nx=nx, ny=ny, k=k)["mesh"]
    n = (k + 1) * (k + 2) // 2
    n_solid = int(np.count_nonzero(md.cell_domain == 1))
    return (md.n_cells - n_solid) * 3 * n + n_solid * 5 * n


def write_traffic_record(captures, out_path=None):
    """profiles/stage_kernel_traffic.json from ncu --csv logs of
    dram__bytes_read.sum, dram__bytes_write.sum and gpu__time_duration.sum.
    ``captures``: (csv path, nx, ny, k) of each capture on the nx x ny
    bilayer.  Per arithmetic (the kernel's template type: double -> k<k>,
    f2x -> f32x2_k<k>, float -> f32_k<k>) and k, the mean over the captured
    ERK stage launches (stage_kernel<T, k, 1>) divided by the captured case's
    cell DOFs, keyed by the current stage sources."""
    import csv
    import collections
    import re
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "ns": 1e-3, "us": 1.0, "usecond": 1.0,
             "msecond": 1e3, "ms": 1e3}
    pat = re.compile(r"stage_kernel<(\w+), ?(?:\(int\))?(\d), ?(?:\(int\))?1>")
    out = {}
    for path, nx, ny, k in captures:
        nx, ny, k = int(nx), int(ny), int(k)
        dofs = bilayer_cell_dofs(nx, ny, k)
        rows = [r for r in csv.reader(open(path)) if len(r) > 10]
        hdr, data = rows[0], rows[1:]
        ki, mi, vi, ui, ii = (hdr.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit", "ID"))
        per = collections.defaultdict(dict)
        for r in data:
            per[(r[ii], r[ki])][r[mi]] = float(r[vi].replace(",", "")) * scale.get(r[ui], 1.0)
        by_key = collections.defaultdict(list)
        for (_, name), m in per.items():
            g = pat.search(name)
            if g and int(g.group(2)) == k and g.group(1) in TRAFFIC_KEYS:
                by_key[TRAFFIC_KEYS[g.group(1)] % k].append(m)
        for key, ms in by_key.items():
            b = [m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"] for m in ms]
            t = [m["gpu__time_duration.sum"] for m in ms]
            out[key] = {"captured": "bilayer %dx%d, %d cell DOFs, %d stage launches" % (nx, ny, dofs, len(ms)),
                        "dram_bytes_per_launch_mean": sum(b) / len(b),
                        "dram_bytes_per_launch_per_cell_dof": sum(b) / len(b) / dofs,
                        "kernel_time_us_mean_under_ncu": sum(t) / len(t)}
    rec = {"stage_sources_sha256": stage_source_sha(),
           "note": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the ERK stage launches (stage_kernel<T,k,1>), "
                   "mean over the captured launches, divided by the cell DOFs of the captured case; bench.py scales "
                   "by the workload's cell DOFs (one thread per cell, class-sorted SoA: traffic grows in "
                   "proportion). Keys: k<k> FP64 kernel, f32x2_k<k> double-float kernel, f32_k<k> FP32 kernel. "
                   "Written by bench.py --traffic-record."}
    rec.update(out)
    with open(out_path or os.path.join(ROOT, "profiles", "stage_kernel_traffic.json"), "w") as f:
        json.dump(rec, f, indent=1)
    return rec


def fp64_fma_rate():
    import ctypes
    lib = ctypes.CDLL(os.path.join(ROOT, "paper_2505_15771_gb300", "libhho_probe.so"))
    lib.hho_probe_dfma_rate.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    r = ctypes.c_double()
    if lib.hho_probe_dfma_rate(4000, 3, ctypes.byref(r)) != 0:
        return None
    return r.value


CFL_TRIANGLES_ERK4_K3 = 0.045   # below the ERK4 eigenvalue limit of the right-triangle grid at k = 3


def batched_accuracy(a, torch, hho, P, w, dt, n_shots=2, nsteps=500):
    """FP32 batched seismograms and states against the FP64 batched path (which
    equals the oracle shot by shot) on the first shots of the workload, over
    enough steps for the waves to reach receivers on rings of 8 around each
    source (radius 0.3 c_min t: the workload's own receivers are not reached
    within such runs).  Relative L2 per shot, the worst reported."""
    src = [tuple(x) for x in np.asarray(w["sources"], dtype=np.float64)[:n_shots]]
    rho, lam, mu, kappa = (np.asarray(m, dtype=np.float64) for m in w["media"])
    c = np.where(mu > 0, np.sqrt(np.maximum(mu, 1e-300) / rho), np.sqrt(np.maximum(kappa, 1e-300) / rho))
    radius = 0.3 * float(c.min()) * dt * nsteps
    ang = 2 * np.pi * (np.arange(8) + 0.25) / 8
    ring = [(x + radius * np.cos(t), y + radius * np.sin(t)) for (x, y) in src for t in ang]
    P.set_shot_sources(src, [(0.0, 1.0)] * n_shots, np.asarray(w["f0"], dtype=np.float64).reshape(-1)[:n_shots]
                       if np.ndim(w["f0"]) else w["f0"])
    P.set_receivers(ring)
    out = {}
    for name, prec in (("f64", hho.HHO_F64), ("f32", hho.HHO_F32)):
        state, work = P.batch_buffers(4, n_shots, prec)
        seis = torch.zeros((nsteps, n_shots, len(ring), 5), dtype=torch.float32 if prec == hho.HHO_F32 else
                           torch.float64, device=P.dev)
        P.batch_step(state, work, n_shots, 4, 0.0, dt, nsteps, precision=prec, seismogram=seis)
        torch.cuda.synchronize()
        out[name] = (P.batch_to_canonical(state, n_shots, prec), seis.double().cpu().numpy())
        del state, work, seis
    rel = lambda x, y: float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))
    c64, s64 = out["f64"]
    c32, s32 = out["f32"]
    return {"shots": n_shots, "steps": nsteps, "receivers": "rings of 8 at radius %.3g around each source" % radius,
            "seismogram_rel_l2_max": max(rel(s32[:, i], s64[:, i]) for i in range(n_shots)),
            "state_rel_l2_max": max(rel(c32[i], c64[i]) for i in range(n_shots)),
            "against": "the FP64 batched path on the same shots (equal to the FP64 oracle shot by shot)",
            "bar": 1e-5}


def measure_batched(a, torch, hho, solver, hbm_peak):
    """Batched shots on the ~1.2 M-cell hybrid mesh (k = 3): S shots in one
    launch per stage, FP32 (default) or FP64, against FP64 single-shot runs
    on the same mesh (the "S sequential FP64 runs" comparison)."""
    import synth
    S = a.shots
    prec = {"f32": hho.HHO_F32, "f64": hho.HHO_F64, "f32x2": hho.HHO_F32X2, "bf16x3": hho.HHO_BF16X3}[a.batch_precision]
    if a.batch_workload == "c5":
        w = synth.basin_c5(nx=a.batch_nx, ny=a.batch_ny, n_shots=S)
        kk = w["k"]
        desc = ("basin section 20x5 km on %dx%d coarse squares (4x-refined spline basin, hanging-node polygons, "
                "triangles along the basin floor), k=%d, ERK4, water over bedrock with a graded sedimentary basin, "
                "one Ricker point force (f0=15) per shot at a seeded solid point, %d seabed receivers recorded every "
                "step" % (a.batch_nx, a.batch_ny, kk, len(w["receivers"])))
        cfl = CFL_TRIANGLES_ERK4_K3
    else:
        w = synth.hybrid_c3(S, nx=a.batch_nx, ny=a.batch_ny, k=3)
        kk = 3
        desc = ("hybrid %dx%d on [0,2]x[0,1] (quads below y=0.7, triangles above), k=3, ERK4, random-field solid "
                "under water, one Ricker point force per shot at a seeded solid point, 256 receivers recorded every "
                "step" % (a.batch_nx, a.batch_ny))
        cfl = CFL_TRIANGLES_ERK4_K3
    md = w["mesh"]
    P = solver.Problem(md, w["media"], kk)
    P.set_shot_sources(w["sources"], [(0.0, 1.0)] * S, w["f0"])
    P.set_receivers(w["receivers"])
    tab = hho.hho_tableau_erk(4)
    dt = hho.hho_cfl_dt(P.ops, cfl, 0.9)
    ndof = P.layout.n_canonical
    state, work = P.batch_buffers(4, S, prec)
    steps = max(1, a.batch_steps)
    seis = torch.empty((max(steps, 3), S, len(w["receivers"]), 5),
                       dtype=torch.float32 if prec in (hho.HHO_F32, hho.HHO_BF16X3) else torch.float64,
                       device=P.dev)   # FP64 for f32x2
    stream = torch.cuda.current_stream()
    P.batch_step(state, work, S, 4, 0.0, dt, 3, precision=prec, seismogram=seis)
    torch.cuda.synchronize()
    hho.hho_profile_enable(P.ops, True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    P.batch_step(state, work, S, 4, 3 * dt, dt, steps, precision=prec, seismogram=seis)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    stage_ms, nl = hho.hho_profile_read(P.ops)
    hho.hho_profile_enable(P.ops, False)
    value = S * ndof * 4 * steps / (ms * 1e-3)
    finite = bool(torch.isfinite(seis[:steps]).all().item())
    # the same steps replayed as one captured graph per step (stage kernels,
    # receiver record, clock increment); the profiled run above uses stream
    # launches with an event pair around every stage kernel
    P.set_launch_mode(hho.HHO_LAUNCH_GRAPH)
    P.batch_step(state, work, S, 4, 0.0, dt, 2, precision=prec, seismogram=seis)   # capture
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    P.batch_step(state, work, S, 4, 3 * dt, dt, steps, precision=prec, seismogram=seis)
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1)
    P.set_launch_mode(hho.HHO_LAUNCH_AUTO)
    # the same shots with the dense local products on the tcgen05 tensor
    # cores (split BF16, FP32 accumulation), from the same start
    tensor_core = None
    if prec == hho.HHO_F32:
        xf, wf = P.batch_buffers(4, S, hho.HHO_F32)   # the FP32 trajectory of the same schedule
        P.batch_step(xf, wf, S, 4, 0.0, dt, 3, precision=hho.HHO_F32)
        P.batch_step(xf, wf, S, 4, 3 * dt, dt, steps, precision=hho.HHO_F32)
        canon32 = P.batch_to_canonical(xf, S, hho.HHO_F32)[0]
        del xf, wf
        xt, wt = P.batch_buffers(4, S, hho.HHO_BF16X3)
        P.batch_step(xt, wt, S, 4, 0.0, dt, 3, precision=hho.HHO_BF16X3)
        torch.cuda.synchronize()
        hho.hho_profile_enable(P.ops, True)
        t0e = torch.cuda.Event(enable_timing=True)
        t1e = torch.cuda.Event(enable_timing=True)
        t0e.record(stream)
        P.batch_step(xt, wt, S, 4, 3 * dt, dt, steps, precision=hho.HHO_BF16X3)
        t1e.record(stream)
        torch.cuda.synchronize()
        tc_ms = t0e.elapsed_time(t1e)
        tc_stage_ms, tc_nl = hho.hho_profile_read(P.ops)
        hho.hho_profile_enable(P.ops, False)
        canon_tc = P.batch_to_canonical(xt, S, hho.HHO_BF16X3)[0]
        tc_err = hho.hho_tc_error(P.ops)
        tc_avg = tc_stage_ms * 1e-3 / max(tc_nl, 1)
        _, bmin, _ = hho.hho_stage_cost(P.ops, tab)
        tc_bytes = bmin / 8 * 4 * S / 4
        tensor_core = {"precision": "bf16x3", "value": S * ndof * 4 * steps / (tc_ms * 1e-3),
                       "ms_per_step": tc_ms / steps, "avg_launch_ms": tc_avg * 1e3,
                       "over_fp32": (S * ndof * 4 * steps / (tc_ms * 1e-3)) / value,
                       "rel_diff_vs_fp32_shot0": float(np.linalg.norm(canon_tc - canon32) /
                                                      max(np.linalg.norm(canon32), 1e-300)),
                       "mma_wait_error": tc_err,
                       "roofline": {"bound": "hbm", "achieved": tc_bytes / tc_avg / 1e9, "peak": hbm_peak,
                                    "unit": "GB/s", "frac": tc_bytes / tc_avg / 1e9 / hbm_peak,
                                    "kernel": "stage_tc_kernel<%d,1>" % kk},
                       "note": "lift and trace products of every face as two tcgen05 GEMMs per stage per block of "
                               "32 cells x 4 shots, operands split into BF16 hi + lo, three MMAs per K step"}
        del xt, wt
    # FP64 single shot on the same mesh
    x1 = P.empty_state()
    w1 = P.work(tab)
    hho.hho_erk_step(P.ops, tab, 0.0, dt, 2, x1.data_ptr(), w1.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    hho.hho_erk_step(P.ops, tab, 0.0, dt, steps, x1.data_ptr(), w1.data_ptr(), stream.cuda_stream)
    f1.record(stream)
    torch.cuda.synchronize()
    v64 = ndof * 4 * steps / (f0.elapsed_time(f1) * 1e-3)
    accuracy = batched_accuracy(a, torch, hho, P, w, dt) if prec == hho.HHO_F32 else None
    _, bytes_min, bytes_kernel = hho.hho_stage_cost(P.ops, tab)
    elt = 4 if prec in (hho.HHO_F32, hho.HHO_BF16X3) else 8
    per_launch = bytes_min / 8 * elt * S / 4
    avg = stage_ms * 1e-3 / max(nl, 1)
    out = {"metric": "shot-cell-DOF updates/s per ERK stage", "value": value, "unit": "shot-cell-DOF-stage/s",
           "precision": a.batch_precision, "shots": S, "steps": steps, "ms_per_step": ms / steps,
           "workload": desc,
           "cells": int(md.n_cells), "cell_dofs": int(ndof), "dt": dt, "seismograms_finite": finite,
           "tensor_core": tensor_core, "fp32_accuracy": accuracy,
           "graph_replay": {"value": S * ndof * 4 * steps / (graph_ms * 1e-3), "ms_per_step": graph_ms / steps,
                            "launch": "one captured graph per step (s stage kernels + record + clock)"},
           "fp64_single_shot_same_mesh": v64, "speedup_vs_sequential_fp64": value / v64,
           "roofline": {"bound": "hbm", "achieved": per_launch / avg / 1e9, "peak": hbm_peak, "unit": "GB/s",
                        "frac": per_launch / avg / 1e9 / hbm_peak,
                        "algorithmic_bytes_per_launch": per_launch, "avg_launch_ms": avg * 1e3,
                        "kernel": "stage_kernel<%s,%d,1>" % ({hho.HHO_F32: "float", hho.HHO_F64: "double",
                                                               hho.HHO_F32X2: "f2x"}[prec], kk)}}
    P.close()
    return out


def measure_adjoint(a, torch, hho):
    """Discrete adjoint on the 256 x 256 two-layer workload (k = 2, ERK4,
    800 steps, checkpoints every 50, 128 interface receivers): one shot's
    misfit gradient w.r.t. every cell's (rho, kappa, lambda, mu), timed with
    CUDA events against the forward run with trace recording."""
    import synth
    w = synth.adjoint_c4()
    md = w["mesh"]
    nc = md.n_cells
    k, nsteps, ckpt = w["k"], a.adjoint_steps, 50
    stream = torch.cuda.current_stream()
    tab = hho.hho_tableau_erk(4)
    mesh = hho.hho_mesh_create(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain)
    ops = hho.hho_operators_build(mesh, k, *w["background"])
    hho.hho_mesh_destroy(mesh)
    hho.hho_sources_set(ops, [w["sources"][0]], [(0.0, 1.0)], [w["f0"]], [1.0 / w["f0"]], [1.0])
    hho.hho_receivers_set(ops, w["receivers"])
    dt = hho.hho_cfl_dt(ops, CFL_SQUARES_ERK4[k], 0.9)
    lay = hho.hho_state_layout(ops)
    x = torch.zeros(lay.n_state, dtype=torch.float64, device="cuda")
    wk = torch.empty(hho.hho_work_size(ops, tab), dtype=torch.float64, device="cuda")
    seis = torch.zeros((nsteps, len(w["receivers"]), 5), dtype=torch.float64, device="cuda")
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    hho.hho_erk_step_record(ops, tab, 0.0, dt, min(nsteps, 3), x.data_ptr(), wk.data_ptr(), seis.data_ptr(),
                            stream.cuda_stream)
    x.zero_()
    torch.cuda.synchronize()
    e[0].record(stream)
    hho.hho_erk_step_record(ops, tab, 0.0, dt, nsteps, x.data_ptr(), wk.data_ptr(), seis.data_ptr(),
                            stream.cuda_stream)
    e[1].record(stream)
    torch.cuda.synchronize()
    fwd_ms = e[0].elapsed_time(e[1])
    g = (0.01 * seis).contiguous()   # cotangent: a residual of 1 % of the traces
    x0 = torch.zeros_like(x)
    nw = hho.hho_adjoint_work_size(ops, tab, nsteps, ckpt)
    aw = torch.empty(nw, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e[2].record(stream)
    grad, _ = hho.hho_adjoint_vjp(ops, tab, 0.0, dt, nsteps, ckpt, x0.data_ptr(), g.data_ptr(), aw.data_ptr(), nw,
                                  nc, n_src=1, stream=stream.cuda_stream)
    e[3].record(stream)
    torch.cuda.synchronize()
    adj_ms = e[2].elapsed_time(e[3])
    # the FP32 reverse mode on the same problem and cotangent
    nw32 = hho.hho_adjoint_work_size_f32(ops, tab, nsteps, ckpt)
    aw32 = torch.empty(nw32, dtype=torch.float32, device="cuda")
    x32, g32c = x0.float(), g.float().contiguous()
    del aw
    torch.cuda.synchronize()
    e[2].record(stream)
    grad32, _ = hho.hho_adjoint_vjp_f32(ops, tab, 0.0, dt, nsteps, ckpt, x32.data_ptr(), g32c.data_ptr(),
                                        aw32.data_ptr(), nw32, nc, n_src=1, stream=stream.cuda_stream)
    e[3].record(stream)
    torch.cuda.synchronize()
    adj32_ms = e[2].elapsed_time(e[3])
    ndof = lay.n_canonical
    out = {"metric": "adjoint cell-DOF-stages/s (forward-equivalent work / gradient time)",
           "value": ndof * 4 * nsteps / (adj_ms * 1e-3), "unit": "cell-DOF-stage/s",
           "workload": "256x256 quads, two-layer (water over solid), k=2, ERK4, %d steps, checkpoints every %d, "
                       "one Ricker shot, 128 interface receivers, gradient w.r.t. per-cell rho/kappa/lambda/mu"
                       % (nsteps, ckpt),
           "cells": int(nc), "cell_dofs": int(ndof), "steps": nsteps, "gradient_ms": adj_ms,
           "forward_record_ms": fwd_ms, "adjoint_over_forward": adj_ms / fwd_ms,
           "gradient_finite": bool(np.isfinite(grad).all()), "dtype": "f64",
           "fp32": {"gradient_ms": adj32_ms, "value": ndof * 4 * nsteps / (adj32_ms * 1e-3),
                    "rel_diff_vs_fp64": float(np.linalg.norm(grad32 - grad) / np.linalg.norm(grad)),
                    "note": "hho_adjoint_vjp_f32: FP32 stage kernels and adjoint vectors, FP64 gradient sums"}}
    hho.hho_ops_destroy(ops)
    return out


def measure_small(a, torch, hho, solver):
    """The small academic configuration (512 right triangles, k = 1, ERK4,
    200 steps, Ricker source, 8 interface receivers recorded every step),
    whose stage kernels are too short to hide launch overhead: FP64, timed
    with CUDA events over the 200 steps, stream launches against replayed
    step graphs."""
    import synth
    w = synth.academic_c1()
    dt = json.load(open(os.path.join(ROOT, "tests", "golden", "c1_dt.json")))["dt"]
    P = solver.Problem(w["mesh"], w["media"], w["k"])
    P.set_sources([w["source"]], [(0.0, 1.0)], w["f0"])
    P.set_receivers(w["receivers"])
    tab = hho.hho_tableau_erk(4)
    n = P.layout.n_canonical
    nsteps = w["nsteps"]
    seis = torch.zeros((nsteps, len(w["receivers"]), 5), dtype=torch.float64, device=P.dev)
    sp = torch.cuda.current_stream().cuda_stream
    res = {}
    for name, mode in (("stream", hho.HHO_LAUNCH_STREAM), ("graph", hho.HHO_LAUNCH_GRAPH)):
        P.set_launch_mode(mode)
        x = P.to_device(np.zeros(n))
        hho.hho_erk_step_record(P.ops, tab, 0.0, dt, nsteps, x.data_ptr(), P.work(tab).data_ptr(), seis.data_ptr(),
                                sp)   # warm-up (and graph capture)
        best = None
        for _ in range(3):
            x.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            hho.hho_erk_step_record(P.ops, tab, 0.0, dt, nsteps, x.data_ptr(), P.work(tab).data_ptr(),
                                    seis.data_ptr(), sp)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        res[name] = {"ms_per_run": best, "us_per_step": 1e3 * best / nsteps,
                     "value": n * 4 * nsteps / (best * 1e-3)}
    P.close()
    return {"metric": METRIC, "unit": UNIT,
            "workload": "academic: 512 right triangles on the unit square, k=1, ERK4, 200 steps, Ricker source, "
                        "8 interface receivers recorded every step, FP64 (best of 3 runs)",
            "cell_dofs": int(n), "stream": res["stream"], "graph": res["graph"],
            "graph_speedup": res["stream"]["ms_per_run"] / res["graph"]["ms_per_run"]}


def measure_sdirk(a, torch, hho, solver):
    """Implicit SDIRK(3,4) (matrix-free GMRES on the stage systems,
    block-Jacobi preconditioned) against ERK4 over the same simulated time on
    the bilayer at 256 x 128, k = 2: SDIRK at 4 x the ERK4 square CFL step,
    tol 1e-8, restart 10; the same SDIRK run without the preconditioner
    beside it.  The first timed SDIRK call includes the preconditioner build
    (the warm-up call builds it for the same step, so it is reused)."""
    import synth
    w = synth.bilayer_c2(nx=256, ny=128, k=2)
    P = solver.Problem(w["mesh"], w["media"], 2)
    P.set_sources([w["source"]], [(0.0, 1.0)], 10.0)
    n = P.layout.n_canonical
    dt_erk = hho.hho_cfl_dt(P.ops, CFL_SQUARES_ERK4[2], 0.9)
    ratio, n_sdirk = 4, 4
    x = P.to_device(np.zeros(n))
    P.sdirk_step(x, 3, 0.0, ratio * dt_erk, 1, tol=1e-8, restart=10, max_iter=5000)   # warm-up
    P.step(x, 4, 0.0, dt_erk, 3)
    x.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its = P.sdirk_step(x, 3, 0.0, ratio * dt_erk, n_sdirk, tol=1e-8, restart=10, max_iter=5000)
    torch.cuda.synchronize()
    t_sd = time.perf_counter() - t0
    e_sd = P.energy(x)
    y = P.to_device(np.zeros(n))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    P.step(y, 4, 0.0, dt_erk, ratio * n_sdirk)
    e1.record()
    torch.cuda.synchronize()
    t_erk = e0.elapsed_time(e1) * 1e-3
    diff = float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y))
    stages = 3 * n_sdirk
    # the same SDIRK steps without the preconditioner
    hho.hho_sdirk_set_preconditioner(P.ops, 0)
    z = P.to_device(np.zeros(n))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    its0 = P.sdirk_step(z, 3, 0.0, ratio * dt_erk, n_sdirk, tol=1e-8, restart=10, max_iter=5000)
    torch.cuda.synchronize()
    t_sd0 = time.perf_counter() - t0
    hho.hho_sdirk_set_preconditioner(P.ops, 1)
    out = {"metric": "wall time for the same simulated interval, SDIRK(3,4) vs ERK4",
           "workload": "bilayer 256x128 on [0,2]x[0,1], k=2, Ricker source, SDIRK(3,4) dt = %d x ERK4 dt, "
                       "%d SDIRK steps, GMRES tol 1e-8 restart 10, FP64" % (ratio, n_sdirk),
           "cell_dofs": int(n), "sdirk_wall_s": t_sd, "erk4_s": t_erk, "sdirk_over_erk4": t_sd / t_erk,
           "gmres_applications": int(its), "applications_per_stage": its / stages,
           "rel_diff_vs_erk4": diff, "energy_sdirk": e_sd,
           "unpreconditioned": {"sdirk_wall_s": t_sd0, "sdirk_over_erk4": t_sd0 / t_erk,
                                "applications_per_stage": its0 / stages},
           "note": "wall clock (GMRES synchronises once per Krylov vector); block-Jacobi right preconditioner "
                   "(exact cell blocks of the stage matrix, the local solves of Eq. sc2)"}
    P.close()
    return out


def measure_arith(a, torch, hho, P, tab, dt, state, work, seis, stream, U0, arith, hbm_peak, peak_fma, world,
                  clocks=None, dist=None):
    """One arithmetic of the stage path on the headline workload: W warm-up
    steps, then exactly K timed steps (CUDA events on the launching stream),
    starting from the seeded random state U0 (packed on the device, so the
    rate is measured on non-zero data).  Returns the timing, the stage
    kernel's per-launch time (library profiler: events around every stage
    launch on the same stream) and its rooflines."""
    P.set_arithmetic(arith)
    ndof = P.layout.n_canonical
    x0 = P.to_device(U0, stream)

    def run(nsteps, t0):
        hho.hho_erk_step_record(P.ops, tab, t0, dt, nsteps, state.data_ptr(), work.data_ptr(), seis.data_ptr(),
                                stream.cuda_stream)

    state.copy_(x0)
    run(max(a.warmup, 3), 0.0)          # warm-up (also the first touch of every buffer)
    torch.cuda.synchronize()
    e_warm = P.energy(state)
    hho.hho_profile_enable(P.ops, True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.start()
        time.sleep(0.3)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    run(a.steps, a.warmup * dt)
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks is not None else None
    if world > 1:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    stage_ms, n_launch = hho.hho_profile_read(P.ops)
    hho.hho_profile_enable(P.ops, False)
    e_end = P.energy(state)
    fp64_ops, bytes_min, bytes_kernel = hho.hho_stage_cost(P.ops, tab)
    avg_launch_s = stage_ms * 1e-3 / max(n_launch, 1)
    ops_per_launch = fp64_ops / a.stages
    name = "f64" if arith == hho.HHO_F64 else "f32x2"
    kern = "stage_kernel<%s,%d,1>" % ("double" if arith == hho.HHO_F64 else "f2x", a.k)
    hbm = {"bound": "hbm", "achieved": bytes_min / a.stages / avg_launch_s / 1e9, "peak": hbm_peak, "unit": "GB/s",
           "frac": bytes_min / a.stages / avg_launch_s / 1e9 / hbm_peak,
           "algorithmic_bytes_per_launch": bytes_min / a.stages,
           "traffic": measured_traffic(a.k, ndof, name), "kernel": kern, "avg_launch_ms": avg_launch_s * 1e3,
           "launches_timed": n_launch, "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)"}
    alu = {"bound": "alu", "achieved": ops_per_launch / avg_launch_s / 1e12,
           "peak": (peak_fma / 1e12) if peak_fma else None, "unit": "T FP64 lane-ops/s (multiply-add = 1)",
           "frac": (ops_per_launch / avg_launch_s / peak_fma) if peak_fma else None,
           "fp64_lane_ops_per_launch": ops_per_launch, "kernel": kern, "avg_launch_ms": avg_launch_s * 1e3,
           "launches_timed": n_launch, "peak_source": "live DFMA probe (libhho_probe.so), best of 3, same run"}
    if arith == hho.HHO_F64:
        # FP64 instructions: the FP64 pipe binds (about 13 lane-ops per cell
        # DOF per stage against 32 bytes); HBM is the view beside it
        roofline = dict(alu)
        roofline["traffic"] = hbm["traffic"]
        roofline["hbm_view"] = {k2: hbm[k2] for k2 in ("achieved", "peak", "unit", "frac",
                                                        "algorithmic_bytes_per_launch", "peak_source")}
    else:
        # double-float: no FP64 instruction; the FP32 pipes have headroom, so
        # the bound is HBM, with the FP64-equivalent lane-op rate as a view
        roofline = dict(hbm)
        roofline["alu_view"] = {k2: alu[k2] for k2 in ("achieved", "peak", "unit", "frac", "peak_source")}
        roofline["alu_view"]["note"] = ("FP64-equivalent lane-ops of the cost model per second, against the FP64 "
                                        "DFMA probe")
    return {"arith": name, "ms": ms, "units": ndof * a.stages * a.steps, "clocks": clk, "roofline": roofline,
            "energy_after_warmup": e_warm, "energy_after_timed": e_end}


def measure_e2e(a, torch, hho, P, dt, stream, arith, world):
    """End to end through hho_erk_run_host with the state in pinned host
    memory: every step reads it from and writes it back to host memory
    inside the timed region."""
    P.set_arithmetic(arith)
    ndof = P.layout.n_canonical
    h = torch.zeros(ndof, dtype=torch.float64, pin_memory=True)
    hn = h.numpy()
    hn[:] = synth_random_state(ndof)
    P.run_host(hn, a.stages, 0.0, dt, 1, stream)       # warm (allocates its buffers)
    ne = max(3, min(a.steps, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(ne):
        P.run_host(hn, a.stages, i * dt, dt, 1, stream)
    el = time.perf_counter() - t0
    return {"value": world * ndof * a.stages * ne / el, "unit": UNIT, "h2d_bytes_per_step": 8 * ndof,
            "d2h_bytes_per_step": 8 * ndof, "steps": ne, "arith": "f64" if arith == hho.HHO_F64 else "f32x2",
            "path": "hho_erk_run_host on a pinned host buffer: the pack kernel reads the canonical state from "
                    "host memory (NVLink-C2C), 1 ERK step, the unpack kernel writes it back to host memory, "
                    "stream sync"}


RANDOM_STATE_SEED = 11


def synth_random_state(n):
    import synth
    return synth.random_state(n, RANDOM_STATE_SEED)


def main():
    a = parse()
    if a.traffic_record:
        if len(a.traffic_record) % 4:
            raise SystemExit("--traffic-record takes groups of four: CSV NX NY K")
        t = a.traffic_record
        rec = write_traffic_record([tuple(t[i:i + 4]) for i in range(0, len(t), 4)])
        print(json.dumps({k: v["dram_bytes_per_launch_per_cell_dof"] for k, v in rec.items() if isinstance(v, dict)}))
        return
    if a.batch_nx is None:
        a.batch_nx = 2860 if a.batch_workload == "c5" else 1360
    if a.batch_ny is None:
        a.batch_ny = 715 if a.batch_workload == "c5" else 680
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    import synth
    from paper_2505_15771_gb300 import hho, solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(hho.LIB_PATH):
        raise RuntimeError("libhho.so is not built; run __graft_entry__.build() first")

    w = synth.bilayer_c2(nx=a.nx, ny=a.ny, k=a.k)
    md, media = w["mesh"], w["media"]
    P = solver.Problem(md, media, a.k)
    P.set_sources([w["source"]], [(0.0, 1.0)], 10.0)
    P.set_receivers(w["receivers"])
    ARITH = {"f64": hho.HHO_F64, "f32x2": hho.HHO_F32X2}
    tab = hho.hho_tableau_erk(a.stages)
    # CFL-limited dt (Eq. CFL): 0.9 x the ERK4 eigenvalue limit of the stage
    # operator on squares (c# dt / h = 0.233, 0.122, 0.082 for k = 1, 2, 3)
    dt = hho.hho_cfl_dt(P.ops, CFL_SQUARES_ERK4[a.k], 0.9)
    ndof = P.layout.n_canonical
    U0 = synth_random_state(ndof)
    state = P.empty_state()
    work = P.work(tab)
    seis = torch.empty((max(a.steps, a.warmup, 3), len(w["receivers"]), 5), dtype=torch.float64, device=P.dev)
    stream = torch.cuda.current_stream()
    peak_fma = fp64_fma_rate()
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    head = measure_arith(a, torch, hho, P, tab, dt, state, work, seis, stream, U0, ARITH[a.arith], hbm_peak,
                         peak_fma, world, ClockSampler(local), dist)
    ms, total_units = replica_reduce(head["ms"], head["units"], world, dist, P.dev)
    value = total_units / (ms * 1e-3)

    # the other arithmetic on the same workload and initial state, with its own rooflines and e2e
    other_name = "f64" if a.arith == "f32x2" else "f32x2"
    oth = measure_arith(a, torch, hho, P, tab, dt, state, work, seis, stream, U0, ARITH[other_name], hbm_peak,
                        peak_fma, 1)
    alternative = {"arith": other_name, "value": oth["units"] / (oth["ms"] * 1e-3), "unit": UNIT,
                   "ms_per_step": oth["ms"] / a.steps, "roofline": oth["roofline"],
                   "energy_after_timed": oth["energy_after_timed"],
                   "note": ("double-float pairs on the FP32 pipes (about 48 significand bits, FP32 exponent range), "
                            "same FP64-oracle parity bar" if other_name == "f32x2" else "FP64 instructions")}
    e2e = None
    if not a.no_e2e:
        e2e = measure_e2e(a, torch, hho, P, dt, stream, ARITH[a.arith], world)
        alternative["e2e"] = measure_e2e(a, torch, hho, P, dt, stream, ARITH[other_name], 1)
    P.set_arithmetic(ARITH[a.arith])

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        rate, desc, n, el = oracle_sample(a, seconds=10.0)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

    work_mb = 8e-6 * work.numel()
    state_mb = 8e-6 * P.layout.n_state
    batched = None
    if rank == 0 and not a.no_batched:
        P.close()
        del state, work, seis
        torch.cuda.empty_cache()
        batched = measure_batched(a, torch, hho, solver, hbm_peak)
    small = None
    if rank == 0:
        small = measure_small(a, torch, hho, solver)
    sdirk = None
    if rank == 0 and not a.no_sdirk:
        torch.cuda.empty_cache()
        sdirk = measure_sdirk(a, torch, hho, solver)
    adjoint = None
    if rank == 0 and not a.no_adjoint:
        torch.cuda.empty_cache()
        adjoint = measure_adjoint(a, torch, hho)

    # stages + receiver records (+ the state's conversion to and from pairs)
    launches = a.stages * a.steps + a.steps + 1 + (2 if a.arith == "f32x2" else 0)
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": a.arith, "data": "synthetic",
                "config": {"workload": workload_name(a), "cells": int(md.n_cells), "cell_dofs": int(ndof),
                           "k": a.k, "tableau": "erk%d" % a.stages, "dt": dt,
                           "initial_state": "seeded standard-normal canonical state (seed %d)"
                                            % RANDOM_STATE_SEED,
                           "l2": "inputs larger than L2 (state %.0f MB, work %.0f MB per GPU)" % (state_mb, work_mb),
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "energy_after_warmup": head["energy_after_warmup"],
                           "energy_after_timed": head["energy_after_timed"]},
                "roofline": head["roofline"], "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": head["clocks"], "alternative": alternative, "batched": batched, "adjoint": adjoint,
                "sdirk": sdirk, "small": small}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
