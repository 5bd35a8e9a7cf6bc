"""Build-time tuner of the stage kernels' launch parameters.

The ERK stage kernel of each arithmetic (FP64, double-float, FP32) and
degree k has four compile-time parameters, kept in csrc/stage_tuning.h:
the resident blocks per SM asked of the register allocator, whether the
cell's rate accumulators live in shared memory, the mask of L2 prefetch
hints, and whether a rectangle's faces are traced by one body per
orientation looped over its two faces or by four unrolled bodies.  Which combination is fastest depends on the GPU, the arithmetic, k
and the workload, and is not predictable from the register counts alone
(for instance, on GB300 shared accumulators lose without prefetch hints and
win with them).  This tool measures it:

* candidates are full builds of the stage kernels with one table entry
  changed (build.build_stage_variant, compiled in parallel);
* each candidate runs in a fresh process (HHO_LIB points the binding at its
  build) on a workload of the benchmark's shape, timed with CUDA events
  after warm-up;
* the search is coordinate descent from the current entry, one parameter
  at a time, for a given number of passes;
* --write stores the winner in csrc/stage_tuning.h.

    python -m paper_2505_15771_gb300.tune --arith f2x --k 2 --workload bilayer
    python -m paper_2505_15771_gb300.tune --arith f32 --k 3 --workload hybrid --write

Workloads: bilayer (the 1024 x 512 two-layer mesh, one shot, FP64 or
double-float, hho_erk_step), hybrid (the 1.2 M-cell quad/triangle mesh, 16
shots, batched FP32) and basin (the 3.3 M-cell basin with hanging nodes, 32
shots, batched FP32).  The library must have been built in-tree first.
"""
import argparse
import concurrent.futures
import json
import os
import re
import subprocess
import sys
import tempfile

from . import build as B

HEADER = os.path.join(B.CSRC, "stage_tuning.h")
TABLE = {"f64": "TUNED_F64", "f32": "TUNED_F32", "f2x": "TUNED_F2X"}
AXES = {"min_blocks": [4, 5, 6, 8, 10, 12], "acc_smem": [0, 1], "prefetch": [0, 16, 48, 50], "rect_loop": [0, 1]}
FIELDS = ("min_blocks", "acc_smem", "prefetch", "rect_loop")
_TABLE_RE = r"constexpr StageTuning %s = \{\{([^}]*)\}, \{([^}]*)\}, \{([^}]*)\}, \{([^}]*)\}\};"


def read_tables(text):
    """{arith: {field: [k1, k2, k3]}} from the header text."""
    out = {}
    for arith, name in TABLE.items():
        m = re.search(_TABLE_RE % name, text)
        if not m:
            raise ValueError("table %s not found in stage_tuning.h" % name)
        out[arith] = {f: [int(v) for v in m.group(i + 1).split(",")] for i, f in enumerate(FIELDS)}
    return out


def write_tables(text, tables):
    for arith, name in TABLE.items():
        t = tables[arith]
        line = "constexpr StageTuning %s = {%s};" % (
            name, ", ".join("{%s}" % ", ".join(map(str, t[f])) for f in FIELDS))
        text = re.sub(_TABLE_RE % name, line, text)
    return text


def with_entry(tables, arith, k, entry):
    t = json.loads(json.dumps(tables))
    for f in FIELDS:
        t[arith][f][k - 1] = entry.get(f, t[arith][f][k - 1])
    return t


# ---- timing in a fresh process -------------------------------------------------------

def time_workload(arith, k, workload, steps, warmup):
    """Stage updates per second of the loaded library on the workload."""
    import torch
    import synth
    from . import hho, solver
    tab = hho.hho_tableau_erk(4)
    # CFL-limited steps as in the benchmark: 0.9 x the ERK4 limit of the
    # stage operator on squares, and a margin below it on the right-triangle
    # grids
    if workload == "bilayer":
        w = synth.bilayer_c2(nx=1024, ny=512, k=k)
        P = solver.Problem(w["mesh"], w["media"], k)
        P.set_sources([w["source"]], [(0.0, 1.0)], 10.0)
        P.set_arithmetic(hho.HHO_F64 if arith == "f64" else hho.HHO_F32X2)
        state, work = P.empty_state(), P.work(tab)
        dt = hho.hho_cfl_dt(P.ops, {1: 0.233, 2: 0.122, 3: 0.082}[k], 0.9)
        stream = torch.cuda.current_stream()
        run = lambda n, t0: hho.hho_erk_step(P.ops, tab, t0, dt, n, state.data_ptr(), work.data_ptr(),
                                             stream.cuda_stream)
        units = P.layout.n_canonical * 4
    else:
        S = 16 if workload == "hybrid" else 32
        w = synth.hybrid_c3(S, nx=1360, ny=680, k=k) if workload == "hybrid" else \
            synth.basin_c5(nx=2860, ny=715, k=k, n_shots=S)
        P = solver.Problem(w["mesh"], w["media"], k)
        P.set_shot_sources(w["sources"], [(0.0, 1.0)] * S, w["f0"])
        prec = {"f32": hho.HHO_F32, "f64": hho.HHO_F64, "f2x": hho.HHO_F32X2}[arith]
        state, work = P.batch_buffers(4, S, prec)
        dt = hho.hho_cfl_dt(P.ops, 0.045, 0.9)
        run = lambda n, t0: P.batch_step(state, work, S, 4, t0, dt, n, precision=prec)
        units = P.layout.n_canonical * 4 * S
    run(warmup, 0.0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    run(steps, warmup * dt)
    e1.record()
    torch.cuda.synchronize()
    return units * steps / (e0.elapsed_time(e1) * 1e-3)


def measure(lib, arith, k, workload, steps, warmup):
    env = dict(os.environ, HHO_LIB=lib)
    code = ("import json, sys; from paper_2505_15771_gb300 import tune; "
            "print(json.dumps(tune.time_workload(%r, %d, %r, %d, %d)))" % (arith, k, workload, steps, warmup))
    r = subprocess.run([sys.executable, "-c", code], cwd=B.ROOT, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("timing failed for %s:\n%s" % (lib, r.stderr[-2000:]))
    return float(r.stdout.strip().splitlines()[-1])


# ---- search ----------------------------------------------------------------------------

def describe(entry):
    return " ".join("%s=%d" % (f, entry[f]) for f in FIELDS)


def tune(arith, k, workload, steps=20, warmup=3, passes=1, jobs=4, log=print, header_text=None, build_fn=None,
         measure_fn=None):
    """Coordinate descent over AXES from the table's current (arith, k)
    entry.  Returns (best entry, {(min_blocks, acc_smem, prefetch,
    rect_loop): rate}, tables).  build_fn(header_text, out_dir) -> library path and
    measure_fn(library, arith, k, workload, steps, warmup) -> rate default to
    a candidate build and a timing in a fresh process."""
    base_text = header_text if header_text is not None else open(HEADER).read()
    build_fn = build_fn or B.build_stage_variant
    measure_fn = measure_fn or measure
    tables = read_tables(base_text)
    best = {f: tables[arith][f][k - 1] for f in FIELDS}
    results = {}
    key = lambda e: tuple(e[f] for f in FIELDS)
    with tempfile.TemporaryDirectory(prefix="hho_tune_") as tmp:
        def build(entry):
            d = os.path.join(tmp, "mb%d_acc%d_pf%d_rl%d" % key(entry))
            return build_fn(write_tables(base_text, with_entry(tables, arith, k, entry)), d)

        for _ in range(passes):
            for axis in FIELDS:
                cands = [dict(best, **{axis: v}) for v in AXES[axis]]
                cands = [c for c in cands if key(c) not in results]
                with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
                    libs = list(ex.map(build, cands))
                for c, lib in zip(cands, libs):
                    results[key(c)] = measure_fn(lib, arith, k, workload, steps, warmup)
                    log("  %-52s %.4e" % (describe(c), results[key(c)]))
                best = max((dict(zip(FIELDS, kk)) for kk in results), key=lambda e: results[key(e)])
    return best, results, tables


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--arith", required=True, choices=sorted(TABLE))
    ap.add_argument("--k", type=int, required=True, choices=[1, 2, 3])
    ap.add_argument("--workload", required=True, choices=["bilayer", "hybrid", "basin"])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--passes", type=int, default=1)
    ap.add_argument("--jobs", type=int, default=4, help="candidate builds in parallel")
    ap.add_argument("--write", action="store_true", help="store the winner in csrc/stage_tuning.h")
    a = ap.parse_args(argv)
    if a.workload == "bilayer" and a.arith == "f32":
        ap.error("the bilayer workload is single-shot: FP64 or double-float")
    if a.workload != "bilayer" and a.arith != "f32":
        ap.error("the batched workloads are timed in FP32")
    print("tuning %s k=%d on %s" % (a.arith, a.k, a.workload))
    best, results, tables = tune(a.arith, a.k, a.workload, a.steps, a.warmup, a.passes, a.jobs)
    cur = {f: tables[a.arith][f][a.k - 1] for f in FIELDS}
    ck = tuple(cur[f] for f in FIELDS)
    print("current %s: %s" % (describe(cur), "%.4e" % results[ck] if ck in results else "not timed"))
    print("best    %s: %.4e" % (describe(best), results[tuple(best[f] for f in FIELDS)]))
    if a.write:
        text = write_tables(open(HEADER).read(), with_entry(tables, a.arith, a.k, best))
        with open(HEADER, "w") as f:
            f.write(text)
        print("written to", HEADER)


if __name__ == "__main__":
    main()
