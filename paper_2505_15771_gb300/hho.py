"""Thin ctypes binding of libhho.so (declared in include/hho.h).

Argument marshalling only: every step of the path runs in the library's
kernels.  Functions keep the C names.  Device pointers are plain integers
(e.g. ``tensor.data_ptr()`` of a CUDA tensor) and streams are
``torch.cuda.Stream.cuda_stream`` integers (0 = legacy default stream).

The library must have been built in-tree (``__graft_entry__.build()`` or
``python paper_2505_15771_gb300/build.py``); loading fails loudly otherwise.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HHO_LIB names another build of the library (tune.py times its candidate
# builds this way); by default the in-tree one is loaded.
LIB_PATH = os.environ.get("HHO_LIB") or os.path.join(_HERE, "libhho.so")

HHO_F64, HHO_F32, HHO_F32X2, HHO_BF16X3 = 0, 1, 2, 3
HHO_FIELD_RICKER = 0
HHO_LAUNCH_STREAM, HHO_LAUNCH_GRAPH, HHO_LAUNCH_AUTO = 0, 1, 2
(HHO_OK, HHO_EINVAL, HHO_EMESH, HHO_EMATERIAL, HHO_EDEGREE, HHO_ECFL, HHO_EUNSTABLE, HHO_ECUDA, HHO_ENOMEM,
 HHO_ENOCONV) = range(10)


class HHOError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hho error %d: %s" % (code, msg))
        self.code = code


class MeshInfo(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("n_cells", C.c_int64), ("n_faces", C.c_int64),
                ("n_fluid_cells", C.c_int64), ("n_solid_cells", C.c_int64),
                ("n_faces_by_type", C.c_int64 * 5), ("n_classes", C.c_int32), ("n_colours", C.c_int32),
                ("max_faces_per_cell", C.c_int32), ("reserved", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("eta_f", C.c_double), ("eta_s", C.c_double), ("stab_speed", C.c_int32), ("tau_over_k", C.c_int32)]


class Layout(C.Structure):
    _fields_ = [("n_state", C.c_int64), ("n_canonical", C.c_int64), ("n_fluid_pad", C.c_int64),
                ("n_solid_pad", C.c_int64), ("n", C.c_int32), ("f", C.c_int32), ("n_classes", C.c_int32),
                ("reserved", C.c_int32)]


class Tableau(C.Structure):
    _fields_ = [("s", C.c_int32), ("reserved", C.c_int32), ("a", (C.c_double * 6) * 6), ("b", C.c_double * 6),
                ("c", C.c_double * 6)]


_P = C.c_void_p
_I32, _I64, _D = C.c_int32, C.c_int64, C.c_double
_SIGS = {
    "hho_last_error": (C.c_int, [C.c_char_p, C.c_size_t]),
    "hho_mesh_create": (C.c_int, [_P, _I64, _P, _P, _I64, _P, _P, C.POINTER(_P)]),
    "hho_mesh_query": (C.c_int, [_P, C.POINTER(MeshInfo)]),
    "hho_mesh_tables": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "hho_mesh_destroy": (None, [_P]),
    "hho_params_default": (None, [C.POINTER(Params)]),
    "hho_operators_build": (C.c_int, [_P, _I32, _P, _P, _P, _P, C.POINTER(Params), C.POINTER(_P)]),
    "hho_ops_destroy": (None, [_P]),
    "hho_operators_build_tau": (C.c_int, [_P, _I32, _P, _P, _P, _P, C.POINTER(Params), _P, C.POINTER(_P)]),
    "hho_ops_tau": (C.c_int, [_P, _P]),
    "hho_state_layout": (C.c_int, [_P, C.POINTER(Layout)]),
    "hho_state_pack": (C.c_int, [_P, _P, _P, _P]),
    "hho_state_unpack": (C.c_int, [_P, _P, _P, _P]),
    "hho_project_field": (C.c_int, [_P, _I32, _P, _I32, _P]),
    "hho_tableau_erk": (C.c_int, [_I32, C.POINTER(Tableau)]),
    "hho_work_size": (C.c_int, [_P, C.POINTER(Tableau), C.POINTER(_I64)]),
    "hho_sources_set": (C.c_int, [_P, _I32, _P, _P, _P, _P, _P]),
    "hho_sources_set_samples": (C.c_int, [_P, _I32, _P, _P, _D, _D, _I64, _I32, _P]),
    "hho_mesh_submesh": (C.c_int, [_P, _I64, _P, C.POINTER(_P)]),
    "hho_locate_points": (C.c_int, [_P, _I64, _P, _P]),
    "hho_tc_gemm_check": (C.c_int, [_I32, _I32, _P, _P, _P, _P]),
    "hho_f2x_check": (C.c_int, [_I32, _P, _P]),
    "hho_tc_error": (C.c_int, [_P, _P]),
    "hho_adjoint_work_size_f32": (C.c_int, [_P, C.POINTER(Tableau), _I64, _I64, C.POINTER(_I64)]),
    "hho_adjoint_vjp_f32": (C.c_int, [_P, C.POINTER(Tableau), _D, _D, _I64, _I64, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "hho_erk_traces": (C.c_int, [_P, C.POINTER(Tableau), _P, _P, _P]),
    "hho_erk_stage": (C.c_int, [_P, C.POINTER(Tableau), _I64, _I32, _D, _D, _P, _P, _P]),
    "hho_trace_buffer_offset": (C.c_int, [_P, C.POINTER(Tableau), _I32, C.POINTER(_I64)]),
    "hho_trace_offsets": (C.c_int, [_P, _I64, _P, _P, _P]),
    "hho_halo_gather": (C.c_int, [_P, _P, _I64, _P, _P]),
    "hho_halo_scatter": (C.c_int, [_P, _P, _I64, _P, _P]),
    "hho_ricker_samples": (C.c_int, [C.POINTER(Tableau), _D, _D, _I64, _D, _D, _D, _P]),
    "hho_erk_step": (C.c_int, [_P, C.POINTER(Tableau), _D, _D, _I64, _P, _P, _P]),
    "hho_set_arithmetic": (C.c_int, [_P, _I32]),
    "hho_set_launch_mode": (C.c_int, [_P, _I32]),
    "hho_tableau_sdirk": (C.c_int, [_I32, C.POINTER(Tableau)]),
    "hho_sdirk_work_size": (C.c_int, [_P, C.POINTER(Tableau), _I32, C.POINTER(_I64)]),
    "hho_sdirk_set_preconditioner": (C.c_int, [_P, _I32]),
    "hho_sdirk_step": (C.c_int, [_P, C.POINTER(Tableau), _D, _D, _I64, _D, _I32, _I32, _P, _P, C.POINTER(_I64),
                                 _P]),
    "hho_erk_run_host": (C.c_int, [_P, C.POINTER(Tableau), _D, _D, _I64, _P, _P]),
    "hho_apply": (C.c_int, [_P, _D, _P, _P, _P, _P]),
    "hho_receivers_set": (C.c_int, [_P, _I32, _P]),
    "hho_record": (C.c_int, [_P, _P, _P, _P]),
    "hho_energy": (C.c_int, [_P, _P, _P, C.POINTER(_D), _P]),
    "hho_cfl_dt": (C.c_int, [_P, _D, _D, C.POINTER(_D)]),
    "hho_erk_step_record": (C.c_int, [_P, C.POINTER(Tableau), _D, _D, _I64, _P, _P, _P, _P]),
    "hho_stage_cost": (C.c_int, [_P, C.POINTER(Tableau), C.POINTER(_I64), C.POINTER(_I64), C.POINTER(_I64)]),
    "hho_profile_enable": (C.c_int, [_P, _I32]),
    "hho_profile_read": (C.c_int, [_P, C.POINTER(_D), C.POINTER(_I64)]),
    "hho_energy_static": (C.c_int, [_P, _P, _P, _P]),
    "hho_cfl_bracket": (C.c_int, [_P, C.POINTER(Tableau), _P, _D, _I64, _D, _D, _I64, _P, _P, C.POINTER(_I64),
                                  C.POINTER(_I64), _P]),
    "hho_adjoint_work_size": (C.c_int, [_P, C.POINTER(Tableau), _I64, _I64, C.POINTER(_I64)]),
    "hho_adjoint_vjp": (C.c_int, [_P, C.POINTER(Tableau), _D, _D, _I64, _I64, _P, _P, _P, _I64, _P, _P, _P, _P]),
    "hho_batch_sizes": (C.c_int, [_P, C.POINTER(Tableau), _I32, _I32, C.POINTER(_I64), C.POINTER(_I64)]),
    "hho_batch_pack": (C.c_int, [_P, _I32, _I32, _P, _P, _P]),
    "hho_batch_unpack": (C.c_int, [_P, _I32, _I32, _P, _P, _P]),
    "hho_batch_sources_set": (C.c_int, [_P, _I32, _P, _P, _D, _D, _D]),
    "hho_batch_erk_step": (C.c_int, [_P, C.POINTER(Tableau), _I32, _I32, _D, _D, _I64, _P, _P, _P, _P]),
}
EXPORTED = sorted(_SIGS)

_lib = None


def lib():
    """Loads libhho.so once; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libhho.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().hho_last_error(buf, 1024)
    return buf.value.decode()


def _check(rc):
    if rc != HHO_OK:
        raise HHOError(rc, last_error())


def _ptr(a):
    """Host numpy array -> void*; ints pass through (device pointers)."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    return a.ctypes.data_as(_P)


def _arr(x, dtype):
    return np.ascontiguousarray(x, dtype=dtype)


# ---- same-named entry points ------------------------------------------------------------

def hho_mesh_create(xy, cell_ptr, cell_vtx, cell_domain, vertex_rep=None):
    xy = _arr(xy, np.float64).reshape(-1, 2)
    cp = _arr(cell_ptr, np.int64)
    cv = _arr(cell_vtx, np.int64)
    cd = _arr(cell_domain, np.uint8)
    vr = None if vertex_rep is None else _arr(vertex_rep, np.int64)
    out = _P()
    _check(lib().hho_mesh_create(_ptr(xy), xy.shape[0], _ptr(cp), _ptr(cv), len(cp) - 1, _ptr(cd), _ptr(vr),
                                 C.byref(out)))
    return out


def hho_mesh_query(mesh):
    info = MeshInfo()
    _check(lib().hho_mesh_query(mesh, C.byref(info)))
    return info


def hho_mesh_tables(mesh):
    info = hho_mesh_query(mesh)
    nc, nf = info.n_cells, info.n_faces
    face_cells = np.empty((nf, 2), np.int64)
    cfp = np.empty(nc + 1, np.int64)
    lib().hho_mesh_tables(mesh, None, _ptr(cfp), None, None, None, None)
    cf = np.empty(int(cfp[-1]), np.int64)
    ft = np.empty(nf, np.int32)
    col = np.empty(nf, np.int32)
    cls = np.empty(nc, np.int32)
    _check(lib().hho_mesh_tables(mesh, _ptr(face_cells), _ptr(cfp), _ptr(cf), _ptr(ft), _ptr(col), _ptr(cls)))
    return {"face_cells": face_cells, "cell_faces_ptr": cfp, "cell_faces": cf, "face_type": ft,
            "face_colour": col, "cell_class": cls}


def hho_mesh_destroy(mesh):
    lib().hho_mesh_destroy(mesh)


def hho_params_default():
    p = Params()
    lib().hho_params_default(C.byref(p))
    return p


def hho_operators_build(mesh, k, rho, lam, mu, kappa, params=None):
    arrs = [_arr(a, np.float64) for a in (rho, lam, mu, kappa)]
    p = hho_params_default() if params is None else params
    out = _P()
    _check(lib().hho_operators_build(mesh, int(k), *[_ptr(a) for a in arrs], C.byref(p), C.byref(out)))
    return out


def hho_operators_build_tau(mesh, k, rho, lam, mu, kappa, tau, params=None):
    arrs = [_arr(a, np.float64) for a in (rho, lam, mu, kappa)]
    t = None if tau is None else _arr(tau, np.float64)
    p = hho_params_default() if params is None else params
    out = _P()
    _check(lib().hho_operators_build_tau(mesh, int(k), *[_ptr(a) for a in arrs], C.byref(p), _ptr(t), C.byref(out)))
    return out


def hho_ops_tau(ops, n_cells):
    t = np.empty(n_cells, np.float64)
    _check(lib().hho_ops_tau(ops, _ptr(t)))
    return t


def hho_project_field(ops, kind, params):
    """Canonical FP64 vector (host) of an initial field projected onto the cell spaces."""
    lay = hho_state_layout(ops)
    out = np.empty(lay.n_canonical, np.float64)
    p = np.ascontiguousarray(params, dtype=np.float64)
    _check(lib().hho_project_field(ops, int(kind), _ptr(p), len(p), _ptr(out)))
    return out


def hho_ops_destroy(ops):
    lib().hho_ops_destroy(ops)


def hho_state_layout(ops):
    lay = Layout()
    _check(lib().hho_state_layout(ops, C.byref(lay)))
    return lay


def hho_state_pack(ops, d_canonical, d_state, stream=0):
    _check(lib().hho_state_pack(ops, d_canonical, d_state, stream))


def hho_state_unpack(ops, d_state, d_canonical, stream=0):
    _check(lib().hho_state_unpack(ops, d_state, d_canonical, stream))


def hho_tableau_erk(s):
    t = Tableau()
    _check(lib().hho_tableau_erk(int(s), C.byref(t)))
    return t


def hho_work_size(ops, tab):
    n = _I64()
    _check(lib().hho_work_size(ops, C.byref(tab), C.byref(n)))
    return n.value


def hho_sources_set(ops, xy, direction, f0, t0, amp):
    xy = _arr(xy, np.float64).reshape(-1, 2)
    d = _arr(direction, np.float64).reshape(-1, 2)
    a = [_arr(v, np.float64).reshape(-1) for v in (f0, t0, amp)]
    _check(lib().hho_sources_set(ops, xy.shape[0], _ptr(xy), _ptr(d), *[_ptr(v) for v in a]))


def hho_sources_set_samples(ops, xy, direction, t_start, dt, samples):
    """Point sources with sampled time functions; samples: [n_src, nsteps, s] (one value per step and stage)."""
    xy = _arr(xy, np.float64).reshape(-1, 2)
    d = _arr(direction, np.float64).reshape(-1, 2)
    w = _arr(samples, np.float64)
    if w.ndim != 3 or w.shape[0] != xy.shape[0]:
        raise ValueError("samples must have shape [n_src, nsteps, s]")
    _check(lib().hho_sources_set_samples(ops, xy.shape[0], _ptr(xy), _ptr(d), float(t_start), float(dt),
                                         w.shape[1], w.shape[2], _ptr(w)))


def hho_mesh_submesh(parent, cells):
    """Sub-mesh of the listed parent cells (in that order), with the parent's class geometry."""
    c = _arr(cells, np.int64)
    out = _P()
    _check(lib().hho_mesh_submesh(parent, len(c), _ptr(c), C.byref(out)))
    return out


def hho_locate_points(ops, xy):
    """Owning cell (lowest-index containing cell, input order) of every point; -1 outside."""
    p = _arr(xy, np.float64).reshape(-1, 2)
    out = np.empty(p.shape[0], np.int64)
    _check(lib().hho_locate_points(ops, p.shape[0], _ptr(p), _ptr(out)))
    return out


def hho_tc_gemm_check(A, B):
    """D = A B (A [128, K], B [K, N], float32) through the split-BF16 tcgen05 path; returns (D, status)."""
    A = _arr(A, np.float32)
    B = _arr(B, np.float32)
    D = np.zeros((128, B.shape[1]), np.float32)
    st = C.c_int32(0)
    _check(lib().hho_tc_gemm_check(int(A.shape[1]), int(B.shape[1]), _ptr(A), _ptr(B), _ptr(D), C.byref(st)))
    return D, st.value


def hho_f2x_check(pairs):
    """Double-float operations on the GPU: pairs [n, 3, 2] float32 (x, y, z as hi, lo) ->
    [n, 6, 2] float32 pairs of x+y, x-y, x*y, x*y+z, x/y, ((x z + y) z + x) z + y."""
    p = _arr(pairs, np.float32).reshape(-1, 3, 2)
    out = np.zeros((p.shape[0], 6, 2), np.float32)
    _check(lib().hho_f2x_check(int(p.shape[0]), _ptr(p), _ptr(out)))
    return out


def hho_tc_error(ops):
    """Reads and clears the tensor-core stage's error flag (1: an MMA wait gave up)."""
    v = C.c_int32(0)
    _check(lib().hho_tc_error(ops, C.byref(v)))
    return v.value


def hho_erk_traces(ops, tab, d_state, d_work, stream=0):
    _check(lib().hho_erk_traces(ops, C.byref(tab), d_state, d_work, stream))


def hho_erk_stage(ops, tab, n, j, tn, dt, d_state, d_work, stream=0):
    _check(lib().hho_erk_stage(ops, C.byref(tab), int(n), int(j), float(tn), float(dt), d_state, d_work, stream))


def hho_trace_buffer_offset(ops, tab, which):
    o = _I64()
    _check(lib().hho_trace_buffer_offset(ops, C.byref(tab), int(which), C.byref(o)))
    return o.value


def hho_trace_offsets(ops, f, cells, faces):
    """[n, 2f] offsets (within one trace buffer) of the traces each (cell, local face) publishes; -1 padded."""
    c = _arr(cells, np.int64)
    j = _arr(faces, np.int32)
    out = np.full((len(c), 2 * f), -1, np.int64)
    _check(lib().hho_trace_offsets(ops, len(c), _ptr(c), _ptr(j), _ptr(out)))
    return out


def hho_halo_gather(d_src, d_idx, n, d_dst, stream=0):
    _check(lib().hho_halo_gather(d_src, d_idx, int(n), d_dst, stream))


def hho_halo_scatter(d_src, d_idx, n, d_dst, stream=0):
    _check(lib().hho_halo_scatter(d_src, d_idx, int(n), d_dst, stream))


def hho_ricker_samples(tab, t_start, dt, nsteps, f0, t0, amp):
    """[nsteps, s] Ricker values at the tableau's stage times (the rounding of the ERK loops)."""
    out = np.zeros((int(nsteps), tab.s), np.float64)
    _check(lib().hho_ricker_samples(C.byref(tab), float(t_start), float(dt), int(nsteps), float(f0), float(t0),
                                    float(amp), _ptr(out)))
    return out


def hho_tableau_sdirk(s):
    """SDIRK tableau: s = 1, 2 (as printed), 3 (SDIRK(3,4)) or 23 (order-3 2-stage)."""
    t = Tableau()
    _check(lib().hho_tableau_sdirk(int(s), C.byref(t)))
    return t


def hho_sdirk_work_size(ops, tab, restart):
    n = _I64()
    _check(lib().hho_sdirk_work_size(ops, C.byref(tab), int(restart), C.byref(n)))
    return n.value


def hho_sdirk_set_preconditioner(ops, kind):
    """GMRES preconditioner of hho_sdirk_step: 1 block Jacobi (default), 0 none."""
    _check(lib().hho_sdirk_set_preconditioner(ops, int(kind)))


def hho_sdirk_step(ops, tab, t0, dt, nsteps, tol, restart, max_iter, d_state, d_work, stream=0):
    """Returns the number of GMRES operator applications."""
    its = _I64()
    _check(lib().hho_sdirk_step(ops, C.byref(tab), float(t0), float(dt), int(nsteps), float(tol), int(restart),
                                int(max_iter), _ptr(d_state), _ptr(d_work), C.byref(its), _ptr(stream)))
    return its.value


def hho_set_launch_mode(ops, mode):
    """HHO_LAUNCH_STREAM, HHO_LAUNCH_GRAPH or HHO_LAUNCH_AUTO (default) for the ERK loops."""
    _check(lib().hho_set_launch_mode(ops, int(mode)))


def hho_set_arithmetic(ops, arith):
    """HHO_F64 (default) or HHO_F32X2 (double-float) for the single-shot stepping calls."""
    _check(lib().hho_set_arithmetic(ops, int(arith)))


def hho_erk_step(ops, tab, t0, dt, nsteps, d_state, d_work, stream=0):
    _check(lib().hho_erk_step(ops, C.byref(tab), float(t0), float(dt), int(nsteps), d_state, d_work, stream))


def hho_erk_run_host(ops, tab, t0, dt, nsteps, h_canonical, stream=0):
    """h_canonical: numpy float64 array (or a host pointer int), updated in place."""
    _check(lib().hho_erk_run_host(ops, C.byref(tab), float(t0), float(dt), int(nsteps), _ptr(h_canonical), stream))


def hho_apply(ops, t, d_state, d_rate, d_work, stream=0):
    _check(lib().hho_apply(ops, float(t), d_state, d_rate, d_work, stream))


def hho_receivers_set(ops, xy):
    xy = _arr(xy, np.float64).reshape(-1, 2)
    _check(lib().hho_receivers_set(ops, xy.shape[0], _ptr(xy)))


def hho_record(ops, d_state, d_out, stream=0):
    _check(lib().hho_record(ops, d_state, d_out, stream))


def hho_energy(ops, d_state, d_work, stream=0):
    e = _D()
    _check(lib().hho_energy(ops, d_state, d_work, C.byref(e), stream))
    return e.value


def hho_cfl_dt(ops, cfl_star, safety=1.0):
    dt = _D()
    _check(lib().hho_cfl_dt(ops, float(cfl_star), float(safety), C.byref(dt)))
    return dt.value


def hho_erk_step_record(ops, tab, t0, dt, nsteps, d_state, d_work, d_seismogram, stream=0):
    _check(lib().hho_erk_step_record(ops, C.byref(tab), float(t0), float(dt), int(nsteps), d_state, d_work,
                                     d_seismogram, stream))


def hho_stage_cost(ops, tab):
    a, b, c = _I64(), _I64(), _I64()
    _check(lib().hho_stage_cost(ops, C.byref(tab), C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def hho_profile_enable(ops, on=True):
    _check(lib().hho_profile_enable(ops, 1 if on else 0))


def hho_profile_read(ops):
    ms, n = _D(), _I64()
    _check(lib().hho_profile_read(ops, C.byref(ms), C.byref(n)))
    return ms.value, n.value


def hho_energy_static(ops, d_state, d_energy, stream=0):
    """Energy into the device double at d_energy; the library allocates nothing."""
    _check(lib().hho_energy_static(ops, d_state, d_energy, stream))


def hho_batch_sizes(ops, tab, n_shots, precision):
    a, b = _I64(), _I64()
    _check(lib().hho_batch_sizes(ops, C.byref(tab), int(n_shots), int(precision), C.byref(a), C.byref(b)))
    return a.value, b.value


def hho_batch_pack(ops, n_shots, precision, d_canonical, d_state, stream=0):
    _check(lib().hho_batch_pack(ops, int(n_shots), int(precision), d_canonical, d_state, stream))


def hho_batch_unpack(ops, n_shots, precision, d_state, d_canonical, stream=0):
    _check(lib().hho_batch_unpack(ops, int(n_shots), int(precision), d_state, d_canonical, stream))


def hho_batch_sources_set(ops, xy, direction, f0, t0, amp=1.0):
    xy = _arr(xy, np.float64).reshape(-1, 2)
    d = _arr(direction, np.float64).reshape(-1, 2)
    _check(lib().hho_batch_sources_set(ops, xy.shape[0], _ptr(xy), _ptr(d), float(f0), float(t0), float(amp)))


def hho_batch_erk_step(ops, tab, n_shots, precision, t0, dt, nsteps, d_state, d_work, d_seismogram=None, stream=0):
    _check(lib().hho_batch_erk_step(ops, C.byref(tab), int(n_shots), int(precision), float(t0), float(dt),
                                    int(nsteps), d_state, d_work, d_seismogram, stream))


def hho_cfl_bracket(ops, tab, d_state0, T_f, N0, eps, delta, max_trials, d_state, d_work, stream=0):
    """Algorithm 1 of Sec. 5.1 on the GPU; returns (N_last_stable, N_first_unstable), -1 where absent."""
    a, b = _I64(), _I64()
    _check(lib().hho_cfl_bracket(ops, C.byref(tab), d_state0, float(T_f), int(N0), float(eps), float(delta),
                                 int(max_trials), d_state, d_work, C.byref(a), C.byref(b), stream))
    return a.value, b.value


def hho_adjoint_work_size(ops, tab, nsteps, checkpoint_every):
    n = _I64()
    _check(lib().hho_adjoint_work_size(ops, C.byref(tab), int(nsteps), int(checkpoint_every), C.byref(n)))
    return n.value


def hho_adjoint_vjp(ops, tab, t0, dt, nsteps, checkpoint_every, d_state0, d_cotangent, d_work, work_doubles,
                    n_cells, n_src=0, stream=0, with_tau=False):
    """Returns (grad_cell [n_cells, 4] = dL/d(rho, kappa, lambda, mu), grad_wavelet [nsteps, s, n_src] or None),
    and dL/dtau [n_cells] as a third value when with_tau."""
    g = np.zeros((n_cells, 4), np.float64)
    w = np.zeros((int(nsteps), tab.s, n_src), np.float64) if n_src > 0 else None
    gt = np.zeros(n_cells, np.float64) if with_tau else None
    _check(lib().hho_adjoint_vjp(ops, C.byref(tab), float(t0), float(dt), int(nsteps), int(checkpoint_every),
                                 d_state0, d_cotangent, d_work, int(work_doubles), _ptr(g),
                                 None if w is None else _ptr(w), None if gt is None else _ptr(gt), stream))
    return (g, w, gt) if with_tau else (g, w)


def hho_adjoint_work_size_f32(ops, tab, nsteps, checkpoint_every):
    n = _I64()
    _check(lib().hho_adjoint_work_size_f32(ops, C.byref(tab), int(nsteps), int(checkpoint_every), C.byref(n)))
    return n.value


def hho_adjoint_vjp_f32(ops, tab, t0, dt, nsteps, checkpoint_every, d_state0, d_cotangent, d_work, work_floats,
                        n_cells, n_src=0, stream=0, with_tau=False):
    """FP32 reverse mode (float32 state, cotangent and work); outputs as hho_adjoint_vjp."""
    g = np.zeros((n_cells, 4), np.float64)
    w = np.zeros((int(nsteps), tab.s, n_src), np.float64) if n_src > 0 else None
    gt = np.zeros(n_cells, np.float64) if with_tau else None
    _check(lib().hho_adjoint_vjp_f32(ops, C.byref(tab), float(t0), float(dt), int(nsteps), int(checkpoint_every),
                                     d_state0, d_cotangent, d_work, int(work_floats), _ptr(g),
                                     None if w is None else _ptr(w), None if gt is None else _ptr(gt), stream))
    return (g, w, gt) if with_tau else (g, w)
