"""Test helpers: build the library if needed, and run the oracle on synth meshes."""
import os
import threading

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_lock = threading.Lock()


def ensure_built():
    from paper_2505_15771_gb300 import build, hho
    with _lock:
        if not os.path.exists(hho.LIB_PATH):
            build.build()
    return hho


def oracle_system(md, k, media, **kw):
    from oracle import assemble as A
    from oracle import mesh as M
    m = M.build_mesh(md.xy, md.cell_ptr, md.cell_vtx, md.cell_domain, md.vertex_rep)
    return A.System(m, k, *media, **kw)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))
