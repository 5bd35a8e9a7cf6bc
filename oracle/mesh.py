"""Mesh description (Sec. 3.1 of the paper) and the canonical tables.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's mesh is a polygonal mesh aligned with the fluid/solid partition;
hanging nodes are ordinary polygon vertices (Sec. 3.1, Fig. "mesh").  Its
faces split into interior fluid faces, interior solid faces, interface faces
on Gamma, and boundary faces of each subdomain.

Canonical conventions (they have to agree bit for bit with the GPU library's
own host code, which implements them separately):

1. Faces are the edges between consecutive polygon vertices.  A face is keyed
   by the unordered pair of the two vertices' *representative* ids
   (``vertex_rep``; identity unless periodic images are identified).  Faces
   are numbered in order of first encounter, scanning cells 0..N-1 and local
   edges j = 0..nv-1 (edge j joins local vertex j to j+1).  (A periodic
   direction therefore needs at least three cells, or two distinct edges
   would share a key.)
2. A face's cell 0 is the first cell that meets it; cell 1 is the other one,
   or -1 on the boundary.
3. The face tangent runs from the endpoint with the smaller representative id
   to the one with the larger id, using cell 0's vertex coordinates; the face
   normal is n_F = (t_y, -t_x) / |t|.
4. Colours: greedy in face order, the smallest colour not used by an earlier
   face that shares a cell with this face.
5. Cell class key: (domain, number of vertices, the vertex coordinates
   relative to the centroid divided by the diameter, each multiplied by 2**40
   and rounded half-to-even).  Classes are numbered by first appearance.
6. Centroid and diameter are computed in the fixed order written below
   (relative to vertex 0, no fused multiply-add), so that two codes that
   follow this order produce identical bits.

Face types: 0 fluid interior, 1 solid interior, 2 interface (Gamma),
3 fluid boundary, 4 solid boundary.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

FLUID, SOLID = 0, 1
FT_FLUID, FT_SOLID, FT_IFACE, FT_BND_FLUID, FT_BND_SOLID = 0, 1, 2, 3, 4


def cell_geometry(px, py):
    """Area, centroid and diameter of a CCW polygon given by coordinate lists.

    Operation order is fixed (convention 6): relative coordinates d_i = p_i - p_0,
    cross_i = dx_i*dy_{i+1} - dx_{i+1}*dy_i, A2 = sum cross_i,
    cx = sum (dx_i + dx_{i+1}) * cross_i, centroid = p_0 + cx / (3*A2).
    """
    nv = len(px)
    dx = [px[i] - px[0] for i in range(nv)]
    dy = [py[i] - py[0] for i in range(nv)]
    a2 = 0.0
    cx = 0.0
    cy = 0.0
    for i in range(nv):
        j = (i + 1) % nv
        cr = dx[i] * dy[j] - dx[j] * dy[i]
        a2 = a2 + cr
        cx = cx + (dx[i] + dx[j]) * cr
        cy = cy + (dy[i] + dy[j]) * cr
    offx = cx / (3.0 * a2)
    offy = cy / (3.0 * a2)
    h = 0.0
    for i in range(nv):
        for j in range(i + 1, nv):
            ex = px[i] - px[j]
            ey = py[i] - py[j]
            d = math.sqrt(ex * ex + ey * ey)
            if d > h:
                h = d
    return 0.5 * a2, (px[0] + offx, py[0] + offy), h, (dx, dy, offx, offy)


@dataclass
class Mesh:
    xy: np.ndarray                 # (nv, 2)
    cell_ptr: np.ndarray           # (nc+1,)
    cell_vtx: np.ndarray           # concatenated CCW vertex ids
    cell_domain: np.ndarray        # (nc,) 0 fluid / 1 solid
    vertex_rep: np.ndarray         # (nv,) representative ids for face matching
    # derived
    n_cells: int = 0
    n_faces: int = 0
    face_cells: np.ndarray = None  # (nF, 2) int64, -1 on the boundary
    face_type: np.ndarray = None   # (nF,)
    face_colour: np.ndarray = None
    cell_faces: list = field(default_factory=list)   # per cell: list of face ids (local order)
    face_local: np.ndarray = None  # (nF, 2) local edge index in cell 0 / cell 1
    face_ends: np.ndarray = None   # (nF, 2, 2) endpoints (canonical orientation, cell-0 coords)
    cell_area: np.ndarray = None
    cell_centroid: np.ndarray = None
    cell_diam: np.ndarray = None
    cell_class: np.ndarray = None


def cell_vertices(mesh: Mesh, c: int) -> np.ndarray:
    return mesh.cell_vtx[mesh.cell_ptr[c]:mesh.cell_ptr[c + 1]]


def build_mesh(xy, cell_ptr, cell_vtx, cell_domain, vertex_rep=None) -> Mesh:
    """Derive faces, face types, colours, geometry and classes (conventions 1-6)."""
    xy = np.asarray(xy, dtype=np.float64)
    cell_ptr = np.asarray(cell_ptr, dtype=np.int64)
    cell_vtx = np.asarray(cell_vtx, dtype=np.int64)
    cell_domain = np.asarray(cell_domain, dtype=np.uint8)
    nv = xy.shape[0]
    rep = np.arange(nv, dtype=np.int64) if vertex_rep is None else np.asarray(vertex_rep, dtype=np.int64)
    m = Mesh(xy=xy, cell_ptr=cell_ptr, cell_vtx=cell_vtx, cell_domain=cell_domain, vertex_rep=rep)
    nc = len(cell_ptr) - 1
    m.n_cells = nc

    key_to_face = {}
    face_cells = []
    face_local = []
    face_ends = []
    cell_faces = []
    for c in range(nc):
        vs = cell_vertices(m, c)
        k = len(vs)
        faces_c = []
        for j in range(k):
            a, b = int(vs[j]), int(vs[(j + 1) % k])
            ra, rb = int(rep[a]), int(rep[b])
            key = (min(ra, rb), max(ra, rb))
            if key not in key_to_face:
                fid = len(face_cells)
                key_to_face[key] = fid
                face_cells.append([c, -1])
                face_local.append([j, -1])
                lo, hi = (a, b) if ra < rb else (b, a)
                face_ends.append([xy[lo].copy(), xy[hi].copy()])
            else:
                fid = key_to_face[key]
                if face_cells[fid][1] != -1:
                    raise ValueError("edge shared by more than two cells")
                face_cells[fid][1] = c
                face_local[fid][1] = j
            faces_c.append(fid)
        cell_faces.append(faces_c)
    m.n_faces = len(face_cells)
    m.face_cells = np.array(face_cells, dtype=np.int64).reshape(-1, 2)
    m.face_local = np.array(face_local, dtype=np.int64).reshape(-1, 2)
    m.face_ends = np.array(face_ends, dtype=np.float64).reshape(-1, 2, 2)
    m.cell_faces = cell_faces

    ft = np.empty(m.n_faces, dtype=np.int64)
    for f in range(m.n_faces):
        c0, c1 = m.face_cells[f]
        d0 = int(cell_domain[c0])
        if c1 < 0:
            ft[f] = FT_BND_FLUID if d0 == FLUID else FT_BND_SOLID
        else:
            d1 = int(cell_domain[c1])
            if d0 != d1:
                ft[f] = FT_IFACE
            else:
                ft[f] = FT_FLUID if d0 == FLUID else FT_SOLID
    m.face_type = ft

    colour = np.full(m.n_faces, -1, dtype=np.int64)
    for f in range(m.n_faces):
        used = set()
        for c in m.face_cells[f]:
            if c < 0:
                continue
            for g in cell_faces[c]:
                if g < f:
                    used.add(int(colour[g]))
        col = 0
        while col in used:
            col += 1
        colour[f] = col
    m.face_colour = colour

    area = np.empty(nc)
    cen = np.empty((nc, 2))
    diam = np.empty(nc)
    classes = np.empty(nc, dtype=np.int64)
    class_keys = {}
    for c in range(nc):
        vs = cell_vertices(m, c)
        px = [float(xy[v, 0]) for v in vs]
        py = [float(xy[v, 1]) for v in vs]
        a, (x0, y0), h, (dx, dy, offx, offy) = cell_geometry(px, py)
        if not a > 0.0:
            raise ValueError("cell %d is not counter-clockwise or is degenerate" % c)
        area[c] = a
        cen[c] = (x0, y0)
        diam[c] = h
        key = [int(cell_domain[c]), len(vs)]
        for i in range(len(vs)):
            key.append(int(round(math.ldexp((dx[i] - offx) / h, 40))))
            key.append(int(round(math.ldexp((dy[i] - offy) / h, 40))))
        key = tuple(key)
        if key not in class_keys:
            class_keys[key] = len(class_keys)
        classes[c] = class_keys[key]
    m.cell_area = area
    m.cell_centroid = cen
    m.cell_diam = diam
    m.cell_class = classes
    return m


def face_geometry(mesh: Mesh, f: int):
    """Midpoint, half-tangent (B-A)/2, length and unit normal n_F = (t_y, -t_x)."""
    a, b = mesh.face_ends[f]
    mid = 0.5 * (a + b)
    half = 0.5 * (b - a)
    length = float(np.hypot(b[0] - a[0], b[1] - a[1]))
    t = (b - a) / length
    n = np.array([t[1], -t[0]])
    return mid, half, length, n


def face_in_cell(mesh: Mesh, f: int, c: int):
    """Face f as seen from cell c: (A, B, length, n_T).

    A -> B is the canonical orientation (smaller representative id first),
    taken from cell c's own vertex coordinates (periodic images may be
    translated copies).  n_T is the unit normal pointing out of c: local edge
    j runs v_j -> v_{j+1} counter-clockwise, so the outward normal of that
    direction is (t_y, -t_x).
    """
    j = mesh.face_local[f, 0] if mesh.face_cells[f, 0] == c else mesh.face_local[f, 1]
    vs = cell_vertices(mesh, c)
    a, b = int(vs[j]), int(vs[(j + 1) % len(vs)])
    pa, pb = mesh.xy[a], mesh.xy[b]
    tc = pb - pa
    length = float(np.hypot(tc[0], tc[1]))
    n_out = np.array([tc[1], -tc[0]]) / length
    if mesh.vertex_rep[a] > mesh.vertex_rep[b]:
        pa, pb = pb, pa
    return pa.copy(), pb.copy(), length, n_out


def tables(mesh: Mesh):
    """The integer tables that the GPU library must reproduce bit for bit."""
    cfp = np.zeros(mesh.n_cells + 1, dtype=np.int64)
    for c in range(mesh.n_cells):
        cfp[c + 1] = cfp[c] + len(mesh.cell_faces[c])
    cf = np.array([f for fl in mesh.cell_faces for f in fl], dtype=np.int64)
    return {
        "face_cells": mesh.face_cells.copy(),
        "cell_faces_ptr": cfp,
        "cell_faces": cf,
        "face_type": mesh.face_type.copy(),
        "face_colour": mesh.face_colour.copy(),
        "cell_class": mesh.cell_class.copy(),
    }
