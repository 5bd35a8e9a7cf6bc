"""Seeded synthetic inputs: meshes, media, sources, receivers, states.

This module holds none of the numerical method's arithmetic.  It only builds
inputs (vertex coordinates, CCW cell polygons, subdomain tags, per-cell
material arrays, point positions, random DOF vectors) that both the CPU
oracle and the GPU library consume.

Workload shapes follow the paper's academic bilayer (Sec. 5.2: fluid over
solid, flat interface) and its basin case (Sec. 5.3: water over a solid with a
sedimentary basin); the sizes are synthetic stand-ins with the paper's
shapes, because the paper's meshes, gmsh files and SEM3D traces are not
available.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

FLUID, SOLID = 0, 1


@dataclass
class MeshData:
    xy: np.ndarray          # (nv, 2) float64
    cell_ptr: np.ndarray    # (nc+1,) int64
    cell_vtx: np.ndarray    # int64, CCW
    cell_domain: np.ndarray  # (nc,) uint8
    vertex_rep: np.ndarray | None = None

    @property
    def n_cells(self):
        return len(self.cell_ptr) - 1

    def centroids_approx(self):
        """Vertex averages (only used to tag subdomains and sample media)."""
        cnt = np.diff(self.cell_ptr)
        sx = np.add.reduceat(self.xy[self.cell_vtx, 0], self.cell_ptr[:-1])
        sy = np.add.reduceat(self.xy[self.cell_vtx, 1], self.cell_ptr[:-1])
        return np.stack([sx / cnt, sy / cnt], axis=1)


def _grid_vertices(nx, ny, x0, x1, y0, y1):
    xs = x0 + (x1 - x0) * np.arange(nx + 1) / nx
    ys = y0 + (y1 - y0) * np.arange(ny + 1) / ny
    X, Y = np.meshgrid(xs, ys, indexing="xy")          # (ny+1, nx+1)
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    vid = lambda i, j: j * (nx + 1) + i
    return xy, vid


def _finish(xy, polys, y_interface, vertex_rep=None):
    cell_ptr = np.zeros(len(polys) + 1, dtype=np.int64)
    cell_ptr[1:] = np.cumsum([len(p) for p in polys])
    cell_vtx = np.array([v for p in polys for v in p], dtype=np.int64)
    md = MeshData(xy=np.asarray(xy, dtype=np.float64), cell_ptr=cell_ptr, cell_vtx=cell_vtx,
                  cell_domain=np.zeros(len(polys), dtype=np.uint8), vertex_rep=vertex_rep)
    cen = md.centroids_approx()
    md.cell_domain = np.where(cen[:, 1] < y_interface, SOLID, FLUID).astype(np.uint8)
    return md


def tri_grid(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, y_interface=0.5, periodic_x=False):
    """Squares split by the diagonal in the (1, 1) direction: 2 nx ny right triangles."""
    xy, vid = _grid_vertices(nx, ny, x0, x1, y0, y1)
    polys = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            polys.append([a, b, c])
            polys.append([a, c, d])
    rep = _periodic_rep(nx, ny, vid) if periodic_x else None
    return _finish(xy, polys, y_interface, rep)


def quad_grid(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, y_interface=0.5, periodic_x=False):
    """nx * ny axis-aligned rectangles (vertices bottom-left first, counter-clockwise)."""
    xy, vid = _grid_vertices(nx, ny, x0, x1, y0, y1)
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    a = (J * (nx + 1) + I).ravel()
    quads = np.stack([a, a + 1, a + nx + 2, a + nx + 1], axis=1)
    rep = _periodic_rep(nx, ny, vid) if periodic_x else None
    return _finish_array(xy, quads, y_interface, rep)


def hybrid_grid(nx, ny, x0, x1, y0, y1, y_split, y_interface):
    """Quads below y_split, each square split into two triangles above it
    (row by row, so cells stay in row order)."""
    xy, vid = _grid_vertices(nx, ny, x0, x1, y0, y1)
    ptr = [0]
    vtx = []
    for j in range(ny):
        yc = y0 + (y1 - y0) * (j + 0.5) / ny
        a = j * (nx + 1) + np.arange(nx)
        b, c, d = a + 1, a + nx + 2, a + nx + 1
        if yc < y_split:
            cells = np.stack([a, b, c, d], axis=1).ravel()
            vtx.append(cells)
            ptr.extend(ptr[-1] + 4 * np.arange(1, nx + 1))
        else:
            cells = np.stack([a, b, c, a, c, d], axis=1).ravel()
            vtx.append(cells)
            ptr.extend(ptr[-1] + 3 * np.arange(1, 2 * nx + 1))
    md = MeshData(xy=np.asarray(xy, dtype=np.float64), cell_ptr=np.array(ptr, dtype=np.int64),
                  cell_vtx=np.concatenate(vtx).astype(np.int64), cell_domain=None)
    md.cell_domain = np.zeros(md.n_cells, dtype=np.uint8)
    cen = md.centroids_approx()
    md.cell_domain = np.where(cen[:, 1] < y_interface, SOLID, FLUID).astype(np.uint8)
    return md


def hanging_node_patch(nx, ny, x0=0.0, x1=1.0, y0=0.0, y1=1.0, y_interface=0.5, refine_rows=(0,)):
    """Quad grid where the listed rows are refined 2x; the coarse neighbours of
    refined cells become pentagons/hexagons (hanging nodes as vertices)."""
    # Build a fine vertex lattice (2nx x 2ny) and pick the vertices each cell uses.
    fx, fy = 2 * nx, 2 * ny
    xy, vid = _grid_vertices(fx, fy, x0, x1, y0, y1)
    refined = set(refine_rows)
    polys = []
    used = set()
    for j in range(ny):
        for i in range(nx):
            if j in refined:
                for jj in range(2):
                    for ii in range(2):
                        I, J = 2 * i + ii, 2 * j + jj
                        p = [vid(I, J), vid(I + 1, J), vid(I + 1, J + 1), vid(I, J + 1)]
                        polys.append(p)
                continue
            I, J = 2 * i, 2 * j
            p = [vid(I, J)]
            if (j - 1) in refined:
                p.append(vid(I + 1, J))            # hanging node on the bottom edge
            p.append(vid(I + 2, J))
            p.append(vid(I + 2, J + 2))
            if (j + 1) in refined:
                p.append(vid(I + 1, J + 2))        # hanging node on the top edge
            p.append(vid(I, J + 2))
            polys.append(p)
    for p in polys:
        used.update(p)
    # compact the vertex numbering
    order = sorted(used)
    remap = {v: n for n, v in enumerate(order)}
    polys = [[remap[v] for v in p] for p in polys]
    return _finish(xy[order], polys, y_interface)


def _finish_array(xy, cells, y_interface, vertex_rep=None):
    nc, nvc = cells.shape
    md = MeshData(xy=np.asarray(xy, dtype=np.float64), cell_ptr=np.arange(nc + 1, dtype=np.int64) * nvc,
                  cell_vtx=cells.ravel().astype(np.int64), cell_domain=np.zeros(nc, dtype=np.uint8),
                  vertex_rep=vertex_rep)
    cen = md.centroids_approx()
    md.cell_domain = np.where(cen[:, 1] < y_interface, SOLID, FLUID).astype(np.uint8)
    return md


def _periodic_rep(nx, ny, vid):
    rep = np.arange((nx + 1) * (ny + 1), dtype=np.int64)
    for j in range(ny + 1):
        rep[vid(nx, j)] = vid(0, j)
    return rep


# ---- media -------------------------------------------------------------------

def lame_from_speeds(rho, vp, vs):
    mu = rho * vs * vs
    lam = rho * vp * vp - 2.0 * mu
    return lam, mu


def layered_media(md: MeshData, fluid=(1.0, 1.5), solid=(2.5, 3.0, 1.7)):
    """Per-cell (rho, lam, mu, kappa): homogeneous fluid (rho, c) over solid (rho, vp, vs)."""
    fl = md.cell_domain == FLUID
    ls, ms = lame_from_speeds(solid[0], solid[1], solid[2])
    rho = np.where(fl, fluid[0], solid[0]).astype(np.float64)
    kappa = np.where(fl, fluid[0] * fluid[1] ** 2, 0.0)
    lam = np.where(fl, 0.0, ls)
    mu = np.where(fl, 0.0, ms)
    return rho, lam, mu, kappa


def gaussian_random_field(seed, x0, x1, y0, y1, corr=0.05, spacing=1.0 / 256):
    """Seeded white noise on a grid convolved with a Gaussian (std ``corr``),
    normalised to max |g| = 1.  Returns a sampler g(x, y) (nearest grid point)."""
    rng = np.random.default_rng(seed)
    nx = int(round((x1 - x0) / spacing)) + 1
    ny = int(round((y1 - y0) / spacing)) + 1
    noise = rng.standard_normal((ny, nx))
    kx = np.fft.fftfreq(nx, d=spacing)
    ky = np.fft.fftfreq(ny, d=spacing)
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    filt = np.exp(-2.0 * (np.pi * corr) ** 2 * (KX ** 2 + KY ** 2))
    g = np.real(np.fft.ifft2(np.fft.fft2(noise) * filt))
    g /= np.max(np.abs(g))

    def sample(x, y):
        i = np.clip(np.rint((np.asarray(x) - x0) / spacing).astype(int), 0, nx - 1)
        j = np.clip(np.rint((np.asarray(y) - y0) / spacing).astype(int), 0, ny - 1)
        return g[j, i]
    return sample


def random_field_media(md: MeshData, seeds=(1, 2), base=(2.5, 3.0, 1.7), amp=0.2,
                       fluid=(1.0, 1.5), box=(0.0, 2.0, 0.0, 1.0)):
    """Solid: vp, vs share field g1 (keeps vp/vs fixed, lambda > 0), rho uses g2;
    value = base * (1 + amp * g).  Fluid: homogeneous water (rho, c)."""
    g1 = gaussian_random_field(seeds[0], *box)
    g2 = gaussian_random_field(seeds[1], *box)
    cen = md.centroids_approx()
    a = g1(cen[:, 0], cen[:, 1])
    b = g2(cen[:, 0], cen[:, 1])
    fl = md.cell_domain == FLUID
    r = base[0] * (1.0 + amp * b)
    vp = base[1] * (1.0 + amp * a)
    vs = base[2] * (1.0 + amp * a)
    ls, ms = lame_from_speeds(r, vp, vs)
    rho = np.where(fl, fluid[0], r)
    kappa = np.where(fl, fluid[0] * fluid[1] ** 2, 0.0)
    lam = np.where(fl, 0.0, ls)
    mu = np.where(fl, 0.0, ms)
    return rho, lam, mu, kappa


# ---- points and states -----------------------------------------------------------

def seeded_point(seed, x0, x1, y0, y1, margin=0.05):
    rng = np.random.default_rng(seed)
    return (x0 + margin + (x1 - x0 - 2 * margin) * rng.random(),
            y0 + margin + (y1 - y0 - 2 * margin) * rng.random())


def receivers_on_line(n, x0, x1, y):
    """n points evenly inside (x0, x1) at height y: x = x0 + (i + 1/2)(x1 - x0)/n."""
    return [(x0 + (i + 0.5) * (x1 - x0) / n, y) for i in range(n)]


def random_state(n_values, seed):
    """Seeded standard-normal DOF vector (canonical layout)."""
    return np.random.default_rng(seed).standard_normal(n_values)


def ricker(t, f0, t0=None, amp=1.0):
    """Ricker wavelet w(t) = amp (1 - 2 pi^2 f0^2 (t-t0)^2) exp(-pi^2 f0^2 (t-t0)^2), t0 = 1/f0."""
    t0 = 1.0 / f0 if t0 is None else t0
    a = (np.pi * f0 * (t - t0)) ** 2
    return amp * (1.0 - 2.0 * a) * np.exp(-a)


# ---- the named workloads ----------------------------------------------------------

def academic_c1():
    """512 right triangles on the unit square, solid below y = 0.5 (rho 2.5,
    vp 3.0, vs 1.7), water above (rho 1, c 1.5); k = 1, ERK4, 200 steps,
    Ricker f0 = 10 point force (e_y) at a seeded solid point, 8 receivers on
    the interface y = 0.5."""
    md = tri_grid(16, 16)
    media = layered_media(md)
    src = seeded_point(0, 0.0, 1.0, 0.0, 0.5)
    rec = receivers_on_line(8, 0.0, 1.0, 0.5)
    return dict(mesh=md, media=media, k=1, tableau="erk4", nsteps=200, cfl_star=0.265,
                h=1.0 / 16, c_max=3.0, source=src, f0=10.0, receivers=rec)


def hybrid_c3(n_shots, nx=1360, ny=680, k=3):
    """[0,2]x[0,1]: squares below y = 0.7, each split into two triangles above
    (647,360 quads + 554,880 triangles at 1360x680); solid below y = 0.5 with
    the seeded random field (seeds 1, 2), water above; n_shots Ricker point
    forces at seeded solid points (seed 100 + shot); 256 receivers at y = 0.75."""
    md = hybrid_grid(nx, ny, 0.0, 2.0, 0.0, 1.0, 0.7, 0.5)
    media = random_field_media(md, seeds=(1, 2))
    srcs = [seeded_point(100 + s, 0.0, 2.0, 0.0, 0.5) for s in range(n_shots)]
    rec = receivers_on_line(256, 0.0, 2.0, 0.75)
    return dict(mesh=md, media=media, k=k, sources=srcs, f0=10.0, receivers=rec, h=1.0 / ny)


def gaussian_anomaly(md: MeshData, centre, radius, amplitude):
    """Per-cell multiplicative factor 1 + amplitude exp(-|x - centre|^2 / radius^2)."""
    cen = md.centroids_approx()
    r2 = (cen[:, 0] - centre[0]) ** 2 + (cen[:, 1] - centre[1]) ** 2
    return 1.0 + amplitude * np.exp(-r2 / radius ** 2)


def adjoint_c4(n=256, k=2, n_shots=8, n_rec=128):
    """Two-layer medium on [0,1]^2, 256 x 256 quads, solid below y = 0.5
    (rho 2.5, vp 3.0, vs 1.7), water above (rho 1, c 1.5).  The true model has
    a +10 % Gaussian anomaly in v_S (radius 0.06) at a seeded solid point
    (seed 4, y in [0.3, 0.45]); the current model is the smooth background.
    n_shots Ricker point forces (f0 = 30) at seeded solid points (seeds 5,
    6, ...; y in [0.3, 0.45]) and n_rec receivers on the interface y = 0.5,
    so that 800 CFL-limited steps (t = 0.11) record the scattered field."""
    md = quad_grid(n, n, 0.0, 1.0, 0.0, 1.0, 0.5)
    bg = layered_media(md)
    c = seeded_point(4, 0.2, 0.8, 0.3, 0.45, margin=0.0)
    f = gaussian_anomaly(md, c, 0.06, 0.10)
    rho = bg[0]
    sol = md.cell_domain == SOLID
    vp = np.where(sol, 3.0, 0.0)
    vs = np.where(sol, 1.7 * f, 0.0)
    lam_t, mu_t = lame_from_speeds(rho, vp, vs)
    true = (rho, np.where(sol, lam_t, 0.0), np.where(sol, mu_t, 0.0), bg[3])
    srcs = [seeded_point(5 + s, 0.05, 0.95, 0.3, 0.45, margin=0.0) for s in range(n_shots)]
    rec = receivers_on_line(n_rec, 0.0, 1.0, 0.5)
    return dict(mesh=md, true=true, background=bg, k=k, sources=srcs, receivers=rec, f0=30.0, anomaly_centre=c)


# Boundary slots of a coarse cell on the 4x finer lattice, counter-clockwise
# from the bottom-left corner: corners 0, 4, 8, 12; slots 1-3 bottom, 5-7
# right, 9-11 top, 13-15 left (the possible hanging nodes).
_SLOT_OFF = np.array([(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (4, 1), (4, 2), (4, 3),
                      (4, 4), (3, 4), (2, 4), (1, 4), (0, 4), (0, 3), (0, 2), (0, 1)], dtype=np.int64)
_SLOT_SIDE = np.array([-1, 0, 0, 0, -1, 1, 1, 1, -1, 2, 2, 2, -1, 3, 3, 3])
# slot lists of the polygons a coarse cell can become
_POLY_SLOTS = {
    "quad": list(range(16)),
    "tri_d0_a": [0, 1, 2, 3, 4, 5, 6, 7, 8],          # split along bottom-left -> top-right
    "tri_d0_b": [0, 8, 9, 10, 11, 12, 13, 14, 15],
    "tri_d1_a": [0, 1, 2, 3, 4, 12, 13, 14, 15],      # split along bottom-right -> top-left
    "tri_d1_b": [4, 5, 6, 7, 8, 9, 10, 11, 12],
}


def basin_floor(seed, xa, xb, n_ctrl=7, dmin=0.3, dmax=0.8):
    """Seeded basin depth d(x) >= 0: a clamped cubic spline through n_ctrl
    equally spaced control points on [xa, xb] (zero at both ends, interior
    depths uniform in [dmin, dmax]); zero outside (xa, xb)."""
    from scipy.interpolate import CubicSpline
    rng = np.random.default_rng(seed)
    xc = np.linspace(xa, xb, n_ctrl)
    dc = np.concatenate([[0.0], dmin + (dmax - dmin) * rng.random(n_ctrl - 2), [0.0]])
    cs = CubicSpline(xc, dc, bc_type="clamped")

    def depth(x):
        x = np.asarray(x, dtype=np.float64)
        d = np.where((x > xa) & (x < xb), cs(np.clip(x, xa, xb)), 0.0)
        return np.maximum(d, 0.0)
    return depth


def basin_mesh(nx, ny, x0, x1, y0, y1, y_sea, depth):
    """Coarse nx x ny squares; those whose centre lies in the basin
    (y_sea - depth(x) < y < y_sea) are refined 4 x 4; their unrefined
    neighbours keep the shared sides' 3 hanging nodes as vertices (7- to
    13-vertex polygons); unrefined solid cells crossed by the basin floor are
    split into two triangles (diagonal along the floor's slope), hanging nodes
    included.  Cells: plain/hanging coarse cells row by row, then the
    triangles, then the fine squares in fine-lattice row order."""
    hx, hy = (x1 - x0) / nx, (y1 - y0) / ny
    FX = 4 * nx + 1
    J, I = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    xl, yb = x0 + I * hx, y0 + J * hy
    xc, yc = xl + 0.5 * hx, yb + 0.5 * hy
    floor_c = y_sea - depth(xc)
    refined = (depth(xc) > 0) & (yc > floor_c) & (yc < y_sea)
    fl, fm, fr = y_sea - depth(xl), floor_c, y_sea - depth(xl + hx)
    lo = np.minimum(np.minimum(fl, fm), fr)
    hi = np.maximum(np.maximum(fl, fm), fr)
    touches = (depth(xl) > 0) | (depth(xc) > 0) | (depth(xl + hx) > 0)
    split = ~refined & touches & (yb + hy <= y_sea) & (lo < yb + hy) & (hi > yb)
    diag1 = (fr - fl) < 0            # floor rising to the left: split bottom-right -> top-left
    pad = np.zeros((ny + 2, nx + 2), dtype=bool)
    pad[1:-1, 1:-1] = refined
    hang = np.stack([pad[:-2, 1:-1], pad[1:-1, 2:], pad[2:, 1:-1], pad[1:-1, :-2]], axis=-1) & ~refined[..., None]
    # fine-lattice vertex ids of each coarse cell's 16 boundary slots
    base = (4 * J)[..., None] * FX + (4 * I)[..., None]
    slot_vid = base + _SLOT_OFF[:, 1] * FX + _SLOT_OFF[:, 0]          # (ny, nx, 16)
    slot_on = np.where(_SLOT_SIDE < 0, True, False)[None, None, :] | \
        np.take_along_axis(hang, np.clip(_SLOT_SIDE, 0, 3)[None, None, :].repeat(ny, 0).repeat(nx, 1), axis=2) & \
        (_SLOT_SIDE >= 0)[None, None, :]
    ptr_parts, vtx_parts = [], []

    def emit(mask_cells, slots):
        sv = slot_vid[mask_cells][:, slots]
        so = slot_on[mask_cells][:, slots]
        ptr_parts.append(so.sum(axis=1))
        vtx_parts.append(sv[so])

    emit(~refined & ~split, _POLY_SLOTS["quad"])
    if split.any():
        # the two triangles of each split cell, in cell order
        for a_key, b_key, m in (("tri_d0_a", "tri_d0_b", split & ~diag1), ("tri_d1_a", "tri_d1_b", split & diag1)):
            if not m.any():
                continue
            sa, sb = _POLY_SLOTS[a_key], _POLY_SLOTS[b_key]
            va, oa = slot_vid[m][:, sa], slot_on[m][:, sa]
            vb, ob = slot_vid[m][:, sb], slot_on[m][:, sb]
            cnt = np.stack([oa.sum(1), ob.sum(1)], axis=1).ravel()
            v = np.concatenate([va, vb], axis=1)
            o = np.concatenate([oa, ob], axis=1)
            ptr_parts.append(cnt)
            vtx_parts.append(v[o])
    # fine squares of the refined cells, fine-lattice row order
    fJ, fI = np.nonzero(np.repeat(np.repeat(refined, 4, axis=0), 4, axis=1))
    a = fJ.astype(np.int64) * FX + fI
    ptr_parts.append(np.full(len(a), 4))
    vtx_parts.append(np.stack([a, a + 1, a + FX + 1, a + FX], axis=1).ravel())
    counts = np.concatenate(ptr_parts).astype(np.int64)
    vtx = np.concatenate(vtx_parts).astype(np.int64)
    used, inv = np.unique(vtx, return_inverse=True)
    xy = np.stack([x0 + (used % FX) * (hx / 4), y0 + (used // FX) * (hy / 4)], axis=1)
    cell_ptr = np.zeros(len(counts) + 1, dtype=np.int64)
    cell_ptr[1:] = np.cumsum(counts)
    md = MeshData(xy=xy, cell_ptr=cell_ptr, cell_vtx=inv.astype(np.int64), cell_domain=np.zeros(len(counts), np.uint8))
    cen = md.centroids_approx()
    md.cell_domain = np.where(cen[:, 1] < y_sea, SOLID, FLUID).astype(np.uint8)
    return md


def basin_c5(nx=2860, ny=715, k=2, n_shots=32, n_rec=512):
    """A 20 x 5 km section (units km, s): water (rho 1.0, c 1.5) above the
    seabed y = 4, bedrock below (rho 2.7, vp 5.5, vs 3.2) holding a
    sedimentary basin between x = 6 and 14 km whose floor is a seeded spline
    (seed 8, depth 0.3-0.8 km).  Basin media grow linearly with the relative
    depth z in [0, 1] below the seabed: vs 0.4 + 0.4 z, vp 1.6 + 0.4 z,
    rho 1.8 + 0.3 z.  Mesh: basin_mesh on nx x ny squares (2860 x 715: about
    3.3 M cells).  n_shots Ricker point forces (f0 = 15 Hz) at seeded solid
    points (seed 9) with x in [4, 16], y in [3.2, 3.95]; n_rec receivers on the
    seabed."""
    x0, x1, y0, y1, y_sea = 0.0, 20.0, 0.0, 5.0, 4.0
    depth = basin_floor(8, 6.0, 14.0)
    md = basin_mesh(nx, ny, x0, x1, y0, y1, y_sea, depth)
    cen = md.centroids_approx()
    d = depth(cen[:, 0])
    sol = md.cell_domain == SOLID
    in_basin = sol & (d > 0) & (cen[:, 1] > y_sea - d)
    z = np.clip((y_sea - cen[:, 1]) / np.where(d > 0, d, 1.0), 0.0, 1.0)
    rho = np.where(sol, np.where(in_basin, 1.8 + 0.3 * z, 2.7), 1.0)
    vp = np.where(in_basin, 1.6 + 0.4 * z, 5.5)
    vs = np.where(in_basin, 0.4 + 0.4 * z, 3.2)
    ls, ms = lame_from_speeds(rho, vp, vs)
    lam = np.where(sol, ls, 0.0)
    mu = np.where(sol, ms, 0.0)
    kappa = np.where(sol, 0.0, 1.0 * 1.5 ** 2)
    rng = np.random.default_rng(9)
    srcs = [(4.0 + 12.0 * rng.random(), 3.2 + 0.75 * rng.random()) for _ in range(n_shots)]
    rec = receivers_on_line(n_rec, x0, x1, y_sea)
    return dict(mesh=md, media=(rho, lam, mu, kappa), k=k, sources=srcs, f0=15.0, receivers=rec,
                in_basin=in_basin, depth=depth)


def ricker_academic(n=64, k=2):
    """Sec. 5.2.1 (academic properties): L = H = 1, fluid (rho 1, c_P 1) over
    solid (rho 1, c_P sqrt 3, c_S 1), so lambda = mu = kappa = 1; n x n
    squares.  The paper puts the pulse at x_c = 0 and the interface sensor at
    x = -0.3, so the domain is read as x in (-L/2, L/2): fluid y in (0, 0.5),
    solid y in (-0.5, 0).  Initial Ricker pulse on m (Eq. ricker_ic) at
    (0, 0.125) with theta = 1, lambda = c_P^f / f_c = 0.1 (f_c = 10); no
    source term; T_f = 1.  Sensors S^f, S^s read off the figure of the
    domain, S^i = (-0.3, 0) from the text."""
    md = quad_grid(n, n, -0.5, 0.5, -0.5, 0.5, y_interface=0.0)
    sol = md.cell_domain == SOLID
    nc = md.n_cells
    rho = np.ones(nc)
    lam = np.where(sol, 1.0, 0.0)     # rho (c_P^2 - 2 c_S^2) = 3 - 2
    mu = np.where(sol, 1.0, 0.0)
    kappa = np.where(sol, 0.0, 1.0)
    return dict(mesh=md, media=(rho, lam, mu, kappa), k=k, pulse=(0.0, 0.125, 1.0, 0.1),
                sensors=[(-0.25, 0.15), (-0.25, -0.25), (-0.3, 0.0)], T_f=1.0, c_max=np.sqrt(3.0), h=1.0 / n)


def granite_water(h=0.025, k=2):
    """Sec. 5.2.2 (granite under water) in km, s and g/cm^3: L = 3.8, fluid
    height 1 (rho 1.025, c_P 1.5), solid height 1.6 (rho 2.69, c_P 6, c_S 3),
    domain x in (-1.9, 1.9), y in (-1.6, 1); squares of side h (25 m: the
    paper's 23.6 m does not divide the layer heights).  Pulse on m (Eq.
    ricker_ic) at (0, 0.2) with theta = 1, lambda = 1.5 / 10 = 0.15;
    T_f = 0.5.  Sensors S^f = (-0.5, 0.2), S^s = (-1.0, -0.5) and
    S^i = (-0.4, 0) as printed with the run's sensor table."""
    nx, ny = int(round(3.8 / h)), int(round(2.6 / h))
    md = quad_grid(nx, ny, -1.9, 1.9, -1.6, 1.0, y_interface=0.0)
    sol = md.cell_domain == SOLID
    rho = np.where(sol, 2.69, 1.025)
    ls, ms = lame_from_speeds(2.69, 6.0, 3.0)
    lam = np.where(sol, ls, 0.0)
    mu = np.where(sol, ms, 0.0)
    kappa = np.where(sol, 0.0, 1.025 * 1.5 ** 2)
    return dict(mesh=md, media=(rho, lam, mu, kappa), k=k, pulse=(0.0, 0.2, 1.0, 0.15),
                sensors=[(-0.5, 0.2), (-1.0, -0.5), (-0.4, 0.0)], T_f=0.5, c_max=6.0, h=h)


def bilayer_c2(nx=1024, ny=512, k=2):
    """[0,2]x[0,1] quads, solid below y = 0.5 with a seeded +-20 % random field
    (vp, vs share g1 seed 1, rho g2 seed 2), water above; 256 receivers at y = 0.75."""
    md = quad_grid(nx, ny, 0.0, 2.0, 0.0, 1.0, 0.5)
    media = random_field_media(md, seeds=(1, 2))
    src = seeded_point(3, 0.0, 2.0, 0.0, 0.5)
    rec = receivers_on_line(256, 0.0, 2.0, 0.75)
    return dict(mesh=md, media=media, k=k, source=src, f0=10.0, receivers=rec,
                h=1.0 / ny, c_max=float(np.sqrt((media[1] + 2 * media[2]) / media[0]).max()))
