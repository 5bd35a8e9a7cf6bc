// Mesh construction (Sec. 3.1): faces, face sets, colours, cell classes.
//
// Canonical rules (documented in hho.h) are implemented here on their own;
// this file must be compiled without floating-point contraction
// (-ffp-contract=off) so that centroids, diameters and class keys are the
// same bits on every host.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>

#include "hho_internal.h"

static thread_local char g_err[512];

void hho_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" int hho_last_error(char* buf, size_t len) {
    size_t n = strlen(g_err);
    if (buf && len > 0) {
        size_t m = n < len - 1 ? n : len - 1;
        memcpy(buf, g_err, m);
        buf[m] = 0;
    }
    return (int)n;
}

namespace {

struct PairHash {
    size_t operator()(const std::pair<int64_t, int64_t>& p) const {
        uint64_t h = (uint64_t)p.first * 0x9E3779B97F4A7C15ull;
        h ^= (uint64_t)p.second + 0x632BE59BD9B4E019ull + (h << 6) + (h >> 2);
        return (size_t)h;
    }
};

// Area, centroid and diameter of a CCW polygon in the fixed operation order:
// d_i = p_i - p_0; cross_i = dx_i dy_{i+1} - dx_{i+1} dy_i; A2 = sum cross_i;
// cx = sum (dx_i + dx_{i+1}) cross_i; centroid = p_0 + cx / (3 A2);
// diameter = max_{i<j} sqrt(ex*ex + ey*ey).
struct Geo {
    double area, cx, cy, h, offx, offy;
    std::vector<double> dx, dy;
};

Geo polygon_geometry(const double* px, const double* py, int nv) {
    Geo g;
    g.dx.resize(nv);
    g.dy.resize(nv);
    for (int i = 0; i < nv; ++i) {
        g.dx[i] = px[i] - px[0];
        g.dy[i] = py[i] - py[0];
    }
    double a2 = 0.0, cx = 0.0, cy = 0.0;
    for (int i = 0; i < nv; ++i) {
        int j = (i + 1) % nv;
        double t1 = g.dx[i] * g.dy[j];
        double t2 = g.dx[j] * g.dy[i];
        double cr = t1 - t2;
        a2 = a2 + cr;
        cx = cx + (g.dx[i] + g.dx[j]) * cr;
        cy = cy + (g.dy[i] + g.dy[j]) * cr;
    }
    g.offx = cx / (3.0 * a2);
    g.offy = cy / (3.0 * a2);
    g.area = 0.5 * a2;
    g.cx = px[0] + g.offx;
    g.cy = py[0] + g.offy;
    double h = 0.0;
    for (int i = 0; i < nv; ++i)
        for (int j = i + 1; j < nv; ++j) {
            double ex = px[i] - px[j];
            double ey = py[i] - py[j];
            double d = std::sqrt(ex * ex + ey * ey);
            if (d > h) h = d;
        }
    g.h = h;
    return g;
}

}  // namespace

extern "C" int hho_mesh_create(const double* h_xy, int64_t n_vertices, const int64_t* h_cell_ptr,
                               const int64_t* h_cell_vtx, int64_t n_cells, const uint8_t* h_cell_domain,
                               const int64_t* h_vertex_rep, hho_mesh** out) {
    if (!h_xy || !h_cell_ptr || !h_cell_vtx || !h_cell_domain || !out || n_vertices <= 0 || n_cells <= 0) {
        hho_set_error("hho_mesh_create: null pointer or non-positive size");
        return HHO_EINVAL;
    }
    *out = nullptr;
    if (n_cells > (int64_t)1 << 30 || n_vertices > (int64_t)1 << 40) {
        hho_set_error("hho_mesh_create: mesh too large");
        return HHO_EINVAL;
    }
    hho_mesh* m = new (std::nothrow) hho_mesh();
    if (!m) {
        hho_set_error("hho_mesh_create: out of host memory");
        return HHO_ENOMEM;
    }
    m->nv = n_vertices;
    m->nc = n_cells;
    m->xy.assign(h_xy, h_xy + 2 * n_vertices);
    m->cell_ptr.assign(h_cell_ptr, h_cell_ptr + n_cells + 1);
    if (m->cell_ptr[0] != 0) {
        hho_set_error("hho_mesh_create: cell_ptr[0] must be 0");
        delete m;
        return HHO_EINVAL;
    }
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t k = m->cell_ptr[c + 1] - m->cell_ptr[c];
        if (k < 3) {
            hho_set_error("hho_mesh_create: cell %lld has %lld vertices (< 3)", (long long)c, (long long)k);
            delete m;
            return HHO_EMESH;
        }
        if (k > 32) {
            hho_set_error("hho_mesh_create: cell %lld has %lld vertices (> 32)", (long long)c, (long long)k);
            delete m;
            return HHO_EMESH;
        }
    }
    int64_t nvtx = m->cell_ptr[n_cells];
    m->cell_vtx.assign(h_cell_vtx, h_cell_vtx + nvtx);
    for (int64_t i = 0; i < nvtx; ++i)
        if (m->cell_vtx[i] < 0 || m->cell_vtx[i] >= n_vertices) {
            hho_set_error("hho_mesh_create: vertex id %lld out of range", (long long)m->cell_vtx[i]);
            delete m;
            return HHO_EINVAL;
        }
    m->domain.assign(h_cell_domain, h_cell_domain + n_cells);
    for (int64_t c = 0; c < n_cells; ++c)
        if (m->domain[c] > 1) {
            hho_set_error("hho_mesh_create: cell %lld has domain %d (must be 0 or 1)", (long long)c, (int)m->domain[c]);
            delete m;
            return HHO_EINVAL;
        }
    m->rep.resize(n_vertices);
    for (int64_t v = 0; v < n_vertices; ++v) {
        m->rep[v] = h_vertex_rep ? h_vertex_rep[v] : v;
        if (m->rep[v] < 0 || m->rep[v] >= n_vertices) {
            hho_set_error("hho_mesh_create: vertex_rep[%lld] out of range", (long long)v);
            delete m;
            return HHO_EINVAL;
        }
    }

    // Rule 1-2: faces by first encounter, keyed by representative pairs.
    std::unordered_map<std::pair<int64_t, int64_t>, int64_t, PairHash> key_to_face;
    key_to_face.reserve((size_t)(nvtx));
    m->cell_faces.resize(nvtx);
    m->face_cells.reserve(nvtx + 16);
    m->face_local.reserve(nvtx + 16);
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t b = m->cell_ptr[c];
        int64_t k = m->cell_ptr[c + 1] - b;
        if (k > m->max_nf) m->max_nf = (int32_t)k;
        for (int64_t j = 0; j < k; ++j) {
            int64_t va = m->cell_vtx[b + j], vb = m->cell_vtx[b + (j + 1) % k];
            int64_t ra = m->rep[va], rb = m->rep[vb];
            if (ra == rb) {
                hho_set_error("hho_mesh_create: cell %lld has a zero-length edge", (long long)c);
                delete m;
                return HHO_EMESH;
            }
            std::pair<int64_t, int64_t> key(ra < rb ? ra : rb, ra < rb ? rb : ra);
            auto it = key_to_face.find(key);
            int64_t fid;
            if (it == key_to_face.end()) {
                fid = (int64_t)(m->face_cells.size() / 2);
                key_to_face.emplace(key, fid);
                m->face_cells.push_back(c);
                m->face_cells.push_back(-1);
                m->face_local.push_back((int32_t)j);
                m->face_local.push_back(-1);
            } else {
                fid = it->second;
                if (m->face_cells[2 * fid + 1] != -1) {
                    hho_set_error("hho_mesh_create: an edge of cell %lld is shared by more than two cells", (long long)c);
                    delete m;
                    return HHO_EMESH;
                }
                if (m->face_cells[2 * fid] == c) {
                    hho_set_error("hho_mesh_create: cell %lld meets itself across an edge", (long long)c);
                    delete m;
                    return HHO_EMESH;
                }
                m->face_cells[2 * fid + 1] = c;
                m->face_local[2 * fid + 1] = (int32_t)j;
            }
            m->cell_faces[b + j] = fid;
        }
    }
    m->nf = (int64_t)(m->face_cells.size() / 2);

    // Face types.
    m->face_type.resize(m->nf);
    for (int64_t F = 0; F < m->nf; ++F) {
        int64_t c0 = m->face_cells[2 * F], c1 = m->face_cells[2 * F + 1];
        int d0 = m->domain[c0];
        if (c1 < 0)
            m->face_type[F] = d0 == 0 ? FT_BND_FLUID : FT_BND_SOLID;
        else if (m->domain[c1] != d0)
            m->face_type[F] = FT_IFACE;
        else
            m->face_type[F] = d0 == 0 ? FT_FLUID : FT_SOLID;
    }

    // Rule 4: greedy colouring in face order.
    m->face_colour.assign(m->nf, -1);
    std::vector<int32_t> used;
    for (int64_t F = 0; F < m->nf; ++F) {
        used.clear();
        for (int s = 0; s < 2; ++s) {
            int64_t c = m->face_cells[2 * F + s];
            if (c < 0) continue;
            for (int64_t i = m->cell_ptr[c]; i < m->cell_ptr[c + 1]; ++i) {
                int64_t G = m->cell_faces[i];
                if (G < F) used.push_back(m->face_colour[G]);
            }
        }
        int32_t col = 0;
        for (;;) {
            bool taken = false;
            for (int32_t u : used)
                if (u == col) { taken = true; break; }
            if (!taken) break;
            ++col;
        }
        m->face_colour[F] = col;
        if (col + 1 > m->n_colours) m->n_colours = col + 1;
    }

    // Geometry and rule 5: classes.
    m->centroid.resize(2 * n_cells);
    m->diam.resize(n_cells);
    m->area.resize(n_cells);
    m->cell_class.resize(n_cells);
    std::map<std::vector<int64_t>, int32_t> class_of_key;
    std::vector<double> px, py;
    std::vector<int64_t> key;
    for (int64_t c = 0; c < n_cells; ++c) {
        int64_t b = m->cell_ptr[c];
        int nv = (int)(m->cell_ptr[c + 1] - b);
        px.resize(nv);
        py.resize(nv);
        for (int i = 0; i < nv; ++i) {
            px[i] = m->xy[2 * m->cell_vtx[b + i]];
            py[i] = m->xy[2 * m->cell_vtx[b + i] + 1];
        }
        Geo g = polygon_geometry(px.data(), py.data(), nv);
        if (!(g.area > 0.0)) {
            hho_set_error("hho_mesh_create: cell %lld is clockwise or degenerate (area %g)", (long long)c, g.area);
            delete m;
            return HHO_EMESH;
        }
        m->area[c] = g.area;
        m->centroid[2 * c] = g.cx;
        m->centroid[2 * c + 1] = g.cy;
        m->diam[c] = g.h;
        key.assign({(int64_t)m->domain[c], (int64_t)nv});
        for (int i = 0; i < nv; ++i) {
            double rx = (g.dx[i] - g.offx) / g.h;
            double ry = (g.dy[i] - g.offy) / g.h;
            key.push_back((int64_t)std::nearbyint(std::ldexp(rx, 40)));
            key.push_back((int64_t)std::nearbyint(std::ldexp(ry, 40)));
        }
        auto it = class_of_key.find(key);
        if (it == class_of_key.end()) {
            int32_t id = (int32_t)class_of_key.size();
            class_of_key.emplace(key, id);
            m->class_first.push_back(c);
            m->cell_class[c] = id;
            m->class_ref_off.push_back((int64_t)m->class_ref.size());
            for (int i = 0; i < nv; ++i) {
                m->class_ref.push_back((px[i] - g.cx) / g.h);
                m->class_ref.push_back((py[i] - g.cy) / g.h);
            }
        } else {
            m->cell_class[c] = it->second;
        }
    }
    m->n_classes = (int32_t)class_of_key.size();
    m->class_ref_off.push_back((int64_t)m->class_ref.size());
    *out = m;
    return HHO_OK;
}

extern "C" int hho_mesh_submesh(const hho_mesh* parent, int64_t n_cells, const int64_t* h_cells, hho_mesh** out) {
    if (!parent || !h_cells || !out || n_cells <= 0 || n_cells > parent->nc) {
        hho_set_error("hho_mesh_submesh: null pointer or bad cell count");
        return HHO_EINVAL;
    }
    *out = nullptr;
    std::vector<int64_t> vloc(parent->nv, -1), vlist;
    std::vector<char> seen(parent->nc, 0);
    auto use = [&](int64_t v) {
        if (vloc[v] < 0) {
            vloc[v] = (int64_t)vlist.size();
            vlist.push_back(v);
        }
    };
    std::vector<int64_t> ptr(1, 0), vtx;
    std::vector<uint8_t> dom;
    for (int64_t i = 0; i < n_cells; ++i) {
        const int64_t c = h_cells[i];
        if (c < 0 || c >= parent->nc || seen[c]) {
            hho_set_error("hho_mesh_submesh: cell %lld out of range or repeated", (long long)c);
            return HHO_EINVAL;
        }
        seen[c] = 1;
        for (int64_t e = parent->cell_ptr[c]; e < parent->cell_ptr[c + 1]; ++e) {
            use(parent->cell_vtx[e]);
            vtx.push_back(vloc[parent->cell_vtx[e]]);
        }
        ptr.push_back((int64_t)vtx.size());
        dom.push_back(parent->domain[c]);
    }
    // identified (periodic) vertices keep their representative
    const size_t nused = vlist.size();
    for (size_t i = 0; i < nused; ++i) use(parent->rep[vlist[i]]);
    std::vector<double> xy(2 * vlist.size());
    std::vector<int64_t> rep(vlist.size());
    for (size_t i = 0; i < vlist.size(); ++i) {
        xy[2 * i] = parent->xy[2 * vlist[i]];
        xy[2 * i + 1] = parent->xy[2 * vlist[i] + 1];
        rep[i] = vloc[parent->rep[vlist[i]]];
    }
    hho_mesh* m = nullptr;
    int rc = hho_mesh_create(xy.data(), (int64_t)vlist.size(), ptr.data(), vtx.data(), n_cells, dom.data(),
                             rep.data(), &m);
    if (rc) return rc;
    // class reference geometry from the parent's classes
    m->class_ref.clear();
    m->class_ref_off.clear();
    for (int32_t cl = 0; cl < m->n_classes; ++cl) {
        const int32_t pcl = parent->cell_class[h_cells[m->class_first[cl]]];
        const int64_t a = parent->class_ref_off[pcl], b = parent->class_ref_off[pcl + 1];
        m->class_ref_off.push_back((int64_t)m->class_ref.size());
        m->class_ref.insert(m->class_ref.end(), parent->class_ref.begin() + a, parent->class_ref.begin() + b);
    }
    m->class_ref_off.push_back((int64_t)m->class_ref.size());
    *out = m;
    return HHO_OK;
}

extern "C" int hho_mesh_query(const hho_mesh* m, hho_mesh_info* out) {
    if (!m || !out) {
        hho_set_error("hho_mesh_query: null pointer");
        return HHO_EINVAL;
    }
    memset(out, 0, sizeof(*out));
    out->n_vertices = m->nv;
    out->n_cells = m->nc;
    out->n_faces = m->nf;
    for (int64_t c = 0; c < m->nc; ++c) {
        if (m->domain[c] == 0) out->n_fluid_cells++;
        else out->n_solid_cells++;
    }
    for (int64_t F = 0; F < m->nf; ++F) out->n_faces_by_type[m->face_type[F]]++;
    out->n_classes = m->n_classes;
    out->n_colours = m->n_colours;
    out->max_faces_per_cell = m->max_nf;
    return HHO_OK;
}

extern "C" int hho_mesh_tables(const hho_mesh* m, int64_t* face_cells, int64_t* cell_faces_ptr,
                               int64_t* cell_faces, int32_t* face_type, int32_t* face_colour,
                               int32_t* cell_class) {
    if (!m) {
        hho_set_error("hho_mesh_tables: null mesh");
        return HHO_EINVAL;
    }
    if (face_cells) memcpy(face_cells, m->face_cells.data(), sizeof(int64_t) * 2 * m->nf);
    if (cell_faces_ptr) memcpy(cell_faces_ptr, m->cell_ptr.data(), sizeof(int64_t) * (m->nc + 1));
    if (cell_faces) memcpy(cell_faces, m->cell_faces.data(), sizeof(int64_t) * m->cell_ptr[m->nc]);
    if (face_type) memcpy(face_type, m->face_type.data(), sizeof(int32_t) * m->nf);
    if (face_colour) memcpy(face_colour, m->face_colour.data(), sizeof(int32_t) * m->nf);
    if (cell_class) memcpy(cell_class, m->cell_class.data(), sizeof(int32_t) * m->nc);
    return HHO_OK;
}

extern "C" void hho_mesh_destroy(hho_mesh* m) { delete m; }
