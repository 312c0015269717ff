// mesh.cpp -- mesh ingestion on the host: face matching (including periodic
// pairing), face normals and areas, cell volumes and vertex means.
//
// The paper's domain is any mix of triangles and quadrilaterals in 2D or
// hexahedra (among others) in 3D (Sec. 2); each element is one index.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <string>
#include <unordered_map>

#include "hfv_internal.h"

namespace hfv {

static const int kTriFaces[3][2] = {{0, 1}, {1, 2}, {2, 0}};
static const int kQuadFaces[4][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 0}};
static const int kHexFaces[6][4] = {{0, 3, 2, 1}, {4, 5, 6, 7}, {0, 1, 5, 4},
                                    {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};
// tetrahedron v0 v1 v2 v3 of positive volume: face k is opposite vertex k,
// listed so that (p1 - p0) x (p2 - p0) points outward
static const int kTetFaces[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
// prism: triangles v0 v1 v2 (counter-clockwise seen from the other end) and
// v3 v4 v5 (v3 joined to v0); pyramid: base v0..v3 counter-clockwise seen
// from the apex v4.  Triangular faces first, quadrilaterals after.
static const int kPrismFaces[5][4] = {{0, 2, 1, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
static const int kPyramidFaces[5][4] = {{0, 1, 4, -1}, {1, 2, 4, -1}, {2, 3, 4, -1}, {3, 0, 4, -1}, {0, 3, 2, 1}};

int type_nverts(int t)
{
    return t == HFV_TRI ? 3 : t == HFV_QUAD ? 4 : t == HFV_TET ? 4 : t == HFV_HEX ? 8 : t == HFV_PRISM ? 6 : t == HFV_PYRAMID ? 5 : 0;
}
int type_nfaces(int t)
{
    return t == HFV_TRI ? 3 : t == HFV_QUAD ? 4 : t == HFV_TET ? 4 : t == HFV_HEX ? 6 : t == HFV_PRISM || t == HFV_PYRAMID ? 5 : 0;
}
int face_nverts(int t, int f)
{
    if (t == HFV_TRI || t == HFV_QUAD) return 2;
    if (t == HFV_TET) return 3;
    if (t == HFV_PRISM) return f < 2 ? 3 : 4;
    if (t == HFV_PYRAMID) return f < 4 ? 3 : 4;
    return 4;
}
int element_family(const hfv_mesh* m)
{
    if (m->dim == 2) return 0;
    bool hex = true, tet = true;
    for (uint8_t t : m->type) {
        hex = hex && t == HFV_HEX;
        tet = tet && t == HFV_TET;
    }
    return hex ? 0 : tet ? 1 : 2;
}
int type_face_vertex(int t, int f, int k)
{
    if (t == HFV_TRI) return kTriFaces[f][k];
    if (t == HFV_QUAD) return kQuadFaces[f][k];
    if (t == HFV_TET) return kTetFaces[f][k];
    if (t == HFV_PRISM) return kPrismFaces[f][k];
    if (t == HFV_PYRAMID) return kPyramidFaces[f][k];
    return kHexFaces[f][k];
}

namespace {

struct Key4 {
    int64_t v[4];
    bool operator==(const Key4& o) const { return std::memcmp(v, o.v, sizeof v) == 0; }
};
struct Key4Hash {
    size_t operator()(const Key4& k) const
    {
        uint64_t h = 1469598103934665603ull;
        for (int i = 0; i < 4; ++i) {
            h ^= (uint64_t)k.v[i] + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
            h *= 1099511628211ull;
        }
        return (size_t)h;
    }
};

inline const double* node(const hfv_mesh* m, int64_t c, int k) { return &m->xyz[3 * (int64_t)m->cidx[m->cptr[c] + k]]; }

// outward area vector of local face f of cell c, from c's own vertices
void area_vector(const hfv_mesh* m, int64_t c, int f, double A[3])
{
    int t = m->type[c];
    const int fnv = face_nverts(t, f);
    if (fnv == 2) {
        const double* a = node(m, c, type_face_vertex(t, f, 0));
        const double* b = node(m, c, type_face_vertex(t, f, 1));
        A[0] = b[1] - a[1];
        A[1] = a[0] - b[0];
        A[2] = 0.0;
        return;
    }
    const double* p0 = node(m, c, type_face_vertex(t, f, 0));
    const double* p1 = node(m, c, type_face_vertex(t, f, 1));
    const double* p2 = node(m, c, type_face_vertex(t, f, 2));
    if (fnv == 3) {
        double e[3], g[3];
        for (int k = 0; k < 3; ++k) { e[k] = p1[k] - p0[k]; g[k] = p2[k] - p0[k]; }
        A[0] = 0.5 * (e[1] * g[2] - e[2] * g[1]);
        A[1] = 0.5 * (e[2] * g[0] - e[0] * g[2]);
        A[2] = 0.5 * (e[0] * g[1] - e[1] * g[0]);
        return;
    }
    const double* p3 = node(m, c, type_face_vertex(t, f, 3));
    double e[3], g[3];
    for (int k = 0; k < 3; ++k) { e[k] = p2[k] - p0[k]; g[k] = p3[k] - p1[k]; }
    A[0] = 0.5 * (e[1] * g[2] - e[2] * g[1]);
    A[1] = 0.5 * (e[2] * g[0] - e[0] * g[2]);
    A[2] = 0.5 * (e[0] * g[1] - e[1] * g[0]);
}

// |V| = (1/3) sum_f int_f x . dA over the faces (triangles flat, quadrilaterals
// bilinear), relative to vertex 0; the integrand of a bilinear face has
// degree <= 2 per direction, so the 2x2 Gauss rule is exact
double divergence_measure(const hfv_mesh* m, int64_t c)
{
    const int t = m->type[c];
    const double* o = node(m, c, 0);
    const double g = 0.5 / std::sqrt(3.0);
    const double pts[2] = {0.5 - g, 0.5 + g};
    double vol = 0.0;
    for (int f = 0; f < type_nfaces(t); ++f) {
        double p[4][3];
        const int fnv = face_nverts(t, f);
        for (int a = 0; a < fnv; ++a)
            for (int k = 0; k < 3; ++k) p[a][k] = node(m, c, type_face_vertex(t, f, a))[k] - o[k];
        if (fnv == 3) {
            double e[3], h[3];
            for (int k = 0; k < 3; ++k) { e[k] = p[1][k] - p[0][k]; h[k] = p[2][k] - p[0][k]; }
            const double A[3] = {0.5 * (e[1] * h[2] - e[2] * h[1]), 0.5 * (e[2] * h[0] - e[0] * h[2]),
                                 0.5 * (e[0] * h[1] - e[1] * h[0])};
            for (int k = 0; k < 3; ++k) vol += (p[0][k] + p[1][k] + p[2][k]) / 3.0 * A[k] / 3.0;
            continue;
        }
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                const double s = pts[i], u = pts[j];
                double x[3], xs[3], xu[3];
                for (int k = 0; k < 3; ++k) {
                    x[k] = (1 - s) * (1 - u) * p[0][k] + s * (1 - u) * p[1][k] + s * u * p[2][k] + (1 - s) * u * p[3][k];
                    xs[k] = (1 - u) * (p[1][k] - p[0][k]) + u * (p[2][k] - p[3][k]);
                    xu[k] = (1 - s) * (p[3][k] - p[0][k]) + s * (p[2][k] - p[1][k]);
                }
                const double n[3] = {xs[1] * xu[2] - xs[2] * xu[1], xs[2] * xu[0] - xs[0] * xu[2], xs[0] * xu[1] - xs[1] * xu[0]};
                vol += 0.25 * (x[0] * n[0] + x[1] * n[1] + x[2] * n[2]) / 3.0;
            }
    }
    return vol;
}

// cell measure: triangle cross product, quadrilateral shoelace, tetrahedron
// triple product, hexahedron 2x2x2 Gauss rule on the trilinear map (exact:
// det J has degree <= 2 per direction), prism and pyramid by the divergence
// theorem over their faces
double cell_measure(const hfv_mesh* m, int64_t c)
{
    int t = m->type[c];
    if (t == HFV_PRISM || t == HFV_PYRAMID) return divergence_measure(m, c);
    if (t == HFV_TET) {
        const double* o = node(m, c, 0);
        double a[3], b[3], q[3];
        for (int k = 0; k < 3; ++k) {
            a[k] = node(m, c, 1)[k] - o[k];
            b[k] = node(m, c, 2)[k] - o[k];
            q[k] = node(m, c, 3)[k] - o[k];
        }
        return (a[0] * (b[1] * q[2] - b[2] * q[1]) - a[1] * (b[0] * q[2] - b[2] * q[0]) +
                a[2] * (b[0] * q[1] - b[1] * q[0])) / 6.0;
    }
    if (t == HFV_TRI) {
        const double *a = node(m, c, 0), *b = node(m, c, 1), *q = node(m, c, 2);
        return 0.5 * ((b[0] - a[0]) * (q[1] - a[1]) - (b[1] - a[1]) * (q[0] - a[0]));
    }
    if (t == HFV_QUAD) {
        // shoelace on coordinates relative to v0 (absolute coordinates would
        // cancel catastrophically for small cells far from the origin)
        const double* o = node(m, c, 0);
        double s = 0.0;
        for (int k = 1; k < 3; ++k) {
            const double *a = node(m, c, k), *b = node(m, c, k + 1);
            s += (a[0] - o[0]) * (b[1] - o[1]) - (b[0] - o[0]) * (a[1] - o[1]);
        }
        return 0.5 * s;
    }
    const double g = 0.5 / std::sqrt(3.0);
    const double pts[2] = {0.5 - g, 0.5 + g};
    static const int corner[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                     {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
    double vol = 0.0;
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j)
            for (int k = 0; k < 2; ++k) {
                double u[3] = {pts[i], pts[j], pts[k]};
                double J[3][3] = {};
                for (int a = 0; a < 8; ++a) {
                    double w[3], dw[3];
                    for (int q = 0; q < 3; ++q) {
                        w[q] = corner[a][q] ? u[q] : 1.0 - u[q];
                        dw[q] = corner[a][q] ? 1.0 : -1.0;
                    }
                    double grad[3] = {dw[0] * w[1] * w[2], w[0] * dw[1] * w[2], w[0] * w[1] * dw[2]};
                    const double* x = node(m, c, a);
                    const double* x0 = node(m, c, 0);
                    for (int r = 0; r < 3; ++r)
                        for (int q = 0; q < 3; ++q) J[r][q] += (x[r] - x0[r]) * grad[q];   // the gradients sum to 0
                }
                double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                             J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
                vol += 0.125 * det;
            }
    return vol;
}

// a descriptor's cell types, CSR offsets (non-negative, each cell's count
// that of its type), vertex ids, node coordinates and periods, checked before
// anything is read through the offsets
int check_desc(const hfv_mesh_desc& d, const std::string& who)
{
    const int64_t* ptr = d.cell_node_ptr;
    if (ptr[0] < 0) {
        set_error(who + ": cell_node_ptr[0] is negative");
        return HFV_ERR_MESH;
    }
    for (int64_t c = 0; c < d.n_cells; ++c) {
        const int t = d.cell_type[c];
        const bool ok = ((d.dim == 2 && (t == HFV_TRI || t == HFV_QUAD)) ||
                         (d.dim == 3 && (t == HFV_HEX || t == HFV_TET || t == HFV_PRISM || t == HFV_PYRAMID))) &&
                        ptr[c + 1] == ptr[c] + type_nverts(t);   // ptr[c] <= ptr[0] + 8c: no overflow
        if (!ok) {
            set_error(who + ": cell " + std::to_string(c) + " has an unsupported type or a vertex count not its type's");
            return HFV_ERR_MESH;
        }
    }
    for (int64_t k = ptr[0]; k < ptr[d.n_cells]; ++k)
        if (d.cell_node_idx[k] < 0 || d.cell_node_idx[k] >= d.n_nodes) {
            set_error(who + ": cell_node_idx[" + std::to_string(k) + "] is not a node id");
            return HFV_ERR_MESH;
        }
    for (int64_t i = 0; i < d.n_nodes * d.dim; ++i)
        if (!std::isfinite(d.node_xyz[i])) {
            set_error(who + ": node " + std::to_string(i / d.dim) + " has a non-finite coordinate");
            return HFV_ERR_MESH;
        }
    for (int k = 0; k < d.dim; ++k)
        if (!(std::isfinite(d.period[k]) && d.period[k] >= 0.0)) {
            set_error(who + ": periods must be finite and non-negative");
            return HFV_ERR_ARG;
        }
    return HFV_OK;
}

}  // namespace
}  // namespace hfv

using namespace hfv;

extern "C" int hfv_mesh_create(const hfv_mesh_desc* d, hfv_mesh** out)
{
    if (!d || !out || (d->dim != 2 && d->dim != 3) || d->n_cells <= 0 || d->n_nodes <= 0 || !d->node_xyz ||
        !d->cell_type || !d->cell_node_ptr || !d->cell_node_idx || !d->period || d->n_cells >= (int64_t(1) << 31)) {
        set_error("hfv_mesh_create: invalid descriptor");
        return HFV_ERR_ARG;
    }
    *out = nullptr;
    const int chk = check_desc(*d, "hfv_mesh_create");
    if (chk != HFV_OK) return chk;
    hfv_mesh* m = nullptr;
    try {
        m = new hfv_mesh();
        m->dim = d->dim;
        m->nn = d->n_nodes;
        m->nc = d->n_cells;
        const int64_t nc = m->nc;
        m->xyz.assign(3 * m->nn, 0.0);
        for (int64_t i = 0; i < m->nn; ++i)
            for (int k = 0; k < d->dim; ++k) m->xyz[3 * i + k] = d->node_xyz[d->dim * i + k];
        m->type.assign(d->cell_type, d->cell_type + nc);
        m->cptr.assign(d->cell_node_ptr, d->cell_node_ptr + nc + 1);
        m->cidx.assign(d->cell_node_idx, d->cell_node_idx + m->cptr[nc]);   // offsets checked above
        for (int k = 0; k < 3; ++k) m->period[k] = k < d->dim ? d->period[k] : 0.0;
        m->nbr.assign(nc * kMaxFaces, -1);
        m->nbrf.assign(nc * kMaxFaces, -1);
        m->nshift.assign(nc * kMaxFaces * 3, 0);
        m->own.assign(nc * kMaxFaces, 0);
        m->fnorm.assign(nc * kMaxFaces * 3, 0.0);
        m->farea.assign(nc * kMaxFaces, 0.0);

        // topological matching: sorted vertex ids -> first half-face seen
        std::unordered_map<Key4, int64_t, Key4Hash> open;
        open.reserve((size_t)(nc * 2));
        auto link = [&](int64_t c, int f, int64_t c2, int f2) {
            m->nbr[c * kMaxFaces + f] = (int32_t)c2;
            m->nbrf[c * kMaxFaces + f] = (int8_t)f2;
            m->nbr[c2 * kMaxFaces + f2] = (int32_t)c;
            m->nbrf[c2 * kMaxFaces + f2] = (int8_t)f;
        };
        for (int64_t c = 0; c < nc; ++c) {
            int t = m->type[c];
            for (int f = 0; f < type_nfaces(t); ++f) {
                Key4 k{{-1, -1, -1, -1}};
                int fn = face_nverts(t, f);
                for (int q = 0; q < fn; ++q) k.v[q] = m->cidx[m->cptr[c] + type_face_vertex(t, f, q)];
                std::sort(k.v, k.v + fn);
                auto it = open.find(k);
                if (it == open.end()) {
                    open.emplace(k, c * kMaxFaces + f);
                } else {
                    int64_t other = it->second;
                    if (other < 0) {
                        set_error("hfv_mesh_create: a face is shared by more than two cells");
                        delete m;
                        return HFV_ERR_MESH;
                    }
                    link(other / kMaxFaces, (int)(other % kMaxFaces), c, f);
                    it->second = -1;
                }
            }
        }
        // periodic pairing of still-open faces by their wrapped, quantised centres
        bool periodic = m->period[0] > 0 || m->period[1] > 0 || m->period[2] > 0;
        if (periodic) {
            std::unordered_map<Key4, int64_t, Key4Hash> wrap;
            for (auto& kv : open) {
                if (kv.second < 0) continue;
                int64_t c = kv.second / kMaxFaces;
                int f = (int)(kv.second % kMaxFaces);
                int t = m->type[c];
                double x[3] = {0, 0, 0};
                for (int q = 0; q < face_nverts(t, f); ++q)
                    for (int k = 0; k < 3; ++k) x[k] += node(m, c, type_face_vertex(t, f, q))[k];
                Key4 key{{0, 0, 0, 0}};
                for (int k = 0; k < 3; ++k) {
                    double xc = x[k] / face_nverts(t, f);
                    const int64_t S = int64_t(1) << 30;
                    if (m->period[k] > 0) {
                        int64_t q = std::llround(xc / m->period[k] * (double)S) % S;
                        key.v[k] = q < 0 ? q + S : q;
                    } else {
                        key.v[k] = std::llround(xc * (double)S);
                    }
                }
                auto it = wrap.find(key);
                if (it == wrap.end()) {
                    wrap.emplace(key, kv.second);
                } else {
                    int64_t c2 = it->second / kMaxFaces;
                    int f2 = (int)(it->second % kMaxFaces);
                    if (c2 == c) {
                        set_error("hfv_mesh_create: a cell is its own periodic neighbour (mesh too coarse)");
                        delete m;
                        return HFV_ERR_MESH;
                    }
                    link(c2, f2, c, f);
                    double y[3] = {0, 0, 0};
                    int t2 = m->type[c2];
                    for (int q = 0; q < face_nverts(t2, f2); ++q)
                        for (int k = 0; k < 3; ++k) y[k] += node(m, c2, type_face_vertex(t2, f2, q))[k];
                    for (int k = 0; k < 3; ++k) {
                        // x_c2 + s * period lies next to c  (s integer)
                        int s = 0;
                        if (m->period[k] > 0)
                            s = (int)std::lround((x[k] / face_nverts(t, f) - y[k] / face_nverts(t2, f2)) / m->period[k]);
                        if (s < -127 || s > 127) {
                            set_error("hfv_mesh_create: periodic faces more than 127 periods apart");
                            delete m;
                            return HFV_ERR_MESH;
                        }
                        m->nshift[(c * kMaxFaces + f) * 3 + k] = (int8_t)s;
                        m->nshift[(c2 * kMaxFaces + f2) * 3 + k] = (int8_t)(-s);
                    }
                    wrap.erase(it);
                }
            }
        }
        // ownership, normals, areas, volumes, vertex means
        m->vol.assign(nc, 0.0);
        m->vmean.assign(nc * 3, 0.0);
        int64_t nface = 0;
        for (int64_t c = 0; c < nc; ++c) {
            int t = m->type[c];
            for (int f = 0; f < type_nfaces(t); ++f) {
                int32_t j = m->nbr[c * kMaxFaces + f];
                if (j == c) {
                    set_error("hfv_mesh_create: a cell is its own neighbour");
                    delete m;
                    return HFV_ERR_MESH;
                }
                bool own = j < 0 || j > c;
                m->own[c * kMaxFaces + f] = own;
                if (own) {
                    ++nface;
                    double A[3];
                    area_vector(m, c, f, A);
                    double a = std::sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
                    if (!(a > 0)) {
                        set_error("hfv_mesh_create: zero-area face on cell " + std::to_string(c));
                        delete m;
                        return HFV_ERR_MESH;
                    }
                    m->farea[c * kMaxFaces + f] = a;
                    for (int k = 0; k < 3; ++k) m->fnorm[(c * kMaxFaces + f) * 3 + k] = A[k] / a;
                    if (j >= 0) {
                        int f2 = m->nbrf[c * kMaxFaces + f];
                        m->farea[(int64_t)j * kMaxFaces + f2] = a;
                        for (int k = 0; k < 3; ++k) m->fnorm[((int64_t)j * kMaxFaces + f2) * 3 + k] = -A[k] / a;
                    }
                }
            }
            double v = cell_measure(m, c);
            if (!(v > 0)) {
                set_error("hfv_mesh_create: cell " + std::to_string(c) + " has non-positive measure (vertex order?)");
                delete m;
                return HFV_ERR_MESH;
            }
            m->vol[c] = v;
            int nvx = type_nverts(t);
            for (int q = 0; q < nvx; ++q)
                for (int k = 0; k < 3; ++k) m->vmean[3 * c + k] += node(m, c, q)[k];
            for (int k = 0; k < 3; ++k) m->vmean[3 * c + k] /= nvx;
        }
        m->nface = nface;
        m->seg_off = {0, nc};
    } catch (const std::bad_alloc&) {
        delete m;
        set_error("hfv_mesh_create: out of host memory");
        return HFV_ERR_OOM;
    }
    *out = m;
    return HFV_OK;
}

extern "C" int hfv_mesh_create_batch(const hfv_mesh_desc* descs, int n_meshes, hfv_mesh** out)
{
    if (!descs || !out || n_meshes <= 0) {
        set_error("hfv_mesh_create_batch: invalid arguments");
        return HFV_ERR_ARG;
    }
    *out = nullptr;
    // one descriptor holding every mesh, node and cell ids offset per mesh:
    // no face is shared between meshes, so stencils and fluxes never couple them
    int64_t nn = 0, nc = 0, nidx = 0;
    const int dim = descs[0].dim;
    for (int k = 0; k < n_meshes; ++k) {
        const hfv_mesh_desc& d = descs[k];
        if (d.dim != dim || d.n_cells <= 0 || d.n_nodes <= 0 || !d.node_xyz || !d.cell_type || !d.cell_node_ptr ||
            !d.cell_node_idx || !d.period) {
            set_error("hfv_mesh_create_batch: descriptor " + std::to_string(k) + " is invalid or of another dimension");
            return HFV_ERR_ARG;
        }
        const int chk = check_desc(d, "hfv_mesh_create_batch: descriptor " + std::to_string(k));
        if (chk != HFV_OK) return chk;
        for (int a = 0; a < dim; ++a)
            if (d.period[a] != 0.0) {
                set_error("hfv_mesh_create_batch: descriptor " + std::to_string(k) + " is periodic; batched meshes are open");
                return HFV_ERR_ARG;
            }
        nn += d.n_nodes;
        nc += d.n_cells;
        nidx += d.cell_node_ptr[d.n_cells] - d.cell_node_ptr[0];
    }
    if (nn >= (int64_t(1) << 31) || nc >= (int64_t(1) << 31)) {
        set_error("hfv_mesh_create_batch: more than 2^31 nodes or cells");
        return HFV_ERR_ARG;
    }
    std::vector<int64_t> seg(n_meshes + 1, 0);
    std::vector<double> xyz, period(dim, 0.0);
    std::vector<uint8_t> type;
    std::vector<int64_t> ptr;
    std::vector<int32_t> idx;
    try {
        xyz.reserve(nn * dim);
        type.reserve(nc);
        ptr.reserve(nc + 1);
        idx.reserve(nidx);
        ptr.push_back(0);
        int64_t node0 = 0;
        for (int k = 0; k < n_meshes; ++k) {
            const hfv_mesh_desc& d = descs[k];
            xyz.insert(xyz.end(), d.node_xyz, d.node_xyz + d.n_nodes * dim);
            type.insert(type.end(), d.cell_type, d.cell_type + d.n_cells);
            const int64_t base = ptr.back();
            for (int64_t c = 0; c < d.n_cells; ++c) ptr.push_back(base + d.cell_node_ptr[c + 1] - d.cell_node_ptr[0]);
            for (int64_t i = d.cell_node_ptr[0]; i < d.cell_node_ptr[d.n_cells]; ++i)
                idx.push_back((int32_t)(d.cell_node_idx[i] + node0));   // ids checked by check_desc
            node0 += d.n_nodes;
            seg[k + 1] = seg[k] + d.n_cells;
        }
    } catch (const std::bad_alloc&) {
        set_error("hfv_mesh_create_batch: out of host memory");
        return HFV_ERR_OOM;
    }
    hfv_mesh_desc all;
    all.dim = dim;
    all.n_nodes = nn;
    all.n_cells = nc;
    all.node_xyz = xyz.data();
    all.cell_type = type.data();
    all.cell_node_ptr = ptr.data();
    all.cell_node_idx = idx.data();
    all.period = period.data();
    hfv_mesh* m = nullptr;
    int rc = hfv_mesh_create(&all, &m);
    if (rc != HFV_OK) return rc;
    m->seg_off = seg;
    *out = m;
    return HFV_OK;
}

extern "C" int hfv_mesh_segments(const hfv_mesh* m, int* n_segments, int64_t* cell_offsets)
{
    if (!m || !n_segments) { set_error("hfv_mesh_segments: NULL argument"); return HFV_ERR_ARG; }
    *n_segments = (int)m->seg_off.size() - 1;
    if (cell_offsets) std::memcpy(cell_offsets, m->seg_off.data(), m->seg_off.size() * sizeof(int64_t));
    return HFV_OK;
}

extern "C" int hfv_mesh_volumes(const hfv_mesh* m, double* vol)
{
    if (!m || !vol) { set_error("hfv_mesh_volumes: NULL argument"); return HFV_ERR_ARG; }
    std::memcpy(vol, m->vol.data(), m->vol.size() * sizeof(double));
    return HFV_OK;
}

extern "C" int hfv_mesh_info(const hfv_mesh* m, int64_t* n_cells, int64_t* n_faces, int* dim)
{
    if (!m) { set_error("hfv_mesh_info: NULL mesh"); return HFV_ERR_ARG; }
    if (n_cells) *n_cells = m->nc;
    if (n_faces) *n_faces = m->nface;
    if (dim) *dim = m->dim;
    return HFV_OK;
}

extern "C" int hfv_mesh_connectivity(const hfv_mesh* m, int32_t* nbr, int8_t* nbrf)
{
    if (!m || !nbr || !nbrf) { set_error("hfv_mesh_connectivity: NULL argument"); return HFV_ERR_ARG; }
    std::memcpy(nbr, m->nbr.data(), m->nbr.size() * sizeof(int32_t));
    std::memcpy(nbrf, m->nbrf.data(), m->nbrf.size());
    return HFV_OK;
}

extern "C" void hfv_mesh_destroy(hfv_mesh* m) { delete m; }
