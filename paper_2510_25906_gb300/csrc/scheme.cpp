// scheme.cpp -- stencil construction on the host (deterministic, integer keys).
//
// Central stencil (Sec. 2.1): M = stencil_factor * K(r, d) cells besides the
// cell itself, K(r, d) = prod_{l=1..d}(r + l) / d!.  Neighbouring elements
// are included recursively: face-adjacency layers are taken whole while they
// fit; the first layer that does not fit is ordered by the quantised squared
// distance of vertex means, llround(|x_j - x_i|^2 / h_i^2 * 2^20) with
// h_i^2 = |V_i| (2D) or |V_i|^(2/3) (3D), then by cell id.  The stored order
// is (layer, distance key, id).
//
// Directional stencils (Sec. 2.3), one per face f: the central-stencil cells
// whose vertex mean lies strictly beyond the cell's vertex mean along the
// face's outward normal (quantised to h_i / 2^20), in stencil order, at most
// Md = 2 K(1, d); with fewer than d + 1 such cells the first Md central
// cells are used instead.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <thread>
#include <vector>

#include "hfv_internal.h"

namespace hfv {

namespace {

int binom_K(int r, int d)
{
    long num = 1, den = 1;
    for (int l = 1; l <= d; ++l) { num *= (r + l); den *= l; }
    return (int)(num / den);
}

struct Cand {
    int layer;
    int64_t key;
    int32_t id;
    int8_t k[3];
    bool operator<(const Cand& o) const
    {
        if (layer != o.layer) return layer < o.layer;
        if (key != o.key) return key < o.key;
        return id < o.id;
    }
};

}  // namespace

int build_stencils(hfv_scheme* s)
{
    const hfv_mesh* m = s->mesh;
    const int d = m->dim;
    s->d = d;
    s->nv = d + 2;
    s->r = s->p.order - 1;
    s->N = binom_K(s->r, d) - 1;
    s->M = (int)std::llround(s->p.stencil_factor * binom_K(s->r, d));
    s->Md = 2 * binom_K(1, d);
    // Gauss points per face direction, exact to degree >= r: ceil((r+1)/2) on
    // edges and on the quadrilaterals of hexahedral meshes, ceil((r+2)/2) per
    // direction of the collapsed rule on triangles (exact to degree
    // 2 nq - 2), used on every face of a mesh with triangular faces so that
    // all faces carry nq^2 points
    s->fam = element_family(m);
    s->nfmax = d == 2 || s->fam == 1 ? 4 : 6;
    s->nq = s->fam ? (s->r + 3) / 2 : (s->r + 2) / 2;
    s->nfp = d == 2 ? s->nq : s->nq * s->nq;
    if (s->M < s->N || s->M < s->Md || s->M > 255) {
        set_error("hfv_scheme_create: stencil size out of range");
        return HFV_ERR_ARG;
    }
    const int64_t nc = m->nc;
    const int M = s->M, Md = s->Md;
    // face-point data live at a fixed stride per cell (the largest face count
    // of the dimension times the points per face): rows past a cell's own
    // face points are never read, so the padding costs memory, not traffic
    const int64_t qs = (int64_t)s->nfmax * s->nfp;
    s->qoff.assign(nc + 1, 0);
    for (int64_t c = 0; c <= nc; ++c) s->qoff[c] = c * qs;
    s->qtot = s->qoff[nc];
    // L: compact per-cell blocks of Q_c x M values, each padded to 16 bytes so
    // that a run of consecutive cells is one aligned bulk copy
    const int per16 = s->p.precision == HFV_FP32 ? 4 : 2;
    s->nc_pad = (nc + 191) / 192 * 192;   // a whole number of tiles of every tile size (8-64 cells, 48)
    s->loff.assign(s->nc_pad + 1, 0);
    for (int64_t c = 0; c < s->nc_pad; ++c) {
        int64_t blk = c < nc ? (int64_t)type_nfaces(m->type[c]) * s->nfp * M : 0;
        s->loff[c + 1] = s->loff[c] + (blk + per16 - 1) / per16 * per16;
    }
    s->ltot = s->loff[s->nc_pad];
    s->sten.assign(nc * M, 0);
    s->sshift.assign(nc * M * 3, 0);
    s->dir.assign(nc * kMaxFaces * Md, 0);
    s->nd.assign(nc * kMaxFaces, 0);
    s->n1.assign(nc, 0);

    // cells are independent: contiguous ranges on host threads, each with
    // its own BFS marks; the first failing cell (in cell order) is reported
    struct Work {
        std::vector<Cand> layer, next, chosen;
        std::vector<int32_t> mark;   // last cell whose BFS visited this cell
        int64_t fail = -1;
    };
    auto one = [&](int64_t i, Work& w) -> bool {
        std::vector<Cand>& layer = w.layer;
        std::vector<Cand>& next = w.next;
        std::vector<Cand>& chosen = w.chosen;
        std::vector<int32_t>& mark = w.mark;
        const double* xi = &m->vmean[3 * i];
        double h2 = d == 2 ? m->vol[i] : std::cbrt(m->vol[i]) * std::cbrt(m->vol[i]);
        layer.clear();
        chosen.clear();
        layer.push_back(Cand{0, 0, (int32_t)i, {0, 0, 0}});
        mark[i] = (int32_t)i;
        for (int L = 1; L <= 16 && (int)chosen.size() < M; ++L) {
            next.clear();
            for (const Cand& a : layer) {
                int t = m->type[a.id];
                for (int f = 0; f < type_nfaces(t); ++f) {
                    int32_t j = m->nbr[(int64_t)a.id * kMaxFaces + f];
                    if (j < 0 || mark[j] == (int32_t)i) continue;
                    mark[j] = (int32_t)i;
                    Cand e;
                    e.layer = L;
                    e.id = j;
                    double dist2 = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        e.k[k] = (int8_t)(a.k[k] + m->nshift[((int64_t)a.id * kMaxFaces + f) * 3 + k]);
                        double dx = m->vmean[3 * (int64_t)j + k] + e.k[k] * m->period[k] - xi[k];
                        dist2 += dx * dx;
                    }
                    e.key = std::llround(dist2 / h2 * 1048576.0);
                    next.push_back(e);
                }
            }
            if (next.empty()) break;
            std::sort(next.begin(), next.end());
            size_t room = (size_t)M - chosen.size();
            size_t take = std::min(room, next.size());
            chosen.insert(chosen.end(), next.begin(), next.begin() + take);
            layer.swap(next);
        }
        if ((int)chosen.size() < M) return false;
        std::sort(chosen.begin(), chosen.end());
        int first_layer = 0;
        for (int a = 0; a < M; ++a) first_layer += chosen[a].layer == 1;
        s->n1[i] = (uint8_t)first_layer;
        for (int a = 0; a < M; ++a) {
            s->sten[i * M + a] = chosen[a].id;
            for (int k = 0; k < 3; ++k) s->sshift[(i * M + a) * 3 + k] = chosen[a].k[k];
        }
        // directional stencils
        double h = d == 2 ? std::sqrt(m->vol[i]) : std::cbrt(m->vol[i]);
        int nf = type_nfaces(m->type[i]);
        for (int f = 0; f < nf; ++f) {
            const double* n = &m->fnorm[(i * kMaxFaces + f) * 3];
            uint8_t* out = &s->dir[(i * kMaxFaces + f) * Md];
            int cnt = 0;
            for (int a = 0; a < M && cnt < Md; ++a) {
                int32_t j = chosen[a].id;
                double sd = 0.0;
                for (int k = 0; k < 3; ++k)
                    sd += (m->vmean[3 * (int64_t)j + k] + chosen[a].k[k] * m->period[k] - xi[k]) * n[k];
                if (std::llround(sd / h * 1048576.0) > 0) out[cnt++] = (uint8_t)a;
            }
            if (cnt < d + 1) {
                for (int a = 0; a < Md; ++a) out[a] = (uint8_t)a;
                cnt = Md;
            }
            for (int a = cnt; a < Md; ++a) out[a] = 0;
            s->nd[i * kMaxFaces + f] = (uint8_t)cnt;
        }
        return true;
    };
    const unsigned hw = std::thread::hardware_concurrency();
    const int nt = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(hw ? hw : 1), 16, nc / 4096}));
    std::vector<Work> work(nt);
    auto range = [&](int t) {
        Work& w = work[t];
        w.mark.assign(nc, -1);
        const int64_t lo = nc * t / nt, hi = nc * (t + 1) / nt;
        for (int64_t i = lo; i < hi; ++i)
            if (!one(i, w)) { w.fail = i; return; }
    };
    if (nt == 1) {
        range(0);
    } else {
        std::vector<std::thread> th;
        for (int t = 0; t < nt; ++t) th.emplace_back(range, t);
        for (auto& x : th) x.join();
    }
    for (const Work& w : work)
        if (w.fail >= 0) {
            set_error("hfv_scheme_create: cell " + std::to_string(w.fail) + " reaches fewer than M = " +
                      std::to_string(M) + " cells within 16 face layers");
            return HFV_ERR_STENCIL;
        }
    return HFV_OK;
}

}  // namespace hfv
