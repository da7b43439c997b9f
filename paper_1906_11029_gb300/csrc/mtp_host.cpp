// Host side of the MTP library: mesh construction, tent pitching, C ABI.
//
// Built with -ffp-contract=off: the pitcher's arithmetic is specified operation by
// operation (see mtp_pitch_tents in mtp.h) and must not be contracted into FMAs, so
// its tent list is reproducible bit for bit on any IEEE-754 host.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "mtp_internal.h"

namespace mtp {

static thread_local std::string g_error;

int set_error(int code, const std::string& msg) {
    g_error = msg;
    return code;
}

// ---------------------------------------------------------------------------------
// reference tables, cached per (dim, p)
// ---------------------------------------------------------------------------------
static const RefTables& ref_tables(int dim, int p) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, std::unique_ptr<RefTables>> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto key = std::make_pair(dim, p);
    auto it = cache.find(key);
    if (it == cache.end()) it = cache.emplace(key, std::make_unique<RefTables>(build_ref_tables(dim, p))).first;
    return *it->second;
}

// ---------------------------------------------------------------------------------
// mesh
// ---------------------------------------------------------------------------------
static int build_mesh(int dim, int64_t nv, const double* X, int64_t ne, const int32_t* E,
                      const double* eps, const double* mu, const mtp_options& o, Mesh& m) {
    m.dim = dim;
    m.p = o.p;
    m.q = o.q > 0 ? o.q : o.p + 1;
    m.m = o.m > 0 ? o.m : 2 * o.p;
    m.precision = o.precision;
    m.n_rhs = o.n_rhs > 0 ? o.n_rhs : 1;
    m.flags = o.flags;
    m.nf = n_fields(dim);
    m.nb = n_basis(dim, o.p);
    m.nfb = n_face_basis(dim, o.p);
    m.nv = nv;
    m.ne = ne;
    const int nvert = dim + 1;
    m.verts.assign(X, X + nv * dim);
    for (int64_t i = 0; i < nv * dim; ++i)
        if (!std::isfinite(X[i])) return set_error(MTP_EINVAL, "non-finite vertex coordinate");
    m.elems.resize(ne * nvert);
    m.eps.assign(eps, eps + ne);
    m.mu.assign(mu, mu + ne);
    for (int64_t e = 0; e < ne; ++e) {
        if (!(eps[e] > 0) || !(mu[e] > 0) || !std::isfinite(eps[e]) || !std::isfinite(mu[e]))
            return set_error(MTP_EINVAL, "eps and mu must be positive and finite (element " + std::to_string(e) + ")");
        int32_t* el = &m.elems[e * nvert];
        for (int i = 0; i < nvert; ++i) {
            int32_t v = E[e * nvert + i];
            if (v < 0 || v >= nv) return set_error(MTP_EINVAL, "element " + std::to_string(e) + " has a vertex id out of range");
            el[i] = v;
        }
        std::sort(el, el + nvert);
        for (int i = 1; i < nvert; ++i)
            if (el[i] == el[i - 1]) return set_error(MTP_EMESH, "element " + std::to_string(e) + " repeats a vertex");
    }
    // geometry
    m.geo.assign(ne * kGeoStride, 0.0);
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* el = &m.elems[e * nvert];
        double P[4][3] = {};
        for (int i = 0; i < nvert; ++i)
            for (int c = 0; c < dim; ++c) P[i][c] = X[(int64_t)el[i] * dim + c];
        double J[3][3] = {}, Ji[3][3] = {};   // J columns = edges P_l - P_0
        for (int l = 0; l < dim; ++l)
            for (int c = 0; c < dim; ++c) J[c][l] = P[l + 1][c] - P[0][c];
        double det;
        if (dim == 2) {
            det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
            Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
            Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
        } else {
            double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
            double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
            double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
            det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
            Ji[0][0] = c00 / det;
            Ji[1][0] = c01 / det;
            Ji[2][0] = c02 / det;
            Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
            Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
            Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
            Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
            Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
            Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
        }
        double scale = 0;
        for (int l = 0; l < dim; ++l)
            for (int c = 0; c < dim; ++c) scale = std::fmax(scale, std::fabs(J[c][l]));
        if (!(std::fabs(det) > 1e-13 * std::pow(scale, dim)))
            return set_error(MTP_EMESH, "element " + std::to_string(e) + " is degenerate");
        double* g = &m.geo[e * kGeoStride];
        double gl[4][3] = {};
        for (int l = 0; l < dim; ++l)
            for (int c = 0; c < dim; ++c) gl[l + 1][c] = Ji[l][c];
        for (int c = 0; c < dim; ++c) {
            double s = 0;
            for (int l = 1; l <= dim; ++l) s += gl[l][c];
            gl[0][c] = -s;
        }
        double adet = std::fabs(det);
        for (int i = 0; i < nvert; ++i) {
            double n2 = 0;
            for (int c = 0; c < 3; ++c) n2 += gl[i][c] * gl[i][c];
            double nn = std::sqrt(n2);
            for (int c = 0; c < 3; ++c) {
                g[3 * i + c] = gl[i][c];
                g[12 + 3 * i + c] = -gl[i][c] / nn;
            }
            g[24 + i] = adet * nn;          // (dim-1)! |F_i|
        }
        g[28] = 1.0 / std::sqrt(adet);
        g[29] = eps[e];
        g[30] = mu[e];
        g[31] = std::sqrt(mu[e] / eps[e]);
    }
    // facets: sort (facet key, element, local facet)
    struct FK { int32_t v[3]; int64_t e; int f; };
    std::vector<FK> keys;
    keys.reserve(ne * nvert);
    for (int64_t e = 0; e < ne; ++e)
        for (int f = 0; f < nvert; ++f) {
            FK k{{-1, -1, -1}, e, f};
            int n = 0;
            for (int i = 0; i < nvert; ++i)
                if (i != f) k.v[n++] = m.elems[e * nvert + i];
            keys.push_back(k);
        }
    std::sort(keys.begin(), keys.end(), [](const FK& a, const FK& b) {
        if (a.v[0] != b.v[0]) return a.v[0] < b.v[0];
        if (a.v[1] != b.v[1]) return a.v[1] < b.v[1];
        if (a.v[2] != b.v[2]) return a.v[2] < b.v[2];
        return a.e < b.e;
    });
    m.nbr.assign(ne * nvert, -1);
    m.nbr_face.assign(ne * nvert, -1);
    auto same = [](const FK& a, const FK& b) { return a.v[0] == b.v[0] && a.v[1] == b.v[1] && a.v[2] == b.v[2]; };
    for (size_t i = 0; i < keys.size();) {
        size_t j = i + 1;
        while (j < keys.size() && same(keys[i], keys[j])) ++j;
        if (j - i > 2) return set_error(MTP_EMESH, "a facet is shared by more than two elements");
        if (j - i == 2) {
            const FK &a = keys[i], &b = keys[i + 1];
            m.nbr[a.e * nvert + a.f] = (int32_t)b.e;
            m.nbr_face[a.e * nvert + a.f] = (int8_t)b.f;
            m.nbr[b.e * nvert + b.f] = (int32_t)a.e;
            m.nbr_face[b.e * nvert + b.f] = (int8_t)a.f;
        }
        i = j;
    }
    // vertex patches
    m.patch_ptr.assign(nv + 1, 0);
    for (int64_t e = 0; e < ne; ++e)
        for (int i = 0; i < nvert; ++i) m.patch_ptr[m.elems[e * nvert + i] + 1]++;
    for (int64_t v = 0; v < nv; ++v) m.patch_ptr[v + 1] += m.patch_ptr[v];
    m.patch_elem.assign(m.patch_ptr[nv], 0);
    {
        std::vector<int64_t> fill(m.patch_ptr.begin(), m.patch_ptr.end() - 1);
        for (int64_t e = 0; e < ne; ++e)
            for (int i = 0; i < nvert; ++i) m.patch_elem[fill[m.elems[e * nvert + i]]++] = (int32_t)e;
    }
    m.max_patch = 0;
    m.patch_info.assign(m.patch_elem.size() * 12, 0);
    // order each patch by (local index of V, element id): elements sharing the lambda_V-weighted
    // reference tables are adjacent, so the tent kernel can pair them
    auto local_index = [&](int32_t e, int64_t v) {
        int j = 0;
        while (m.elems[(int64_t)e * nvert + j] != v) ++j;
        return j;
    };
    for (int64_t v = 0; v < nv; ++v)
        std::stable_sort(m.patch_elem.begin() + m.patch_ptr[v], m.patch_elem.begin() + m.patch_ptr[v + 1],
                         [&](int32_t x, int32_t y) {
                             const int jx = local_index(x, v), jy = local_index(y, v);
                             return jx != jy ? jx < jy : x < y;
                         });
    for (int64_t v = 0; v < nv; ++v) {
        int64_t b = m.patch_ptr[v], n = m.patch_ptr[v + 1] - b;
        m.max_patch = std::max<int>(m.max_patch, (int)n);
        for (int64_t k = 0; k < n; ++k) {
            int32_t e = m.patch_elem[b + k];
            int8_t* info = &m.patch_info[(b + k) * 12];
            int j = 0;
            while (m.elems[(int64_t)e * nvert + j] != v) ++j;
            info[0] = (int8_t)j;
            for (int f = 0; f < nvert; ++f) {
                int8_t slot = -2, nf = -1;
                if (f != j) {
                    int32_t e2 = m.nbr[(int64_t)e * nvert + f];
                    if (e2 < 0) {
                        slot = -1;
                    } else {
                        for (int64_t k2 = 0; k2 < n; ++k2)
                            if (m.patch_elem[b + k2] == e2) slot = (int8_t)k2;
                        if (slot < 0) return set_error(MTP_EMESH, "facet neighbour outside the vertex patch (non-conforming mesh)");
                        nf = m.nbr_face[(int64_t)e * nvert + f];
                    }
                }
                info[4 + f] = slot;
                info[8 + f] = nf;
            }
        }
    }
    // vertex adjacency: the other vertices of the elements in each patch
    m.adj_ptr.assign(nv + 1, 0);
    {
        std::vector<std::vector<int32_t>> nb(nv);
        for (int64_t v = 0; v < nv; ++v) {
            for (int64_t q = m.patch_ptr[v]; q < m.patch_ptr[v + 1]; ++q) {
                const int32_t e = m.patch_elem[q];
                for (int i = 0; i < nvert; ++i)
                    if (m.elems[(int64_t)e * nvert + i] != v) nb[v].push_back(m.elems[(int64_t)e * nvert + i]);
            }
            std::sort(nb[v].begin(), nb[v].end());
            nb[v].erase(std::unique(nb[v].begin(), nb[v].end()), nb[v].end());
            m.adj_ptr[v + 1] = m.adj_ptr[v] + (int64_t)nb[v].size();
        }
        m.adj.reserve(m.adj_ptr[nv]);
        for (int64_t v = 0; v < nv; ++v) m.adj.insert(m.adj.end(), nb[v].begin(), nb[v].end());
    }
    const int cap = dim == 2 ? kMaxPatch2D : kMaxPatch3D;
    if (m.max_patch > cap)
        return set_error(MTP_EUNSUPPORTED, "largest vertex patch has " + std::to_string(m.max_patch) +
                                               " elements; the library is compiled for patches of up to " + std::to_string(cap));
    m.ref = ref_tables(dim, o.p);
    return MTP_OK;
}

// ---------------------------------------------------------------------------------
// pitcher (see mtp_pitch_tents in mtp.h for the rule)
// ---------------------------------------------------------------------------------
int pitch_graph(const Mesh& m, const double* wavespeed, double cf, PitchGraph& g) {
    const int d = m.dim, nvert = d + 1;
    const int64_t nv = m.nv, ne = m.ne;
    std::vector<double> k(nv, INFINITY), c(ne);
    for (int64_t e = 0; e < ne; ++e) {
        c[e] = wavespeed ? wavespeed[e] : 1.0 / std::sqrt(m.eps[e] * m.mu[e]);
        if (!(c[e] > 0) || !std::isfinite(c[e])) return set_error(MTP_EINVAL, "wave speeds must be positive and finite");
    }
    // element heights on the sorted vertex order, operation order fixed
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* el = &m.elems[e * nvert];
        double P[4][3] = {};
        for (int i = 0; i < nvert; ++i)
            for (int q = 0; q < d; ++q) P[i][q] = m.verts[(int64_t)el[i] * d + q];
        double H[4];
        if (d == 2) {
            double det = (P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) - (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]);
            double adet = std::fabs(det);
            for (int i = 0; i < 3; ++i) {
                int a = i == 0 ? 1 : 0, b = i == 2 ? 1 : 2;
                double dx = P[b][0] - P[a][0];
                double dy = P[b][1] - P[a][1];
                H[i] = adet / std::sqrt(dx * dx + dy * dy);
            }
        } else {
            double e1[3], e2[3], e3[3];
            for (int q = 0; q < 3; ++q) {
                e1[q] = P[1][q] - P[0][q];
                e2[q] = P[2][q] - P[0][q];
                e3[q] = P[3][q] - P[0][q];
            }
            double det = ((e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0])) +
                          e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]));
            double adet = std::fabs(det);
            for (int i = 0; i < 4; ++i) {
                int idx[3], n = 0;
                for (int q = 0; q < 4; ++q)
                    if (q != i) idx[n++] = q;
                double u[3], w[3];
                for (int q = 0; q < 3; ++q) {
                    u[q] = P[idx[1]][q] - P[idx[0]][q];
                    w[q] = P[idx[2]][q] - P[idx[0]][q];
                }
                double cx = u[1] * w[2] - u[2] * w[1];
                double cy = u[2] * w[0] - u[0] * w[2];
                double cz = u[0] * w[1] - u[1] * w[0];
                H[i] = adet / std::sqrt((cx * cx + cy * cy) + cz * cz);
            }
        }
        for (int i = 0; i < nvert; ++i) k[el[i]] = std::fmin(k[el[i]], H[i]);
    }
    // edges: (a < b) -> max wave speed; then directed CSR sorted by (src, dst)
    std::vector<std::pair<int64_t, double>> ekeys;   // key = a * nv + b
    ekeys.reserve(ne * nvert * d / 2);
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* el = &m.elems[e * nvert];
        for (int i = 0; i < nvert; ++i)
            for (int j = i + 1; j < nvert; ++j) ekeys.emplace_back((int64_t)el[i] * nv + el[j], c[e]);
    }
    std::sort(ekeys.begin(), ekeys.end());
    std::vector<int64_t>& ptr = g.ptr;
    ptr.assign(nv + 1, 0);
    std::vector<std::pair<int64_t, double>> edges;   // unique, with max c
    for (size_t i = 0; i < ekeys.size();) {
        size_t j = i;
        double cm = ekeys[i].second;
        while (j < ekeys.size() && ekeys[j].first == ekeys[i].first) { cm = std::fmax(cm, ekeys[j].second); ++j; }
        edges.emplace_back(ekeys[i].first, cm);
        i = j;
    }
    for (auto& ed : edges) { ptr[ed.first / nv + 1]++; ptr[ed.first % nv + 1]++; }
    for (int64_t v = 0; v < nv; ++v) ptr[v + 1] += ptr[v];
    std::vector<int32_t>& dst = g.dst;
    std::vector<double>& bnd = g.bnd;
    dst.assign(ptr[nv], 0);
    bnd.assign(ptr[nv], 0.0);
    {
        std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
        for (auto& ed : edges) {
            int64_t a = ed.first / nv, b = ed.first % nv;
            double bab = (cf * std::fmin(k[a], k[b])) / ((double)d * ed.second);
            dst[fill[a]] = (int32_t)b; bnd[fill[a]++] = bab;
            dst[fill[b]] = (int32_t)a; bnd[fill[b]++] = bab;
        }
        for (int64_t v = 0; v < nv; ++v) {   // sort each row by dst
            std::vector<std::pair<int32_t, double>> row;
            for (int64_t q = ptr[v]; q < ptr[v + 1]; ++q) row.emplace_back(dst[q], bnd[q]);
            std::sort(row.begin(), row.end());
            for (int64_t q = ptr[v]; q < ptr[v + 1]; ++q) { dst[q] = row[q - ptr[v]].first; bnd[q] = row[q - ptr[v]].second; }
        }
    }
    return MTP_OK;
}

int pitch(const Mesh& m, const double* wavespeed, double cf, double T, Tents& out) {
    const int64_t nv = m.nv;
    PitchGraph g;
    int rc = pitch_graph(m, wavespeed, cf, g);
    if (rc != MTP_OK) return rc;
    const std::vector<int64_t>& ptr = g.ptr;
    const std::vector<int32_t>& dst = g.dst;
    const std::vector<double>& bnd = g.bnd;
    // rounds
    std::vector<double> tau(nv, 0.0);
    std::vector<int64_t> last(nv, -1);
    std::vector<int32_t> tv, tl;
    std::vector<double> tb, tt;
    std::vector<char> dirty(nv, 1), is_sel(nv, 0);
    std::vector<int32_t> cand_list, sel;
    for (int64_t v = 0; v < nv; ++v) cand_list.push_back((int32_t)v);
    std::vector<double> newt;
    std::vector<int64_t> newl;
    while (true) {
        sel.clear();
        for (int32_t v : cand_list) {
            dirty[v] = 0;
            if (!(tau[v] < T)) continue;
            bool mn = true;
            for (int64_t q = ptr[v]; q < ptr[v + 1]; ++q) {
                int32_t w = dst[q];
                bool less = (tau[v] < tau[w]) || (tau[v] == tau[w] && v < w);
                if (!less) { mn = false; break; }
            }
            if (mn) sel.push_back(v);
        }
        if (sel.empty()) break;
        std::sort(sel.begin(), sel.end());
        newt.assign(sel.size(), 0);
        newl.assign(sel.size(), 0);
        for (size_t i = 0; i < sel.size(); ++i) {
            int32_t v = sel[i];
            double cm = INFINITY;
            int64_t lm = last[v];
            for (int64_t q = ptr[v]; q < ptr[v + 1]; ++q) {
                double x = tau[dst[q]] + bnd[q];
                if (x < cm) cm = x;
                if (last[dst[q]] > lm) lm = last[dst[q]];
            }
            newt[i] = std::fmin(T, cm);
            newl[i] = 1 + lm;
        }
        cand_list.clear();
        for (size_t i = 0; i < sel.size(); ++i) {
            int32_t v = sel[i];
            tv.push_back(v);
            tb.push_back(tau[v]);
            tt.push_back(newt[i]);
            tl.push_back((int32_t)newl[i]);
            tau[v] = newt[i];
            last[v] = newl[i];
            if (!dirty[v]) { dirty[v] = 1; cand_list.push_back(v); }
            for (int64_t q = ptr[v]; q < ptr[v + 1]; ++q)
                if (!dirty[dst[q]]) { dirty[dst[q]] = 1; cand_list.push_back(dst[q]); }
        }
    }
    for (int64_t v = 0; v < nv; ++v)
        if (tau[v] != T) return set_error(MTP_ECAUSAL, "pitching stalled before reaching T");
    // counting sort by (layer, vertex): within a layer, vertices ascending
    int64_t nl = 0;
    for (int32_t l : tl) nl = std::max<int64_t>(nl, (int64_t)l + 1);
    const size_t n = tv.size();
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) {
        if (tl[a] != tl[b]) return tl[a] < tl[b];
        return tv[a] < tv[b];
    });
    out.vertex.resize(n); out.layer.resize(n); out.t_bot.resize(n); out.t_top.resize(n);
    for (size_t i = 0; i < n; ++i) {
        out.vertex[i] = tv[order[i]]; out.layer[i] = tl[order[i]];
        out.t_bot[i] = tb[order[i]]; out.t_top[i] = tt[order[i]];
    }
    out.layer_ptr.assign(nl + 1, 0);
    for (size_t i = 0; i < n; ++i) out.layer_ptr[out.layer[i] + 1]++;
    for (int64_t l = 0; l < nl; ++l) out.layer_ptr[l + 1] += out.layer_ptr[l];
    pitch_finish(m, T, cf, out);
    return MTP_OK;
}

void pitch_finish(const Mesh& m, double T, double cf, Tents& out) {
    double dofs = 0;
    for (size_t i = 0; i < out.vertex.size(); ++i) {
        int32_t v = out.vertex[i];
        dofs += (double)(m.patch_ptr[v + 1] - m.patch_ptr[v]);
    }
    out.spacetime_dofs = dofs * m.nf * m.nb * (double)m.m * (double)m.q * m.n_rhs;
    out.T = T;
    out.cf = cf;
}

}  // namespace mtp

// =================================================================================
// C ABI
// =================================================================================
using namespace mtp;

struct mtp_mesh { Mesh m; };
struct mtp_tents { Tents t; };
struct mtp_batch { Batch b; };

#define MTP_GUARD_BEGIN try {
#define MTP_GUARD_END                                                        \
    }                                                                        \
    catch (const std::bad_alloc&) { return set_error(MTP_ENOMEM, "host allocation failed"); } \
    catch (const std::exception& ex) { return set_error(MTP_EINVAL, ex.what()); }

extern "C" {

int mtp_mesh_create(int dim, int64_t n_verts, const double* vertices, int64_t n_elems,
                    const int32_t* elements, const double* eps, const double* mu,
                    const mtp_options* opts, mtp_mesh_t* out) {
    MTP_GUARD_BEGIN
    if (!out) return set_error(MTP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!vertices || !elements || !eps || !mu || !opts) return set_error(MTP_EINVAL, "NULL input array");
    if (dim != 2 && dim != 3) return set_error(MTP_EINVAL, "dim must be 2 or 3");
    if (n_verts < dim + 1 || n_elems < 1) return set_error(MTP_EINVAL, "mesh too small");
    if (n_verts > INT32_MAX || n_elems > INT32_MAX) return set_error(MTP_EINVAL, "mesh too large for int32 ids");
    if (opts->p < 1 || opts->p > kMaxDegree) return set_error(MTP_EUNSUPPORTED, "p must be in 1..5");
    const bool tc = opts->precision == MTP_TF32 || opts->precision == MTP_TF32X3;
    if (tc && opts->p > 4) return set_error(MTP_EUNSUPPORTED, "tensor-core precisions are built for p <= 4");
    if (opts->q < 0 || opts->m < 0 || opts->q > 8 || opts->m > 64) return set_error(MTP_EINVAL, "q must be in 0..8 and m in 0..64");
    if (opts->precision < MTP_FP64 || opts->precision > MTP_FP32_SPLIT) return set_error(MTP_EINVAL, "unknown precision");
    if (tc && dim != 3) return set_error(MTP_EUNSUPPORTED, "tensor-core precisions are built for 3D meshes");
    if (opts->n_rhs < 0 || opts->n_rhs > 4096) return set_error(MTP_EINVAL, "n_rhs must be in 0..4096");
    if (opts->flags & ~(MTP_FLAG_LAYER_LAUNCHES | MTP_FLAG_TEST_STALL | MTP_FLAG_SUBSTITUTED_RK4))
        return set_error(MTP_EINVAL, "unknown flag bits");
    if ((opts->flags & MTP_FLAG_SUBSTITUTED_RK4) && opts->precision != MTP_FP64)
        return set_error(MTP_EUNSUPPORTED, "MTP_FLAG_SUBSTITUTED_RK4 is built for MTP_FP64");
    auto h = std::make_unique<mtp_mesh>();
    int rc = build_mesh(dim, n_verts, vertices, n_elems, elements, eps, mu, *opts, h->m);
    if (rc != MTP_OK) return rc;
    *out = h.release();
    return MTP_OK;
    MTP_GUARD_END
}

void mtp_mesh_destroy(mtp_mesh_t mesh) {
    if (!mesh) return;
    device_mesh_free(mesh->m);
    delete mesh;
}

int mtp_mesh_info(mtp_mesh_t mesh, int* dim, int* nf, int* nb, int64_t* ne, int64_t* nv, int* max_patch) {
    if (!mesh) return set_error(MTP_EINVAL, "mesh is NULL");
    const Mesh& m = mesh->m;
    if (dim) *dim = m.dim;
    if (nf) *nf = m.nf;
    if (nb) *nb = m.nb;
    if (ne) *ne = m.ne;
    if (nv) *nv = m.nv;
    if (max_patch) *max_patch = m.max_patch;
    return MTP_OK;
}

int mtp_pitch_tents(mtp_mesh_t mesh, const double* wavespeed, double cf, double T, mtp_tents_t* out) {
    MTP_GUARD_BEGIN
    if (!out) return set_error(MTP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh) return set_error(MTP_EINVAL, "mesh is NULL");
    if (!(cf > 0 && cf < 1)) return set_error(MTP_EINVAL, "causality factor must be in (0, 1)");
    if (!(T > 0) || !std::isfinite(T)) return set_error(MTP_EINVAL, "T must be positive and finite");
    auto h = std::make_unique<mtp_tents>();
    h->t.mesh = &mesh->m;
    int rc = pitch(mesh->m, wavespeed, cf, T, h->t);
    if (rc != MTP_OK) return rc;
    *out = h.release();
    return MTP_OK;
    MTP_GUARD_END
}

int mtp_pitch_tents_device(mtp_mesh_t mesh, const double* wavespeed, double cf, double T, mtp_tents_t* out,
                           void* stream) {
    MTP_GUARD_BEGIN
    if (!out) return set_error(MTP_EINVAL, "out is NULL");
    *out = nullptr;
    if (!mesh) return set_error(MTP_EINVAL, "mesh is NULL");
    if (!(cf > 0 && cf < 1)) return set_error(MTP_EINVAL, "causality factor must be in (0, 1)");
    if (!(T > 0) || !std::isfinite(T)) return set_error(MTP_EINVAL, "T must be positive and finite");
    auto h = std::make_unique<mtp_tents>();
    h->t.mesh = &mesh->m;
    PitchGraph g;
    int rc = pitch_graph(mesh->m, wavespeed, cf, g);
    if (rc != MTP_OK) return rc;
    rc = device_pitch(mesh->m, g, T, h->t, stream);
    if (rc != MTP_OK) return rc;
    pitch_finish(mesh->m, T, cf, h->t);
    *out = h.release();
    return MTP_OK;
    MTP_GUARD_END
}

void mtp_tents_destroy(mtp_tents_t tents) {
    if (!tents) return;
    device_tents_free(tents->t);
    delete tents;
}

int mtp_tents_info(mtp_tents_t tents, int64_t* n_tents, int64_t* n_layers, double* st_dofs) {
    if (!tents) return set_error(MTP_EINVAL, "tents is NULL");
    const Tents& t = tents->t;
    if (n_tents) *n_tents = (int64_t)t.vertex.size();
    if (n_layers) *n_layers = (int64_t)t.layer_ptr.size() - 1;
    if (st_dofs) *st_dofs = t.spacetime_dofs;
    return MTP_OK;
}

int mtp_tents_get(mtp_tents_t tents, int32_t* vertex, double* t_bot, double* t_top, int32_t* layer,
                  int64_t* layer_ptr) {
    if (!tents) return set_error(MTP_EINVAL, "tents is NULL");
    const Tents& t = tents->t;
    const size_t n = t.vertex.size();
    if (vertex) std::memcpy(vertex, t.vertex.data(), n * sizeof(int32_t));
    if (t_bot) std::memcpy(t_bot, t.t_bot.data(), n * sizeof(double));
    if (t_top) std::memcpy(t_top, t.t_top.data(), n * sizeof(double));
    if (layer) std::memcpy(layer, t.layer.data(), n * sizeof(int32_t));
    if (layer_ptr) std::memcpy(layer_ptr, t.layer_ptr.data(), t.layer_ptr.size() * sizeof(int64_t));
    return MTP_OK;
}

int mtp_state_from_lattice(mtp_mesh_t mesh, const double* vals, void* state, void* stream) {
    MTP_GUARD_BEGIN
    if (!mesh || !vals || !state) return set_error(MTP_EINVAL, "NULL argument");
    return device_from_lattice(mesh->m, vals, state, stream);
    MTP_GUARD_END
}

int mtp_state_to_lattice(mtp_mesh_t mesh, const void* state, double* vals, void* stream) {
    MTP_GUARD_BEGIN
    if (!mesh || !vals || !state) return set_error(MTP_EINVAL, "NULL argument");
    return device_to_lattice(mesh->m, state, vals, stream);
    MTP_GUARD_END
}

int mtp_evolve(mtp_tents_t tents, void* state, double T, void* stream) {
    MTP_GUARD_BEGIN
    if (!tents || !state) return set_error(MTP_EINVAL, "NULL argument");
    if (T != tents->t.T) return set_error(MTP_EINVAL, "T differs from the T the tents were pitched to");
    return device_evolve(tents->t, state, 0, (int64_t)tents->t.layer_ptr.size() - 1, true, stream);
    MTP_GUARD_END
}

int mtp_evolve_layers(mtp_tents_t tents, void* state, int64_t lb, int64_t le, void* stream) {
    MTP_GUARD_BEGIN
    if (!tents || !state) return set_error(MTP_EINVAL, "NULL argument");
    const int64_t nl = (int64_t)tents->t.layer_ptr.size() - 1;
    if (lb < 0 || le > nl || lb > le) return set_error(MTP_EINVAL, "layer range out of bounds");
    return device_evolve(tents->t, state, lb, le, false, stream);
    MTP_GUARD_END
}

int mtp_evolve_host(mtp_tents_t tents, const void* in, void* out, double T, void* stream) {
    MTP_GUARD_BEGIN
    if (!tents || !in || !out) return set_error(MTP_EINVAL, "NULL argument");
    if (T != tents->t.T) return set_error(MTP_EINVAL, "T differs from the T the tents were pitched to");
    return device_evolve_host(tents->t, in, out, stream);
    MTP_GUARD_END
}

int mtp_adjoint(mtp_tents_t tents, const void* state0, const void* lamT, void* lam0, double* geps, double* gmu,
                int64_t checkpoint_every, void* stream) {
    MTP_GUARD_BEGIN
    if (!tents || !state0 || !lamT || !lam0 || !geps || !gmu) return set_error(MTP_EINVAL, "NULL argument");
    if (checkpoint_every < 0) return set_error(MTP_EINVAL, "checkpoint_every must be >= 0");
    return device_adjoint(tents->t, state0, lamT, lam0, geps, gmu, checkpoint_every, stream);
    MTP_GUARD_END
}

int mtp_tents_set_launch(mtp_tents_t tents, int launch) {
    if (!tents) return set_error(MTP_EINVAL, "tents is NULL");
    if (launch < 0 || launch > 2) return set_error(MTP_EINVAL, "launch must be 0, 1 or 2");
    tents->t.launch = launch;
    return MTP_OK;
}

int mtp_tents_set_variant(mtp_tents_t tents, int variant) {
    if (!tents) return set_error(MTP_EINVAL, "tents is NULL");
    if (variant < 0 || variant > 4) return set_error(MTP_EINVAL, "variant must be 0 .. 4");
    const Mesh& m = *tents->t.mesh;
    if (variant > 0 && (m.precision != MTP_FP32 || (m.flags & MTP_FLAG_SUBSTITUTED_RK4)))
        return set_error(MTP_EUNSUPPORTED, "kernel variants 1 .. 4 are built for MTP_FP32 SAT meshes");
    if (variant >= 3 && (m.dim != 3 || m.p < 2 || m.p > 4))
        return set_error(MTP_EUNSUPPORTED, "kernel variants 3 and 4 (tcgen05 volume term) are built for 3D, p = 2..4");
    if (variant >= 3 && m.max_patch * m.nf > 256)
        return set_error(MTP_EUNSUPPORTED, "kernel variants 3 and 4 take patches of at most 42 tetrahedra");
    tents->t.variant = variant;
    return MTP_OK;
}

int mtp_tents_autotune(mtp_tents_t tents, void* scratch_state, int64_t lb, int64_t le, int* best, double* ms_out,
                       void* stream) {
    MTP_GUARD_BEGIN
    if (!tents || !scratch_state) return set_error(MTP_EINVAL, "NULL argument");
    const int64_t nl = (int64_t)tents->t.layer_ptr.size() - 1;
    if (lb < 0 || le > nl || lb >= le) return set_error(MTP_EINVAL, "layer window out of bounds or empty");
    return device_autotune(tents->t, scratch_state, lb, le, best, ms_out, stream);
    MTP_GUARD_END
}

int mtp_batch_create(int64_t n, const mtp_tents_t* tents, mtp_batch_t* out) {
    MTP_GUARD_BEGIN
    if (!out) return set_error(MTP_EINVAL, "out is NULL");
    *out = nullptr;
    if (n < 1 || !tents) return set_error(MTP_EINVAL, "need at least one instance");
    auto h = std::make_unique<mtp_batch>();
    for (int64_t i = 0; i < n; ++i) {
        if (!tents[i]) return set_error(MTP_EINVAL, "NULL tents handle in the batch");
        const Mesh& m = *tents[i]->t.mesh;
        const Mesh& m0 = *tents[0]->t.mesh;
        if (m.dim != m0.dim || m.precision != m0.precision)
            return set_error(MTP_EINVAL, "all instances of a batch need the same dimension and precision");
        if (m.q != m.p + 1 || m.m != 2 * m.p)
            return set_error(MTP_EUNSUPPORTED, "batched instances use the default q = p + 1, m = 2p");
        h->b.inst.push_back(&tents[i]->t);
        h->b.spacetime_dofs += tents[i]->t.spacetime_dofs;
    }
    // tickets: all tents ordered by (layer, instance, vertex)
    int64_t nt = 0, nl = 0;
    for (Tents* t : h->b.inst) {
        nt += (int64_t)t->vertex.size();
        nl = std::max<int64_t>(nl, (int64_t)t->layer_ptr.size() - 1);
    }
    h->b.ticket_inst.reserve(nt);
    h->b.ticket_tent.reserve(nt);
    for (int64_t l = 0; l < nl; ++l)
        for (int64_t i = 0; i < n; ++i) {
            const Tents& t = *h->b.inst[i];
            if (l + 1 >= (int64_t)t.layer_ptr.size()) continue;
            for (int64_t q = t.layer_ptr[l]; q < t.layer_ptr[l + 1]; ++q) {
                h->b.ticket_inst.push_back((int32_t)i);
                h->b.ticket_tent.push_back(q);
            }
        }
    *out = h.release();
    return MTP_OK;
    MTP_GUARD_END
}

void mtp_batch_destroy(mtp_batch_t batch) {
    if (!batch) return;
    device_batch_free(batch->b);
    delete batch;
}

int mtp_batch_info(mtp_batch_t batch, int64_t* n_instances, int64_t* n_tents, double* spacetime_dofs) {
    if (!batch) return set_error(MTP_EINVAL, "batch is NULL");
    if (n_instances) *n_instances = (int64_t)batch->b.inst.size();
    if (n_tents) *n_tents = (int64_t)batch->b.ticket_inst.size();
    if (spacetime_dofs) *spacetime_dofs = batch->b.spacetime_dofs;
    return MTP_OK;
}

int mtp_batch_evolve(mtp_batch_t batch, void* const* states, void* stream) {
    MTP_GUARD_BEGIN
    if (!batch || !states) return set_error(MTP_EINVAL, "NULL argument");
    for (size_t i = 0; i < batch->b.inst.size(); ++i)
        if (!states[i]) return set_error(MTP_EINVAL, "NULL state for instance " + std::to_string(i));
    return device_batch_evolve(batch->b, states, stream);
    MTP_GUARD_END
}

int mtp_energy(mtp_mesh_t mesh, const void* state, double* out_host, void* stream) {
    MTP_GUARD_BEGIN
    if (!mesh || !state || !out_host) return set_error(MTP_EINVAL, "NULL argument");
    return device_energy(mesh->m, state, out_host, stream);
    MTP_GUARD_END
}

const char* mtp_last_error(void) { return g_error.c_str(); }

}  // extern "C"
