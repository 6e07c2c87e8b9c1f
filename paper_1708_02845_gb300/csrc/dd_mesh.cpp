// Host-side mesh topology and cotangent Laplacian (Section IV).
//
// Boundary vertices are the endpoints of edges with one incident triangle;
// the caller's loops must list exactly those vertices, consecutive ones joined
// by a boundary edge, and their concatenation fixes the column order of the
// Poisson kernel.  Interior vertices keep ascending id order (the I block of
// Eq. 18).  The Laplacian weight of an edge is half the sum of the cotangents
// of the angles opposite it (one angle on a boundary edge).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "dd_internal.h"

namespace {

struct HalfEdge {
    uint64_t key;   // (min << 32) | max
    int32_t t;      // triangle
    int32_t c;      // local index of the corner opposite the edge
    int32_t a, b;   // directed edge a -> b in the triangle's orientation
};

inline uint64_t edge_key(int32_t a, int32_t b) {
    uint32_t lo = (uint32_t)std::min(a, b), hi = (uint32_t)std::max(a, b);
    return ((uint64_t)lo << 32) | hi;
}

dd_status fail(std::string &err, const char *fmt, long long a = 0, long long b = 0) {
    char buf[256];
    std::snprintf(buf, sizeof buf, fmt, a, b);
    err = buf;
    return DD_EINVAL;
}

}  // namespace

dd_status build_host_mesh(const double *xy, int64_t n_v, const int32_t *tri, int64_t n_t,
                          const int32_t *loop_idx, const int64_t *loop_off, int32_t n_loops,
                          HostMesh &M, std::string &err) {
    if (!xy || !tri || !loop_idx || !loop_off) return fail(err, "null mesh pointer");
    if (n_v < 3 || n_t < 1) return fail(err, "mesh needs at least 3 vertices and 1 triangle");
    if (n_v > (int64_t)INT32_MAX || n_t > (int64_t)INT32_MAX / 3) return fail(err, "mesh too large");
    if (n_loops < 1) return fail(err, "need at least one boundary loop");
    if (loop_off[0] != 0) return fail(err, "loop_off[0] must be 0");
    for (int32_t l = 0; l < n_loops; ++l)
        if (loop_off[l + 1] - loop_off[l] < 3) return fail(err, "loop %lld has fewer than 3 vertices", l);
    const int64_t k = loop_off[n_loops];

    M.n_v = n_v;
    M.n_t = n_t;
    M.xy.assign(xy, xy + 2 * n_v);
    M.tri.assign(tri, tri + 3 * n_t);
    for (int64_t i = 0; i < 2 * n_v; ++i)
        if (!std::isfinite(xy[i])) return fail(err, "non-finite coordinate at vertex %lld", i / 2);

    // triangles: ids, orientation, gradient basis of the hat functions
    M.gphi.resize(6 * n_t);
    for (int64_t t = 0; t < n_t; ++t) {
        const int32_t *v = tri + 3 * t;
        for (int c = 0; c < 3; ++c)
            if (v[c] < 0 || v[c] >= n_v) return fail(err, "triangle %lld has vertex id out of range", t);
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) return fail(err, "triangle %lld repeats a vertex", t);
        double p[3][2];
        for (int c = 0; c < 3; ++c) {
            p[c][0] = xy[2 * v[c]];
            p[c][1] = xy[2 * v[c] + 1];
        }
        double a2 = (p[1][0] - p[0][0]) * (p[2][1] - p[0][1]) - (p[1][1] - p[0][1]) * (p[2][0] - p[0][0]);
        if (!(a2 > 0.0)) return fail(err, "triangle %lld is not counter-clockwise with positive area", t);
        for (int c = 0; c < 3; ++c) {
            // grad(phi_c) = J e_c / (2A), e_c = p[c+2] - p[c+1], J = +90 degree rotation
            const double *pa = p[(c + 1) % 3], *pb = p[(c + 2) % 3];
            M.gphi[6 * t + 2 * c] = (float)(-(pb[1] - pa[1]) / a2);
            M.gphi[6 * t + 2 * c + 1] = (float)((pb[0] - pa[0]) / a2);
        }
    }

    // half-edges sorted by undirected key
    std::vector<HalfEdge> he(3 * n_t);
    for (int64_t t = 0; t < n_t; ++t)
        for (int c = 0; c < 3; ++c) {
            int32_t a = tri[3 * t + (c + 1) % 3], b = tri[3 * t + (c + 2) % 3];
            he[3 * t + c] = HalfEdge{edge_key(a, b), (int32_t)t, c, a, b};
        }
    std::sort(he.begin(), he.end(), [](const HalfEdge &x, const HalfEdge &y) {
        return x.key < y.key || (x.key == y.key && x.t < y.t);
    });

    M.tnbr.assign(3 * n_t, -1);
    std::vector<uint64_t> bkeys;            // boundary edge keys (sorted)
    std::vector<std::pair<int32_t, int32_t>> edges;
    std::vector<double> weight;
    std::vector<uint8_t> is_b(n_v, 0);
    for (size_t i = 0; i < he.size();) {
        size_t j = i;
        while (j < he.size() && he[j].key == he[i].key) ++j;
        const size_t cnt = j - i;
        if (cnt > 2) return fail(err, "edge (%lld,%lld) has more than two triangles",
                                 (long long)(he[i].key >> 32), (long long)(he[i].key & 0xffffffffu));
        double w = 0.0;
        for (size_t q = i; q < j; ++q) {
            // cotangent of the angle at the corner opposite the edge
            const int32_t *v = tri + 3 * he[q].t;
            int32_t kc = v[he[q].c], a = he[q].a, b = he[q].b;
            double ux = xy[2 * a] - xy[2 * kc], uy = xy[2 * a + 1] - xy[2 * kc + 1];
            double vx = xy[2 * b] - xy[2 * kc], vy = xy[2 * b + 1] - xy[2 * kc + 1];
            double dot = ux * vx + uy * vy, cross = std::fabs(ux * vy - uy * vx);
            w += 0.5 * dot / cross;
        }
        if (cnt == 2) {
            if (!(he[i].a == he[i + 1].b && he[i].b == he[i + 1].a))
                return fail(err, "triangles %lld and %lld are inconsistently oriented", he[i].t, he[i + 1].t);
            M.tnbr[3 * he[i].t + he[i].c] = he[i + 1].t;
            M.tnbr[3 * he[i + 1].t + he[i + 1].c] = he[i].t;
        } else {
            bkeys.push_back(he[i].key);
            is_b[he[i].a] = 1;
            is_b[he[i].b] = 1;
        }
        edges.emplace_back((int32_t)(he[i].key >> 32), (int32_t)(he[i].key & 0xffffffffu));
        weight.push_back(w);
        i = j;
    }
    M.n_edges = (int64_t)edges.size();

    // every vertex used
    {
        std::vector<uint8_t> used(n_v, 0);
        for (int64_t i = 0; i < 3 * n_t; ++i) used[tri[i]] = 1;
        for (int64_t v = 0; v < n_v; ++v)
            if (!used[v]) return fail(err, "vertex %lld is not used by any triangle", v);
    }

    // loops must cover exactly the topological boundary
    M.col_of.assign(n_v, -1);
    M.B.assign(loop_idx, loop_idx + k);
    int64_t nb = 0;
    for (int64_t v = 0; v < n_v; ++v) nb += is_b[v];
    if (nb != k) return fail(err, "loops list %lld vertices but the boundary has %lld", k, nb);
    for (int64_t i = 0; i < k; ++i) {
        int32_t v = loop_idx[i];
        if (v < 0 || v >= n_v) return fail(err, "loop vertex id %lld out of range", v);
        if (!is_b[v]) return fail(err, "loop vertex %lld is not on the boundary", v);
        if (M.col_of[v] >= 0) return fail(err, "loop vertex %lld appears twice", v);
        M.col_of[v] = (int32_t)i;
    }
    for (int32_t l = 0; l < n_loops; ++l) {
        const int64_t lo = loop_off[l], hi = loop_off[l + 1];
        if (hi < lo || hi > k) return fail(err, "bad loop offsets at loop %lld", l);
        for (int64_t i = lo; i < hi; ++i) {
            int32_t a = loop_idx[i], b = loop_idx[i + 1 < hi ? i + 1 : lo];
            if (!std::binary_search(bkeys.begin(), bkeys.end(), edge_key(a, b)))
                return fail(err, "loop step %lld -> %lld is not a boundary edge", a, b);
        }
    }
    M.k = k;
    M.row_of.assign(n_v, -1);
    M.I.clear();
    for (int64_t v = 0; v < n_v; ++v)
        if (!is_b[v]) {
            M.row_of[v] = (int32_t)M.I.size();
            M.I.push_back((int32_t)v);
        }
    M.m = (int64_t)M.I.size();

    // vertex -> triangles (ascending triangle id)
    M.vt_off.assign(n_v + 1, 0);
    for (int64_t i = 0; i < 3 * n_t; ++i) M.vt_off[tri[i] + 1]++;
    for (int64_t v = 0; v < n_v; ++v) M.vt_off[v + 1] += M.vt_off[v];
    M.vt.resize(3 * n_t);
    {
        std::vector<int32_t> fill(M.vt_off.begin(), M.vt_off.end() - 1);
        for (int64_t t = 0; t < n_t; ++t)
            for (int c = 0; c < 3; ++c) M.vt[fill[tri[3 * t + c]]++] = (int32_t)t;
    }
    // vertex -> neighbours (ascending) and edge weights per vertex
    M.vn_off.assign(n_v + 1, 0);
    for (auto &e : edges) {
        M.vn_off[e.first + 1]++;
        M.vn_off[e.second + 1]++;
    }
    for (int64_t v = 0; v < n_v; ++v) M.vn_off[v + 1] += M.vn_off[v];
    M.vn.resize(2 * edges.size());
    std::vector<double> vw(2 * edges.size());
    {
        std::vector<int32_t> fill(M.vn_off.begin(), M.vn_off.end() - 1);
        // edges are sorted by (min, max): appending in that order keeps each list ascending
        // for the "max" side; sort every list afterwards to be exact.
        for (size_t e = 0; e < edges.size(); ++e) {
            int32_t a = edges[e].first, b = edges[e].second;
            vw[fill[a]] = weight[e];
            M.vn[fill[a]++] = b;
            vw[fill[b]] = weight[e];
            M.vn[fill[b]++] = a;
        }
        for (int64_t v = 0; v < n_v; ++v) {
            int32_t lo = M.vn_off[v], hi = M.vn_off[v + 1];
            std::vector<std::pair<int32_t, double>> tmp;
            for (int32_t q = lo; q < hi; ++q) tmp.emplace_back(M.vn[q], vw[q]);
            std::sort(tmp.begin(), tmp.end());
            for (int32_t q = lo; q < hi; ++q) {
                M.vn[q] = tmp[q - lo].first;
                vw[q] = tmp[q - lo].second;
            }
        }
    }

    // A = -L_II in CSR (interior numbering, columns ascending) and L_IB entries
    M.a_off.assign(M.m + 1, 0);
    M.a_col.clear();
    M.a_val.clear();
    M.a_diag.assign(M.m, 0.0);
    M.rb_row.clear();
    M.rb_col.clear();
    M.rb_val.clear();
    for (int64_t r = 0; r < M.m; ++r) {
        const int32_t v = M.I[r];
        double diag = 0.0;
        for (int32_t q = M.vn_off[v]; q < M.vn_off[v + 1]; ++q) diag += vw[q];
        std::vector<std::pair<int32_t, double>> row;
        row.emplace_back((int32_t)r, diag);
        for (int32_t q = M.vn_off[v]; q < M.vn_off[v + 1]; ++q) {
            int32_t u = M.vn[q];
            if (M.row_of[u] >= 0) {
                if (vw[q] != 0.0) row.emplace_back(M.row_of[u], -vw[q]);
            } else if (vw[q] != 0.0) {
                M.rb_row.push_back((int32_t)r);
                M.rb_col.push_back(M.col_of[u]);
                M.rb_val.push_back(vw[q]);
            }
        }
        std::sort(row.begin(), row.end());
        for (auto &e : row) {
            M.a_col.push_back(e.first);
            M.a_val.push_back(e.second);
        }
        M.a_diag[r] = diag;
        if (!(diag > 0.0)) return fail(err, "interior vertex %lld has a non-positive Laplacian diagonal", v);
        M.a_off[r + 1] = (int64_t)M.a_col.size();
    }
    return DD_OK;
}
