// Triangle-based gradient-descent path tracing, Section IV ("Gradient-descent
// path generation"), one thread per (target, source) pair.
//
// The field is piecewise linear, so triangle tau has the constant gradient
// g = (f0 - f2) grad(phi_0) + (f1 - f2) grad(phi_1) and the path follows -g.
// The walk, made precise from the paper's prose:
//  * vertex v: stop at the target; if v neighbours the target, the path lies
//    on an edge incident on it: append the target and stop.  Otherwise follow
//    the steepest incident triangle whose descent direction enters it from v
//    (inside the corner wedge; ties to the lowest triangle id) to the opposite
//    edge.  With no such triangle take the incident edge of largest positive
//    slope (f_v - f_u)/|v - u| to its other end; none means a local minimum.
//  * edge (a, b) left from triangle tau: an edge incident on the target ends
//    the path at the target.  Otherwise enter the triangle across; if its
//    descent direction points into it, cross to the exit edge; if not (valley
//    edge) or there is no triangle across (boundary edge), slide along the
//    edge to its lower endpoint (ties to the lower id).
//  * an exit whose barycentric coordinate is <= kEpsBary lands on the vertex.
// Geometry and gradients are FP32; the hat-function gradients are computed in
// FP64 on the host and rounded once.
//
// Work split for latency.  What a vertex state decides depends only on the
// field and the vertex (the best triangle is the steepest, ties by id, so the
// order in which the incident triangles are examined does not matter), so it
// is computed for every vertex of every field before the walk
// (vertex_decision_kernel), after the barycentric rates of every triangle
// (rates_kernel).  Both are stored field-minor ([triangle][field],
// [vertex][field]): a warp of the decision kernel handles one vertex for 32
// fields, so the triangle records it reads are shared by all its lanes and
// the rates it reads are contiguous.  The walk then does one thing per iteration: cross one
// triangle from an edge (one 64-byte record and one 16-byte rate load, both
// addressed by the id the previous step found), apply one vertex decision
// (one 48-byte load), or slide along a valley or boundary edge.
#include <cfloat>
#include <cstring>
#include <cstdlib>
#include <algorithm>
#include <cmath>
#include <random>
#include <vector>

#include "dd_internal.h"

namespace {

constexpr float kEpsBary = 1e-6f;    // barycentric snap to a vertex
constexpr float kEpsWedge = 1e-6f;   // relative tolerance of the wedge / entry tests
constexpr int32_t kDenseMinPaths = 128;   // paths per field from which decisions are precomputed

// Triangle record (64 bytes): vertex ids, the ids of the triangles across the
// edges opposite each vertex (-1 on the boundary), the squared norms q_i of
// the hat gradients, and the vertex positions.
struct Tri {
    int v0, v1, v2, n0, n1, n2;
    float q0, q1, q2;
    float2 p0, p1, p2;
};

__device__ __forceinline__ Tri load_tri(const int4 *__restrict__ rec, int t) {
    const int4 a = __ldg(rec + 4 * t), b = __ldg(rec + 4 * t + 1);
    const float4 c = __ldg(reinterpret_cast<const float4 *>(rec) + 4 * t + 2);
    const float4 d = __ldg(reinterpret_cast<const float4 *>(rec) + 4 * t + 3);
    Tri T;
    T.v0 = a.x;
    T.v1 = a.y;
    T.v2 = a.z;
    T.n0 = a.w;
    T.n1 = b.x;
    T.n2 = b.y;
    T.q0 = __int_as_float(b.z);
    T.q1 = __int_as_float(b.w);
    T.q2 = c.x;
    T.p0 = make_float2(c.z, c.w);
    T.p1 = make_float2(d.x, d.y);
    T.p2 = make_float2(d.z, d.w);
    return T;
}

__device__ __forceinline__ int vid(const Tri &T, int i) { return i == 0 ? T.v0 : (i == 1 ? T.v1 : T.v2); }
__device__ __forceinline__ float2 pos(const Tri &T, int i) { return i == 0 ? T.p0 : (i == 1 ? T.p1 : T.p2); }
__device__ __forceinline__ int local_of(const Tri &T, int x) { return T.v0 == x ? 0 : (T.v1 == x ? 1 : 2); }
__device__ __forceinline__ float sel3f(int i, float a, float b, float c) { return i == 0 ? a : (i == 1 ? b : c); }
__device__ __forceinline__ int sel3i(int i, int a, int b, int c) { return i == 0 ? a : (i == 1 ? b : c); }

// Per (field, triangle): (r0, r1, r2, |g|^2) with r_i = -grad(phi_i) . g the
// rate of change of barycentric coordinate i along the descent direction -g.
// g = f0 grad(phi_0) + f1 grad(phi_1) + f2 grad(phi_2) = (f0 - f2) g0 + (f1 - f2) g1.
__device__ __forceinline__ float4 tri_rates(const float4 *__restrict__ gphi, const int4 *__restrict__ rec, int64_t t,
                                            const float *__restrict__ f) {
    const int4 a = __ldg(rec + 4 * t);
    const float4 h = __ldg(gphi + 2 * t);                 // (g0x, g0y, g1x, g1y)
    const float f2 = f[a.z], d0 = f[a.x] - f2, d1 = f[a.y] - f2;
    const float gx = d0 * h.x + d1 * h.z, gy = d0 * h.y + d1 * h.w;
    const float r0 = -(h.x * gx + h.y * gy), r1 = -(h.z * gx + h.w * gy);
    return make_float4(r0, r1, -(r0 + r1), gx * gx + gy * gy);
}

// rates[t * T + a] for every triangle t and field a (field-minor)
__global__ void rates_kernel(const float4 *__restrict__ gphi, const int4 *__restrict__ rec, int64_t n_t, int32_t T,
                             const float *__restrict__ fields, int64_t field_stride, float4 *__restrict__ rates) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_t * T) return;
    const int64_t t = i / T;
    const int a = (int)(i - t * T);
    rates[i] = tri_rates(gphi, rec, t, fields + (int64_t)a * field_stride);
}

// What the walk does at a vertex (48 bytes)
enum { kVCross = 0, kVVertex = 1, kVAdjacent = 2, kVStuck = 3 };
struct VDec {
    int4 h;      // kind, then: cross (ea, eb, t_next) | vertex (u, -, -) | adjacent (target, -, -)
    float4 w;    // cross (la, lb, point) | vertex, adjacent (position, -, -)
    float4 e;    // cross: positions of ea and eb
};

struct TraceDom {
    const int4 *rec;
    const float4 *gphi;
    const float2 *xy;
    const int32_t *vt_off, *vt;
    int64_t n_t, n_v;
};

// The vertex state at v, one incident triangle at a time: add() examines a
// triangle of v's fan, finish() turns the fan's best candidate into the
// decision.  Both the decision kernel (a whole fan in one call) and the walk
// without precomputed decisions (one triangle per iteration) use it, so the
// two give the same decision bit for bit.
struct FanScan {
    bool adj;
    int best, b_vj, b_vk, b_next;
    float best_g2, baj, bak;
    float2 b_pj, b_pk;

    __device__ __forceinline__ void begin() {
        adj = false;
        best = -1;
        b_vj = b_vk = 0;
        b_next = -1;
        best_g2 = baj = bak = 0.f;
        b_pj = b_pk = make_float2(0.f, 0.f);
    }

    // triangle tl (record T, rates R of the field) incident on v
    __device__ __forceinline__ void add(int v, int target, int tl, const Tri &T, const float4 &R) {
        const float eps2 = kEpsWedge * kEpsWedge;
        // rotated view: v is local vertex L, then X and Y counter-clockwise; the exit edge is X-Y
        const int L = local_of(T, v), X = L == 2 ? 0 : L + 1, Y = L == 0 ? 2 : L - 1;
        const float rX = sel3f(X, R.x, R.y, R.z), rY = sel3f(Y, R.x, R.y, R.z);
        const float qX = sel3f(X, T.q0, T.q1, T.q2), qY = sel3f(Y, T.q0, T.q1, T.q2);
        const int vX = sel3i(X, T.v0, T.v1, T.v2), vY = sel3i(Y, T.v0, T.v1, T.v2);
        const float gg = R.w;
        adj |= (vX == target) | (vY == target);
        const float tol2 = eps2 * gg * fmaxf(qX, qY);
        const bool in_x = rX >= 0.f || rX * rX <= tol2;
        const bool in_y = rY >= 0.f || rY * rY <= tol2;
        if (gg > 0.f && in_x && in_y && rX + rY > 0.f && (gg > best_g2 || (gg == best_g2 && tl < best))) {
            best = tl;
            best_g2 = gg;
            baj = fmaxf(rX, 0.f);
            bak = fmaxf(rY, 0.f);
            b_vj = vX;
            b_vk = vY;
            b_pj = pos(T, X);
            b_pk = pos(T, Y);
            b_next = sel3i(L, T.n0, T.n1, T.n2);
        }
    }

    __device__ __forceinline__ VDec finish(const TraceDom &p, const float *__restrict__ f, int target, int v) const {
        VDec d;
        d.e = make_float4(0.f, 0.f, 0.f, 0.f);
        if (adj) {                                   // v lies on an edge incident on the target
            const float2 pt = p.xy[target];
            d.h = make_int4(kVAdjacent, target, 0, 0);
            d.w = make_float4(pt.x, pt.y, 0.f, 0.f);
            return d;
        }
        if (best >= 0) {
            const float s = __fdividef(1.0f, baj + bak);
            const float lj = s * baj, lk = s * bak;
            if (lj <= kEpsBary) {
                d.h = make_int4(kVVertex, b_vk, 0, 0);
                d.w = make_float4(b_pk.x, b_pk.y, 0.f, 0.f);
            } else if (lk <= kEpsBary) {
                d.h = make_int4(kVVertex, b_vj, 0, 0);
                d.w = make_float4(b_pj.x, b_pj.y, 0.f, 0.f);
            } else {
                d.h = make_int4(kVCross, b_vj, b_vk, b_next);
                d.w = make_float4(lj, lk, lj * b_pj.x + lk * b_pk.x, lj * b_pj.y + lk * b_pk.y);
                d.e = make_float4(b_pj.x, b_pj.y, b_pk.x, b_pk.y);
            }
            return d;
        }
        // no descending triangle: the incident edge of largest positive slope (ties to the lower id)
        int best_u = -1;
        float best_s = 0.f;
        float2 best_p = make_float2(0.f, 0.f);
        const float fv = f[v];
        const float2 pv = p.xy[v];
        for (int q = p.vt_off[v]; q < p.vt_off[v + 1]; ++q) {
            const Tri Q = load_tri(p.rec, p.vt[q]);
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const int u = vid(Q, e);
                if (u == v) continue;
                const float2 pu = pos(Q, e);
                const float dx = pv.x - pu.x, dy = pv.y - pu.y;
                const float slope = (fv - f[u]) / sqrtf(dx * dx + dy * dy);
                if (slope > 0.f && (slope > best_s || (slope == best_s && u < best_u))) {
                    best_s = slope;
                    best_u = u;
                    best_p = pu;
                }
            }
        }
        if (best_u < 0) {
            d.h = make_int4(kVStuck, 0, 0, 0);
            d.w = make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            d.h = make_int4(kVVertex, best_u, 0, 0);
            d.w = make_float4(best_p.x, best_p.y, 0.f, 0.f);
        }
        return d;
    }
};

// the vertex state's decision at v for field f (rates of that field at
// `rates`, one entry per triangle every `rstride`)
__device__ __forceinline__ VDec vertex_decision(const TraceDom &p, const float *__restrict__ f,
                                                const float4 *__restrict__ rates, int64_t rstride, int target, int v) {
    FanScan fs;
    fs.begin();
    for (int q = p.vt_off[v], q1 = p.vt_off[v + 1]; q < q1; ++q) {
        const int tl = p.vt[q];
        fs.add(v, target, tl, load_tri(p.rec, tl), __ldg(rates + (int64_t)tl * rstride));
    }
    return fs.finish(p, f, target, v);
}

// one warp per (vertex, group of 32 fields), lane = field: dec[v * T + a]
__global__ void vertex_decision_kernel(const TraceDom p, int32_t T, const float *__restrict__ fields,
                                       int64_t field_stride, const float4 *__restrict__ rates,
                                       const int32_t *__restrict__ targets, VDec *__restrict__ dec) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int groups = (T + 31) >> 5;
    const int64_t v = w / groups;
    const int a = (int)(w - v * groups) * 32 + (threadIdx.x & 31);
    if (v >= p.n_v || a >= T) return;
    dec[v * T + a] = vertex_decision(p, fields + (int64_t)a * field_stride, rates + a, T, targets[a], (int)v);
}

// One path: walk from `source` to `target` on field f, with that field's
// triangle rates and vertex decisions.  The warp votes at the top of every
// iteration, so its threads reconverge once per step; finished threads (and
// padding lanes) idle there until the last path of the warp ends.
// (rates of this field start at `rates`, one entry per triangle every
// `rstride`; its decisions at `dec`, one per vertex every `dstride`.  With
// dec == nullptr a vertex state computes its decision itself -- the same
// function, so the same result -- which pays when few paths share a field.
// With rates == nullptr the walk computes each triangle's rates from the
// field where it needs them, by the same function as rates_kernel, so again
// with the same result: few paths per field touch a small share of the
// triangles, and a pass over all of them would cost more than the walk.)
__device__ __forceinline__ void trace_path(const TraceDom &p, const float *__restrict__ f,
                                           const float4 *__restrict__ rates, int64_t rstride,
                                           const VDec *__restrict__ dec, int64_t dstride, int target, int source,
                                           float2 *__restrict__ out, int32_t max_pts, int32_t max_steps,
                                           int32_t *len_out, int32_t *status_out, bool active) {
    const float eps2 = kEpsWedge * kEpsWedge;
    int len = 0;
    int status = DD_TRACE_STEP_LIMIT;
    int states = 1;                // vertex and edge states entered (the step cap counts these)
    bool fin = !active;
    bool at_vertex = true;
    int v = source;
    // fan scan of the current vertex when decisions are not precomputed: one
    // incident triangle (from the vertex's triangle list) per iteration
    FanScan fs;
    fs.begin();
    int scan_q = 0, scan_end = 0;
    if (active && !dec) {
        scan_q = p.vt_off[v];
        scan_end = p.vt_off[v + 1];
    }
    // edge state: the path sits on edge (ea, eb) at weights (la, lb) and enters
    // t_next (the triangle across that edge, -1 on the boundary)
    int t_next = -1, ea = 0, eb = 0;
    float la = 0.f, lb = 0.f;
    float2 pa = make_float2(0.f, 0.f), pb = pa;
    if (active) {
        out[len++] = p.xy[v];
        if (v == target) {
            status = DD_TRACE_OK;
            fin = true;
        }
    }

// The macros end the current iteration with `continue` when the path ends;
// they are used as statements inside braces (no do-while wrapper, so that
// `continue` reaches the walk loop).
#define DD_PUSH(pt)                              \
    if (len >= max_pts) {                        \
        status = DD_TRACE_TRUNCATED;             \
        fin = true;                              \
        continue;                                \
    }                                            \
    out[len++] = (pt);
#define DD_ENTER_VERTEX(vert)                    \
    v = (vert);                                  \
    at_vertex = true;                            \
    if (!dec) {                                  \
        fs.begin();                              \
        scan_q = p.vt_off[v];                    \
        scan_end = p.vt_off[v + 1];              \
    }                                            \
    if (++states > max_steps) {                  \
        fin = true;                              \
        continue;                                \
    }                                            \
    if (v == target) {                           \
        status = DD_TRACE_OK;                    \
        fin = true;                              \
        continue;                                \
    }
#define DD_SLIDE()                                                     \
    {                                                                  \
        const float fa = f[ea], fb = f[eb];                            \
        const bool a_low = fa < fb || (fa == fb && ea < eb);           \
        DD_PUSH(a_low ? pa : pb);                                      \
        DD_ENTER_VERTEX(a_low ? ea : eb);                              \
    }

    const int64_t iter_cap = 4LL * max_steps + 16;
    for (int64_t iter = 0;; ++iter) {
        if (!fin && iter >= iter_cap) fin = true;
        if (!__any_sync(0xffffffffu, !fin)) break;
        if (fin) continue;
        if (at_vertex) {
            // ---- vertex state: apply the decision (precomputed, or scanned here one
            // incident triangle per iteration, so the warp's other lanes wait little)
            const VDec *dv = dec ? dec + (int64_t)v * dstride : nullptr;
            VDec own;
            if (!dv) {
                if (scan_q < scan_end) {
                    const int tl = p.vt[scan_q++];
                    fs.add(v, target, tl, load_tri(p.rec, tl),
                           rates ? __ldg(rates + (int64_t)tl * rstride) : tri_rates(p.gphi, p.rec, tl, f));
                    continue;
                }
                own = fs.finish(p, f, target, v);
            }
            const int4 h = dv ? __ldg(&dv->h) : own.h;
            const float4 w = dv ? __ldg(&dv->w) : own.w;
            const int kind = h.x;
            if (kind == kVStuck) {
                status = DD_TRACE_STUCK;
                fin = true;
                continue;
            }
            const bool cross = kind == kVCross;
            DD_PUSH(make_float2(cross ? w.z : w.x, cross ? w.w : w.y));
            if (kind == kVAdjacent) {
                status = DD_TRACE_OK;
                fin = true;
                continue;
            }
            if (!cross) {
                DD_ENTER_VERTEX(h.y);
                continue;
            }
            const float4 e = dv ? __ldg(&dv->e) : own.e;
            at_vertex = false;
            ea = h.y;
            eb = h.z;
            t_next = h.w;
            la = w.x;
            lb = w.y;
            pa = make_float2(e.x, e.y);
            pb = make_float2(e.z, e.w);
            if (++states > max_steps) fin = true;
            continue;
        }
        if (t_next < 0) {                // boundary edge: slide to the lower endpoint
            DD_SLIDE();
            continue;
        }
        // ---- edge state: entering T across (ea, eb); in T's counter-clockwise order
        // eb is local vertex L, ea is X, and the opposite vertex is Y
        const int tl = t_next;
        const Tri T = load_tri(p.rec, tl);
        const float4 Rt = rates ? __ldg(rates + (int64_t)tl * rstride) : tri_rates(p.gphi, p.rec, tl, f);
        const int L = local_of(T, eb), X = L == 2 ? 0 : L + 1, Y = L == 0 ? 2 : L - 1;
        const float ra = sel3f(X, Rt.x, Rt.y, Rt.z), rb = sel3f(L, Rt.x, Rt.y, Rt.z), rc = sel3f(Y, Rt.x, Rt.y, Rt.z);
        const float qY = sel3f(Y, T.q0, T.q1, T.q2);
        const bool enters = rc > 0.f && rc * rc > eps2 * Rt.w * qY;
        const float sa = ra < 0.f ? __fdividef(la, -ra) : INFINITY;
        const float sb = rb < 0.f ? __fdividef(lb, -rb) : INFINITY;
        if (!enters || !(fminf(sa, sb) < INFINITY)) {   // valley edge (or no exit): lower endpoint
            DD_SLIDE();
            continue;
        }
        const int vY = sel3i(Y, T.v0, T.v1, T.v2);
        const float2 pY = pos(T, Y);
        const bool via_a = sa <= sb;                      // exit through the edge opposite a (the Y-R edge)
        const float s = via_a ? sa : sb;
        float lkeep = fmaxf(via_a ? lb + s * rb : la + s * ra, 0.f);
        float lc2 = fmaxf(s * rc, 0.f);
        const float inv = __fdividef(1.0f, lkeep + lc2);
        lkeep *= inv;
        lc2 *= inv;
        const int keep_v = via_a ? eb : ea;
        const float2 keep_p = via_a ? pb : pa;
        if (lkeep <= kEpsBary) {
            DD_PUSH(pY);
            DD_ENTER_VERTEX(vY);
            continue;
        }
        if (lc2 <= kEpsBary) {
            DD_PUSH(keep_p);
            DD_ENTER_VERTEX(keep_v);
            continue;
        }
        DD_PUSH(make_float2(lkeep * keep_p.x + lc2 * pY.x, lkeep * keep_p.y + lc2 * pY.y));
        // new edge in T's counter-clockwise order: via a -> (Y, R) = (c, b); via b -> (X, Y) = (a, c)
        if (via_a) {
            t_next = sel3i(X, T.n0, T.n1, T.n2);
            ea = vY;
            eb = keep_v;
            pa = pY;
            pb = keep_p;
            la = lc2;
            lb = lkeep;
        } else {
            t_next = sel3i(L, T.n0, T.n1, T.n2);
            ea = keep_v;
            eb = vY;
            pa = keep_p;
            pb = pY;
            la = lkeep;
            lb = lc2;
        }
        if (++states > max_steps) {
            fin = true;
            continue;
        }
        if (ea == target || eb == target) {   // an edge incident on the target
            DD_PUSH(p.xy[target]);
            status = DD_TRACE_OK;
            fin = true;
            continue;
        }
    }
#undef DD_PUSH
#undef DD_ENTER_VERTEX
#undef DD_SLIDE
    if (active) {
        *len_out = len;
        *status_out = status;
    }
}

struct TraceParams {
    TraceDom d;
    const float4 *rates;           // [n_t][T]
    const VDec *dec;               // [n_v][T]
    const float *fields;
    int64_t field_stride;
    const int32_t *targets, *sources;
    int64_t total;
    int32_t S, max_pts, max_steps, T;
    float2 *out_xy;
    int32_t *out_len, *out_status;
};

__global__ void __launch_bounds__(128) trace_kernel(const TraceParams p) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = gid < p.total;       // padding lanes stay in the warp's walk loop, idle
    const int64_t id = active ? gid : 0;
    const int a = (int)(id / p.S);
    trace_path(p.d, p.fields + (int64_t)a * p.field_stride, p.rates ? p.rates + a : nullptr, p.T,
               p.dec ? p.dec + a : nullptr, p.T,
               p.targets[a], p.sources[id], p.out_xy + id * p.max_pts, p.max_pts, p.max_steps, p.out_len + id,
               p.out_status + id, active);
}

// ---- several meshes in one launch: global target g belongs to domain tdom[g] (local index tloc[g])
struct BatchTraceDom {
    TraceDom d;
    const float *fields;      // [T_d][n_v]
    float4 *rates;            // [T_d][n_t] (decisions are computed by the walk itself)
    int32_t max_steps, T;
};

__global__ void batch_rates_kernel(const BatchTraceDom *__restrict__ doms, const int32_t *__restrict__ tdom,
                                   const int32_t *__restrict__ tloc) {
    const int g = blockIdx.y;
    const BatchTraceDom q = doms[tdom[g]];
    const int a = tloc[g];
    const float *f = q.fields + (int64_t)a * q.d.n_v;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < q.d.n_t; t += (int64_t)gridDim.x * blockDim.x)
        q.rates[(int64_t)a * q.d.n_t + t] = tri_rates(q.d.gphi, q.d.rec, t, f);
}

// path id -> global target: id / S, or path_target[id] when sources per target vary
__global__ void __launch_bounds__(64) batch_trace_kernel(const BatchTraceDom *__restrict__ doms,
                                                        const int32_t *__restrict__ tdom,
                                                        const int32_t *__restrict__ tloc,
                                                        const int32_t *__restrict__ targets,
                                                        const int32_t *__restrict__ sources,
                                                        const int32_t *__restrict__ path_target, int64_t total,
                                                        int32_t S, int32_t max_pts, float2 *__restrict__ out_xy,
                                                        int32_t *__restrict__ out_len, int32_t *__restrict__ out_status) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = gid < total;         // padding lanes stay in the warp's walk loop, idle
    const int64_t id = active ? gid : 0;
    const int g = path_target ? path_target[id] : (int)(id / S);
    const BatchTraceDom q = doms[tdom[g]];
    const int a = tloc[g];
    trace_path(q.d, q.fields + (int64_t)a * q.d.n_v, q.rates + (int64_t)a * q.d.n_t, 1, nullptr, 0, targets[g],
               sources[id], out_xy + id * max_pts, max_pts, q.max_steps, out_len + id, out_status + id, active);
}

TraceDom make_dom(const DevMesh &m) {
    TraceDom d;
    d.rec = m.trec;
    d.gphi = m.gphi;
    d.xy = m.xy;
    d.vt_off = m.vt_off;
    d.vt = m.vt;
    d.n_t = m.n_t;
    d.n_v = m.n_v;
    return d;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int32_t step_cap(const DevMesh &m) {
    const int64_t cap = 4 * m.n_t;
    return cap > (int64_t)INT32_MAX ? INT32_MAX : (int32_t)cap;
}

}  // namespace

size_t trace_scratch_bytes(const DevMesh &m, int32_t T, bool decisions) {
    return align256((size_t)T * m.n_t * sizeof(float4)) +
           (decisions ? align256((size_t)T * m.n_v * sizeof(VDec)) : 0);
}

// Vertex decisions for every (field, vertex) before the walk pay off when
// many paths share a field (they are reused); with few paths each vertex
// state computes its own.  DD_TRACE_DECISIONS=dense|lazy overrides the choice
// (for measurements).
bool trace_dense_decisions(int32_t S) {
    static int mode = -1;
    if (mode < 0) {
        const char *e = getenv("DD_TRACE_DECISIONS");
        mode = (e && !strcmp(e, "dense")) ? 1 : (e && !strcmp(e, "lazy")) ? 0 : 2;
    }
    return mode == 2 ? S >= kDenseMinPaths : mode == 1;
}

void launch_trace(const DevMesh &m, const float *fields, int64_t field_stride, const int32_t *targets,
                  const int32_t *sources, int32_t T, int32_t S, int32_t max_pts, float2 *out_xy, int32_t *out_len,
                  int32_t *out_status, void *scratch, cudaStream_t s) {
    const bool dense = trace_dense_decisions(S);
    TraceParams p;
    // the rates of every triangle only where vertex decisions are precomputed (many
    // paths per field); with few, the walk forms the rates it needs itself
    float4 *rates = dense ? reinterpret_cast<float4 *>(scratch) : nullptr;
    VDec *dec = dense ? reinterpret_cast<VDec *>(reinterpret_cast<char *>(scratch) +
                                                 align256((size_t)T * m.n_t * sizeof(float4)))
                      : nullptr;
    p.d = make_dom(m);
    p.rates = rates;
    p.dec = dec;
    p.fields = fields;
    p.field_stride = field_stride;
    p.targets = targets;
    p.sources = sources;
    p.total = (int64_t)T * S;
    p.S = S;
    p.max_pts = max_pts;
    p.max_steps = step_cap(m);
    p.T = T;
    p.out_xy = out_xy;
    p.out_len = out_len;
    p.out_status = out_status;
    if (p.total == 0) return;
    if (dense) {
        {
            KMark km_("rates_kernel", s);
            rates_kernel<<<(unsigned)((m.n_t * T + 255) / 256), 256, 0, s>>>(m.gphi, m.trec, m.n_t, T, fields,
                                                                              field_stride, rates);
        }
        const int64_t warps = m.n_v * ((T + 31) / 32);
        {
            KMark km_("vertex_decision_kernel", s);
            vertex_decision_kernel<<<(unsigned)((warps + 3) / 4), 128, 0, s>>>(p.d, T, fields, field_stride, rates,
                                                                                targets, dec);
        }
    }
    {
        KMark km_("trace_kernel", s);
        trace_kernel<<<(unsigned)((p.total + 127) / 128), 128, 0, s>>>(p);   // 128: measured best of 64/128/256
    }
}

size_t batch_trace_dom_bytes() { return sizeof(BatchTraceDom); }

// host-side builder of one domain descriptor (into a byte buffer uploaded by the
// caller); scratch: trace_scratch_bytes(m, T) bytes of device memory
void fill_batch_trace_dom(void *dst, const DevMesh &m, const float *fields, int32_t T, void *scratch) {
    BatchTraceDom q;
    q.d = make_dom(m);
    q.fields = fields;
    q.rates = reinterpret_cast<float4 *>(scratch);
    q.max_steps = step_cap(m);
    q.T = T;
    std::memcpy(dst, &q, sizeof q);
}

void launch_batch_trace(const void *d_doms, const int32_t *d_tdom, const int32_t *d_tloc, const int32_t *d_targets,
                        const int32_t *d_sources, int32_t n_targets, int32_t S, int64_t max_nt, int64_t max_nv,
                        int32_t max_pts, float2 *out_xy, int32_t *out_len, int32_t *out_status, cudaStream_t s,
                        const int32_t *d_path_target, int64_t n_paths) {
    if (n_targets <= 0) return;
    const BatchTraceDom *doms = reinterpret_cast<const BatchTraceDom *>(d_doms);
    const int64_t total = d_path_target ? n_paths : (int64_t)n_targets * S;
    if (total == 0) return;
    dim3 gr((unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (max_nt + 255) / 256)), (unsigned)n_targets);
    {
        KMark km_("batch_rates_kernel", s);
        batch_rates_kernel<<<gr, 256, 0, s>>>(doms, d_tdom, d_tloc);
    }
    (void)max_nv;
    {
        KMark km_("batch_trace_kernel", s);
        batch_trace_kernel<<<(unsigned)((total + 63) / 64), 64, 0, s>>>(doms, d_tdom, d_tloc, d_targets, d_sources,
                                                                        d_path_target, total, S, max_pts, out_xy, out_len,
                                                                        out_status);
    }
}

namespace {
// one warp per path: its first len points.  MODE 2: point pairs as 16-byte
// stores (rows 16-byte aligned at both ends); 1: one point (8 bytes) per
// store; 0: one float per store (any 4-byte aligned buffer).
template <int MODE>
__global__ void copy_paths_kernel(const float2 *__restrict__ src, const int32_t *__restrict__ len, int64_t n,
                                  int32_t max_pts, float2 *__restrict__ dst) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= n) return;
    const int L = min(max(len[w], 0), max_pts);
    const float2 *a = src + w * (int64_t)max_pts;
    float2 *b = dst + w * (int64_t)max_pts;
    if (MODE == 2) {
        const float4 *a4 = reinterpret_cast<const float4 *>(a);
        float4 *b4 = reinterpret_cast<float4 *>(b);
        for (int i = lane; 2 * i + 1 < L; i += 32) b4[i] = __ldcs(a4 + i);
        if ((L & 1) && lane == 0) b[L - 1] = a[L - 1];
    } else if (MODE == 1) {
        for (int i = lane; i < L; i += 32) b[i] = a[i];
    } else {
        const float *af = reinterpret_cast<const float *>(a);
        float *bf = reinterpret_cast<float *>(b);
        for (int i = lane; i < 2 * L; i += 32) bf[i] = af[i];
    }
}
}  // namespace

void launch_copy_paths(const float2 *src, const int32_t *len, int64_t n, int32_t max_pts, float2 *dst,
                       cudaStream_t s) {
    if (n <= 0) return;
    const uintptr_t d = reinterpret_cast<uintptr_t>(dst);
    const unsigned grid = (unsigned)((n + 7) / 8);
    KMark km_("copy_paths_kernel", s);
    if ((max_pts & 1) == 0 && (d & 15) == 0)
        copy_paths_kernel<2><<<grid, 256, 0, s>>>(src, len, n, max_pts, dst);
    else if ((d & 7) == 0)
        copy_paths_kernel<1><<<grid, 256, 0, s>>>(src, len, n, max_pts, dst);
    else
        copy_paths_kernel<0><<<grid, 256, 0, s>>>(src, len, n, max_pts, dst);
}

// ------------------------------------------------------------------ dependent-load latency
// The walk's floor is a chain of dependent gathers.  This measures the
// latency of one such gather: one thread follows a random cycle through a
// buffer, one 4-byte index at the head of every 128-byte line, each load's
// address the value of the one before (loads at L2, bypassing L1).
namespace {
// steps loads from the position *pos, which is left where the chase ended
__global__ void load_chase_kernel(const int32_t *__restrict__ a, int64_t steps, int32_t *__restrict__ pos) {
    int32_t j = *pos;
    for (int64_t i = 0; i < steps; ++i) j = __ldcg(a + j);
    *pos = j;
}
}  // namespace

dd_status measure_load_latency(int64_t bytes, int32_t steps, cudaStream_t s, double *ns, std::string &err) {
    const int64_t n = bytes / 128;            // lines
    // a single cycle over all lines in a seeded random order
    std::vector<int64_t> perm((size_t)n);
    for (int64_t i = 0; i < n; ++i) perm[(size_t)i] = i;
    std::mt19937_64 rng(0x5eedULL);
    for (int64_t i = n - 1; i > 0; --i) {
        const int64_t j = (int64_t)(rng() % (uint64_t)(i + 1));
        std::swap(perm[(size_t)i], perm[(size_t)j]);
    }
    std::vector<int32_t> next((size_t)n);
    for (int64_t i = 0; i < n; ++i) next[(size_t)perm[(size_t)i]] = (int32_t)(perm[(size_t)((i + 1) % n)] * 32);
    int32_t *d = nullptr, *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    dd_status st = DD_OK;
    auto fail = [&](dd_status code, const char *what) {
        cudaGetLastError();
        err = what;
        st = code;
    };
    if (cudaMalloc(&d, (size_t)n * 128) != cudaSuccess || cudaMalloc(&sink, sizeof(int32_t)) != cudaSuccess) {
        fail(DD_ENOMEM, "allocation of the latency buffer failed");
    } else if (cudaMemcpy2DAsync(d, 128, next.data(), sizeof(int32_t), sizeof(int32_t), (size_t)n,
                                 cudaMemcpyHostToDevice, s) != cudaSuccess ||
               cudaMemsetAsync(sink, 0, sizeof(int32_t), s) != cudaSuccess ||
               cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        fail(DD_ECUDA, "latency buffer set-up failed");
    } else {
        // warm-up: the whole cycle when it is short (the timed loads then hit
        // L2), else its first 2^18 lines (the timed loads go on to lines not
        // yet visited)
        load_chase_kernel<<<1, 1, 0, s>>>(d, std::min<int64_t>(n, 1 << 18), sink);
        cudaEventRecord(e0, s);
        load_chase_kernel<<<1, 1, 0, s>>>(d, steps, sink);
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            fail(DD_ECUDA, "latency kernel failed");
        else
            *ns = (double)ms * 1e6 / steps;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (d) cudaFree(d);
    if (sink) cudaFree(sink);
    return st;
}
