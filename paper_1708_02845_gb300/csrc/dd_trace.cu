// Triangle-based gradient-descent path tracing, Section IV ("Gradient-descent
// path generation"), one thread per (target, source) pair.
//
// The field is piecewise linear, so triangle tau has the constant gradient
// g = (f1 - f0) grad(phi_1) + (f2 - f0) grad(phi_2) and the path follows -g.
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
// Layout for latency: every triangle is one 64-byte record (vertex ids,
// neighbour ids, hat gradients of vertices 0 and 1 -- the third is minus their
// sum -- and vertex positions), and the per-field triangle gradients are
// computed once per field by tri_grad_kernel.  Crossing a triangle then needs
// a single dependent load level: the record and gradient of the next triangle,
// whose id sits in the current record.
#include <cfloat>
#include <cstring>
#include <algorithm>
#include <cmath>

#include "dd_internal.h"

namespace {

constexpr float kEpsBary = 1e-6f;    // barycentric snap to a vertex
constexpr float kEpsWedge = 1e-6f;   // relative tolerance of the wedge / entry tests

struct TraceParams {
    const int4 *rec;               // [n_t][4] triangle records
    const float2 *grads;           // [T][n_t] per-field triangle gradients
    const float2 *xy;
    const int32_t *vt_off, *vt;
    const float *fields;
    int64_t field_stride, n_t;
    const int32_t *targets, *sources;
    int64_t total;
    int32_t S, max_pts, max_steps;
    float2 *out_xy;
    int32_t *out_len, *out_status;
};

struct Tri {
    int v0, v1, v2, n0, n1, n2;
    float2 g0, g1, p0, p1, p2;
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
    T.g0 = make_float2(__int_as_float(b.z), __int_as_float(b.w));
    T.g1 = make_float2(c.x, c.y);
    T.p0 = make_float2(c.z, c.w);
    T.p1 = make_float2(d.x, d.y);
    T.p2 = make_float2(d.z, d.w);
    return T;
}

__device__ __forceinline__ int vid(const Tri &T, int i) { return i == 0 ? T.v0 : (i == 1 ? T.v1 : T.v2); }
__device__ __forceinline__ float2 pos(const Tri &T, int i) { return i == 0 ? T.p0 : (i == 1 ? T.p1 : T.p2); }
__device__ __forceinline__ int local_of(const Tri &T, int x) { return T.v0 == x ? 0 : (T.v1 == x ? 1 : 2); }
__device__ __forceinline__ float dot2(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }

// g = f0 grad(phi_0) + f1 grad(phi_1) + f2 grad(phi_2) = (f0 - f2) g0 + (f1 - f2) g1
__global__ void tri_grad_kernel(const int4 *__restrict__ rec, int64_t n_t, const float *__restrict__ fields,
                                int64_t field_stride, float2 *__restrict__ grads) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_t) return;
    const int a = blockIdx.y;
    const Tri T = load_tri(rec, (int)t);
    const float *f = fields + (int64_t)a * field_stride;
    const float f2 = f[T.v2], d0 = f[T.v0] - f2, d1 = f[T.v1] - f2;
    grads[(int64_t)a * n_t + t] = make_float2(d0 * T.g0.x + d1 * T.g1.x, d0 * T.g0.y + d1 * T.g1.y);
}

// Loop structure: every iteration loads one triangle record (and its field
// gradient) and advances one thread's state by it, so the threads of a warp
// issue their loads together.  A vertex state walks the fan of triangles
// around the vertex through the neighbour links (counter-clockwise from a
// known incident triangle, then clockwise from it if the fan is open),
// evaluating one triangle per iteration.  Both states share one rotated view
// of the loaded triangle: a reference vertex R (the fan vertex, or the
// second endpoint b of the entry edge) and the two that follow it
// counter-clockwise, X and Y.  For an entry edge (a, b) of the previous
// triangle, consistent orientation puts a at X and the opposite vertex at Y.
// Quantities on the critical path use squared norms and approximate
// reciprocals; the decisions they feed carry relative tolerances.
__device__ __forceinline__ float sel3f(int i, float a, float b, float c) { return i == 0 ? a : (i == 1 ? b : c); }
__device__ __forceinline__ int sel3i(int i, int a, int b, int c) { return i == 0 ? a : (i == 1 ? b : c); }

struct TraceDom {
    const int4 *rec;
    const float2 *xy;
    const int32_t *vt_off, *vt;
    int64_t n_t;
};

// one path: walk from `source` to `target` on field f (triangle gradients `grads`)
__device__ __forceinline__ void trace_path(const TraceDom &p, const float *__restrict__ f,
                                           const float2 *__restrict__ grads, int target, int source,
                                           float2 *__restrict__ out, int32_t max_pts, int32_t max_steps,
                                           int32_t *len_out, int32_t *status_out, bool active) {
    const float eps2 = kEpsWedge * kEpsWedge;
    int v = source;
    int len = 0;
    int status = DD_TRACE_STEP_LIMIT;
    int states = 1;                // vertex and edge states entered (the step cap counts these)
    bool fin = !active;            // finished (or a padding lane): idles until the warp is done
    if (active) out[len++] = p.xy[v];

    // vertex (fan-scan) state
    bool scanning = true;
    int t0 = active ? p.vt[p.vt_off[v]] : 0;
    int scan_t = t0, t0_cw = -1;
    bool ccw = true, adj = false;
    int best = -1;
    float best_g2 = 0.f, baj = 0.f, bak = 0.f;
    int b_vj = 0, b_vk = 0, b_next = -1;
    float2 b_pj = make_float2(0.f, 0.f), b_pk = b_pj;
    // edge state: the path sits on edge (ea, eb) of triangle cur_id, weights (la, lb),
    // and enters t_next (the triangle across that edge, -1 on the boundary)
    int cur_id = -1, t_next = -1, ea = 0, eb = 0;
    float la = 0.f, lb = 0.f;
    float2 pa = make_float2(0.f, 0.f), pb = pa;

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
#define DD_ENTER_VERTEX(vert, tri_id)            \
    v = (vert);                                  \
    scanning = true;                             \
    t0 = (tri_id);                               \
    scan_t = t0;                                 \
    t0_cw = -1;                                  \
    ccw = true;                                  \
    adj = false;                                 \
    best = -1;                                   \
    best_g2 = 0.f;                               \
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
        DD_ENTER_VERTEX(a_low ? ea : eb, cur_id);                      \
    }

    if (active && v == target) {
        status = DD_TRACE_OK;
        fin = true;
    }
    // The warp votes at the top of every iteration, so its threads reconverge
    // once per step instead of drifting into different iterations; finished
    // threads idle here until the last path of the warp ends.
    const int64_t iter_cap = 16LL * max_steps;
    for (int64_t iter = 0;; ++iter) {
        if (!fin && iter >= iter_cap) fin = true;
        if (!__any_sync(0xffffffffu, !fin)) break;
        if (fin) continue;
        if (!scanning && t_next < 0) {     // boundary edge: slide to the lower endpoint
            DD_SLIDE();
            continue;
        }
        const int tl = scanning ? scan_t : t_next;
        const Tri T = load_tri(p.rec, tl);
        const float2 g = grads[tl];
        // ---- shared rotated view: R = reference vertex, X = R+1, Y = R+2 (counter-clockwise)
        const int refv = scanning ? v : eb;
        const int L = local_of(T, refv), X = L == 2 ? 0 : L + 1, Y = L == 0 ? 2 : L - 1;
        const float r0 = -dot2(T.g0, g), r1 = -dot2(T.g1, g), r2 = -(r0 + r1);   // d(lambda_i)/ds along -g
        const float2 g2v = make_float2(-(T.g0.x + T.g1.x), -(T.g0.y + T.g1.y));
        const float q0 = dot2(T.g0, T.g0), q1 = dot2(T.g1, T.g1), q2 = dot2(g2v, g2v);
        const float gg = dot2(g, g);
        const float rX = sel3f(X, r0, r1, r2), rY = sel3f(Y, r0, r1, r2);
        const float qX = sel3f(X, q0, q1, q2), qY = sel3f(Y, q0, q1, q2);
        const int vX = sel3i(X, T.v0, T.v1, T.v2), vY = sel3i(Y, T.v0, T.v1, T.v2);
        const float2 pY = make_float2(sel3f(Y, T.p0.x, T.p1.x, T.p2.x), sel3f(Y, T.p0.y, T.p1.y, T.p2.y));
        const int nL = sel3i(L, T.n0, T.n1, T.n2), nX = sel3i(X, T.n0, T.n1, T.n2), nY = sel3i(Y, T.n0, T.n1, T.n2);
        if (scanning) {
            // ---- one triangle of the fan around v (v = R, the candidate exit edge is X-Y)
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
                b_pj = make_float2(sel3f(X, T.p0.x, T.p1.x, T.p2.x), sel3f(X, T.p0.y, T.p1.y, T.p2.y));
                b_pk = pY;
                b_next = nL;
            }
            if (tl == t0) t0_cw = nY;
            int next = ccw ? nX : nY;
            if (ccw && next == t0) {
                next = -1;                       // closed fan: done
            } else if (ccw && next < 0) {
                ccw = false;                     // open fan: continue clockwise from t0
                next = t0_cw;
            }
            if (next >= 0) {
                scan_t = next;
                continue;
            }
            // ---- fan complete
            if (adj) {                           // v lies on an edge incident on the target
                DD_PUSH(p.xy[target]);
                status = DD_TRACE_OK;
                fin = true;
                continue;
            }
            if (best >= 0) {
                const float s = __fdividef(1.0f, baj + bak);
                const float lj = s * baj, lk = s * bak;
                if (lj <= kEpsBary) {
                    DD_PUSH(b_pk);
                    DD_ENTER_VERTEX(b_vk, best);
                } else if (lk <= kEpsBary) {
                    DD_PUSH(b_pj);
                    DD_ENTER_VERTEX(b_vj, best);
                } else {
                    DD_PUSH(make_float2(lj * b_pj.x + lk * b_pk.x, lj * b_pj.y + lk * b_pk.y));
                    scanning = false;
                    cur_id = best;
                    t_next = b_next;
                    ea = b_vj;
                    eb = b_vk;
                    pa = b_pj;
                    pb = b_pk;
                    la = lj;
                    lb = lk;
                    if (++states > max_steps) {
                        fin = true;
                        continue;
                    }
                }
                continue;
            }
            // no descending triangle: the incident edge of largest positive slope
            // (ties to the lower id); rare, so it walks the vertex's triangle list
            {
                int best_u = -1, best_ut = -1;
                float best_s = 0.f;
                float2 best_p = make_float2(0.f, 0.f);
                const float fv = f[v];
                const float2 pv = p.xy[v];
                for (int q = p.vt_off[v]; q < p.vt_off[v + 1]; ++q) {
                    const int tq = p.vt[q];
                    const Tri Q = load_tri(p.rec, tq);
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
                            best_ut = tq;
                        }
                    }
                }
                if (best_u < 0) {
                    status = DD_TRACE_STUCK;
                    fin = true;
                    continue;
                }
                DD_PUSH(best_p);
                DD_ENTER_VERTEX(best_u, best_ut);
                continue;
            }
        }
        // ---- edge state: entering T across (ea, eb); ea = X, eb = R, the opposite vertex is Y
        {
            const float ra = rX, rb = sel3f(L, r0, r1, r2), rc = rY;
            const bool enters = rc > 0.f && rc * rc > eps2 * gg * qY;
            const float sa = ra < 0.f ? __fdividef(la, -ra) : INFINITY;
            const float sb = rb < 0.f ? __fdividef(lb, -rb) : INFINITY;
            if (!enters || !(fminf(sa, sb) < INFINITY)) {   // valley edge (or no exit): lower endpoint
                DD_SLIDE();
                continue;
            }
            const bool via_a = sa <= sb;                      // exit through the edge opposite a (= Y-R edge)
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
                DD_ENTER_VERTEX(vY, tl);
                continue;
            }
            if (lc2 <= kEpsBary) {
                DD_PUSH(keep_p);
                DD_ENTER_VERTEX(keep_v, tl);
                continue;
            }
            DD_PUSH(make_float2(lkeep * keep_p.x + lc2 * pY.x, lkeep * keep_p.y + lc2 * pY.y));
            // new edge in T's counter-clockwise order: via a -> (Y, R) = (c, b); via b -> (X, Y) = (a, c)
            cur_id = tl;
            if (via_a) {
                t_next = nX;
                ea = vY;
                eb = keep_v;
                pa = pY;
                pb = keep_p;
                la = lc2;
                lb = lkeep;
            } else {
                t_next = nL;
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
    }
#undef DD_PUSH
#undef DD_ENTER_VERTEX
#undef DD_SLIDE
    if (active) {
        *len_out = len;
        *status_out = status;
    }
}

__global__ void __launch_bounds__(64) trace_kernel(const TraceParams p) {
    const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = gid < p.total;       // padding lanes stay in the warp's walk loop, idle
    const int64_t id = active ? gid : 0;
    const int a = (int)(id / p.S);
    TraceDom d;
    d.rec = p.rec;
    d.xy = p.xy;
    d.vt_off = p.vt_off;
    d.vt = p.vt;
    d.n_t = p.n_t;
    trace_path(d, p.fields + (int64_t)a * p.field_stride, p.grads + (int64_t)a * p.n_t, p.targets[a], p.sources[id],
               p.out_xy + id * p.max_pts, p.max_pts, p.max_steps, p.out_len + id, p.out_status + id, active);
}

// ---- several meshes in one launch: global target g belongs to domain tdom[g] (local index tloc[g])
struct BatchTraceDom {
    TraceDom d;
    const float *fields;      // [T_d][n_v]
    float2 *grads;            // [T_d][n_t]
    int64_t n_v;
    int32_t max_steps, pad;
};

__global__ void batch_grad_kernel(const BatchTraceDom *__restrict__ doms, const int32_t *__restrict__ tdom,
                                  const int32_t *__restrict__ tloc) {
    const int g = blockIdx.y;
    const BatchTraceDom q = doms[tdom[g]];
    const int a = tloc[g];
    const float *f = q.fields + (int64_t)a * q.n_v;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < q.d.n_t; t += (int64_t)gridDim.x * blockDim.x) {
        const Tri T = load_tri(q.d.rec, (int)t);
        const float f2 = f[T.v2], d0 = f[T.v0] - f2, d1 = f[T.v1] - f2;
        q.grads[(int64_t)a * q.d.n_t + t] = make_float2(d0 * T.g0.x + d1 * T.g1.x, d0 * T.g0.y + d1 * T.g1.y);
    }
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
    trace_path(q.d, q.fields + (int64_t)a * q.n_v, q.grads + (int64_t)a * q.d.n_t, targets[g], sources[id],
               out_xy + id * max_pts, max_pts, q.max_steps, out_len + id, out_status + id, active);
}

}  // namespace

void launch_trace(const DevMesh &m, const float *fields, int64_t field_stride, const int32_t *targets,
                  const int32_t *sources, int32_t T, int32_t S, int32_t max_pts, float2 *out_xy, int32_t *out_len,
                  int32_t *out_status, float2 *grads, cudaStream_t s) {
    TraceParams p;
    p.rec = m.trec;
    p.grads = grads;
    p.xy = m.xy;
    p.vt_off = m.vt_off;
    p.vt = m.vt;
    p.fields = fields;
    p.field_stride = field_stride;
    p.n_t = m.n_t;
    p.targets = targets;
    p.sources = sources;
    p.total = (int64_t)T * S;
    p.S = S;
    p.max_pts = max_pts;
    const int64_t cap = 4 * m.n_t;
    p.max_steps = cap > (int64_t)INT32_MAX ? INT32_MAX : (int32_t)cap;
    p.out_xy = out_xy;
    p.out_len = out_len;
    p.out_status = out_status;
    if (p.total == 0) return;
    dim3 gg((unsigned)((m.n_t + 255) / 256), (unsigned)T);
    tri_grad_kernel<<<gg, 256, 0, s>>>(m.trec, m.n_t, fields, field_stride, grads);
    trace_kernel<<<(unsigned)((p.total + 63) / 64), 64, 0, s>>>(p);
}

size_t batch_trace_dom_bytes() { return sizeof(BatchTraceDom); }

// host-side builder of one domain descriptor (into a byte buffer uploaded by the caller)
void fill_batch_trace_dom(void *dst, const DevMesh &m, const float *fields, float2 *grads) {
    BatchTraceDom q;
    q.d.rec = m.trec;
    q.d.xy = m.xy;
    q.d.vt_off = m.vt_off;
    q.d.vt = m.vt;
    q.d.n_t = m.n_t;
    q.fields = fields;
    q.grads = grads;
    q.n_v = m.n_v;
    const int64_t cap = 4 * m.n_t;
    q.max_steps = cap > (int64_t)INT32_MAX ? INT32_MAX : (int32_t)cap;
    q.pad = 0;
    std::memcpy(dst, &q, sizeof q);
}

void launch_batch_trace(const void *d_doms, const int32_t *d_tdom, const int32_t *d_tloc, const int32_t *d_targets,
                        const int32_t *d_sources, int32_t n_targets, int32_t S, int64_t max_nt, int32_t max_pts,
                        float2 *out_xy, int32_t *out_len, int32_t *out_status, cudaStream_t s,
                        const int32_t *d_path_target, int64_t n_paths) {
    if (n_targets <= 0) return;
    const BatchTraceDom *doms = reinterpret_cast<const BatchTraceDom *>(d_doms);
    dim3 gg((unsigned)std::max<int64_t>(1, std::min<int64_t>(64, (max_nt + 255) / 256)), (unsigned)n_targets);
    batch_grad_kernel<<<gg, 256, 0, s>>>(doms, d_tdom, d_tloc);
    const int64_t total = d_path_target ? n_paths : (int64_t)n_targets * S;
    if (total == 0) return;
    batch_trace_kernel<<<(unsigned)((total + 63) / 64), 64, 0, s>>>(doms, d_tdom, d_tloc, d_targets, d_sources,
                                                                    d_path_target, total, S, max_pts, out_xy, out_len,
                                                                    out_status);
}
