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
#include <cfloat>
#include <cmath>

#include "dd_internal.h"

namespace {

constexpr float kEpsBary = 1e-6f;    // barycentric snap to a vertex
constexpr float kEpsWedge = 1e-6f;   // relative tolerance of the wedge / entry tests

struct TraceParams {
    const int4 *tri;
    const int4 *tnbr;
    const float4 *gphi;
    const float2 *xy;
    const int32_t *vt_off, *vt, *vn_off, *vn;
    const float *fields;
    int64_t field_stride;
    const int32_t *targets, *sources;
    int64_t total;
    int32_t S, max_pts, max_steps;
    float2 *out_xy;
    int32_t *out_len, *out_status;
};

__device__ __forceinline__ int comp(const int4 v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

__device__ __forceinline__ int local_of(const int4 v, int x) { return v.x == x ? 0 : (v.y == x ? 1 : 2); }

__device__ __forceinline__ void load_gphi(const float4 *gphi, int t, float2 g[3]) {
    const float4 a = gphi[2 * t], b = gphi[2 * t + 1];
    g[0] = make_float2(a.x, a.y);
    g[1] = make_float2(a.z, a.w);
    g[2] = make_float2(b.x, b.y);
}

__device__ __forceinline__ float dot2(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }

__device__ __forceinline__ float2 tri_grad(const float *f, const int4 tv, const float2 g[3]) {
    const float f0 = f[tv.x], d1 = f[tv.y] - f0, d2 = f[tv.z] - f0;
    return make_float2(d1 * g[1].x + d2 * g[2].x, d1 * g[1].y + d2 * g[2].y);
}

__global__ void __launch_bounds__(128) trace_kernel(const TraceParams p) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= p.total) return;
    const int a = (int)(id / p.S);
    const int target = p.targets[a];
    const float *f = p.fields + (int64_t)a * p.field_stride;
    float2 *out = p.out_xy + id * p.max_pts;
    int v = p.sources[id];
    int len = 0;
    int status = DD_TRACE_STEP_LIMIT;
    out[len++] = p.xy[v];
    bool at_vertex = true;
    int tc = -1, ic = 0;          // edge state: left triangle tc through the edge opposite local ic
    float la = 0.f, lb = 0.f;     // barycentric weights of its endpoints (ic+1, ic+2)

#define DD_PUSH(pt)                              \
    do {                                         \
        if (len >= p.max_pts) {                  \
            status = DD_TRACE_TRUNCATED;         \
            goto done;                           \
        }                                        \
        out[len++] = (pt);                       \
    } while (0)

    for (int step = 0; step < p.max_steps; ++step) {
        if (at_vertex) {
            if (v == target) {
                status = DD_TRACE_OK;
                goto done;
            }
            bool adj = false;
            for (int q = p.vn_off[v]; q < p.vn_off[v + 1]; ++q) adj |= (p.vn[q] == target);
            if (adj) {
                DD_PUSH(p.xy[target]);
                status = DD_TRACE_OK;
                goto done;
            }
            int best = -1, best_i = 0;
            float best_g = 0.f, baj = 0.f, bak = 0.f;
            for (int q = p.vt_off[v]; q < p.vt_off[v + 1]; ++q) {
                const int t = p.vt[q];
                const int4 tv = p.tri[t];
                float2 g3[3];
                load_gphi(p.gphi, t, g3);
                const float2 g = tri_grad(f, tv, g3);
                const float gn = sqrtf(g.x * g.x + g.y * g.y);
                if (!(gn > 0.f)) continue;
                const int i = local_of(tv, v), j = (i + 1) % 3, k = (i + 2) % 3;
                const float aj = -dot2(g3[j], g), ak = -dot2(g3[k], g);
                const float tol = kEpsWedge * gn * fmaxf(sqrtf(dot2(g3[j], g3[j])), sqrtf(dot2(g3[k], g3[k])));
                if (aj >= -tol && ak >= -tol && aj + ak > 0.f && gn > best_g) {
                    best = t;
                    best_i = i;
                    best_g = gn;
                    baj = fmaxf(aj, 0.f);
                    bak = fmaxf(ak, 0.f);
                }
            }
            if (best >= 0) {
                const int4 tv = p.tri[best];
                const int vj = comp(tv, (best_i + 1) % 3), vk = comp(tv, (best_i + 2) % 3);
                const float s = 1.0f / (baj + bak);
                const float lj = s * baj, lk = s * bak;
                if (lj <= kEpsBary) {
                    DD_PUSH(p.xy[vk]);
                    v = vk;
                } else if (lk <= kEpsBary) {
                    DD_PUSH(p.xy[vj]);
                    v = vj;
                } else {
                    const float2 pj = p.xy[vj], pk = p.xy[vk];
                    DD_PUSH(make_float2(lj * pj.x + lk * pk.x, lj * pj.y + lk * pk.y));
                    at_vertex = false;
                    tc = best;
                    ic = best_i;
                    la = lj;
                    lb = lk;
                }
                continue;
            }
            // edge fallback
            int best_u = -1;
            float best_s = 0.f;
            const float fv = f[v];
            const float2 pv = p.xy[v];
            for (int q = p.vn_off[v]; q < p.vn_off[v + 1]; ++q) {
                const int u = p.vn[q];
                const float2 pu = p.xy[u];
                const float dx = pv.x - pu.x, dy = pv.y - pu.y;
                const float slope = (fv - f[u]) / sqrtf(dx * dx + dy * dy);
                if (slope > best_s) {
                    best_s = slope;
                    best_u = u;
                }
            }
            if (best_u < 0) {
                status = DD_TRACE_STUCK;
                goto done;
            }
            DD_PUSH(p.xy[best_u]);
            v = best_u;
            continue;
        }
        // ---- edge state
        {
            const int4 tv = p.tri[tc];
            const int av = comp(tv, (ic + 1) % 3), bv = comp(tv, (ic + 2) % 3);
            if (av == target || bv == target) {
                DD_PUSH(p.xy[target]);
                status = DD_TRACE_OK;
                goto done;
            }
            const int t2 = comp(p.tnbr[tc], ic);
            bool slide = t2 < 0;
            int4 tv2 = make_int4(0, 0, 0, 0);
            float2 g3[3], g2 = make_float2(0.f, 0.f);
            int ia = 0, ib = 0, c2 = 0;
            float rc = 0.f;
            if (!slide) {
                tv2 = p.tri[t2];
                load_gphi(p.gphi, t2, g3);
                g2 = tri_grad(f, tv2, g3);
                ia = local_of(tv2, av);
                ib = local_of(tv2, bv);
                c2 = 3 - ia - ib;
                rc = -dot2(g3[c2], g2);
                const float gn = sqrtf(g2.x * g2.x + g2.y * g2.y);
                const float tol = kEpsWedge * gn * sqrtf(dot2(g3[c2], g3[c2]));
                slide = !(rc > tol);
            }
            if (slide) {
                const float fa = f[av], fb = f[bv];
                const int low = (fa < fb || (fa == fb && av < bv)) ? av : bv;
                DD_PUSH(p.xy[low]);
                v = low;
                at_vertex = true;
                continue;
            }
            const float ra = -dot2(g3[ia], g2), rb = -dot2(g3[ib], g2);
            const float sa = ra < 0.f ? la / -ra : INFINITY;
            const float sb = rb < 0.f ? lb / -rb : INFINITY;
            if (!(fminf(sa, sb) < INFINITY)) {     // no exit edge found: treat as a valley edge
                const float fa = f[av], fb = f[bv];
                const int low = (fa < fb || (fa == fb && av < bv)) ? av : bv;
                DD_PUSH(p.xy[low]);
                v = low;
                at_vertex = true;
                continue;
            }
            const int cv = comp(tv2, c2);
            int exit_local, keep_v;        // exit through the edge opposite exit_local; keep_v stays on it
            float lkeep, lc2;
            if (sa <= sb) {
                lkeep = fmaxf(lb + sa * rb, 0.f);
                lc2 = fmaxf(sa * rc, 0.f);
                exit_local = ia;
                keep_v = bv;
            } else {
                lkeep = fmaxf(la + sb * ra, 0.f);
                lc2 = fmaxf(sb * rc, 0.f);
                exit_local = ib;
                keep_v = av;
            }
            const float tot = lkeep + lc2;
            lkeep /= tot;
            lc2 /= tot;
            if (lkeep <= kEpsBary) {
                DD_PUSH(p.xy[cv]);
                v = cv;
                at_vertex = true;
                continue;
            }
            if (lc2 <= kEpsBary) {
                DD_PUSH(p.xy[keep_v]);
                v = keep_v;
                at_vertex = true;
                continue;
            }
            const int e1 = comp(tv2, (exit_local + 1) % 3), e2 = comp(tv2, (exit_local + 2) % 3);
            const float l1 = e1 == cv ? lc2 : lkeep, l2 = e2 == cv ? lc2 : lkeep;
            const float2 p1 = p.xy[e1], p2 = p.xy[e2];
            DD_PUSH(make_float2(l1 * p1.x + l2 * p2.x, l1 * p1.y + l2 * p2.y));
            tc = t2;
            ic = exit_local;
            la = l1;
            lb = l2;
        }
    }
done:
#undef DD_PUSH
    p.out_len[id] = len;
    p.out_status[id] = status;
}

}  // namespace

void launch_trace(const DevMesh &m, const float *fields, int64_t field_stride, const int32_t *targets,
                  const int32_t *sources, int32_t T, int32_t S, int32_t max_pts, float2 *out_xy, int32_t *out_len,
                  int32_t *out_status, cudaStream_t s) {
    TraceParams p;
    p.tri = m.tri;
    p.tnbr = m.tnbr;
    p.gphi = m.gphi;
    p.xy = m.xy;
    p.vt_off = m.vt_off;
    p.vt = m.vt;
    p.vn_off = m.vn_off;
    p.vn = m.vn;
    p.fields = fields;
    p.field_stride = field_stride;
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
    trace_kernel<<<(unsigned)((p.total + 127) / 128), 128, 0, s>>>(p);
}
