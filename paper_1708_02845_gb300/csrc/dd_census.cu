// Spurious local minima of a distance field (Section V, "Low resolution
// discretizations") and edge-following paths (Section IV, "Gradient-descent
// path generation", the simplest of the two tracers), on the mesh's
// vertex-neighbour lists.
//  * census: an interior vertex v other than the target is a spurious local
//    minimum when no neighbour has a smaller value, f[v] <= f[u] for all u;
//    one thread per (field, vertex), counts by atomic adds.
//  * edge paths: from the source, move to the neighbour of smallest value
//    among those below the current vertex (ties to the lowest id) until the
//    target (OK) or a vertex with no lower neighbour (STUCK); STEP_LIMIT after
//    n_v moves, TRUNCATED when the polyline would exceed max_pts points.
//    One thread per path.  Only comparisons of the given FP32 values are
//    made, so the results are exactly those of the same rule applied to the
//    same values anywhere.
#include "dd_internal.h"

namespace {

__global__ void local_minima_kernel(int64_t n_v, const int32_t *__restrict__ vn_off, const int32_t *__restrict__ vn,
                                    const uint8_t *__restrict__ isb, const float *__restrict__ fields,
                                    const int32_t *__restrict__ targets, uint8_t *__restrict__ flags,
                                    int32_t *__restrict__ counts) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (v >= n_v) return;
    const float *f = fields + (int64_t)a * n_v;
    bool is_min = false;
    if (!isb[v] && v != targets[a]) {
        const float fv = f[v];
        is_min = true;
        for (int32_t q = vn_off[v]; q < vn_off[v + 1] && is_min; ++q) is_min = f[vn[q]] >= fv;
    }
    if (flags) flags[(int64_t)a * n_v + v] = is_min ? 1 : 0;
    if (is_min) atomicAdd(counts + a, 1);
}

__global__ void edge_path_kernel(int64_t n_v, const int32_t *__restrict__ vn_off, const int32_t *__restrict__ vn,
                                 const float2 *__restrict__ xy, const float *__restrict__ fields,
                                 const int32_t *__restrict__ targets, const int32_t *__restrict__ sources, int64_t total,
                                 int32_t S, int32_t max_pts, float2 *__restrict__ out_xy,
                                 int32_t *__restrict__ out_len, int32_t *__restrict__ out_status) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= total) return;
    const int a = (int)(id / S);
    const float *f = fields + (int64_t)a * n_v;
    const int target = targets[a];
    float2 *out = out_xy + id * max_pts;
    int v = sources[id], len = 0, status = DD_TRACE_STEP_LIMIT;
    out[len++] = xy[v];
    if (v == target) {
        status = DD_TRACE_OK;
    } else {
        for (int64_t step = 0; step < n_v; ++step) {
            int best = -1;
            float fb = f[v];
            for (int32_t q = vn_off[v]; q < vn_off[v + 1]; ++q) {   // neighbours in ascending id order
                const int u = vn[q];
                const float fu = f[u];
                if (fu < fb) {
                    fb = fu;
                    best = u;
                }
            }
            if (best < 0) {
                status = DD_TRACE_STUCK;
                break;
            }
            if (len >= max_pts) {
                status = DD_TRACE_TRUNCATED;
                break;
            }
            v = best;
            out[len++] = xy[v];
            if (v == target) {
                status = DD_TRACE_OK;
                break;
            }
        }
    }
    out_len[id] = len;
    out_status[id] = status;
}

}  // namespace

void launch_local_minima(const DevMesh &m, const float *fields, const int32_t *targets, int32_t T, int32_t *counts,
                         uint8_t *flags, cudaStream_t s) {
    local_minima_kernel<<<dim3((unsigned)((m.n_v + 255) / 256), (unsigned)T), 256, 0, s>>>(
        m.n_v, m.vn_off, m.vn, m.isb, fields, targets, flags, counts);
}

void launch_edge_paths(const DevMesh &m, const float *fields, const int32_t *targets, const int32_t *sources, int32_t T,
                       int32_t S, int32_t max_pts, float2 *out_xy, int32_t *out_len, int32_t *out_status,
                       cudaStream_t s) {
    const int64_t total = (int64_t)T * S;
    if (total == 0) return;
    edge_path_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(m.n_v, m.vn_off, m.vn, m.xy, fields, targets,
                                                                      sources, total, S, max_pts, out_xy, out_len,
                                                                      out_status);
}
