// C ABI of libdd: context, mesh upload, Poisson kernel, fields and paths.
// Every entry point returns a dd_status and never lets a C++ exception out.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <tuple>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cmath>

#include "dd_amg.h"
#include "dd_internal.h"

namespace {

dd_status set_err(dd_ctx *c, dd_status s, const std::string &msg) {
    if (c) c->err = msg;
    return s;
}

dd_status cuda_err(dd_ctx *c, cudaError_t e, const char *what) {
    cudaGetLastError();
    return set_err(c, e == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(expr, what)                                   \
    do {                                                 \
        cudaError_t e_ = (expr);                         \
        if (e_ != cudaSuccess) return cuda_err(ctx, e_, what); \
    } while (0)

dd_status select_device(dd_ctx *ctx) {
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_err(ctx, e, "cudaSetDevice");
    return DD_OK;
}

// grow a scratch buffer (synchronises the stream first when it must reallocate)
dd_status ensure_scratch(dd_ctx *ctx, int id, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (ctx->scratch_cap[id] >= bytes) return DD_OK;
    CK(cudaStreamSynchronize(ctx->stream), "synchronize before scratch growth");
    if (ctx->scratch[id]) cudaFree(ctx->scratch[id]);
    ctx->scratch[id] = nullptr;
    ctx->scratch_cap[id] = 0;
    size_t cap = bytes + bytes / 4;
    cudaError_t e = cudaMalloc(&ctx->scratch[id], cap);
    if (e != cudaSuccess) return cuda_err(ctx, e, "scratch allocation");
    ctx->scratch_cap[id] = cap;
    return DD_OK;
}

// copy a small host index array to a scratch buffer through pinned staging
dd_status upload(dd_ctx *ctx, int id, const void *host, size_t bytes) {
    dd_status st = ensure_scratch(ctx, id, bytes);
    if (st != DD_OK) return st;
    if (bytes == 0) return DD_OK;
    // the previous upload from this staging buffer must have left it
    CK(cudaEventSynchronize(ctx->pinned_free[id]), "wait for staging");
    if (ctx->pinned_cap[id] < bytes) {
        if (ctx->pinned[id]) cudaFreeHost(ctx->pinned[id]);
        ctx->pinned[id] = nullptr;
        ctx->pinned_cap[id] = 0;
        size_t cap = bytes + bytes / 4 + 4096;
        CK(cudaMallocHost(&ctx->pinned[id], cap), "pinned staging allocation");
        ctx->pinned_cap[id] = cap;
    }
    std::memcpy(ctx->pinned[id], host, bytes);
    CK(cudaMemcpyAsync(ctx->scratch[id], ctx->pinned[id], bytes, cudaMemcpyHostToDevice, ctx->stream),
       "index upload");
    CK(cudaEventRecord(ctx->pinned_free[id], ctx->stream), "record staging event");
    return DD_OK;
}

// 1 = device memory of this context's device, 0 = host memory, -1 = another device
int pointer_space(const dd_ctx *ctx, const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return a.device == ctx->device ? 1 : -1;
    return 0;
}

// The device address of page-locked (pinned) host memory, which kernels can
// write directly (over NVLink-C2C on Grace), or nullptr for other memory.
void *mapped_alias(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

dd_status ensure_side(dd_ctx *ctx) {
    if (ctx->side) return DD_OK;
    if (cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->side_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->side_ev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->side_ev[2], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return set_err(ctx, DD_ECUDA, "side stream creation failed");
    }
    return DD_OK;
}

dd_status get_mesh(dd_ctx *ctx, int32_t mesh, DevMesh **out) {
    if (!ctx) return DD_EINVAL;
    if (mesh < 0 || mesh >= (int32_t)ctx->meshes.size() || !ctx->meshes[mesh].live)
        return set_err(ctx, DD_EINVAL, "unknown mesh id " + std::to_string(mesh));
    *out = &ctx->meshes[mesh].dev;
    return DD_OK;
}

template <typename T>
dd_status dev_copy(dd_ctx *ctx, DevMesh &m, T **dst, const T *src, size_t count) {
    size_t bytes = (count ? count : 1) * sizeof(T);
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess) return cuda_err(ctx, e, "mesh allocation");
    m.owned.push_back(*dst);
    m.bytes += (int64_t)bytes;
    if (count) {
        e = cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_err(ctx, e, "mesh upload");
    }
    return DD_OK;
}

void free_mesh(DevMesh &m) {
    for (void *p : m.owned) cudaFree(p);
    m = DevMesh();
}

// free one device array of the mesh and forget it
template <typename T>
void release(DevMesh &m, T *&p, int64_t bytes) {
    if (!p) return;
    cudaFree((void *)p);
    m.owned.erase(std::remove(m.owned.begin(), m.owned.end(), (void *)p), m.owned.end());
    m.bytes -= bytes;
    p = nullptr;
}

// the tiled copy of P and of its log2 (the pipelined many-target field pass)
void drop_tiled(DevMesh &m) {
    const int64_t bytes = ((m.n_v + 127) / 128) * 128 * m.pt_kt * (int64_t)sizeof(float);
    release(m, m.pt_p, bytes);
    release(m, m.pt_l, bytes);
    m.pt_kt = 0;
}

void drop_sparse(DevMesh &m) {
    release(m, m.sp_rowsum, m.n_v * (int64_t)sizeof(long long));
    release(m, m.sp_off, (m.n_v + 1) * (int64_t)sizeof(int64_t));
    release(m, m.sp_val, m.sp_kept * (int64_t)sizeof(float));
    release(m, m.sp_col, m.sp_kept * (int64_t)sizeof(uint16_t));
    m.sp_kept = m.sp_bytes = 0;
    m.sp_theta = 0.f;
}

// what was derived from the stored P (the BF16 split, the row entropies, the
// sparse rows) goes when P is recomputed or replaced
void drop_derived(DevMesh &m) {
    release(m, m.LP, m.n_v * m.k_pad * (int64_t)sizeof(float));
    drop_tiled(m);
    release(m, m.p_hi, m.n_v * m.kb * 2);
    release(m, m.p_lo, m.n_v * m.kb * 2);
    release(m, m.ex, m.n_v * (int64_t)sizeof(float));
    m.kb = 0;
    drop_sparse(m);
}

dd_status check_targets(dd_ctx *ctx, const DevMesh &m, const int32_t *ids, int64_t count, bool interior_only,
                        const char *what) {
    if (count > 0 && !ids) return set_err(ctx, DD_EINVAL, std::string(what) + " pointer is null");
    if (count > 0 && pointer_space(ctx, ids) != 0)
        return set_err(ctx, DD_EINVAL, std::string(what) + " must be host memory");
    for (int64_t i = 0; i < count; ++i) {
        int32_t v = ids[i];
        if (v < 0 || v >= m.n_v)
            return set_err(ctx, DD_EINVAL, std::string(what) + " id out of range: " + std::to_string(v));
        if (interior_only && m.is_boundary[v])
            return set_err(ctx, DD_EINVAL, std::string(what) + " must be interior vertices; " + std::to_string(v) +
                                               " is on the boundary");
    }
    return DD_OK;
}

dd_status check_kernel_flag(dd_ctx *ctx) {
    int flag = 0;
    CK(cudaMemcpy(&flag, ctx->d_err, sizeof flag, cudaMemcpyDeviceToHost), "read kernel error flag");
    if (flag) {
        cudaMemset(ctx->d_err, 0, sizeof(int));
        return set_err(ctx, DD_ETIMEOUT, "a bounded device-side wait gave up");
    }
    return DD_OK;
}

// the fields of a mask in bit order (KL, TV, KLT): slot of `bit` in dst [nf][T][n_v]
float *field_slot(float *dst, uint32_t f_mask, uint32_t bit, int64_t stride) {
    if (!(f_mask & bit)) return nullptr;
    int slot = 0;
    for (uint32_t b = 1; b < bit; b <<= 1) slot += (f_mask & b) ? 1 : 0;
    return dst + slot * stride;
}

// The fields of T targets (ids already in device scratch) into dst
// ([fields][T][n_v] by default; stride: the distance between two fields'
// blocks when dst is a block of rows inside a larger output)
// (tile_done: null, or an event recorded once TV is final -- after the FP32
// many-target tile pass, else at the end)
dd_status fields_into(dd_ctx *ctx, DevMesh &m, const int32_t *d_targets, int32_t T, uint32_t f_mask, int32_t prec,
                      float *dst, int64_t stride = -1, cudaEvent_t tile_done = nullptr) {
    if (stride < 0) stride = (int64_t)T * m.n_v;
    float *kl = field_slot(dst, f_mask, DD_F_KL, stride);
    float *tv = field_slot(dst, f_mask, DD_F_TV, stride);
    float *klt = field_slot(dst, f_mask, DD_F_KLT, stride);
    dd_status st;
    if (prec == DD_PREC_BF16X3 && kl) {
        // KL through the split-BF16 tensor-core GEMM; TV and KLT (if asked) stay FP32 below
        std::string err;
        if ((st = prepare_bf16(m, ctx->stream, err)) != DD_OK) return set_err(ctx, st, err);
        if ((st = ensure_scratch(ctx, S_GEMM, gemm_target_scratch_bytes(m, T))) != DD_OK) return st;
        if ((st = launch_kl_gemm(m, d_targets, T, ctx->scratch[S_GEMM], kl, ctx->d_err, ctx->stream, err)) != DD_OK)
            return set_err(ctx, st, err);
        kl = nullptr;
        if (!tv && !klt) return DD_OK;
    }
    if (prec == DD_PREC_SPARSE || prec == DD_PREC_SPARSE_MERGED) {
        if (!m.sp_rowsum) return set_err(ctx, DD_ESTATE, "DD_PREC_SPARSE before dd_sparsify");
        if (sparse_field_smem(m.k_pad) > 200 * 1024)
            return set_err(ctx, DD_EINVAL, "DD_PREC_SPARSE: k too large for the staged target row");
        if (T > 65535) return set_err(ctx, DD_EINVAL, "DD_PREC_SPARSE: at most 65,535 targets per call");
        if ((st = ensure_scratch(ctx, S_STAGE, sparse_stage_bytes(m.k_pad, T))) != DD_OK) return st;
        float4 *stage = reinterpret_cast<float4 *>(ctx->scratch[S_STAGE]);
        launch_stage_targets(m.P, m.n_v, m.k_pad, d_targets, T, stage, ctx->stream);
        launch_sparse_fields(m, d_targets, stage, T, kl, tv, klt, prec == DD_PREC_SPARSE_MERGED, ctx->d_err,
                             ctx->stream);
        CK(cudaGetLastError(), "sparse field kernel launch");
        return DD_OK;
    }
    st = ensure_scratch(ctx, S_STAGE, 4 * (size_t)T * m.k_pad * sizeof(float));
    if (st != DD_OK) return st;
    float4 *stage = reinterpret_cast<float4 *>(ctx->scratch[S_STAGE]);
    launch_stage_targets(m.P, m.n_v, m.k_pad, d_targets, T, stage, ctx->stream, nullptr, m.LP);
    if (kl || tv) {
        // more than two targets: the tiled copy of P (built once per mesh) and the
        // targets staged in the same layout make the pipelined tile available
        TiledArgs ta{};
        const TiledArgs *tiled = nullptr;
        // (without room for them the staged tile shapes, which need none, run instead)
        if (T > 2) {
            std::string err;
            if (prepare_tiled(m, ctx->stream, err) == DD_OK &&
                ensure_scratch(ctx, S_TSTAGE, tiled_target_bytes(m.k_pad, T)) == DD_OK) {
                float *ts = reinterpret_cast<float *>(ctx->scratch[S_TSTAGE]);
                ta = TiledArgs{m.pt_p, m.pt_l, ts, ts + tiled_target_bytes(m.k_pad, T) / (2 * sizeof(float)),
                               m.pt_kt};
                tiled = &ta;
            } else {
                cudaGetLastError();
                ctx->err.clear();
            }
        }
        launch_fields_fp32(m.P, m.n_v, m.k_pad, stage, T, kl, tv, ctx->d_err, ctx->stream, -1, m.LP != nullptr,
                           tiled, tile_done);
    } else if (tile_done) {
        CK(cudaEventRecord(tile_done, ctx->stream), "fields event");
    }
    if (klt) {
        // the target-weighted KL is the reverse-KL member of the f-divergence kernels
        std::string err;
        if ((st = launch_fdiv(m.P, m.n_v, m.k_pad, stage, T, DD_DIV_KL_REVERSE, 0.0, klt, ctx->stream, err,
                              m.LP)) != DD_OK)
            return set_err(ctx, st, err);
    }
    CK(cudaGetLastError(), "field kernel launch");
    return DD_OK;
}

int popcount2(uint32_t f) { return ((f & DD_F_KL) ? 1 : 0) + ((f & DD_F_TV) ? 1 : 0) + ((f & DD_F_KLT) ? 1 : 0); }

}  // namespace

namespace {

struct KTimer {
    std::vector<std::tuple<const char *, cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> pool;
    std::map<std::string, std::pair<int64_t, double>> totals;   // launches, total ms
};

std::mutex g_kt_mutex;
std::map<cudaStream_t, KTimer> g_kt;
std::atomic<int> g_kt_on{0};

cudaEvent_t kt_event(KTimer &t) {
    if (!t.pool.empty()) {
        cudaEvent_t e = t.pool.back();
        t.pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void kt_fold(KTimer &t) {
    for (auto &m : t.pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(std::get<2>(m)) == cudaSuccess &&
            cudaEventElapsedTime(&ms, std::get<1>(m), std::get<2>(m)) == cudaSuccess) {
            auto &tot = t.totals[std::get<0>(m)];
            tot.first += 1;
            tot.second += ms;
        } else {
            cudaGetLastError();
        }
        t.pool.push_back(std::get<1>(m));
        t.pool.push_back(std::get<2>(m));
    }
    t.pending.clear();
}

}  // namespace

KMark::KMark(const char *n, cudaStream_t s) {
    if (!g_kt_on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> lock(g_kt_mutex);
    auto it = g_kt.find(s);
    if (it == g_kt.end()) return;
    cudaEvent_t e = kt_event(it->second);
    if (!e) return;
    if (cudaEventRecord(e, s) != cudaSuccess) {
        cudaGetLastError();
        it->second.pool.push_back(e);
        return;
    }
    name = n;
    stream = s;
    a = e;
}

KMark::~KMark() {
    if (!a) return;
    std::lock_guard<std::mutex> lock(g_kt_mutex);
    auto it = g_kt.find(stream);
    if (it == g_kt.end()) {
        cudaEventDestroy(a);
        return;
    }
    cudaEvent_t b = kt_event(it->second);
    if (!b || cudaEventRecord(b, stream) != cudaSuccess) {
        cudaGetLastError();
        it->second.pool.push_back(a);
        if (b) it->second.pool.push_back(b);
        return;
    }
    it->second.pending.emplace_back(name, a, b);
    if (it->second.pending.size() > 4096) kt_fold(it->second);
}

extern "C" {

int32_t dd_version(void) { return 100; }

dd_status dd_create(dd_ctx **out, int32_t device, void *cuda_stream) {
    if (!out) return DD_EINVAL;
    *out = nullptr;
    try {
        int count = 0;
        if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
            cudaGetLastError();
            return DD_EINVAL;
        }
        dd_ctx *ctx = new dd_ctx();
        ctx->device = device;
        ctx->stream = (cudaStream_t)cuda_stream;
        bool ok = cudaSetDevice(device) == cudaSuccess && cudaMalloc((void **)&ctx->d_err, sizeof(int)) == cudaSuccess &&
                  cudaMemset(ctx->d_err, 0, sizeof(int)) == cudaSuccess;
        for (int i = 0; ok && i < S_COUNT; ++i)
            ok = cudaEventCreateWithFlags(&ctx->pinned_free[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            dd_destroy(ctx);
            return DD_ECUDA;
        }
        *out = ctx;
        return DD_OK;
    } catch (...) {
        return DD_ENOMEM;
    }
}

dd_status dd_set_stream(dd_ctx *ctx, void *cuda_stream) {
    if (!ctx) return DD_EINVAL;
    ctx->stream = (cudaStream_t)cuda_stream;
    return DD_OK;
}

void dd_destroy(dd_ctx *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &s : ctx->meshes)
        if (s.live) free_mesh(s.dev);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    for (cudaEvent_t e : ctx->side_ev)
        if (e) cudaEventDestroy(e);
    for (int i = 0; i < S_COUNT; ++i)
        if (ctx->scratch[i]) cudaFree(ctx->scratch[i]);
    if (ctx->d_err) cudaFree(ctx->d_err);
    for (int i = 0; i < S_COUNT; ++i) {
        if (ctx->pinned[i]) cudaFreeHost(ctx->pinned[i]);
        if (ctx->pinned_free[i]) cudaEventDestroy(ctx->pinned_free[i]);
    }
    delete ctx;
}

const char *dd_last_error(const dd_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

dd_status dd_sync(dd_ctx *ctx) {
    if (!ctx) return DD_EINVAL;
    try {
        dd_status st = select_device(ctx);
        if (st != DD_OK) return st;
        CK(cudaStreamSynchronize(ctx->stream), "stream synchronize");
        return check_kernel_flag(ctx);
    } catch (...) {
        return DD_ENOMEM;
    }
}

dd_status dd_check_mesh(const double *xy, int64_t n_v, const int32_t *tri, int64_t n_t, const int32_t *loop_idx,
                        const int64_t *loop_off, int32_t n_loops, int64_t *info, char *msg, int32_t msg_len) {
    try {
        HostMesh h;
        std::string err;
        dd_status st = build_host_mesh(xy, n_v, tri, n_t, loop_idx, loop_off, n_loops, h, err);
        if (msg && msg_len > 0) {
            std::snprintf(msg, (size_t)msg_len, "%s", st == DD_OK ? "" : err.c_str());
        }
        if (st == DD_OK && info) {
            info[0] = h.n_v;
            info[1] = h.k;
            info[2] = h.m;
            info[3] = h.n_edges;
        }
        return st;
    } catch (const std::bad_alloc &) {
        return DD_ENOMEM;
    } catch (...) {
        return DD_EINVAL;
    }
}

dd_status dd_load_mesh(dd_ctx *ctx, const double *xy, int64_t n_v, const int32_t *tri, int64_t n_t,
                       const int32_t *loop_idx, const int64_t *loop_off, int32_t n_loops, int32_t *mesh_id) {
    if (!ctx || !mesh_id) return DD_EINVAL;
    try {
        dd_status st = select_device(ctx);
        if (st != DD_OK) return st;
        HostMesh h;
        std::string err;
        st = build_host_mesh(xy, n_v, tri, n_t, loop_idx, loop_off, n_loops, h, err);
        if (st != DD_OK) return set_err(ctx, st, err);
        MeshSlot slot;
        DevMesh &m = slot.dev;
        m.n_v = h.n_v;
        m.n_t = h.n_t;
        m.k = h.k;
        m.m = h.m;
        m.k_pad = (h.k + 3) / 4 * 4;
        std::vector<float2> xyf(h.n_v);
        for (int64_t v = 0; v < h.n_v; ++v) xyf[v] = make_float2((float)h.xy[2 * v], (float)h.xy[2 * v + 1]);
        std::vector<int4> tri4(h.n_t), nbr4(h.n_t);
        for (int64_t t = 0; t < h.n_t; ++t) {
            tri4[t] = make_int4(h.tri[3 * t], h.tri[3 * t + 1], h.tri[3 * t + 2], 0);
            nbr4[t] = make_int4(h.tnbr[3 * t], h.tnbr[3 * t + 1], h.tnbr[3 * t + 2], 0);
        }
        std::vector<float4> g4(2 * h.n_t);
        std::vector<int4> rec(4 * h.n_t);
        auto fbits = [](float x) {
            int i;
            std::memcpy(&i, &x, sizeof i);
            return i;
        };
        for (int64_t t = 0; t < h.n_t; ++t) {
            const float *g = &h.gphi[6 * t];
            g4[2 * t] = make_float4(g[0], g[1], g[2], g[3]);
            g4[2 * t + 1] = make_float4(g[4], g[5], 0.f, 0.f);
            const int32_t *v = &h.tri[3 * t], *nb = &h.tnbr[3 * t];
            const float2 p0 = xyf[v[0]], p1 = xyf[v[1]], p2 = xyf[v[2]];
            // squared norms of the three hat gradients (the third is minus the sum of the others)
            const double q0 = (double)g[0] * g[0] + (double)g[1] * g[1];
            const double q1 = (double)g[2] * g[2] + (double)g[3] * g[3];
            const double q2 = (double)g[4] * g[4] + (double)g[5] * g[5];
            rec[4 * t] = make_int4(v[0], v[1], v[2], nb[0]);
            rec[4 * t + 1] = make_int4(nb[1], nb[2], fbits((float)q0), fbits((float)q1));
            rec[4 * t + 2] = make_int4(fbits((float)q2), 0, fbits(p0.x), fbits(p0.y));
            rec[4 * t + 3] = make_int4(fbits(p1.x), fbits(p1.y), fbits(p2.x), fbits(p2.y));
        }
        auto undo = [&](dd_status s2) {
            free_mesh(m);
            return s2;
        };
        if ((st = dev_copy(ctx, m, &m.xy, xyf.data(), xyf.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.tri, tri4.data(), tri4.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.tnbr, nbr4.data(), nbr4.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.gphi, g4.data(), g4.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.trec, rec.data(), rec.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.vt_off, h.vt_off.data(), h.vt_off.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.vt, h.vt.data(), h.vt.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.vn_off, h.vn_off.data(), h.vn_off.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.vn, h.vn.data(), h.vn.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.interior, h.I.data(), h.I.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.boundary, h.B.data(), h.B.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.a_off, h.a_off.data(), h.a_off.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.a_col, h.a_col.data(), h.a_col.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.a_val, h.a_val.data(), h.a_val.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.a_diag, h.a_diag.data(), h.a_diag.size())) != DD_OK) return undo(st);
        m.n_rb = (int64_t)h.rb_row.size();
        if ((st = dev_copy(ctx, m, &m.rb_row, h.rb_row.data(), h.rb_row.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.rb_col, h.rb_col.data(), h.rb_col.size())) != DD_OK) return undo(st);
        if ((st = dev_copy(ctx, m, &m.rb_val, h.rb_val.data(), h.rb_val.size())) != DD_OK) return undo(st);
        m.is_boundary.assign(h.n_v, 0);
        for (int32_t v : h.B) m.is_boundary[v] = 1;
        m.xy_h.assign(h.xy.begin(), h.xy.end());
        if ((st = dev_copy(ctx, m, &m.isb, m.is_boundary.data(), m.is_boundary.size())) != DD_OK) return undo(st);
        slot.live = true;
        ctx->meshes.push_back(slot);
        *mesh_id = (int32_t)ctx->meshes.size() - 1;
        return DD_OK;
    } catch (const std::bad_alloc &) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    } catch (...) {
        return set_err(ctx, DD_EINVAL, "unexpected failure in dd_load_mesh");
    }
}

dd_status dd_unload_mesh(dd_ctx *ctx, int32_t mesh) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    select_device(ctx);
    cudaStreamSynchronize(ctx->stream);
    free_mesh(*m);
    ctx->meshes[mesh].live = false;
    return DD_OK;
}

dd_status dd_mesh_info(dd_ctx *ctx, int32_t mesh, int64_t *info) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    if (!info) return set_err(ctx, DD_EINVAL, "info is null");
    info[0] = m->n_v;
    info[1] = m->n_t;
    info[2] = m->k;
    info[3] = m->m;
    info[4] = m->k_pad;
    info[5] = m->has_P ? 1 : 0;
    info[6] = m->bytes;
    return DD_OK;
}

dd_status dd_poisson_kernel(dd_ctx *ctx, int32_t mesh, double rtol, int32_t max_iter, int32_t *iters,
                            double *resid) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    if (!(rtol > 0.0) || max_iter < 1) return set_err(ctx, DD_EINVAL, "rtol must be > 0 and max_iter >= 1");
    try {
        if ((st = select_device(ctx)) != DD_OK) return st;
        drop_derived(*m);
        std::string err;
        st = run_pcg(*m, rtol, max_iter, ctx->stream, iters, resid, err);
        if (st != DD_OK) set_err(ctx, st, err);
        return st;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_set_poisson_kernel(dd_ctx *ctx, int32_t mesh, const double *P) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    if (!P || pointer_space(ctx, P) != 0) return set_err(ctx, DD_EINVAL, "P must be a host pointer");
    if ((st = select_device(ctx)) != DD_OK) return st;
    drop_derived(*m);
    std::string err;
    st = store_poisson(*m, P, ctx->stream, err);
    if (st != DD_OK) set_err(ctx, st, err);
    return st;
}

dd_status dd_get_poisson_kernel(dd_ctx *ctx, int32_t mesh, float *out) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    if (!m->has_P) return set_err(ctx, DD_ESTATE, "no Poisson kernel stored");
    if (!out) return set_err(ctx, DD_EINVAL, "out is null");
    int sp = pointer_space(ctx, out);
    if (sp < 0) return set_err(ctx, DD_EINVAL, "out is on another device");
    if ((st = select_device(ctx)) != DD_OK) return st;
    CK(cudaMemcpy2DAsync(out, (size_t)m->k * sizeof(float), m->P, (size_t)m->k_pad * sizeof(float),
                         (size_t)m->k * sizeof(float), (size_t)m->n_v, cudaMemcpyDefault, ctx->stream),
       "copy P");
    if (sp == 0) CK(cudaStreamSynchronize(ctx->stream), "copy P");
    return DD_OK;
}

dd_status dd_log_poisson_kernel(dd_ctx *ctx, int32_t mesh, double tol, int32_t max_sweeps, int32_t *sweeps,
                                double *change) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    if (!m->has_P) return set_err(ctx, DD_ESTATE, "dd_log_poisson_kernel before dd_poisson_kernel");
    if (!(tol > 0.0) || max_sweeps < 1) return set_err(ctx, DD_EINVAL, "tol must be > 0 and max_sweeps >= 1");
    try {
        if ((st = select_device(ctx)) != DD_OK) return st;
        // the refined P changes what was derived from the old one
        release(*m, m->p_hi, m->n_v * m->kb * 2);
        release(*m, m->p_lo, m->n_v * m->kb * 2);
        release(*m, m->ex, m->n_v * (int64_t)sizeof(float));
        drop_tiled(*m);
        m->kb = 0;
        drop_sparse(*m);
        std::string err;
        st = refine_log_poisson(*m, tol, max_sweeps, ctx->stream, sweeps, change, err);
        if (st != DD_OK) set_err(ctx, st, err);
        return st;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_get_log_poisson_kernel(dd_ctx *ctx, int32_t mesh, float *out) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    if (!m->LP) return set_err(ctx, DD_ESTATE, "no log P stored (dd_log_poisson_kernel)");
    if (!out) return set_err(ctx, DD_EINVAL, "out is null");
    int sp = pointer_space(ctx, out);
    if (sp < 0) return set_err(ctx, DD_EINVAL, "out is on another device");
    if ((st = select_device(ctx)) != DD_OK) return st;
    CK(cudaMemcpy2DAsync(out, (size_t)m->k * sizeof(float), m->LP, (size_t)m->k_pad * sizeof(float),
                         (size_t)m->k * sizeof(float), (size_t)m->n_v, cudaMemcpyDefault, ctx->stream),
       "copy log P");
    if (sp == 0) CK(cudaStreamSynchronize(ctx->stream), "copy log P");
    return DD_OK;
}

dd_status dd_sparsify(dd_ctx *ctx, int32_t mesh, double theta, int64_t *kept, int64_t *bytes) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    if (!m->has_P) return set_err(ctx, DD_ESTATE, "dd_sparsify before dd_poisson_kernel");
    if (!(theta < 1.0)) return set_err(ctx, DD_EINVAL, "theta must be < 1 (negative: 1/sqrt(n))");
    try {
        if ((st = select_device(ctx)) != DD_OK) return st;
        if (theta < 0.0) theta = 1.0 / std::sqrt((double)m->n_v);
        drop_sparse(*m);
        std::string err;
        if ((st = build_sparse_rows(*m, theta, ctx->stream, kept, bytes, err)) != DD_OK) return set_err(ctx, st, err);
        return DD_OK;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_distance(dd_ctx *ctx, int32_t mesh, const int32_t *targets, int32_t T, uint32_t f_mask, int32_t prec,
                      float *out) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    try {
        if (!m->has_P) return set_err(ctx, DD_ESTATE, "dd_distance before dd_poisson_kernel");
        if (T < 1) return set_err(ctx, DD_EINVAL, "T must be >= 1");
        if (f_mask == 0 || (f_mask & ~(uint32_t)(DD_F_KL | DD_F_TV | DD_F_KLT)))
            return set_err(ctx, DD_EINVAL, "f_mask must be a non-empty combination of DD_F_KL, DD_F_TV, DD_F_KLT");
        if (prec != DD_PREC_FP32 && prec != DD_PREC_BF16X3 && prec != DD_PREC_SPARSE &&
            prec != DD_PREC_SPARSE_MERGED)
            return set_err(ctx, DD_EINVAL, "unsupported precision");
        if (!out) return set_err(ctx, DD_EINVAL, "out is null");
        if ((st = check_targets(ctx, *m, targets, T, true, "targets")) != DD_OK) return st;
        const int sp = pointer_space(ctx, out);
        if (sp < 0) return set_err(ctx, DD_EINVAL, "out is on another device");
        if ((st = select_device(ctx)) != DD_OK) return st;
        if ((st = upload(ctx, S_TARGETS, targets, (size_t)T * sizeof(int32_t))) != DD_OK) return st;
        const size_t out_bytes = (size_t)popcount2(f_mask) * T * m->n_v * sizeof(float);
        float *dst = out;
        if (sp == 0) {
            if ((st = ensure_scratch(ctx, S_FIELDS, out_bytes)) != DD_OK) return st;
            dst = reinterpret_cast<float *>(ctx->scratch[S_FIELDS]);
        }
        st = fields_into(ctx, *m, reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]), T, f_mask, prec, dst);
        if (st != DD_OK) return st;
        if (sp == 0) {
            CK(cudaMemcpyAsync(out, dst, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy fields to host");
            CK(cudaStreamSynchronize(ctx->stream), "fields");
            return check_kernel_flag(ctx);
        }
        return DD_OK;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_trace_fields(dd_ctx *ctx, int32_t mesh, const float *fields, const int32_t *targets, int32_t T,
                          const int32_t *sources, int32_t S, int32_t max_pts, float *out_xy, int32_t *out_len,
                          int32_t *out_status);

dd_status dd_divergence(dd_ctx *ctx, int32_t mesh, const int32_t *targets, int32_t T, int32_t family,
                        double param, float *out) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    try {
        if (!m->has_P) return set_err(ctx, DD_ESTATE, "dd_divergence before dd_poisson_kernel");
        if (T < 1) return set_err(ctx, DD_EINVAL, "T must be >= 1");
        if (family < DD_DIV_CHI2 || family > DD_DIV_KL_REVERSE) return set_err(ctx, DD_EINVAL, "unknown family");
        if (family == DD_DIV_POWER && !(param >= 1.0)) return set_err(ctx, DD_EINVAL, "power family needs p >= 1");
        if (family == DD_DIV_ALPHA && !(std::fabs(std::fabs(param) - 1.0) > 1e-6))
            return set_err(ctx, DD_EINVAL, "alpha family needs |a| != 1");
        if (!out) return set_err(ctx, DD_EINVAL, "out is null");
        if ((st = check_targets(ctx, *m, targets, T, true, "targets")) != DD_OK) return st;
        const int sp = pointer_space(ctx, out);
        if (sp < 0) return set_err(ctx, DD_EINVAL, "out is on another device");
        if ((st = select_device(ctx)) != DD_OK) return st;
        if ((st = upload(ctx, S_TARGETS, targets, (size_t)T * sizeof(int32_t))) != DD_OK) return st;
        const size_t out_bytes = (size_t)T * m->n_v * sizeof(float);
        float *dst = out;
        if (sp == 0) {
            if ((st = ensure_scratch(ctx, S_FIELDS, out_bytes)) != DD_OK) return st;
            dst = reinterpret_cast<float *>(ctx->scratch[S_FIELDS]);
        }
        if ((st = ensure_scratch(ctx, S_STAGE, 4 * (size_t)T * m->k_pad * sizeof(float))) != DD_OK) return st;
        float4 *stage = reinterpret_cast<float4 *>(ctx->scratch[S_STAGE]);
        launch_stage_targets(m->P, m->n_v, m->k_pad, reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]), T,
                             stage, ctx->stream, nullptr, m->LP);
        std::string err;
        if ((st = launch_fdiv(m->P, m->n_v, m->k_pad, stage, T, family, param, dst, ctx->stream, err, m->LP)) !=
            DD_OK)
            return set_err(ctx, st, err);
        CK(cudaGetLastError(), "divergence kernel launch");
        if (sp == 0) {
            CK(cudaMemcpyAsync(out, dst, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy fields to host");
            CK(cudaStreamSynchronize(ctx->stream), "divergence fields");
        }
        return DD_OK;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

namespace {

// paths of T x S (target, source) pairs on device fields [T][n_v]; ids already checked
dd_status trace_into(dd_ctx *ctx, DevMesh &m, const float *d_fields, const int32_t *targets, int32_t T,
                     const int32_t *sources, int32_t S, int32_t max_pts, float *out_xy, int32_t *out_len,
                     int32_t *out_status, bool targets_uploaded, bool edges = false) {
    dd_status st;
    if (!targets_uploaded && (st = upload(ctx, S_TARGETS, targets, (size_t)T * sizeof(int32_t))) != DD_OK) return st;
    if ((st = upload(ctx, S_SOURCES, sources, (size_t)T * S * sizeof(int32_t))) != DD_OK) return st;
    const int sx = pointer_space(ctx, out_xy), sl = pointer_space(ctx, out_len), ss = pointer_space(ctx, out_status);
    if (sx < 0 || sl < 0 || ss < 0) return set_err(ctx, DD_EINVAL, "path outputs on another device");
    const size_t n = (size_t)T * S;
    float2 *dxy = reinterpret_cast<float2 *>(out_xy);
    int32_t *dlen = out_len, *dst = out_status;
    // Host outputs.  Pinned (page-locked) memory has a device address: the
    // walk writes lengths and statuses there itself, and one copy kernel
    // moves each path's defined prefix from device scratch into it with
    // coalesced 16-byte stores (over NVLink-C2C on Grace; measured 0.99 ms
    // per grid140 step against 1.26 ms for the copy-engine path below, while
    // the walk storing points straight into host memory took 1.93 ms).
    // Pageable memory goes through device scratch and the copy engine.
    float2 *xy_alias = nullptr;
    if (sx == 0) {
        xy_alias = reinterpret_cast<float2 *>(mapped_alias(out_xy));
        if ((st = ensure_scratch(ctx, S_XY, n * max_pts * sizeof(float2))) != DD_OK) return st;
        dxy = reinterpret_cast<float2 *>(ctx->scratch[S_XY]);
    }
    const bool xy_copy = sx == 0 && !xy_alias;
    bool len_direct = false, st_direct = false;
    if (sl == 0) {
        if (void *a = mapped_alias(out_len)) {
            dlen = reinterpret_cast<int32_t *>(a);
            len_direct = true;
        } else {
            if ((st = ensure_scratch(ctx, S_LEN, n * sizeof(int32_t))) != DD_OK) return st;
            dlen = reinterpret_cast<int32_t *>(ctx->scratch[S_LEN]);
        }
    }
    if (ss == 0) {
        if (void *a = mapped_alias(out_status)) {
            dst = reinterpret_cast<int32_t *>(a);
            st_direct = true;
        } else {
            if ((st = ensure_scratch(ctx, S_STATUS, n * sizeof(int32_t))) != DD_OK) return st;
            dst = reinterpret_cast<int32_t *>(ctx->scratch[S_STATUS]);
        }
    }
    if (edges) {
        launch_edge_paths(m, d_fields, reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]),
                          reinterpret_cast<const int32_t *>(ctx->scratch[S_SOURCES]), T, S, max_pts, dxy, dlen, dst,
                          ctx->stream);
    } else {
        // rates and vertex decisions of every field are stored only where many paths share a field
        const bool dense = trace_dense_decisions(S);
        if ((st = ensure_scratch(ctx, S_GRAD, dense ? trace_scratch_bytes(m, T, true) : 256)) != DD_OK) return st;
        launch_trace(m, d_fields, m.n_v, reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]),
                     reinterpret_cast<const int32_t *>(ctx->scratch[S_SOURCES]), T, S, max_pts, dxy, dlen, dst,
                     ctx->scratch[S_GRAD], ctx->stream);
    }
    CK(cudaGetLastError(), "trace kernel launch");
    if (xy_alias) {
        launch_copy_paths(dxy, dlen, (int64_t)n, max_pts, xy_alias, ctx->stream);
        CK(cudaGetLastError(), "path copy kernel launch");
    }
    bool host = xy_alias || len_direct || st_direct;
    if (xy_copy) {
        // Only each path's prefix of len points is defined: copy, per chunk of
        // paths, the rows up to the chunk's longest path (one strided copy
        // each) instead of all max_pts points of every path.
        std::vector<int32_t> lens(n);
        int32_t *hl = (sl == 0 && !len_direct) ? out_len : lens.data();
        CK(cudaMemcpyAsync(hl, dlen, n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream), "copy lengths");
        CK(cudaStreamSynchronize(ctx->stream), "path lengths");
        const size_t chunk = 512, pitch = (size_t)max_pts * sizeof(float2);
        for (size_t s0 = 0; s0 < n; s0 += chunk) {
            const size_t s1 = std::min(n, s0 + chunk);
            int32_t L = 0;
            for (size_t i = s0; i < s1; ++i) L = std::max(L, std::min(std::max(hl[i], 0), max_pts));
            if (L == 0) continue;
            CK(cudaMemcpy2DAsync(reinterpret_cast<char *>(out_xy) + s0 * pitch, pitch,
                                 reinterpret_cast<const char *>(dxy) + s0 * pitch, pitch, (size_t)L * sizeof(float2),
                                 s1 - s0, cudaMemcpyDeviceToHost, ctx->stream),
               "copy paths");
        }
        host = true;
    } else if (sl == 0 && !len_direct) {
        CK(cudaMemcpyAsync(out_len, dlen, n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream), "copy lengths");
        host = true;
    }
    if (ss == 0 && !st_direct) {
        CK(cudaMemcpyAsync(out_status, dst, n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
           "copy statuses");
        host = true;
    }
    if (host) {
        CK(cudaStreamSynchronize(ctx->stream), "paths");
        return check_kernel_flag(ctx);
    }
    return DD_OK;
}

dd_status check_path_args(dd_ctx *ctx, int32_t S, int32_t max_pts, const void *a, const void *b, const void *c) {
    if (S < 1) return set_err(ctx, DD_EINVAL, "S must be >= 1");
    if (max_pts < 2) return set_err(ctx, DD_EINVAL, "max_pts must be >= 2");
    if (!a || !b || !c) return set_err(ctx, DD_EINVAL, "null path output");
    return DD_OK;
}

}  // namespace

dd_status dd_trace_fields(dd_ctx *ctx, int32_t mesh, const float *fields, const int32_t *targets, int32_t T,
                          const int32_t *sources, int32_t S, int32_t max_pts, float *out_xy, int32_t *out_len,
                          int32_t *out_status) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    try {
        if (T < 1) return set_err(ctx, DD_EINVAL, "T must be >= 1");
        if ((st = check_path_args(ctx, S, max_pts, out_xy, out_len, out_status)) != DD_OK) return st;
        if (!fields || pointer_space(ctx, fields) != 1)
            return set_err(ctx, DD_EINVAL, "fields must be device memory of the context's device");
        if ((st = check_targets(ctx, *m, targets, T, false, "targets")) != DD_OK) return st;
        if ((st = check_targets(ctx, *m, sources, (int64_t)T * S, false, "sources")) != DD_OK) return st;
        if ((st = select_device(ctx)) != DD_OK) return st;
        return trace_into(ctx, *m, fields, targets, T, sources, S, max_pts, out_xy, out_len, out_status, false);
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_trace_edges(dd_ctx *ctx, int32_t mesh, const float *fields, const int32_t *targets, int32_t T,
                         const int32_t *sources, int32_t S, int32_t max_pts, float *out_xy, int32_t *out_len,
                         int32_t *out_status) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    try {
        if (T < 1) return set_err(ctx, DD_EINVAL, "T must be >= 1");
        if ((st = check_path_args(ctx, S, max_pts, out_xy, out_len, out_status)) != DD_OK) return st;
        if (!fields || pointer_space(ctx, fields) != 1)
            return set_err(ctx, DD_EINVAL, "fields must be device memory of the context's device");
        if ((st = check_targets(ctx, *m, targets, T, false, "targets")) != DD_OK) return st;
        if ((st = check_targets(ctx, *m, sources, (int64_t)T * S, false, "sources")) != DD_OK) return st;
        if ((st = select_device(ctx)) != DD_OK) return st;
        return trace_into(ctx, *m, fields, targets, T, sources, S, max_pts, out_xy, out_len, out_status, false, true);
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_local_minima(dd_ctx *ctx, int32_t mesh, const float *fields, const int32_t *targets, int32_t T,
                          int32_t *counts, uint8_t *flags) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    try {
        if (T < 1) return set_err(ctx, DD_EINVAL, "T must be >= 1");
        if (!counts) return set_err(ctx, DD_EINVAL, "counts is null");
        if (!fields || pointer_space(ctx, fields) != 1)
            return set_err(ctx, DD_EINVAL, "fields must be device memory of the context's device");
        const int sf = flags ? pointer_space(ctx, flags) : 1;
        if (sf < 0) return set_err(ctx, DD_EINVAL, "flags on another device");
        if ((st = check_targets(ctx, *m, targets, T, false, "targets")) != DD_OK) return st;
        if ((st = select_device(ctx)) != DD_OK) return st;
        if ((st = upload(ctx, S_TARGETS, targets, (size_t)T * sizeof(int32_t))) != DD_OK) return st;
        // counts and (for host flags) the flags in one scratch block
        const size_t cbytes = ((size_t)T * sizeof(int32_t) + 255) / 256 * 256;
        const size_t fbytes = (flags && sf == 0) ? (size_t)T * m->n_v : 0;
        if ((st = ensure_scratch(ctx, S_LEN, cbytes + fbytes)) != DD_OK) return st;
        int32_t *dcounts = reinterpret_cast<int32_t *>(ctx->scratch[S_LEN]);
        uint8_t *dflags = flags && sf == 0 ? reinterpret_cast<uint8_t *>(ctx->scratch[S_LEN]) + cbytes : flags;
        CK(cudaMemsetAsync(dcounts, 0, (size_t)T * sizeof(int32_t), ctx->stream), "clear counts");
        launch_local_minima(*m, fields, reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]), T, dcounts, dflags,
                            ctx->stream);
        CK(cudaGetLastError(), "census kernel launch");
        CK(cudaMemcpyAsync(counts, dcounts, (size_t)T * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
           "copy counts");
        if (fbytes)
            CK(cudaMemcpyAsync(flags, dflags, fbytes, cudaMemcpyDeviceToHost, ctx->stream), "copy flags");
        CK(cudaStreamSynchronize(ctx->stream), "census");
        return DD_OK;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_trace(dd_ctx *ctx, int32_t mesh, int32_t target, uint32_t f, const int32_t *sources, int32_t S,
                   int32_t max_pts, float *out_xy, int32_t *out_len, int32_t *out_status) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    try {
        if (!m->has_P) return set_err(ctx, DD_ESTATE, "dd_trace before dd_poisson_kernel");
        if (f != DD_F_KL && f != DD_F_TV) return set_err(ctx, DD_EINVAL, "f must be DD_F_KL or DD_F_TV");
        if ((st = check_path_args(ctx, S, max_pts, out_xy, out_len, out_status)) != DD_OK) return st;
        if ((st = check_targets(ctx, *m, &target, 1, true, "target")) != DD_OK) return st;
        if ((st = check_targets(ctx, *m, sources, S, false, "sources")) != DD_OK) return st;
        if ((st = select_device(ctx)) != DD_OK) return st;
        if ((st = upload(ctx, S_TARGETS, &target, sizeof(int32_t))) != DD_OK) return st;
        if ((st = ensure_scratch(ctx, S_FIELDS, (size_t)m->n_v * sizeof(float))) != DD_OK) return st;
        float *field = reinterpret_cast<float *>(ctx->scratch[S_FIELDS]);
        st = fields_into(ctx, *m, reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]), 1, f, DD_PREC_FP32,
                         field);
        if (st != DD_OK) return st;
        return trace_into(ctx, *m, field, &target, 1, sources, S, max_pts, out_xy, out_len, out_status, true);
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

dd_status dd_query(dd_ctx *ctx, int32_t mesh, const int32_t *targets, int32_t T, const int32_t *sources, int32_t S,
                   uint32_t f_mask, int32_t prec, uint32_t trace_f, int32_t max_pts, float *out_fields,
                   float *out_xy, int32_t *out_len, int32_t *out_status) {
    DevMesh *m = nullptr;
    dd_status st = get_mesh(ctx, mesh, &m);
    if (st != DD_OK) return st;
    try {
        if (!m->has_P) return set_err(ctx, DD_ESTATE, "dd_query before dd_poisson_kernel");
        if (T < 1) return set_err(ctx, DD_EINVAL, "T must be >= 1");
        if (f_mask == 0 || (f_mask & ~(uint32_t)(DD_F_KL | DD_F_TV | DD_F_KLT)))
            return set_err(ctx, DD_EINVAL, "bad f_mask");
        if ((trace_f != DD_F_KL && trace_f != DD_F_TV && trace_f != DD_F_KLT) || !(f_mask & trace_f))
            return set_err(ctx, DD_EINVAL, "trace_f must be one bit of f_mask");
        if (prec != DD_PREC_FP32 && prec != DD_PREC_BF16X3 && prec != DD_PREC_SPARSE &&
            prec != DD_PREC_SPARSE_MERGED)
            return set_err(ctx, DD_EINVAL, "unsupported precision");
        if (!out_fields) return set_err(ctx, DD_EINVAL, "out_fields is null");
        if ((st = check_path_args(ctx, S, max_pts, out_xy, out_len, out_status)) != DD_OK) return st;
        if ((st = check_targets(ctx, *m, targets, T, true, "targets")) != DD_OK) return st;
        if ((st = check_targets(ctx, *m, sources, (int64_t)T * S, false, "sources")) != DD_OK) return st;
        const int sf = pointer_space(ctx, out_fields);
        if (sf < 0) return set_err(ctx, DD_EINVAL, "out_fields is on another device");
        if ((st = select_device(ctx)) != DD_OK) return st;
        if ((st = upload(ctx, S_TARGETS, targets, (size_t)T * sizeof(int32_t))) != DD_OK) return st;
        const size_t out_bytes = (size_t)popcount2(f_mask) * T * m->n_v * sizeof(float);
        float *dst = out_fields;
        if (sf == 0) {
            if ((st = ensure_scratch(ctx, S_FIELDS, out_bytes)) != DD_OK) return st;
            dst = reinterpret_cast<float *>(ctx->scratch[S_FIELDS]);
        }
        const int64_t stride = (int64_t)T * m->n_v;
        const int32_t *d_targets = reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]);
        if (sf == 0) {
            // Host fields: computed in up to four parts of the targets (at
            // least 128 each), each part's rows going back on a side stream
            // while the next is computed, the last one's while the paths are
            // traced; FP32 many-target path only, one part otherwise.  Each
            // part adds its own last partial wave of the tile pass and its own
            // recompute launch, while fewer parts leave more of the copy
            // exposed.  (grid450, 1,024 targets, end to end on one box, two
            // runs each: two parts 20.1k / 18.8k fields/s, four 19.3k / 19.4k,
            // eight 19.5k / 19.3k)
            if ((st = ensure_side(ctx)) != DD_OK) return st;
            const int nf = popcount2(f_mask);
            const int32_t nch = (prec == DD_PREC_FP32 && T >= 256) ? std::min<int32_t>(4, T / 128) : 1;
            const int32_t per = (T + nch - 1) / nch;
            // (TV is final once the tile pass has ended: its copy starts then,
            // while the exact KL recompute runs)
            const int tv_slot = (f_mask & DD_F_TV) ? ((f_mask & DD_F_KL) ? 1 : 0) : -1;
            const bool early_tv = prec == DD_PREC_FP32 && tv_slot >= 0;
            for (int32_t a0 = 0; a0 < T; a0 += per) {
                const int32_t Tc = std::min(per, T - a0);
                st = fields_into(ctx, *m, d_targets + a0, Tc, f_mask, prec, dst + (int64_t)a0 * m->n_v, stride,
                                 early_tv ? ctx->side_ev[2] : nullptr);
                if (st != DD_OK) return st;
                auto copy = [&](int f) {
                    const int64_t o = f * stride + (int64_t)a0 * m->n_v;
                    return cudaMemcpyAsync(out_fields + o, dst + o, (size_t)Tc * m->n_v * sizeof(float),
                                           cudaMemcpyDeviceToHost, ctx->side);
                };
                if (early_tv) {
                    CK(cudaStreamWaitEvent(ctx->side, ctx->side_ev[2], 0), "side wait");
                    CK(copy(tv_slot), "copy fields");
                }
                CK(cudaEventRecord(ctx->side_ev[0], ctx->stream), "fields ready");
                CK(cudaStreamWaitEvent(ctx->side, ctx->side_ev[0], 0), "side wait");
                for (int f = 0; f < nf; ++f)
                    if (!early_tv || f != tv_slot) CK(copy(f), "copy fields");
            }
            CK(cudaEventRecord(ctx->side_ev[1], ctx->side), "fields copied");
        } else {
            st = fields_into(ctx, *m, d_targets, T, f_mask, prec, dst);
            if (st != DD_OK) return st;
        }
        const float *trace_field = field_slot(dst, f_mask, trace_f, stride);
        st = trace_into(ctx, *m, trace_field, targets, T, sources, S, max_pts, out_xy, out_len, out_status, true);
        if (sf == 0) {
            // the next call may reuse the field scratch: the copy must be done
            CK(cudaEventSynchronize(ctx->side_ev[1]), "query fields");
            if (st != DD_OK) return st;
            CK(cudaStreamSynchronize(ctx->stream), "query");
            return check_kernel_flag(ctx);
        }
        return st;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}


namespace {
size_t align256(size_t x) { return (x + 255) / 256 * 256; }
}  // namespace

dd_status dd_query_batch(dd_ctx *ctx, int32_t n_items, const int32_t *mesh_ids, const int32_t *T_per,
                         const int32_t *targets, const int32_t *sources, int32_t S, uint32_t f_mask, uint32_t trace_f,
                         int32_t max_pts, float *out_fields, float *out_xy, int32_t *out_len, int32_t *out_status) {
    if (!ctx) return DD_EINVAL;
    try {
        if (n_items < 1 || !mesh_ids || !T_per) return set_err(ctx, DD_EINVAL, "need at least one item");
        if (f_mask == 0 || (f_mask & ~(uint32_t)(DD_F_KL | DD_F_TV))) return set_err(ctx, DD_EINVAL, "bad f_mask");
        if (S < 0) return set_err(ctx, DD_EINVAL, "S must be >= 0");
        if (S > 0) {
            if ((trace_f != DD_F_KL && trace_f != DD_F_TV) || !(f_mask & trace_f))
                return set_err(ctx, DD_EINVAL, "trace_f must be one bit of f_mask");
            dd_status st = check_path_args(ctx, S, max_pts, out_xy, out_len, out_status);
            if (st != DD_OK) return st;
        }
        if (!out_fields) return set_err(ctx, DD_EINVAL, "out_fields is null");
        const int nf = popcount2(f_mask);
        std::vector<DevMesh *> ms(n_items);
        std::vector<int64_t> foff(n_items + 1, 0), toff(n_items + 1, 0);
        int64_t stage_floats = 0, grad_bytes = 0, max_nt = 0, max_nv = 0, max_k = 0;
        for (int i = 0; i < n_items; ++i) {
            dd_status st = get_mesh(ctx, mesh_ids[i], &ms[i]);
            if (st != DD_OK) return st;
            if (!ms[i]->has_P) return set_err(ctx, DD_ESTATE, "item " + std::to_string(i) + " has no Poisson kernel");
            if (T_per[i] < 1) return set_err(ctx, DD_EINVAL, "every item needs T >= 1");
            toff[i + 1] = toff[i] + T_per[i];
            foff[i + 1] = foff[i] + (int64_t)nf * T_per[i] * ms[i]->n_v;
            stage_floats += 3LL * T_per[i] * ms[i]->k_pad;
            grad_bytes += (int64_t)trace_scratch_bytes(*ms[i], T_per[i], false);
            max_nt = std::max(max_nt, ms[i]->n_t);
            max_nv = std::max(max_nv, ms[i]->n_v);
            max_k = std::max(max_k, ms[i]->k_pad);
        }
        const int32_t nT = (int32_t)toff[n_items];
        if (!targets || pointer_space(ctx, targets) != 0) return set_err(ctx, DD_EINVAL, "targets must be host memory");
        for (int i = 0; i < n_items; ++i) {
            dd_status st = check_targets(ctx, *ms[i], targets + toff[i], T_per[i], true, "targets");
            if (st != DD_OK) return st;
            if (S > 0 && (st = check_targets(ctx, *ms[i], sources + toff[i] * S, (int64_t)T_per[i] * S, false,
                                             "sources")) != DD_OK)
                return st;
        }
        const int sf = pointer_space(ctx, out_fields);
        if (sf < 0) return set_err(ctx, DD_EINVAL, "out_fields is on another device");
        dd_status st = select_device(ctx);
        if (st != DD_OK) return st;

        // metadata block: tprob, tloc, problems, items, trace domains, counter
        std::vector<int32_t> tprob(nT), tloc(nT);
        for (int i = 0; i < n_items; ++i)
            for (int a = 0; a < T_per[i]; ++a) {
                tprob[toff[i] + a] = i;
                tloc[toff[i] + a] = a;
            }
        if ((st = upload(ctx, S_TARGETS, targets, (size_t)nT * sizeof(int32_t))) != DD_OK) return st;
        if (S > 0 && (st = upload(ctx, S_SOURCES, sources, (size_t)nT * S * sizeof(int32_t))) != DD_OK) return st;
        const size_t out_bytes = (size_t)foff[n_items] * sizeof(float);
        float *dfields = out_fields;
        if (sf == 0) {
            if ((st = ensure_scratch(ctx, S_FIELDS, out_bytes)) != DD_OK) return st;
            dfields = reinterpret_cast<float *>(ctx->scratch[S_FIELDS]);
        }
        if ((st = ensure_scratch(ctx, S_STAGE, (size_t)stage_floats * sizeof(float))) != DD_OK) return st;
        if (S > 0 && (st = ensure_scratch(ctx, S_GRAD, (size_t)grad_bytes)) != DD_OK) return st;
        float *stage = reinterpret_cast<float *>(ctx->scratch[S_STAGE]);
        char *grads = reinterpret_cast<char *>(ctx->scratch[S_GRAD]);

        std::vector<BatchProblem> probs(n_items);
        int64_t so = 0;
        for (int i = 0; i < n_items; ++i) {
            BatchProblem &q = probs[i];
            const DevMesh &m = *ms[i];
            const int64_t blk = (int64_t)T_per[i] * m.k_pad;
            q.P = m.P;
            q.n_v = m.n_v;
            q.k_pad = m.k_pad;
            q.sP = stage + so;
            q.sL = stage + so + blk;
            q.sE = stage + so + 2 * blk;
            so += 3 * blk;
            q.T = T_per[i];
            q.variant = 0;
            float *base = dfields + foff[i];
            q.out_kl = (f_mask & DD_F_KL) ? base : nullptr;
            q.out_tv = (f_mask & DD_F_TV) ? base + ((f_mask & DD_F_KL) ? (int64_t)T_per[i] * m.n_v : 0) : nullptr;
        }
        const size_t o_tprob = 0, o_tloc = align256(nT * sizeof(int32_t));
        const size_t o_probs = o_tloc + align256(nT * sizeof(int32_t));
        const size_t o_doms = o_probs + align256(n_items * sizeof(BatchProblem));
        const size_t dom_bytes = batch_trace_dom_bytes();
        const size_t o_counter = o_doms + align256(n_items * dom_bytes);
        const size_t o_items = o_counter + 256;
        // stage all targets first (the autotuner times shapes on the staged data)
        std::vector<uint8_t> meta(o_items);
        std::memcpy(meta.data() + o_tprob, tprob.data(), nT * sizeof(int32_t));
        std::memcpy(meta.data() + o_tloc, tloc.data(), nT * sizeof(int32_t));
        std::memcpy(meta.data() + o_probs, probs.data(), n_items * sizeof(BatchProblem));
        if ((st = upload(ctx, S_META, meta.data(), meta.size())) != DD_OK) return st;
        uint8_t *dmeta = reinterpret_cast<uint8_t *>(ctx->scratch[S_META]);
        launch_batch_stage(reinterpret_cast<const BatchProblem *>(dmeta + o_probs),
                           reinterpret_cast<const int32_t *>(dmeta + o_tprob),
                           reinterpret_cast<const int32_t *>(dmeta + o_tloc),
                           reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]), nT, max_k, ctx->stream);
        CK(cudaGetLastError(), "batch staging launch");
        for (int i = 0; i < n_items; ++i)
            probs[i].variant = tile_variant_for(probs[i].P, probs[i].n_v, probs[i].k_pad, probs[i].sP, probs[i].sL,
                                                probs[i].sE, probs[i].T, probs[i].out_kl, probs[i].out_tv, ctx->stream);
        // items: every output tile, larger row extents first for balance
        std::vector<std::pair<int64_t, BatchItem>> order;
        for (int i = 0; i < n_items; ++i) {
            const int tr = tile_rows(probs[i].variant), tt = tile_targets(probs[i].variant);
            const int64_t cost = ms[i]->k_pad * tr * (int64_t)tt;
            for (int64_t xt = 0; xt * tr < ms[i]->n_v; ++xt)
                for (int at = 0; at * tt < T_per[i]; ++at) order.push_back({cost, BatchItem{i, (int32_t)xt, at, 0}});
        }
        std::stable_sort(order.begin(), order.end(),
                         [](const std::pair<int64_t, BatchItem> &x, const std::pair<int64_t, BatchItem> &y) {
                             return x.first > y.first;
                         });
        // the pipelined launch: every mesh's tiled copy of P (built once per
        // mesh; without room for it the batch stays staged), every problem's
        // targets in the tiled layout, items of 128 rows x 64 targets
        bool pipe_ok = true;
        int64_t tstage_bytes = 0, max_tiles = 0;
        for (int i = 0; i < n_items && pipe_ok; ++i) {
            std::string err;
            if (prepare_tiled(*ms[i], ctx->stream, err) != DD_OK) pipe_ok = false;
            tstage_bytes += (int64_t)tiled_target_bytes(ms[i]->k_pad, T_per[i]);
            max_tiles = std::max<int64_t>(max_tiles, (T_per[i] + 63) / 64 * (tiled_k32(ms[i]->k_pad) / 32));
        }
        if (pipe_ok && ensure_scratch(ctx, S_TSTAGE, (size_t)tstage_bytes) != DD_OK) {
            cudaGetLastError();
            pipe_ok = false;
        }
        std::vector<std::pair<int64_t, BatchItem>> order_pipe;
        if (pipe_ok) {
            float *ts = reinterpret_cast<float *>(ctx->scratch[S_TSTAGE]);
            for (int i = 0; i < n_items; ++i) {
                BatchProblem &q = probs[i];
                const DevMesh &m = *ms[i];
                const int64_t half = (int64_t)tiled_target_bytes(m.k_pad, T_per[i]) / (2 * sizeof(float));
                q.PT = m.pt_p;
                q.LT = m.pt_l;
                q.kt = m.pt_kt;
                q.TQ = ts;
                q.TL = ts + half;
                ts += 2 * half;
                for (int64_t xt = 0; xt * 128 < m.n_v; ++xt)
                    for (int at = 0; at * 64 < T_per[i]; ++at)
                        order_pipe.push_back({m.pt_kt, BatchItem{i, (int32_t)xt, at, 0}});
            }
            std::stable_sort(order_pipe.begin(), order_pipe.end(),
                             [](const std::pair<int64_t, BatchItem> &x, const std::pair<int64_t, BatchItem> &y) {
                                 return x.first > y.first;
                             });
        }
        const size_t o_items_pipe = o_items + align256(order.size() * sizeof(BatchItem));
        meta.resize(o_items_pipe + order_pipe.size() * sizeof(BatchItem));
        std::memcpy(meta.data() + o_probs, probs.data(), n_items * sizeof(BatchProblem));
        // trace domains; gradients per item in consecutive blocks [T_i][n_t_i]
        {
            int64_t go = 0;
            for (int i = 0; i < n_items; ++i) {
                fill_batch_trace_dom(meta.data() + o_doms + i * dom_bytes, *ms[i],
                                     (trace_f == DD_F_TV && probs[i].out_tv) ? probs[i].out_tv : probs[i].out_kl,
                                     T_per[i], grads ? grads + go : nullptr);
                go += (int64_t)trace_scratch_bytes(*ms[i], T_per[i], false);
            }
        }
        for (size_t j = 0; j < order.size(); ++j)
            std::memcpy(meta.data() + o_items + j * sizeof(BatchItem), &order[j].second, sizeof(BatchItem));
        for (size_t j = 0; j < order_pipe.size(); ++j)
            std::memcpy(meta.data() + o_items_pipe + j * sizeof(BatchItem), &order_pipe[j].second, sizeof(BatchItem));
        if ((st = upload(ctx, S_META, meta.data(), meta.size())) != DD_OK) return st;
        dmeta = reinterpret_cast<uint8_t *>(ctx->scratch[S_META]);
        int64_t fix_blocks = 0, work = 0;
        for (int i = 0; i < n_items; ++i) {
            if (probs[i].out_kl) fix_blocks += fix_row_blocks(probs[i].n_v);
            work += ms[i]->n_v * ms[i]->k_pad * (int64_t)T_per[i];
        }
        const BatchProblem *dprobs = reinterpret_cast<const BatchProblem *>(dmeta + o_probs);
        int32_t *dcounter = reinterpret_cast<int32_t *>(dmeta + o_counter);
        auto staged = [&]() {
            launch_batch_fields(dprobs, (int32_t)n_items, reinterpret_cast<const BatchItem *>(dmeta + o_items),
                                (int32_t)order.size(), dcounter, ctx->stream, fix_blocks);
        };
        auto pipelined = [&]() {
            launch_batch_fields_pipe(dprobs, (int32_t)n_items, reinterpret_cast<const BatchItem *>(dmeta + o_items_pipe),
                                     (int32_t)order_pipe.size(), dcounter, ctx->d_err, ctx->stream, fix_blocks,
                                     max_tiles, (f_mask & DD_F_KL) != 0, (f_mask & DD_F_TV) != 0);
        };
        if (pipe_ok && batch_launch_choice(n_items, work, f_mask, staged, pipelined, ctx->stream) == 1)
            pipelined();
        else
            staged();
        CK(cudaGetLastError(), "batch field launch");
        bool host = false;
        if (sf == 0) {
            CK(cudaMemcpyAsync(out_fields, dfields, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "copy fields");
            host = true;
        }
        if (S > 0) {
            const int sx = pointer_space(ctx, out_xy), sl = pointer_space(ctx, out_len),
                      ss = pointer_space(ctx, out_status);
            if (sx < 0 || sl < 0 || ss < 0) return set_err(ctx, DD_EINVAL, "path outputs on another device");
            const size_t n = (size_t)nT * S;
            float2 *dxy = reinterpret_cast<float2 *>(out_xy);
            int32_t *dlen = out_len, *dst = out_status;
            if (sx == 0) {
                if ((st = ensure_scratch(ctx, S_XY, n * max_pts * sizeof(float2))) != DD_OK) return st;
                dxy = reinterpret_cast<float2 *>(ctx->scratch[S_XY]);
            }
            if (sl == 0) {
                if ((st = ensure_scratch(ctx, S_LEN, n * sizeof(int32_t))) != DD_OK) return st;
                dlen = reinterpret_cast<int32_t *>(ctx->scratch[S_LEN]);
            }
            if (ss == 0) {
                if ((st = ensure_scratch(ctx, S_STATUS, n * sizeof(int32_t))) != DD_OK) return st;
                dst = reinterpret_cast<int32_t *>(ctx->scratch[S_STATUS]);
            }
            launch_batch_trace(dmeta + o_doms, reinterpret_cast<const int32_t *>(dmeta + o_tprob),
                               reinterpret_cast<const int32_t *>(dmeta + o_tloc),
                               reinterpret_cast<const int32_t *>(ctx->scratch[S_TARGETS]),
                               reinterpret_cast<const int32_t *>(ctx->scratch[S_SOURCES]), nT, S, max_nt, max_nv, max_pts, dxy,
                               dlen, dst, ctx->stream);
            CK(cudaGetLastError(), "batch trace launch");
            if (sx == 0) {
                CK(cudaMemcpyAsync(out_xy, dxy, n * max_pts * sizeof(float2), cudaMemcpyDeviceToHost, ctx->stream),
                   "copy paths");
                host = true;
            }
            if (sl == 0) {
                CK(cudaMemcpyAsync(out_len, dlen, n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream), "copy len");
                host = true;
            }
            if (ss == 0) {
                CK(cudaMemcpyAsync(out_status, dst, n * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream),
                   "copy status");
                host = true;
            }
        }
        if (host) {
            CK(cudaStreamSynchronize(ctx->stream), "batch query");
            return check_kernel_flag(ctx);
        }
        return DD_OK;
    } catch (const std::bad_alloc &) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    } catch (...) {
        return set_err(ctx, DD_EINVAL, "unexpected failure in dd_query_batch");
    }
}

dd_status dd_multigrid_check(const int64_t *a_off, const int32_t *a_col, const double *a_val, int64_t n,
                             const double *b, double *x, double rtol, int32_t max_iter, int32_t *iters,
                             int32_t *levels) {
    if (!a_off || !a_col || !a_val || !b || !x || !iters || !levels || n < 1 || max_iter < 1) return DD_EINVAL;
    try {
        AmgCsr A;
        A.rows = A.cols = n;
        A.off.assign(a_off, a_off + n + 1);
        const int64_t nnz = A.off[n];
        if (nnz < n || A.off[0] != 0) return DD_EINVAL;
        A.col.assign(a_col, a_col + nnz);
        A.val.assign(a_val, a_val + nnz);
        for (int32_t c : A.col)
            if (c < 0 || c >= n) return DD_EINVAL;
        std::vector<double> bb(b, b + n), xx;
        std::string err;
        if (!amg_host_solve(A, bb, xx, rtol, max_iter, iters, levels, err)) return DD_ENOTCONV;
        std::copy(xx.begin(), xx.end(), x);
        return DD_OK;
    } catch (...) {
        return DD_ENOMEM;
    }
}

dd_status dd_check_fast_log(double *spread) {
    if (!spread) return DD_EINVAL;
    try {
        std::string err;
        return fast_log_spread(spread, err);
    } catch (...) {
        return DD_ENOMEM;
    }
}

int32_t dd_kernel_timing(dd_ctx *ctx, int32_t mode, char *buf, int32_t len) {
    if (!ctx || mode < 0 || mode > 2) return DD_EINVAL;
    std::lock_guard<std::mutex> lock(g_kt_mutex);
    auto it = g_kt.find(ctx->stream);
    if (mode == 1) {
        if (it == g_kt.end()) {
            g_kt[ctx->stream];
            g_kt_on.fetch_add(1);
        } else {
            kt_fold(it->second);
            it->second.totals.clear();
        }
        return 0;
    }
    std::string out;
    if (it != g_kt.end()) {
        kt_fold(it->second);
        for (auto &kv : it->second.totals) {
            char line[160];
            std::snprintf(line, sizeof line, "%s %lld %.6f\n", kv.first.c_str(), (long long)kv.second.first,
                          kv.second.second);
            out += line;
        }
        if (mode == 0) {
            for (cudaEvent_t e : it->second.pool) cudaEventDestroy(e);
            g_kt.erase(it);
            g_kt_on.fetch_sub(1);
        }
    }
    if (buf && len > 0) {
        const size_t n = std::min<size_t>(out.size(), (size_t)len - 1);
        std::memcpy(buf, out.data(), n);
        buf[n] = 0;
    }
    return (int32_t)out.size() + 1;
}

dd_status dd_load_latency(dd_ctx *ctx, int64_t bytes, int32_t steps, double *ns_per_load) {
    if (!ctx || !ns_per_load || bytes < 4096 || bytes > (int64_t(1) << 32) || bytes % 128 || steps < 1)
        return ctx ? set_err(ctx, DD_EINVAL, "dd_load_latency: bytes in [4096, 2^32], a multiple of 128; steps >= 1")
                   : DD_EINVAL;
    try {
        dd_status st = select_device(ctx);
        if (st != DD_OK) return st;
        std::string err;
        if ((st = measure_load_latency(bytes, steps, ctx->stream, ns_per_load, err)) != DD_OK)
            return set_err(ctx, st, err);
        return DD_OK;
    } catch (...) {
        return set_err(ctx, DD_ENOMEM, "host allocation failed");
    }
}

int32_t dd_tuning_table(char *buf, int32_t len) {
    try {
        const std::string t = tuning_table();
        if (buf && len > 0) std::snprintf(buf, (size_t)len, "%s", t.c_str());
        return (int32_t)t.size();
    } catch (...) {
        return -1;
    }
}

}  // extern "C"
