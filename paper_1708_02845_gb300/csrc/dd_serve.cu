// Query server: continuous batching of path queries over resident meshes.
//
// A query is (mesh, interior target, S sources) and asks for the S paths
// traced on the target's KL field (Section IV).  A worker thread keeps up to
// n_slots batches in flight, one per CUDA stream.  Whenever a slot is free it
// forms a batch from the queries that have arrived (arrival order, as many as
// fit the slot's device arena and max_batch), groups them by mesh and runs
//   staging of all targets -> one persistent field launch over every mesh's
//   tiles -> one tracer launch over all paths -> copy of each path's
//   defined prefix to pinned host memory,
// all on the slot's stream, so a batch formed from later arrivals overlaps on
// the device with batches already running.  Completion is detected with an
// event; the query's latency is the time from submission to its paths being
// in host memory.  Device arenas and pinned buffers are allocated once when
// the server is created: the HBM budget is split evenly over the slots, and
// a query that cannot fit one slot is refused at submission (DD_EBUDGET).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dd_internal.h"

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

size_t al(size_t x) { return (x + 255) / 256 * 256; }

struct Query {
    int64_t id = 0;
    int32_t mesh = 0, target = 0, S = 0;
    std::vector<int32_t> sources;
    double t_submit = 0, t_done = 0;
    int32_t err = 0;
    std::vector<float> xy;                  // the paths' defined points, path after path (len[s] points each)
    std::vector<int32_t> len, status;       // [S]
    size_t need = 0;                        // device bytes in a batch
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Query *> qs;
    uint8_t *dev = nullptr;
    size_t dev_cap = 0;
    uint8_t *pin_in = nullptr;
    size_t pin_in_cap = 0;
    uint8_t *pin_out = nullptr;
    uint8_t *pin_out_dev = nullptr;         // pin_out's device address (the path copy kernel writes there)
    size_t pin_out_cap = 0;
    size_t out_xy_off = 0, out_len_off = 0, out_st_off = 0;   // within pin_out
};

}  // namespace

struct dd_server {
    dd_ctx *ctx = nullptr;
    int64_t budget = 0;
    int32_t max_pts = 0, max_batch = 0;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Query *> pending;
    struct Done {
        int64_t id;
        int32_t err;
        double latency_ms;
    };
    std::deque<Done> completed;             // not yet reported by poll
    std::unordered_map<int64_t, Query *> finished;
    std::thread worker;
    bool stop = false;
    int in_flight = 0;
    std::string err;
};

namespace {

// device bytes one query needs inside a batch
size_t query_need(const DevMesh &m, int32_t S, int32_t max_pts) {
    return al((size_t)m.n_v * 4) + al((size_t)3 * m.k_pad * 4) + al(trace_scratch_bytes(m, 1, false)) +
           al((size_t)S * ((size_t)max_pts * 8 + 8)) + al((size_t)S * 8) + 4096;
}

// host pinned bytes for a query's outputs
size_t query_out(int32_t S, int32_t max_pts) { return (size_t)S * ((size_t)max_pts * 8 + 8); }

int default_variant(int32_t T) { return T <= 16 ? 2 : (T <= 32 ? 1 : 0); }

// launch one batch on a slot; returns false (and sets q->err) on failure
bool launch_batch(dd_server *sv, Slot &sl) {
    dd_ctx *ctx = sv->ctx;
    std::map<int32_t, std::vector<Query *>> by_mesh;
    for (Query *q : sl.qs) by_mesh[q->mesh].push_back(q);
    std::vector<Query *> order;              // global target order
    std::vector<DevMesh *> ms;
    std::vector<int32_t> Ts;
    for (auto &kv : by_mesh) {
        ms.push_back(&ctx->meshes[kv.first].dev);
        Ts.push_back((int32_t)kv.second.size());
        for (Query *q : kv.second) order.push_back(q);
    }
    const int n_items = (int)ms.size();
    const int32_t nT = (int32_t)order.size();
    int64_t n_paths = 0, max_nt = 0, max_nv = 0, max_k = 0;
    for (Query *q : order) n_paths += q->S;
    for (DevMesh *m : ms) {
        max_nt = std::max(max_nt, m->n_t);
        max_nv = std::max(max_nv, m->n_v);
        max_k = std::max(max_k, m->k_pad);
    }
    // ---- device arena layout
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += al(bytes);
        return r;
    };
    const size_t o_targets = take(nT * 4), o_tprob = take(nT * 4), o_tloc = take(nT * 4);
    const size_t o_sources = take(n_paths * 4), o_ptarget = take(n_paths * 4);
    const size_t o_probs = take(n_items * sizeof(BatchProblem));
    const size_t dom_bytes = batch_trace_dom_bytes();
    const size_t o_doms = take(n_items * dom_bytes);
    const size_t o_counter = take(256);
    size_t n_tiles = 0;
    std::vector<int> var(n_items);
    for (int i = 0; i < n_items; ++i) {
        var[i] = default_variant(Ts[i]);
        n_tiles += (size_t)((ms[i]->n_v + tile_rows(var[i]) - 1) / tile_rows(var[i])) *
                   ((Ts[i] + tile_targets(var[i]) - 1) / tile_targets(var[i]));
    }
    const size_t o_items = take(n_tiles * sizeof(BatchItem));
    const size_t meta_end = o;
    size_t stage_f = 0, field_f = 0, grad_b = 0;
    for (int i = 0; i < n_items; ++i) {
        stage_f += (size_t)3 * Ts[i] * ms[i]->k_pad;
        field_f += (size_t)Ts[i] * ms[i]->n_v;
        grad_b += trace_scratch_bytes(*ms[i], Ts[i], false);
    }
    const size_t o_stage = take(stage_f * 4), o_fields = take(field_f * 4), o_grads = take(grad_b);
    const size_t o_xy = take((size_t)n_paths * sv->max_pts * 8), o_len = take(n_paths * 4), o_st = take(n_paths * 4);
    if (o > sl.dev_cap || meta_end > sl.pin_in_cap) {
        for (Query *q : sl.qs) q->err = DD_EBUDGET;
        return false;
    }
    // ---- metadata in pinned memory
    uint8_t *h = sl.pin_in;
    uint8_t *d = sl.dev;
    int32_t *tg = reinterpret_cast<int32_t *>(h + o_targets), *tp = reinterpret_cast<int32_t *>(h + o_tprob),
            *tl = reinterpret_cast<int32_t *>(h + o_tloc), *src = reinterpret_cast<int32_t *>(h + o_sources),
            *pt = reinterpret_cast<int32_t *>(h + o_ptarget);
    {
        int g = 0;
        int64_t pth = 0;
        for (int i = 0; i < n_items; ++i)
            for (int a = 0; a < Ts[i]; ++a, ++g) {
                Query *q = order[g];
                tg[g] = q->target;
                tp[g] = i;
                tl[g] = a;
                for (int s = 0; s < q->S; ++s, ++pth) {
                    src[pth] = q->sources[s];
                    pt[pth] = g;
                }
            }
    }
    std::vector<BatchProblem> probs(n_items);
    {
        size_t so = 0, fo = 0, go = 0;
        for (int i = 0; i < n_items; ++i) {
            const DevMesh &m = *ms[i];
            BatchProblem &q = probs[i];
            const size_t blk = (size_t)Ts[i] * m.k_pad;
            float *stage = reinterpret_cast<float *>(d + o_stage);
            q.P = m.P;
            q.n_v = m.n_v;
            q.k_pad = m.k_pad;
            q.sP = stage + so;
            q.sL = stage + so + blk;
            q.sE = stage + so + 2 * blk;
            so += 3 * blk;
            q.T = Ts[i];
            q.variant = var[i];
            q.out_kl = reinterpret_cast<float *>(d + o_fields) + fo;
            q.out_tv = nullptr;
            fill_batch_trace_dom(h + o_doms + i * dom_bytes, m, q.out_kl, Ts[i], d + o_grads + go);
            fo += (size_t)Ts[i] * m.n_v;
            go += trace_scratch_bytes(m, Ts[i], false);
        }
        std::memcpy(h + o_probs, probs.data(), n_items * sizeof(BatchProblem));
        size_t j = 0;
        BatchItem *it = reinterpret_cast<BatchItem *>(h + o_items);
        for (int i = 0; i < n_items; ++i) {
            const int tr = tile_rows(var[i]), tt = tile_targets(var[i]);
            for (int64_t xt = 0; xt * tr < ms[i]->n_v; ++xt)
                for (int at = 0; at * tt < Ts[i]; ++at) it[j++] = BatchItem{i, (int32_t)xt, at, 0};
        }
    }
    cudaStream_t s = sl.stream;
    cudaError_t e = cudaMemcpyAsync(d, h, meta_end, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        launch_batch_stage(reinterpret_cast<const BatchProblem *>(d + o_probs), reinterpret_cast<const int32_t *>(d + o_tprob),
                           reinterpret_cast<const int32_t *>(d + o_tloc), reinterpret_cast<const int32_t *>(d + o_targets),
                           nT, max_k, s);
        int64_t fix_blocks = 0;
        for (int i = 0; i < n_items; ++i) fix_blocks += fix_row_blocks(ms[i]->n_v);
        launch_batch_fields(reinterpret_cast<const BatchProblem *>(d + o_probs), (int32_t)n_items,
                            reinterpret_cast<const BatchItem *>(d + o_items), (int32_t)n_tiles,
                            reinterpret_cast<int32_t *>(d + o_counter), s, fix_blocks);
        launch_batch_trace(d + o_doms, reinterpret_cast<const int32_t *>(d + o_tprob),
                           reinterpret_cast<const int32_t *>(d + o_tloc), reinterpret_cast<const int32_t *>(d + o_targets),
                           reinterpret_cast<const int32_t *>(d + o_sources), nT, 0, max_nt, max_nv, sv->max_pts,
                           reinterpret_cast<float2 *>(d + o_xy), reinterpret_cast<int32_t *>(d + o_len),
                           reinterpret_cast<int32_t *>(d + o_st), s, reinterpret_cast<const int32_t *>(d + o_ptarget),
                           n_paths);
        e = cudaGetLastError();
    }
    sl.out_xy_off = 0;
    sl.out_len_off = al((size_t)n_paths * sv->max_pts * 8);
    sl.out_st_off = sl.out_len_off + al(n_paths * 4);
    if (e == cudaSuccess && sl.out_st_off + al(n_paths * 4) > sl.pin_out_cap) e = cudaErrorMemoryAllocation;
    // each path's defined prefix only (one warp per path writes it through the
    // pinned buffer's device address), then the lengths and statuses
    if (e == cudaSuccess) {
        launch_copy_paths(reinterpret_cast<const float2 *>(d + o_xy), reinterpret_cast<const int32_t *>(d + o_len),
                          n_paths, sv->max_pts, reinterpret_cast<float2 *>(sl.pin_out_dev), s);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.pin_out + sl.out_len_off, d + o_len, n_paths * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.pin_out + sl.out_st_off, d + o_st, n_paths * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.done, s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (Query *q : sl.qs) q->err = DD_ECUDA;
        return false;
    }
    sl.qs = order;               // keep the global order for unpacking
    return true;
}

// copy a finished slot's paths into its queries
void retire(dd_server *sv, Slot &sl) {
    const double t = now_ms();
    int64_t pth = 0;
    const float *xy = reinterpret_cast<const float *>(sl.pin_out + sl.out_xy_off);
    const int32_t *ln = reinterpret_cast<const int32_t *>(sl.pin_out + sl.out_len_off);
    const int32_t *st = reinterpret_cast<const int32_t *>(sl.pin_out + sl.out_st_off);
    for (Query *q : sl.qs) {
        size_t pts = 0;
        for (int32_t s = 0; s < q->S; ++s) pts += (size_t)std::max(0, std::min(ln[pth + s], sv->max_pts));
        q->xy.resize(2 * pts);
        float *o = q->xy.data();
        for (int32_t s = 0; s < q->S; ++s) {
            const size_t np = (size_t)std::max(0, std::min(ln[pth + s], sv->max_pts));
            std::memcpy(o, xy + (pth + s) * (size_t)sv->max_pts * 2, np * 2 * sizeof(float));
            o += 2 * np;
        }
        q->len.assign(ln + pth, ln + pth + q->S);
        q->status.assign(st + pth, st + pth + q->S);
        pth += q->S;
        q->t_done = t;
    }
}

void worker_loop(dd_server *sv) {
    cudaSetDevice(sv->ctx->device);
    const size_t slot_cap = sv->slots.empty() ? 0 : sv->slots[0].dev_cap;
    for (;;) {
        // retire finished batches
        bool any_busy = false;
        for (Slot &sl : sv->slots) {
            if (!sl.busy) continue;
            cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            if (q == cudaSuccess) {
                retire(sv, sl);
            } else {
                cudaGetLastError();
                for (Query *x : sl.qs) x->err = DD_ECUDA;
            }
            std::lock_guard<std::mutex> lock(sv->mu);
            for (Query *x : sl.qs) {
                if (x->t_done == 0) x->t_done = now_ms();
                sv->completed.push_back({x->id, x->err, x->t_done - x->t_submit});
                sv->finished[x->id] = x;
            }
            sl.qs.clear();
            sl.busy = false;
            --sv->in_flight;
            sv->cv.notify_all();
        }
        // launch on every free slot while queries wait
        for (Slot &sl : sv->slots) {
            if (sl.busy) continue;
            std::vector<Query *> batch;
            {
                std::lock_guard<std::mutex> lock(sv->mu);
                size_t need = 0, out = 0;
                const size_t out_cap = sl.pin_out_cap * 9 / 10;
                while (!sv->pending.empty() && (int)batch.size() < sv->max_batch) {
                    Query *q = sv->pending.front();
                    const size_t qo = query_out(q->S, sv->max_pts) + 1024;
                    if (!batch.empty() && (need + q->need > slot_cap * 9 / 10 || out + qo > out_cap)) break;
                    need += q->need;
                    out += qo;
                    batch.push_back(q);
                    sv->pending.pop_front();
                }
                // counted in flight from the moment they leave the queue, so that
                // wait_idle never sees an empty queue with a batch not yet launched
                if (!batch.empty()) ++sv->in_flight;
            }
            if (batch.empty()) break;
            sl.qs = batch;
            if (launch_batch(sv, sl)) {
                sl.busy = true;
                any_busy = true;
            } else {
                std::lock_guard<std::mutex> lock(sv->mu);
                for (Query *x : sl.qs) {
                    x->t_done = now_ms();
                    sv->completed.push_back({x->id, x->err, x->t_done - x->t_submit});
                    sv->finished[x->id] = x;
                }
                sl.qs.clear();
                --sv->in_flight;
                sv->cv.notify_all();
            }
        }
        std::unique_lock<std::mutex> lock(sv->mu);
        if (sv->stop && sv->pending.empty() && sv->in_flight == 0) return;
        if (any_busy || sv->in_flight > 0) {
            lock.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
        } else if (sv->pending.empty()) {
            sv->cv.wait_for(lock, std::chrono::milliseconds(2));
        }
    }
}

}  // namespace

extern "C" {

dd_status dd_server_create(dd_ctx *ctx, int64_t budget_bytes, int32_t n_slots, int32_t max_batch, int32_t max_pts,
                           dd_server **out) {
    if (!ctx || !out || n_slots < 1 || n_slots > 16 || max_batch < 1 || max_pts < 2 || budget_bytes < (1 << 20))
        return DD_EINVAL;
    *out = nullptr;
    dd_server *sv = nullptr;
    try {
        if (cudaSetDevice(ctx->device) != cudaSuccess) return DD_ECUDA;
        sv = new dd_server();
        sv->ctx = ctx;
        sv->budget = budget_bytes;
        sv->max_pts = max_pts;
        sv->max_batch = max_batch;
        sv->slots.resize(n_slots);
        const size_t per = (size_t)(budget_bytes / n_slots) / 256 * 256;
        for (Slot &sl : sv->slots) {
            if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaMalloc((void **)&sl.dev, per) != cudaSuccess)
                throw std::bad_alloc();
            sl.dev_cap = per;
            // metadata is small next to the arena; the output copy is bounded by the arena's path share
            sl.pin_in_cap = std::min<size_t>(per, (size_t)64 << 20);
            sl.pin_out_cap = std::min<size_t>(per, (size_t)1 << 30);
            if (cudaMallocHost((void **)&sl.pin_in, sl.pin_in_cap) != cudaSuccess ||
                cudaMallocHost((void **)&sl.pin_out, sl.pin_out_cap) != cudaSuccess ||
                cudaHostGetDevicePointer((void **)&sl.pin_out_dev, sl.pin_out, 0) != cudaSuccess)
                throw std::bad_alloc();
        }
        sv->worker = std::thread(worker_loop, sv);
        *out = sv;
        return DD_OK;
    } catch (...) {
        cudaGetLastError();
        if (sv) {
            for (Slot &sl : sv->slots) {
                if (sl.dev) cudaFree(sl.dev);
                if (sl.pin_in) cudaFreeHost(sl.pin_in);
                if (sl.pin_out) cudaFreeHost(sl.pin_out);
                if (sl.done) cudaEventDestroy(sl.done);
                if (sl.stream) cudaStreamDestroy(sl.stream);
            }
            delete sv;
        }
        return DD_ENOMEM;
    }
}

dd_status dd_server_submit(dd_server *sv, int64_t query_id, int32_t mesh, int32_t target, const int32_t *sources,
                           int32_t S) {
    if (!sv) return DD_EINVAL;
    try {
        dd_ctx *ctx = sv->ctx;
        if (mesh < 0 || mesh >= (int32_t)ctx->meshes.size() || !ctx->meshes[mesh].live) return DD_EINVAL;
        const DevMesh &m = ctx->meshes[mesh].dev;
        if (!m.has_P) return DD_ESTATE;
        if (S < 1 || !sources || target < 0 || target >= m.n_v || m.is_boundary[target]) return DD_EINVAL;
        for (int s = 0; s < S; ++s)
            if (sources[s] < 0 || sources[s] >= m.n_v) return DD_EINVAL;
        Query *q = new Query();
        q->id = query_id;
        q->mesh = mesh;
        q->target = target;
        q->S = S;
        q->sources.assign(sources, sources + S);
        q->need = query_need(m, S, sv->max_pts);
        if (q->need > sv->slots[0].dev_cap * 9 / 10 || query_out(S, sv->max_pts) + 1024 > sv->slots[0].pin_out_cap * 9 / 10) {
            delete q;
            return DD_EBUDGET;
        }
        q->t_submit = now_ms();
        std::lock_guard<std::mutex> lock(sv->mu);
        if (sv->finished.count(query_id)) {
            delete q;
            return DD_EINVAL;
        }
        sv->pending.push_back(q);
        sv->cv.notify_all();
        return DD_OK;
    } catch (...) {
        return DD_ENOMEM;
    }
}

int32_t dd_server_poll(dd_server *sv, int32_t max_n, int64_t *ids, int32_t *statuses, double *latency_ms) {
    if (!sv || max_n < 1 || !ids) return -1;
    std::lock_guard<std::mutex> lock(sv->mu);
    int32_t n = 0;
    while (n < max_n && !sv->completed.empty()) {
        const dd_server::Done d = sv->completed.front();
        sv->completed.pop_front();
        ids[n] = d.id;
        if (statuses) statuses[n] = d.err;
        if (latency_ms) latency_ms[n] = d.latency_ms;
        ++n;
    }
    return n;
}

dd_status dd_server_take(dd_server *sv, int64_t query_id, float *xy, int32_t *len, int32_t *status) {
    if (!sv) return DD_EINVAL;
    Query *q = nullptr;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        auto it = sv->finished.find(query_id);
        if (it == sv->finished.end()) return DD_ESTATE;
        q = it->second;
        sv->finished.erase(it);
    }
    const dd_status st = (dd_status)q->err;
    if (st == DD_OK) {
        if (xy) {
            const float *p = q->xy.data();
            for (int32_t s = 0; s < q->S; ++s) {
                const size_t np = (size_t)std::max(0, std::min(q->len[s], sv->max_pts));
                std::memcpy(xy + (size_t)s * sv->max_pts * 2, p, np * 2 * sizeof(float));
                p += 2 * np;
            }
        }
        if (len) std::memcpy(len, q->len.data(), q->len.size() * sizeof(int32_t));
        if (status) std::memcpy(status, q->status.data(), q->status.size() * sizeof(int32_t));
    }
    delete q;
    return st;
}

dd_status dd_server_wait_idle(dd_server *sv, double timeout_s) {
    if (!sv) return DD_EINVAL;
    std::unique_lock<std::mutex> lock(sv->mu);
    const bool ok = sv->cv.wait_for(lock, std::chrono::duration<double>(timeout_s),
                                    [&] { return sv->pending.empty() && sv->in_flight == 0; });
    return ok ? DD_OK : DD_ETIMEOUT;
}

void dd_server_destroy(dd_server *sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lock(sv->mu);
        sv->stop = true;
        sv->cv.notify_all();
    }
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->ctx->device);
    for (Slot &sl : sv->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaFree(sl.dev);
        cudaFreeHost(sl.pin_in);
        cudaFreeHost(sl.pin_out);
        cudaEventDestroy(sl.done);
        cudaStreamDestroy(sl.stream);
    }
    for (auto &kv : sv->finished) delete kv.second;
    for (Query *q : sv->pending) delete q;
    delete sv;
}

}  // extern "C"
