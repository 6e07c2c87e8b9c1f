// Internal declarations shared by the translation units of libdd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <memory>
#include <functional>
#include <string>
#include <vector>

#include "dd.h"

// ---------------------------------------------------------------- host mesh
// Topology and Laplacian of Section IV, built on the host once per mesh.
struct HostMesh {
    int64_t n_v = 0, n_t = 0, k = 0, m = 0, n_edges = 0;
    std::vector<double> xy;          // [n_v][2]
    std::vector<int32_t> tri;        // [n_t][3] counter-clockwise
    std::vector<int32_t> B;          // boundary vertex ids, column order
    std::vector<int32_t> I;          // interior vertex ids, ascending
    std::vector<int32_t> col_of;     // vertex -> boundary column, or -1
    std::vector<int32_t> row_of;     // vertex -> interior row, or -1
    std::vector<int32_t> tnbr;       // [n_t][3] triangle across the edge opposite local vertex i, or -1
    std::vector<int32_t> vt_off, vt; // vertex -> incident triangles (ascending)
    std::vector<int32_t> vn_off, vn; // vertex -> neighbour vertices (ascending)
    // A = -L_II (symmetric positive definite M-matrix) in CSR, interior numbering
    std::vector<int64_t> a_off;
    std::vector<int32_t> a_col;
    std::vector<double> a_val;
    std::vector<double> a_diag;
    // right-hand sides L_IB: one entry per (interior row, boundary column) edge
    std::vector<int32_t> rb_row, rb_col;
    std::vector<double> rb_val;
    std::vector<float> gphi;         // [n_t][6] gradient of the hat functions
};

// Validate and build; returns DD_OK or DD_EINVAL with a message.
dd_status build_host_mesh(const double *xy, int64_t n_v, const int32_t *tri, int64_t n_t,
                          const int32_t *loop_idx, const int64_t *loop_off, int32_t n_loops,
                          HostMesh &out, std::string &err);

// ---------------------------------------------------------------- device mesh
struct DevMesh {
    int64_t n_v = 0, n_t = 0, k = 0, m = 0, k_pad = 0;
    float2 *xy = nullptr;      // [n_v]
    int4 *tri = nullptr;       // [n_t] (v0, v1, v2, 0)
    int4 *tnbr = nullptr;      // [n_t] (t0, t1, t2, 0)
    float4 *gphi = nullptr;    // [n_t][2]: (g0x, g0y, g1x, g1y), (g2x, g2y, 0, 0)
    int4 *trec = nullptr;      // [n_t][4] tracer records: (v0,v1,v2,n0) (n1,n2,q0,q1) (q2,0,p0x,p0y) (p1x,p1y,p2x,p2y),
                               // q_i = |grad phi_i|^2
    int32_t *vt_off = nullptr, *vt = nullptr;
    int32_t *vn_off = nullptr, *vn = nullptr;
    int32_t *interior = nullptr;   // [m]
    uint8_t *isb = nullptr;        // [n_v] 1 on boundary vertices
    int32_t *boundary = nullptr;   // [k]
    int64_t *a_off = nullptr;
    int32_t *a_col = nullptr;
    double *a_val = nullptr, *a_diag = nullptr;
    int64_t n_rb = 0;
    int32_t *rb_row = nullptr, *rb_col = nullptr;
    double *rb_val = nullptr;
    float *P = nullptr;        // [n_v][k_pad] FP32 Poisson kernel
    float *LP = nullptr;       // [n_v][k_pad] FP32 log2 P to full relative precision (dd_log_poisson_kernel), or null
    bool has_P = false;
    void *p_hi = nullptr, *p_lo = nullptr;   // BF16 split of P, [n_v][kb] (built on first BF16 request)
    float *ex = nullptr;                     // [n_v] sum_b P log P (FP64-accumulated)
    int64_t kb = 0;                          // BF16 row pitch: k rounded up to 64
    // tiled copy of P for the pipelined many-target field pass (built on the
    // first FP32 request for more than two targets): [row tile of 64][column]
    // [row in tile] over an even number of row tiles and k_pad rounded up to
    // 64 columns (pt_kt), zero past n_v and k_pad; pt_l holds the one-number
    // log2 of every entry
    float *pt_p = nullptr, *pt_l = nullptr;
    int64_t pt_kt = 0;
    // sparse fields (dd_sparsify): the threshold relative to the row maximum,
    // the sparsified P as CSR (each row's kept entries in column order), and
    // the exact total of every stored row (for the merged-bin extension)
    int64_t *sp_off = nullptr;               // [n_v + 1] row offsets into sp_val / sp_col
    float *sp_val = nullptr;                 // [sp_kept] kept entries
    uint16_t *sp_col = nullptr;              // [sp_kept] their columns
    long long *sp_rowsum = nullptr;          // [n_v] row totals in 2^-62 fixed point
    int64_t sp_kept = 0, sp_bytes = 0;
    float sp_theta = 0.f;
    int64_t bytes = 0;
    std::vector<void *> owned;
    std::vector<uint8_t> is_boundary;  // host copy: vertex flags
    std::vector<float> xy_h;           // host copy: vertex positions [n_v][2]
    std::vector<int32_t> vn_off_h, vn_h;
};

// ---------------------------------------------------------------- kernels
// Poisson kernel: FP64 Jacobi-PCG over all columns; fills m.P.
dd_status run_pcg(DevMesh &m, double rtol, int32_t max_iter, cudaStream_t s, int32_t *iters,
                  double *resid, std::string &err);
// Store a host FP64 P [n_v][k] into m.P with the same clamp/flush as the solver.
dd_status store_poisson(DevMesh &m, const double *P, cudaStream_t s, std::string &err);
// Refine the stored P to full relative precision in every entry (FP64 sweeps of
// the fixed-point form of Eq. 32, dd_logp.cu) and store log2 P in m.LP.
dd_status refine_log_poisson(DevMesh &m, double tol, int32_t max_sweeps, cudaStream_t s, int32_t *sweeps,
                             double *change, std::string &err);

// Per-target staging of P[t,:] and its split logarithm: four [T][k_pad] float
// arrays back to back -- P[t_a,b], the log-mantissa lm (table), the exponent E
// as the biased float 12582912 + 127 + E (exact; only differences of two are
// used), and the hardware base-2 log of the mantissa (streaming kernel).
// Target ids outside [0, n_v) are not read: their rows are zero-filled and
// *bad_id (if not null) is set to 1.  With LP (log2 P, dd_log_poisson_kernel)
// an entry whose FP32 value is 0 takes its logarithms from LP (finite there)
// instead of the clamp at FLT_MIN.
void launch_stage_targets(const float *P, int64_t n_v, int64_t k_pad, const int32_t *targets, int32_t T,
                          float4 *stage, cudaStream_t s, int *bad_id = nullptr, const float *LP = nullptr);
// FP32 fields.  out_kl / out_tv: [T][n_v] (either may be null).  variant: the
// tile shape for T > 2 (0 .. 3), or -1 for the autotuner's choice (which may
// run timed launches the first time a size class is seen).  staged_logs: the
// staging took logarithms from log2 P (launch_stage_targets with LP), which
// the tile kernel then reads instead of forming them from the staged entries.
// tiled: null, or the tiled copies of P and log2 P (DevMesh::pt_p / pt_l)
// with room for the staged targets in the same layout, which make the
// pipelined tile shape (variant 3) available to the autotuner.
struct TiledArgs {
    const float *PT, *LT;        // [row tiles][kt][64]
    float *TQ, *TL;              // [ceil(T / 64)][kt][64], filled by launch_fields_fp32
    int64_t kt;
};
int64_t tiled_k32(int64_t k_pad);
size_t tiled_target_bytes(int64_t k_pad, int32_t T);
dd_status prepare_tiled(DevMesh &m, cudaStream_t s, std::string &err);
// tile_done: null, or an event recorded on s when the many-target tile pass
// has ended (TV final; KL still to be recomputed near the targets).
void launch_fields_fp32(const float *P, int64_t n_v, int64_t k_pad, const float4 *stage, int32_t T,
                        float *out_kl, float *out_tv, int *err_flag, cudaStream_t s, int variant = -1,
                        bool staged_logs = false, const TiledArgs *tiled = nullptr,
                        cudaEvent_t tile_done = nullptr);
// One problem of a multi-domain field launch, and one output tile of it.
struct BatchProblem {
    const float *P;
    int64_t n_v, k_pad;
    const float *sP, *sL, *sE;   // staged targets [T][k_pad] each
    int32_t T, variant;          // targets; tile shape (0: 64x64, 1: 128x32, 2: 256x16, 3: pipelined)
    float *out_kl, *out_tv;      // [T][n_v] each (either may be null)
    // the pipelined launch: the mesh's tiled copies of P and log2 P and this
    // problem's targets in the same layout (null when the launch is staged)
    const float *PT, *LT;
    float *TQ, *TL;
    int64_t kt;
};
struct BatchItem {
    int32_t prob, x_tile, a_tile, pad;
};
// autotuned tile shape for one problem (may run timed launches the first time)
int tile_variant_for(const float *P, int64_t n_v, int64_t k_pad, const float *sP, const float *sL, const float *sE,
                     int32_t T, float *out_kl, float *out_tv, cudaStream_t s);
int tile_rows(int variant);
int tile_targets(int variant);
void launch_batch_stage(const BatchProblem *d_probs, const int32_t *d_tprob, const int32_t *d_tlocal,
                        const int32_t *d_targets, int32_t n_targets, int64_t k_max, cudaStream_t s);
// tile pass over every item, then the exact recompute by row blocks of every
// problem with KL output (fix_blocks: the sum of their fix_row_blocks(n_v))
void launch_batch_fields(const BatchProblem *d_probs, int32_t n_probs, const BatchItem *d_items, int32_t n_items,
                         int32_t *d_counter, cudaStream_t s, int64_t fix_blocks);
// The pipelined multi-domain launch: every problem carries its tiled arrays
// (PT, LT, TQ, TL, kt) and the items are 128-row x 64-target tiles (BatchItem
// x_tile counts pairs of 64-row tiles); the targets are first put into the
// tiled layout (max_tiles: the largest ceil(T / 64) * kt / 32 of the problems),
// then one persistent launch computes every tile (f_kl / f_tv: which fields
// all problems ask for), then the exact recompute.
void launch_batch_fields_pipe(const BatchProblem *d_probs, int32_t n_probs, const BatchItem *d_items,
                              int32_t n_items, int32_t *d_counter, int *err, cudaStream_t s, int64_t fix_blocks,
                              int64_t max_tiles, bool f_kl, bool f_tv);
int64_t fix_row_blocks(int64_t n_v);
// The autotuner's choice between the staged (0) and the pipelined (1)
// multi-domain launch: the first time a class of batches is seen (the fields
// asked for, problems and n k T work in powers of two) both run (a warm-up
// and two timed launches each, on the caller's stream) and the faster is kept
// for the class.  DD_BATCH_PIPE=0 or 1 pins the choice.
int batch_launch_choice(int32_t n_probs, int64_t work, uint32_t f_mask, const std::function<void()> &staged,
                        const std::function<void()> &pipelined, cudaStream_t s);
std::string tuning_table();
// spurious local minima of T fields [T][n_v] (counts host [T], flags optional [T][n_v])
void launch_local_minima(const DevMesh &m, const float *fields, const int32_t *targets, int32_t T, int32_t *counts,
                         uint8_t *flags, cudaStream_t s);
// edge-following paths (T*S, sources [T][S]) on device fields [T][n_v]
void launch_edge_paths(const DevMesh &m, const float *fields, const int32_t *targets, const int32_t *sources, int32_t T,
                       int32_t S, int32_t max_pts, float2 *out_xy, int32_t *out_len, int32_t *out_status,
                       cudaStream_t s);
// other f-divergence fields [T][n_v] from staged targets (stage_targets_kernel's arrays)
// With LP, the reverse KL takes log P[x,b] from LP where the FP32 entry is 0.
dd_status launch_fdiv(const float *P, int64_t n_v, int64_t k_pad, const float4 *stage, int32_t T, int32_t family,
                      double param, float *out, cudaStream_t s, std::string &err, const float *LP = nullptr);

// Copy the defined prefix of every path (len[i] points of row i, pitch max_pts)
// from device memory to another buffer (e.g. pinned host memory seen through its
// device address), one warp per path, 16-byte stores (dd_trace.cu).
// ns per dependent 4-byte load (L1 bypassed) along a random cycle of 128-byte
// lines through `bytes` of device memory (allocated and freed here)
dd_status measure_load_latency(int64_t bytes, int32_t steps, cudaStream_t s, double *ns, std::string &err);
void launch_copy_paths(const float2 *src, const int32_t *len, int64_t n, int32_t max_pts, float2 *dst,
                       cudaStream_t s);

// Sparse fields (dd_sparse.cu, Section V).  build_sparse_rows fills the sp_*
// members of m from m.P (the caller frees earlier ones; every array it
// allocates is pushed to m.owned).  The sparse stage is the dense stage
// (4 x T x k_pad floats, filled by launch_stage_targets) followed by T block
// lists of sparse_list_pitch(k_pad) uint16, T int32 counts (padded to 16
// bytes) and T doubles M_t; launch_sparse_fields thresholds the staged rows in
// place, lists their blocks, computes M_t and launches the field kernels (one
// target per grid row): KL~ and TV~ from the CSR rows, KLT~ from the dense
// rows at the target's blocks; merged: the merged-bin extension instead.
int64_t sparse_list_pitch(int64_t k_pad);
size_t sparse_stage_bytes(int64_t k_pad, int32_t T);
size_t sparse_field_smem(int64_t k_pad);
dd_status build_sparse_rows(DevMesh &m, double theta, cudaStream_t s, int64_t *kept_out, int64_t *bytes_out,
                            std::string &err);
void launch_sparse_fields(const DevMesh &m, const int32_t *d_targets, float4 *stage, int32_t T, float *out_kl,
                          float *out_tv, float *out_klt, bool merged, int *err_flag, cudaStream_t s);
// spread (max - min) of the hardware mantissa log's error over [1, 2), in base-2 units
dd_status fast_log_spread(double *spread, std::string &err);

// Tracer: when trace_dense_decisions(S), per-field triangle rates and vertex
// decisions into `scratch` (trace_scratch_bytes(m, T, true) bytes), then T*S
// paths; otherwise the walk forms the rates and decisions it needs itself and
// `scratch` is unused.
bool trace_dense_decisions(int32_t S);
size_t trace_scratch_bytes(const DevMesh &m, int32_t T, bool decisions);
void launch_trace(const DevMesh &m, const float *fields, int64_t field_stride, const int32_t *targets,
                  const int32_t *sources, int32_t T, int32_t S, int32_t max_pts, float2 *out_xy,
                  int32_t *out_len, int32_t *out_status, void *scratch, cudaStream_t s);

// Split-BF16 tensor-core KL (tcgen05): BF16 split of P and e_x once per mesh,
// then KL [T][n_v] for T staged targets (scratch: gemm_target_scratch_bytes).
int64_t gemm_kb(int64_t k);
dd_status prepare_bf16(DevMesh &m, cudaStream_t s, std::string &err);
size_t gemm_target_scratch_bytes(const DevMesh &m, int32_t T);
dd_status launch_kl_gemm(const DevMesh &m, const int32_t *d_targets, int32_t T, void *scratch, float *out_kl,
                         int *err_flag, cudaStream_t s, std::string &err);

// Tracer over several meshes in one launch (descriptors built on the host;
// each item's scratch: trace_scratch_bytes(m, T_item, false) bytes; the walk
// computes vertex decisions itself).
size_t batch_trace_dom_bytes();
void fill_batch_trace_dom(void *dst, const DevMesh &m, const float *fields, int32_t T, void *scratch);
void launch_batch_trace(const void *d_doms, const int32_t *d_tdom, const int32_t *d_tloc, const int32_t *d_targets,
                        const int32_t *d_sources, int32_t n_targets, int32_t S, int64_t max_nt, int64_t max_nv,
                        int32_t max_pts, float2 *out_xy, int32_t *out_len, int32_t *out_status, cudaStream_t s,
                        const int32_t *d_path_target = nullptr, int64_t n_paths = 0);

// ---------------------------------------------------------------- context
enum ScratchId { S_TARGETS, S_SOURCES, S_STAGE, S_FIELDS, S_XY, S_LEN, S_STATUS, S_GRAD, S_GEMM, S_META,
                 S_TSTAGE, S_COUNT };

struct MeshSlot {
    bool live = false;
    DevMesh dev;
};

struct dd_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    std::vector<MeshSlot> meshes;
    void *scratch[S_COUNT] = {};
    size_t scratch_cap[S_COUNT] = {};
    int *d_err = nullptr;                     // device error flag written by kernels
    void *pinned[S_COUNT] = {};               // host staging for index uploads, one per scratch id
    size_t pinned_cap[S_COUNT] = {};
    cudaEvent_t pinned_free[S_COUNT] = {};    // recorded after the last upload from pinned[id]
    cudaStream_t side = nullptr;              // copies that overlap the main stream's kernels
    cudaEvent_t side_ev[3] = {};             // fields ready, fields copied, tile pass done
};

// Per-kernel device time (dd_kernel_timing): while timing is enabled for a
// stream, a KMark around a launch on that stream records a CUDA event before
// and after it; totals per kernel name are folded in when read.  Without
// timing enabled a KMark costs one relaxed atomic load.
struct KMark {
    KMark(const char *name, cudaStream_t s);
    ~KMark();
    KMark(const KMark &) = delete;
    KMark &operator=(const KMark &) = delete;
    const char *name = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t a = nullptr;
};

#define DD_CUDA_TRY(expr, errstr)                                                   \
    do {                                                                            \
        cudaError_t e__ = (expr);                                                   \
        if (e__ != cudaSuccess) {                                                   \
            errstr = std::string(#expr) + ": " + cudaGetErrorString(e__);           \
            return DD_ECUDA;                                                        \
        }                                                                           \
    } while (0)
