/*
 * dd.h -- C ABI of the divergence-distance library (libdd.so).
 *
 * Chen, Gotsman & Hormann, "Path Planning with Divergence-Based Distance
 * Functions".  A planar domain is a triangle mesh with n vertices, k of them
 * on the boundary (outer loop plus one loop per obstacle) and m = n - k in the
 * interior (Section IV).  The library
 *   1. builds the cotangent Laplacian L^c (Section IV),
 *   2. solves for the discrete Poisson kernel P = [-L_II^-1 L_IB ; I]
 *      (Eq. 32-33), an n x k non-negative matrix with unit row sums,
 *   3. evaluates the TV and KL divergence fields of a target vertex t over
 *      every vertex x (Eq. 34-35),
 *   4. traces gradient-descent paths through the mesh triangles from source
 *      vertices to t (Section IV, "Gradient-descent path generation").
 *
 * Conventions shared by every call:
 *  - Every function returns a dd_status; on failure a message is available
 *    from dd_last_error(ctx).  No C++ exception or abort crosses the ABI.
 *  - Vertex ids are 0-based int32 in the caller's numbering; rows of P and
 *    entries of every field use that numbering.  Columns of P follow the
 *    boundary loops concatenated in the order given to dd_load_mesh.
 *  - The caller owns every buffer it passes.  The library copies meshes and
 *    owns P, its solver workspace and cached fields until dd_unload_mesh or
 *    dd_destroy.
 *  - Output buffers marked "device or host" may be CUDA device memory on the
 *    context's device (written asynchronously on the context stream) or host
 *    memory (pinned or pageable; the call then stages through device memory
 *    and returns after the copy completed).
 *  - Calls on one context are not thread-safe; use one context per thread.
 *  - All GPU work runs on the context stream, in call order.
 */
#ifndef DD_H
#define DD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dd_ctx dd_ctx;

typedef enum {
    DD_OK = 0,
    DD_EINVAL = -1,    /* bad argument: size, id, pointer space, malformed mesh      */
    DD_ENOMEM = -2,    /* device or host allocation failed                            */
    DD_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed                 */
    DD_ESTATE = -4,    /* call out of order (e.g. a field before the Poisson kernel)  */
    DD_ENOTCONV = -5,  /* the Poisson-kernel solve did not reach rtol in max_iter     */
    DD_ETIMEOUT = -6,  /* a bounded device-side wait gave up (kernel error flag set)  */
    DD_EBUDGET = -7    /* the request exceeds the context's device-memory budget      */
} dd_status;

/* divergence selector bits (Eq. 34: TV, Eq. 35: KL).  Eq. 35's two readings:
 *   DD_F_KL   KL_t(x) = sum_b P[x,b] log(P[x,b]/P[t,b]), weighted by the field
 *             row (the form the tensor-core cross term computes)
 *   DD_F_KLT  KLT_t(x) = sum_b P[t,b] log(P[t,b]/P[x,b]), weighted by the
 *             target row (Eq. 35 with p the target; +inf on boundary rows,
 *             returned as a large finite value >= 50)
 * Fields of a mask are laid out in bit order: KL, TV, KLT. */
enum { DD_F_KL = 1, DD_F_TV = 2, DD_F_KLT = 4 };

/* arithmetic of the field evaluation:
 *  DD_PREC_FP32   FP32 CUDA-core evaluation of Eq. 34-35 term by term in
 *                 two passes.  The exact form splits each log into an exact
 *                 exponent and a table-driven mantissa log.  For one or two
 *                 targets a first pass takes the mantissa logs from the
 *                 hardware base-2 logarithm and is within ln2 *
 *                 DD_FAST_LOG_SPREAD of the exact form (see
 *                 dd_check_fast_log); rows whose KL there is below
 *                 DD_EXACT_BELOW are recomputed in the exact form.  For more
 *                 targets the first pass forms each log2 as one FP32 number
 *                 (exponent plus hardware mantissa log) and is within ln2 *
 *                 DD_FAST_LOG_SPREAD + 2^-24 (2 ln k + 2 KL + 2) of the exact
 *                 form; every (row, target) pair whose KL there is below
 *                 DD_TILE_EXACT_BELOW is recomputed in the exact form.  In
 *                 both cases the rows near the target (x = t among them) come
 *                 from the exact form and every value keeps 1e-5 relative
 *                 accuracy.
 *  DD_PREC_BF16X3 KL cross term sum_b P[x,b] log P[t,b] as a tensor-core GEMM
 *                 of split BF16 hi/lo operands (hi*hi + hi*lo + lo*hi, FP32
 *                 accumulation); TV and KLT are always FP32
 *  DD_PREC_SPARSE the sparse fields of Section V: P sparsified by
 *                 eliminating the entries below a threshold (see
 *                 dd_sparsify), FP32 as DD_PREC_FP32.  Row y keeps
 *                 S_y = {b : P[y,b] >= theta max_b' P[y,b'], P[y,b] > 0}
 *                 (FP32 product), P~ is P with the other entries set to 0.
 *                 In Eq. 35 the weight row's eliminated entries drop their
 *                 terms and the other row enters through its logarithm from
 *                 the full P:
 *                   KLT~_t(x) = sum_{b in S_t} P[t,b] log(P[t,b]/P[x,b])
 *                   KL~_t(x)  = sum_{b in S_x} P[x,b] log(P[x,b]/P[t,b])
 *                   TV~_t(x)  = sum_b |P~[x,b] - P~[t,b]|
 *                 (approximations, not divergences: KL~ and KLT~ can be
 *                 negative; all three are 0 at x = t).  KL~ and TV~ read
 *                 only the sparse copy of P; KLT~ reads the dense P at the
 *                 4-column blocks holding S_t
 *  DD_PREC_SPARSE_MERGED  an extension, not in the paper: S_t decides for
 *                 both rows and the other columns merge into one bin of mass
 *                 M_y = sum_{b not in S_t} P[y,b]:
 *                   KL^_t(x) = sum_{b in S_t} P[x,b] log(P[x,b]/P[t,b])
 *                              + M_x log(M_x / M_t)
 *                   KLT^_t(x) likewise with the roles of x and t swapped
 *                   TV^_t(x) = sum_{b in S_t} |P[x,b] - P[t,b]| + |M_x - M_t|
 *                 (divergences of the coarse-grained harmonic measures:
 *                 0 <= KL^ <= KL, 0 <= TV^ <= TV, all 0 at x = t); each row
 *                 is read only at the 4-column blocks holding S_t */
enum { DD_PREC_FP32 = 0, DD_PREC_BF16X3 = 1, DD_PREC_SPARSE = 2, DD_PREC_SPARSE_MERGED = 3 };
#define DD_FAST_LOG_SPREAD 5.0e-7
#define DD_EXACT_BELOW 0.05
#define DD_TILE_EXACT_BELOW 0.25

/* Measures, on the current device, the spread (maximum minus minimum) of the
 * error of the hardware base-2 logarithm used by the FP32 first pass, over
 * every float mantissa in [1, 2) against an FP64 reference, and writes it to
 * *spread.  The FP32 path's error bound assumes *spread <= DD_FAST_LOG_SPREAD.
 * Allocates and frees 512 KB of device memory.  Errors: DD_EINVAL (null),
 * DD_ENOMEM, DD_ECUDA. */
dd_status dd_check_fast_log(double *spread);

/* Host-only check of the Poisson-kernel solver's preconditioner (no GPU
 * needed): builds the smoothed-aggregation multigrid hierarchy of the SPD
 * matrix A (CSR, n rows, columns ascending, diagonal included) and solves
 * A x = b by conjugate gradients with the same V-cycle the device solver runs,
 * to ||b - A x|| <= rtol ||b||.
 *   a_off [n+1], a_col [nnz], a_val [nnz]   host CSR of A
 *   b [n] host right-hand side; x [n] host output
 *   iters, levels   outputs: CG iterations, hierarchy depth
 * Errors: DD_EINVAL (null or n < 1), DD_ENOTCONV (no hierarchy or no
 * convergence within max_iter). */
dd_status dd_multigrid_check(const int64_t *a_off, const int32_t *a_col, const double *a_val, int64_t n,
                             const double *b, double *x, double rtol, int32_t max_iter, int32_t *iters,
                             int32_t *levels);

/* per-path status written by the tracer */
enum {
    DD_TRACE_OK = 0,          /* reached the target                                   */
    DD_TRACE_STUCK = 1,       /* stopped in a local minimum (no descending edge)      */
    DD_TRACE_STEP_LIMIT = 2,  /* walked 4 * n_triangles states without arriving       */
    DD_TRACE_TRUNCATED = 3    /* the polyline would exceed max_pts points             */
};

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int32_t dd_version(void);

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * (NULL = the legacy default stream) on which all work of the context runs.
 * *out receives the context.  Errors: DD_EINVAL (no such device), DD_ECUDA. */
dd_status dd_create(dd_ctx **out, int32_t device, void *cuda_stream);

/* Replace the context stream; later calls enqueue on it. */
dd_status dd_set_stream(dd_ctx *ctx, void *cuda_stream);

/* Free every device and host resource of the context.  NULL is a no-op. */
void dd_destroy(dd_ctx *ctx);

/* Message of the last failing call on this context (never NULL). */
const char *dd_last_error(const dd_ctx *ctx);

/* Block until all work enqueued by the context has finished. */
dd_status dd_sync(dd_ctx *ctx);

/* Host-only mesh validation (no GPU needed).  Checks: ids in range, every
 * triangle counter-clockwise with positive area, manifold edges (at most two
 * triangles, consistently oriented), every vertex used, and boundary loops
 * that cover exactly the vertices of the edges with one incident triangle,
 * consecutive loop vertices joined by such an edge.
 *   xy        host [n_v][2] float64 coordinates
 *   tri       host [n_t][3] int32 vertex ids, counter-clockwise
 *   loop_idx  host [k] int32 boundary vertex ids, loops concatenated
 *   loop_off  host [n_loops + 1] int64 offsets into loop_idx (loop_off[0] = 0)
 *   info      host [4] int64 out: n_v, k, m, number of edges
 *   msg       host buffer of msg_len bytes for a failure message (may be NULL)
 * Errors: DD_EINVAL with the reason in msg. */
dd_status dd_check_mesh(const double *xy, int64_t n_v, const int32_t *tri, int64_t n_t,
                        const int32_t *loop_idx, const int64_t *loop_off, int32_t n_loops,
                        int64_t *info, char *msg, int32_t msg_len);

/* Validate (as dd_check_mesh) and copy a mesh to the device; builds the
 * triangle adjacency, the vertex-to-triangle and vertex-neighbour lists and
 * the cotangent Laplacian (Section IV).  Arguments as in dd_check_mesh, all
 * host memory.  *mesh_id receives the handle.  Errors: DD_EINVAL, DD_ENOMEM,
 * DD_ECUDA. */
dd_status dd_load_mesh(dd_ctx *ctx, const double *xy, int64_t n_v, const int32_t *tri, int64_t n_t,
                       const int32_t *loop_idx, const int64_t *loop_off, int32_t n_loops,
                       int32_t *mesh_id);

/* Release a mesh and everything computed for it. */
dd_status dd_unload_mesh(dd_ctx *ctx, int32_t mesh);

/* Sizes of a loaded mesh: info[0..6] = n_v, n_t, k, m, k_pad (row pitch of P
 * in floats, a multiple of 4), has_poisson_kernel (0/1), device bytes held. */
dd_status dd_mesh_info(dd_ctx *ctx, int32_t mesh, int64_t *info);

/* Solve for the Poisson kernel, Eq. (32)-(33): (-L_II) X = L_IB for all k
 * right-hand sides at once by conjugate gradients in FP64 on the device,
 * preconditioned by a smoothed-aggregation multigrid V-cycle (the diagonal of
 * -L_II on meshes under 256 interior vertices or where no hierarchy can be
 * built), iterating until every column's residual satisfies
 * ||r_b|| <= rtol * ||L_IB e_b|| or max_iter iterations have run.  The result
 * is stored as FP32 P (row pitch k_pad, boundary rows the identity, negative
 * round-off clamped to 0, values below FLT_MIN flushed to 0).  All columns
 * keep iterating until the slowest one meets rtol, so that small entries of
 * P, whose logarithms enter KL, are accurate well beyond rtol.
 *   rtol      relative residual target, > 0 (1e-15 gives KL within 1e-5)
 *   max_iter  iteration cap, > 0
 *   iters     host out (may be NULL): iterations run
 *   resid     host out (may be NULL): largest relative residual at the end
 * Synchronous.  Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA, DD_ENOTCONV (P is
 * still stored, with the residual reported). */
dd_status dd_poisson_kernel(dd_ctx *ctx, int32_t mesh, double rtol, int32_t max_iter,
                            int32_t *iters, double *resid);

/* Install a Poisson kernel computed elsewhere (e.g. a cached copy keyed by
 * the mesh): P is host [n_v][k] float64 row-major in the mesh's vertex and
 * column order.  It is stored exactly as dd_poisson_kernel stores its own
 * result (FP32, clamp and flush).  Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_set_poisson_kernel(dd_ctx *ctx, int32_t mesh, const double *P);

/* Copy the stored FP32 Poisson kernel out, as [n_v][k] (pitch k, no padding).
 * out: device or host.  Errors: DD_ESTATE if none is stored. */
dd_status dd_get_poisson_kernel(dd_ctx *ctx, int32_t mesh, float *out);

/* The Poisson kernel to full relative precision in every entry, however
 * small, and its logarithm (Section V, Precision: on maze-like domains the
 * kernel spans hundreds of orders of magnitude; the paper computes the
 * vectors log P and combines them in the KL sum).  Refines the stored P by
 * FP64 sweeps of the fixed-point form of Eq. (32),
 *   P[i,b] = (sum_{j interior} w_ij P[j,b] + w_ib) / sum_j w_ij,
 * which add non-negative terms only (so each entry keeps its own relative
 * precision), starting from the solver's values where they are at least
 * 2^-30 and from 0 elsewhere, until the largest relative change of an entry
 * over 32 sweeps is at most tol or max_sweeps have run.  Then stores the
 * refined P as before (FP32, values below FLT_MIN flushed to 0) and log2 P
 * in FP32 for every entry (-inf where P is exactly 0).  Afterwards
 * dd_distance (DD_PREC_FP32), dd_query and dd_divergence (reverse KL) take
 * log P[t,b] (KL) and log P[x,b] (KLT) from log2 P wherever the FP32 entry is
 * 0, instead of evaluating the logarithm at FLT_MIN; the split-BF16, sparse,
 * batch and served paths do not.  Needs non-negative edge weights (grids,
 * Delaunay meshes); entries below about 1e-300 underflow FP64.  Holds one
 * more n_v x k_pad FP32 array; recomputing or replacing P discards it, and
 * it discards the split-BF16 and sparse copies of the old P.
 *   tol         relative change at which the sweeps stop (> 0; 1e-14 is typical)
 *   max_sweeps  sweep cap (>= 1)
 *   sweeps, change  NULL or out: sweeps run (largest over column chunks) and
 *               the last relative change
 * Synchronous.  Errors: DD_ESTATE (no Poisson kernel), DD_EINVAL, DD_ENOMEM,
 * DD_ECUDA, DD_ENOTCONV (not below tol within max_sweeps; the result is still
 * stored). */
dd_status dd_log_poisson_kernel(dd_ctx *ctx, int32_t mesh, double tol, int32_t max_sweeps, int32_t *sweeps,
                                double *change);

/* Copy log2 P out (after dd_log_poisson_kernel), as [n_v][k] FP32 (pitch k),
 * -inf where P is exactly 0.  out: device or host.  Errors: DD_ESTATE if
 * none is stored. */
dd_status dd_get_log_poisson_kernel(dd_ctx *ctx, int32_t mesh, float *out);

/* Prepare DD_PREC_SPARSE and DD_PREC_SPARSE_MERGED on this mesh (Section V:
 * the entries of P below a threshold of 1/sqrt(n) are eliminated before the
 * KL sum, about 90 % of them; the paper does not say relative to what --
 * here, relative to each row's largest entry).  Stores theta, the sparsified
 * P as CSR (each row's kept entries in column order: FP32 values, 16-bit
 * column ids, 64-bit row offsets) and the exact total of every stored row
 * (8 bytes per vertex, for the merged-bin extension).  Recomputing or
 * replacing P (dd_poisson_kernel, dd_set_poisson_kernel) discards it.
 *   theta   threshold relative to the row maximum, < 1; negative: 1/sqrt(n_v)
 *   kept    NULL or out: kept entries over all rows (the sparsity is
 *           1 - kept / (n_v k))
 *   bytes   NULL or out: device bytes of the CSR copy
 * Errors: DD_ESTATE before a Poisson kernel exists, DD_EINVAL (theta >= 1 or
 * NaN, k beyond 65,536 columns), DD_ENOMEM, DD_ECUDA. */
dd_status dd_sparsify(dd_ctx *ctx, int32_t mesh, double theta, int64_t *kept, int64_t *bytes);

/* Divergence fields of T target vertices, Eq. (34)-(35):
 *   TV_t(x)  = sum_b |P[x,b] - P[t,b]|
 *   KL_t(x)  = sum_b P[x,b] log(P[x,b] / P[t,b])     (Eq. 17 with z = x, w = t)
 *   KLT_t(x) = sum_b P[t,b] log(P[t,b] / P[x,b])     (Eq. 35 with p = t)
 * with 0 log 0 = 0, for every vertex x.
 *   targets  host [T] interior vertex ids (a boundary target is DD_EINVAL:
 *            its KL row is infinite)
 *   f_mask   any non-empty combination of DD_F_KL, DD_F_TV, DD_F_KLT
 *   prec     DD_PREC_FP32, DD_PREC_BF16X3, DD_PREC_SPARSE or
 *            DD_PREC_SPARSE_MERGED (the last two after dd_sparsify; DD_ESTATE
 *            before)
 *   out      device or host float32 [nf][T][n_v], nf = number of bits set,
 *            blocks in bit order (KL, TV, KLT)
 * In FP32 a log argument below FLT_MIN is taken as FLT_MIN: where P[t,b] = 0
 * but P[x,b] > 0 (a boundary row x of a column with no interior support) the
 * exact KL is +inf and the result is finite and at least 87; KLT is +inf on
 * every boundary row and the result there is at least 50.
 * Memory: the first DD_PREC_FP32 call with T > 2 on a mesh stores a tiled
 * copy of P and of its log2 beside P (2 x 4 n_v k_pad bytes, rounded up to
 * whole tiles; kept until P is recomputed, refined or replaced or the mesh
 * unloaded), and every such call stages its targets in the same layout
 * (context scratch, 8 T k_pad bytes rounded up): the pipelined tile pass
 * reads them.  When either does not fit, the call runs the staged tile
 * shapes instead, which need neither (same fields, bit for bit).
 * Errors: DD_EINVAL, DD_ESTATE (no Poisson kernel), DD_ENOMEM, DD_ECUDA. */
dd_status dd_distance(dd_ctx *ctx, int32_t mesh, const int32_t *targets, int32_t T,
                      uint32_t f_mask, int32_t prec, float *out);

/* Other f-divergences of Section VI, d_f,t(x) = sum_b P[x,b] f(P[t,b]/P[x,b]),
 * each f taken in its form with f(1) = f'(1) = 0 (the same divergence between
 * probability vectors, with non-negative terms):
 *   DD_DIV_CHI2        (u - 1)^2
 *   DD_DIV_HELLINGER   (sqrt(u) - 1)^2
 *   DD_DIV_POWER       |1 - u|^p, param = p >= 1 (p = 1 is TV, p = 2 chi2)
 *   DD_DIV_ALPHA       4/(1-a^2)(1 - u^((1+a)/2)) + 2/(1-a)(u - 1), param = a,
 *                      |a| != 1 (a -> -1 tends to KL, a -> 1 to the reverse KL)
 *   DD_DIV_KL_REVERSE  u log u: sum_b P[t,b] log(P[t,b] / P[x,b])
 * (KL and TV themselves: dd_distance.)  Evaluated in FP32 with exact split
 * logarithms where a log ratio enters (alpha, reverse KL), so d(t,t) = 0.
 * Where the exact value is +inf (P[x,b] = 0 < P[t,b] on boundary rows x for
 * chi2, p > 1, a > 1) the result is at least 1e30 or +inf; for the reverse
 * KL, whose log argument is taken at FLT_MIN there as in dd_distance, it is
 * finite and at least about 80.
 *   targets  host [T] interior vertex ids
 *   out      device or host float32 [T][n_v]
 * Errors: DD_EINVAL (family, param, ids), DD_ESTATE (no Poisson kernel),
 * DD_ENOMEM, DD_ECUDA. */
enum { DD_DIV_CHI2 = 1, DD_DIV_HELLINGER = 2, DD_DIV_POWER = 3, DD_DIV_ALPHA = 4, DD_DIV_KL_REVERSE = 5 };
dd_status dd_divergence(dd_ctx *ctx, int32_t mesh, const int32_t *targets, int32_t T, int32_t family,
                        double param, float *out);

/* Spurious local minima (Section V, "Low resolution discretizations"): for
 * each of T fields, the interior vertices v other than the target with no
 * mesh neighbour of smaller value (f[v] <= f[u] for every neighbour u), where
 * gradient descent can stop.
 *   fields   device float32 [T][n_v] (e.g. dd_distance output)
 *   targets  host [T] vertex ids
 *   counts   host int32 [T]: number of such vertices per field
 *   flags    NULL, or device or host uint8 [T][n_v]: 1 at those vertices
 * Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_local_minima(dd_ctx *ctx, int32_t mesh, const float *fields, const int32_t *targets, int32_t T,
                          int32_t *counts, uint8_t *flags);

/* Edge-following paths (Section IV, the simpler of the two tracers): from
 * each source, move to the neighbour of smallest value among those below the
 * current vertex (ties to the lowest id) until the target (DD_TRACE_OK) or a
 * vertex with no lower neighbour (DD_TRACE_STUCK); DD_TRACE_STEP_LIMIT after
 * n_v moves.  Arguments and outputs as dd_trace_fields (paths are vertex
 * positions). */
dd_status dd_trace_edges(dd_ctx *ctx, int32_t mesh, const float *fields, const int32_t *targets, int32_t T,
                         const int32_t *sources, int32_t S, int32_t max_pts, float *out_xy, int32_t *out_len,
                         int32_t *out_status);

/* Trace gradient-descent paths from S source vertices to `target` on the
 * field of divergence f (DD_F_KL or DD_F_TV), evaluated in FP32 (Section IV).
 *   sources     host [S] vertex ids
 *   max_pts     capacity of each polyline in points (>= 2)
 *   out_xy      device or host float32 [S][max_pts][2]; path s occupies the
 *               first out_len[s] points, starting at the source vertex and,
 *               when the status is DD_TRACE_OK, ending at the target vertex;
 *               the points past out_len[s] are unspecified (into host memory
 *               only the defined prefixes are copied)
 *   out_len     device or host int32 [S]
 *   out_status  device or host int32 [S], DD_TRACE_* codes
 * Errors: DD_EINVAL, DD_ESTATE, DD_ENOMEM, DD_ECUDA. */
dd_status dd_trace(dd_ctx *ctx, int32_t mesh, int32_t target, uint32_t f,
                   const int32_t *sources, int32_t S, int32_t max_pts,
                   float *out_xy, int32_t *out_len, int32_t *out_status);

/* Trace T x S paths on caller-supplied fields (any scalar per vertex whose
 * minimum is at the target, e.g. a field from dd_distance).
 *   fields      device float32 [T][n_v] (row a is the field of targets[a])
 *   targets     host [T] vertex ids
 *   sources     host [T][S] vertex ids
 *   outputs as dd_trace with T * S paths, path (a, s) at index a * S + s.
 * Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_trace_fields(dd_ctx *ctx, int32_t mesh, const float *fields,
                          const int32_t *targets, int32_t T, const int32_t *sources, int32_t S,
                          int32_t max_pts, float *out_xy, int32_t *out_len, int32_t *out_status);

/* One pass of the whole online path for a batch: the fields of every target
 * (dd_distance with f_mask, prec) and the T x S paths traced on the field of
 * divergence trace_f (one bit of f_mask).  Outputs as dd_distance (fields)
 * and dd_trace_fields (paths); each may be device or host memory.  Host
 * outputs are copied back before the call returns. */
dd_status dd_query(dd_ctx *ctx, int32_t mesh, const int32_t *targets, int32_t T,
                   const int32_t *sources, int32_t S, uint32_t f_mask, int32_t prec,
                   uint32_t trace_f, int32_t max_pts, float *out_fields,
                   float *out_xy, int32_t *out_len, int32_t *out_status);

/* Fields and paths for targets on several loaded meshes in one pass (a batch
 * of uneven domains).  Item i is mesh mesh_ids[i] with T_per[i] targets; the
 * fields of all items are computed by one persistent launch, then the paths
 * of all items by one tracer launch.  The launch is staged (each item in the
 * tile shape the autotuner picks for it) or pipelined (every item in 128 x 64
 * tiles on the meshes' tiled copies of P, as dd_distance builds them: 2 x 4
 * n_v k_pad bytes per mesh, kept with the mesh; without room for them the
 * launch stays staged), whichever the autotuner measured faster for the
 * class of the batch (dd_tuning_table).  Same arithmetic as dd_query with
 * FP32: both launches give the same fields, bit for bit.
 *   n_items   number of items (>= 1)
 *   mesh_ids  host [n_items] loaded meshes with a Poisson kernel
 *   T_per     host [n_items] targets per item (>= 1)
 *   targets   host [sum T] interior vertex ids, item after item
 *   sources   host [sum T][S] vertex ids (ignored when S = 0)
 *   S         sources per target (0: fields only)
 *   f_mask    DD_F_KL | DD_F_TV;  trace_f: one bit of f_mask (when S > 0)
 *   out_fields  device or host float32: item i's block [nf][T_i][n_i] starts
 *             at sum_{j<i} nf T_j n_j
 *   out_xy, out_len, out_status  as dd_trace_fields over sum T x S paths in
 *             target order (may be NULL when S = 0)
 * The first call that meets a new (size, k, T) class runs timed launches of
 * each tile shape before the batch, and the first that meets a new class of
 * batches (f_mask, items and sum n k T in powers of two) a warm-up and two timed
 * runs of each of the two launches, on the context's stream, synchronizing
 * with it.  Errors: DD_EINVAL, DD_ESTATE, DD_ENOMEM, DD_ECUDA, DD_ETIMEOUT. */
dd_status dd_query_batch(dd_ctx *ctx, int32_t n_items, const int32_t *mesh_ids, const int32_t *T_per,
                         const int32_t *targets, const int32_t *sources, int32_t S, uint32_t f_mask,
                         uint32_t trace_f, int32_t max_pts, float *out_fields, float *out_xy,
                         int32_t *out_len, int32_t *out_status);

/* The autotuner's decisions so far as text, one line per size class
 * ("rows<=2^r k_pad<=2^c T<=2^t: 64x64"; "... (tiled copy of P): 128x64
 * pipelined" for single-domain calls that had the tiled copy) and one per
 * class of batches ("batch of problems<=2^p n*k*T<=2^w (KL+TV): pipelined
 * persistent launch").  Writes at most len bytes (NUL terminated) into buf
 * (may be NULL) and returns the full length. */
int32_t dd_tuning_table(char *buf, int32_t len);

/* Per-kernel device time on the context's stream (an observability hook; the
 * paper has no counterpart).  While enabled, every kernel the library
 * launches on that stream is bracketed by two CUDA events; the totals per
 * kernel name are folded in when read.
 *   mode  1: enable (or reset the totals); 2: read; 0: read, then disable
 *   buf   NULL or host text, one line per kernel: "name launches total_ms"
 * Returns the text length + 1 (the size buf needs), DD_EINVAL for a bad mode.
 * Reading synchronizes with the recorded events.  Keyed by the stream the
 * context had when timing was enabled. */
int32_t dd_kernel_timing(dd_ctx *ctx, int32_t mode, char *buf, int32_t len);

/* Latency of one dependent global load (a measurement hook for the floor of
 * the path walk, a chain of dependent gathers; the paper has no counterpart).
 * One thread follows a seeded random cycle through `bytes` of device memory,
 * one 4-byte index at the head of every 128-byte line, each load's address
 * the value the previous one returned, with L1 bypassed: after a warm-up a
 * buffer that fits L2 times an L2 hit, a much larger one a DRAM access.
 * Allocates its buffer (and the host copy of the cycle) and frees both.
 *   bytes        4096 .. 2^32, a multiple of 128
 *   steps        timed loads (>= 1)
 *   ns_per_load  out: CUDA-event time of the timed loads / steps
 * Runs on the context's stream and synchronizes with it.
 * Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_load_latency(dd_ctx *ctx, int64_t bytes, int32_t steps, double *ns_per_load);

/* ---- query server: continuous batching of path queries ------------------
 * A query asks for the paths from S sources to one interior target of a
 * loaded mesh, traced on the target's KL field (Section IV).  A server runs a
 * worker thread that keeps up to n_slots batches in flight, each on its own
 * CUDA stream: whenever a slot is free it takes the queries that have
 * arrived (in arrival order, up to max_batch and what fits the slot), groups
 * them by mesh and runs one staging, one persistent field launch and one
 * tracer launch for all of them, then copies the paths to host memory.
 * Queries arriving while batches run join the next batch, whose work
 * overlaps on the device with the running ones.  The device budget is split
 * evenly over the slots and allocated at creation; nothing is allocated on
 * the device while serving.  While a server runs, meshes of its context must
 * stay loaded and other calls on the context must not run concurrently. */
typedef struct dd_server dd_server;

/* budget_bytes: device memory for the slots (>= 1 MiB); n_slots 1..16;
 * max_batch: queries per batch (>= 1); max_pts: polyline capacity (>= 2).
 * Errors: DD_EINVAL, DD_ENOMEM, DD_ECUDA. */
dd_status dd_server_create(dd_ctx *ctx, int64_t budget_bytes, int32_t n_slots, int32_t max_batch,
                           int32_t max_pts, dd_server **out);

/* Enqueue a query (thread-safe, returns at once).  sources: host [S] vertex
 * ids, copied.  query_id must be unique among unreleased queries.  Errors:
 * DD_EINVAL (ids), DD_ESTATE (no Poisson kernel), DD_EBUDGET (the query can
 * never fit one slot). */
dd_status dd_server_submit(dd_server *sv, int64_t query_id, int32_t mesh, int32_t target,
                           const int32_t *sources, int32_t S);

/* Report up to max_n queries completed since the last poll: ids, their
 * status (DD_OK or an error) and latency in ms from submission to the paths
 * being in host memory.  Returns how many were written (0 if none). */
int32_t dd_server_poll(dd_server *sv, int32_t max_n, int64_t *ids, int32_t *statuses, double *latency_ms);

/* Copy out and release a completed query: xy host [S][max_pts][2] (path s
 * in the first len[s] points of its row; the points past len[s] are left
 * untouched), len and status host [S] (any may be NULL).  Returns the query's
 * status, or DD_ESTATE if it is not complete (or already released). */
dd_status dd_server_take(dd_server *sv, int64_t query_id, float *xy, int32_t *len, int32_t *status);

/* Block until no query is pending or in flight, or timeout_s passed
 * (DD_ETIMEOUT). */
dd_status dd_server_wait_idle(dd_server *sv, double timeout_s);

/* Finish all queries, stop the worker and free the server. */
void dd_server_destroy(dd_server *sv);

/* dd_distance without any device allocation.  The paper has no counterpart:
 * this is a deployment variant of dd_distance for callers that may not call
 * cudaMalloc -- e.g. a robot's real-time control loop that allocates only at
 * start-up, because an allocation can stall the device and overrun the
 * loop's deadline, or a plugin whose host framework owns all device memory.
 * The caller passes everything in its own device memory; no context is used.
 *   P        device float32 [n_v][k_pad] Poisson kernel (e.g. copied from
 *            dd_get_poisson_kernel and padded), k_pad a multiple of 4 with
 *            zero padding columns, 16-byte aligned
 *   targets  device int32 [T] interior vertex ids, 4-byte aligned.  An id
 *            outside [0, n_v) is detected on the device: it is never used
 *            as a row index, and the call returns DD_EINVAL (the output is
 *            then unspecified)
 *   f_mask   DD_F_KL | DD_F_TV as in dd_distance
 *   out      device float32 [nf][T][n_v], layout as in dd_distance, 4-byte
 *            aligned
 *   cuda_stream  stream for the work (NULL = legacy default stream)
 * The fields equal dd_distance's bit for bit.  Nothing is timed or tuned:
 * for T > 2 the tile shape is a fixed function of T (dd_distance's autotuner
 * would run timed launches the first time it meets a size class).
 * Scratch: one fixed device array per GPU (16 MiB, held until the process
 * exits) holds the staged target rows, so T * k_pad must not exceed 1,048,576
 * (DD_EINVAL otherwise).  Every call shares that array: calls whose work
 * overlaps on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The first call on a device looks up the array's
 * device address; make that first call before any stream capture.  The call
 * returns after the work finished (it synchronises the stream).
 * Errors: DD_EINVAL (sizes, alignment, an id out of range), DD_ECUDA,
 * DD_ETIMEOUT (a bounded device wait gave up). */
dd_status dd_distance_noalloc(const float *P, int64_t n_v, int64_t k_pad, const int32_t *targets,
                              int32_t T, uint32_t f_mask, float *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DD_H */
