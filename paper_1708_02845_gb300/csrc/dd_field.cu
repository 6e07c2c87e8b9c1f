// TV and KL divergence fields in FP32, Section IV Eq. (34)-(35).
//
//   TV_t(x) = sum_b |P[x,b] - P[t,b]|
//   KL_t(x) = sum_b P[x,b] (log P[x,b] - log P[t,b])      (Eq. 17, z = x, w = t)
//
// Near the target the two logarithms agree to many digits and KL is a small
// sum of nearly-cancelling terms, so each log is kept as an exact split
//   log p = E ln2 + lm,   E integer,  lm = log(m) for the mantissa m in [1, 2)
// and the difference is formed as (lm_x - lm_t) + (E_x - E_t) ln2: lm < 0.7
// carries an absolute error below 2^-25, the exponent difference is exact,
// and x = t gives exactly 0 (the same code runs on both operands).  lm is
// table driven (Tang, "Table-driven implementation of the logarithm function
// in IEEE floating-point arithmetic", ACM TOMS 1990): a 128-entry table of
// r_j = 1/c_j and log c_j over [1, 2) indexed by the top 7 mantissa bits,
// u = m r_j - 1 (|u| <= 2^-8, one rounding) and log(1 + u) from its degree-3
// Taylor polynomial (truncation |u|^4/4 <= 2^-34, far below the final
// rounding of lm).  The table is computed in FP64 by each CTA.  Every step
// uses explicit round-to-nearest operations so all call sites produce
// bit-identical values.  Target-side arguments below FLT_MIN are evaluated
// at FLT_MIN; row-side terms with P[x,b] = 0 contribute 0 (the 0 log 0 rule).
//
// The kernels:
//  * field_stream (few targets): one warp per group of R rows, lanes along b,
//    16-byte loads of P software-pipelined U float4 per lane and row ahead
//    of the arithmetic, the target row and its logs staged in shared memory
//    by a bulk async copy completing on an mbarrier, a lane-replicated copy
//    of the log table (no bank conflicts), warp-shuffle reductions.
//  * field_tile (many targets): TM rows x TN targets per CTA, b in chunks of
//    32 staged through shared memory, register micro-tiles.  Each P element's
//    base-2 logarithm is formed once per CTA as one FP32 number and reused for
//    TN targets (one subtraction and one multiply-add per KL term).
//  * field_tile_pipe (many targets, one domain) and batch_pipe (many
//    domains): the same sums on a tiled copy of P and of its log2, streamed
//    through shared memory by bulk copies in stages of 64 columns, no
//    staging arithmetic in the loop, FP32x2 over target pairs.
//  * fix_kl_rows: the (row, target) pairs whose first-pass KL lands below
//    DD_TILE_EXACT_BELOW recomputed in the exact split form, by row blocks.
#include <algorithm>
#include <vector>
#include <type_traits>
#include <string>
#include <cstdio>
#include <tuple>
#include <mutex>
#include <map>
#include <cfloat>
#include <cstdint>
#include <cstdlib>

#include "dd_internal.h"
#include "dd_bulk.cuh"
#include "dd_f32x2.cuh"
#include "dd_splitlog.cuh"

namespace {

constexpr float kLn2 = 0.693147180559945309f;

// one term of each sum; accumulators updated in place
__device__ __forceinline__ void accumulate(float px, float lmx, float ex, float pt, float lmt, float et,
                                           float &kl, float &tv) {
    const float d = __fadd_rn(lmx, -lmt);
    const float de = __fadd_rn(ex, -et);
    const float lr = __fmaf_rn(de, kLn2, d);          // log(P_x / P_t)
    kl = __fmaf_rn(px, lr, kl);
    tv = __fadd_rn(tv, fabsf(__fadd_rn(px, -pt)));
}

// the KL term alone (the same operations as in accumulate)
__device__ __forceinline__ void accumulate_kl(float px, float lmx, float ex, float lmt, float et, float &kl) {
    const float d = __fadd_rn(lmx, -lmt);
    const float de = __fadd_rn(ex, -et);
    kl = __fmaf_rn(px, __fmaf_rn(de, kLn2, d), kl);
}

// stage_P / stage_L / stage_E / stage_F: [T][k_pad] target row, its mantissa
// log (table), biased exponent and mantissa log2 (hardware), the target-side
// arguments clamped at FLT_MIN.  One CTA per target, so that the log table
// (FP64, slow on this part) is built once per target row.  A target id
// outside [0, n_v) reads nothing: its staged rows are zero-filled and
// *bad_id (when given) is set to 1.
__global__ void stage_targets_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                     const int32_t *__restrict__ targets, int32_t T, float *__restrict__ sP,
                                     float *__restrict__ sL, float *__restrict__ sE, float *__restrict__ sF,
                                     int *__restrict__ bad_id, const float *__restrict__ LP) {
    __shared__ float tab[2 * kLogTab];
    build_log_table(tab);
    __syncthreads();
    const int a = blockIdx.x;
    if (a >= T) return;
    const int64_t o = (int64_t)a * k_pad;
    const int32_t t = targets[a];
    if (t < 0 || (int64_t)t >= n_v) {
        if (threadIdx.x == 0 && bad_id) atomicExch(bad_id, 1);
        for (int64_t b = threadIdx.x; b < k_pad; b += blockDim.x) sP[o + b] = sL[o + b] = sE[o + b] = sF[o + b] = 0.0f;
        return;
    }
    const float *row = P + (int64_t)t * k_pad;
    const float *lrow = LP ? LP + (int64_t)t * k_pad : nullptr;
    for (int64_t b = threadIdx.x; b < k_pad; b += blockDim.x) {
        const float p = row[b];
        float lm, E, F;
        const float l2 = (lrow && p == 0.0f) ? lrow[b] : -INFINITY;
        if (l2 > -INFINITY) {
            // an entry below FLT_MIN with a known logarithm: log2 p = e + f, e integer, f in [0, 1)
            const float e = floorf(l2);
            F = __fsub_rn(l2, e);
            lm = __fmul_rn(F, kLn2);
            E = __fadd_rn(12583039.0f, e);        // the biased-float exponent of split_log (exact)
        } else {
            split_log<true>(p, tab, lm, E);
            F = lg2_mant(__float_as_int(fmaxf(p, FLT_MIN)));
        }
        sP[o + b] = p;
        sL[o + b] = lm;
        sE[o + b] = E;
        sF[o + b] = F;
    }
}

// ------------------------------------------------------------------ few targets
// streaming 16-byte load, issued where it is written (the asm is volatile and
// ordered against the shared-memory reads that follow it)
__device__ __forceinline__ float4 ld_stream(const float4 *p) {
    float4 v;
    asm volatile("ld.global.cs.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

// Error bound of the fast pass.  DD_FAST_LOG_SPREAD bounds max - min of the
// error of lg2_mant over [1, 2) (base-2 units; about 3.2e-7 measured,
// dd_check_fast_log re-measures it).  A row's fast KL then differs from the
// exact split form by at most ln2 * spread * sum_b P[x,b] = ln2 * spread: the
// constant part of the error cancels between the row and target sides.  Rows
// whose fast KL lies below DD_EXACT_BELOW are recomputed with the table
// logarithm, so every row meets 1e-5 relative: ln2 * 5e-7 / 0.05 = 7e-6.
constexpr float kExactBelow = (float)DD_EXACT_BELOW;
constexpr float kTileExactBelow = (float)DD_TILE_EXACT_BELOW;

// exact (table) KL of row x for one warp, from the staged target arrays
__device__ __forceinline__ float kl_row_exact(const float *__restrict__ P, int64_t x, int64_t k_pad, int nvec,
                                              const float *tP, const float *tL, const float *tE, const float *tab,
                                              int lane) {
    const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
    float k0 = 0.0f, k1 = 0.0f;
#pragma unroll 3
    for (int c = lane; c < nvec; c += 32) {
        const float4 v = __ldcg(row + c);
        const float4 p4 = reinterpret_cast<const float4 *>(tP)[c];
        const float4 l4 = reinterpret_cast<const float4 *>(tL)[c];
        const float4 e4 = reinterpret_cast<const float4 *>(tE)[c];
        const float px[4] = {v.x, v.y, v.z, v.w}, pt[4] = {p4.x, p4.y, p4.z, p4.w};
        const float lt[4] = {l4.x, l4.y, l4.z, l4.w}, et[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float lm, Eb, tvd = 0.0f;
            split_log<false>(px[q], tab, lm, Eb);
            accumulate(px[q], lm, Eb, pt[q], lt[q], et[q], (q & 1) ? k1 : k0, tvd);
        }
    }
    float skl = k0 + k1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) skl += __shfl_xor_sync(0xffffffffu, skl, o);
    return skl;
}

// One target per grid row (blockIdx.y).  Dynamic smem: the target's four
// k_pad arrays (P, lm, E, lg2 m) from one bulk copy each; static smem: the
// log table for the exact recompute.  Each warp streams rows; per (row,
// chunk of 32 U float4 columns) every lane loads U float4.  Two register
// buffers alternate, so the loads of the next (row, chunk) are in flight
// while the current one is computed.
//
// Fast pass per element: log2 P[x,b] - log2 P[t,b] = (lg2 m_x - lg2 m_t) +
// (E_x - E_t), the exponent difference exact and the mantissa logs from the
// hardware (lg2_mant); KL = ln2 * sum.  TV is exact.  A row whose KL is below
// kExactBelow (the rows near the target, x = t among them) is recomputed
// with the exact split form by its warp.
template <int U>
__global__ void __launch_bounds__(256, 2) field_stream_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                                              const float *__restrict__ sP, const float *__restrict__ sL,
                                                              const float *__restrict__ sE, const float *__restrict__ sF,
                                                              int32_t T, float *__restrict__ out_kl,
                                                              float *__restrict__ out_tv, int *__restrict__ err_flag) {
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float tab[2 * kLogTab];
    float *tP = smem;
    float *tL = tP + k_pad;
    float *tE = tL + k_pad;
    float *tF = tE + k_pad;
    const int a = blockIdx.y;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t row_bytes = (uint32_t)(k_pad * sizeof(float));
        mbar_expect_tx(&bar, 4u * row_bytes);
        bulk_g2s(tP, sP + (int64_t)a * k_pad, row_bytes, &bar);
        bulk_g2s(tL, sL + (int64_t)a * k_pad, row_bytes, &bar);
        bulk_g2s(tE, sE + (int64_t)a * k_pad, row_bytes, &bar);
        bulk_g2s(tF, sF + (int64_t)a * k_pad, row_bytes, &bar);
    }
    build_log_table(tab);
    __syncthreads();
    if (!mbar_wait(&bar, 0, err_flag)) {
        // a CTA whose wait gave up must not return while its copies may still land:
        // wait once more (also bounded) before exiting
        mbar_wait(&bar, 0, err_flag);
        return;
    }

    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nvec = (int)(k_pad >> 2);                    // float4 per row
    const int64_t nchunk = (nvec + 32 * U - 1) / (32 * U);
    const int64_t nfull = nvec / (32 * U);                 // chunks with every lane's U float4 in the row
    float *okl = out_kl ? out_kl + (int64_t)a * n_v : nullptr;
    float *otv = out_tv ? out_tv + (int64_t)a * n_v : nullptr;
    const float4 *tP4 = reinterpret_cast<const float4 *>(tP) + lane;
    const float4 *tF4 = reinterpret_cast<const float4 *>(tF) + lane;
    const float4 *tE4 = reinterpret_cast<const float4 *>(tE) + lane;

    float4 buf[2][U];
    f2_t kl = 0ULL, tv = 0ULL;

    auto fetch = [&](float4(&b)[U], int64_t x, int64_t ch) {
        const int c0 = (int)ch * 32 * U;
        const bool full = ch < nfull;
        const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad) + c0 + lane;
#pragma unroll
        for (int u = 0; u < U; ++u)
            b[u] = (full || c0 + u * 32 + lane < nvec) ? ld_stream(row + u * 32) : make_float4(0.f, 0.f, 0.f, 0.f);
    };
    // one item; FULL: every lane's U float4 lie inside the row (no per-u test)
    auto compute = [&](const float4(&b)[U], int64_t ch, auto full_tag) {
        constexpr bool FULL = decltype(full_tag)::value;
        const f2_t mone = pk(-1.0f, -1.0f);
        const int c0 = (int)ch * 32 * U;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!FULL && c0 + u * 32 + lane >= nvec) break;
            const float4 p4 = tP4[c0 + u * 32];
            const float4 f4 = tF4[c0 + u * 32];
            const float4 e4 = tE4[c0 + u * 32];
            const float px[4] = {b[u].x, b[u].y, b[u].z, b[u].w};
            float lf[4], eb[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = __float_as_int(px[q]);
                lf[q] = lg2_mant(i);
                eb[q] = __int_as_float((int)__funnelshift_r((unsigned)i, (unsigned)kMagicHi, 23));
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const f2_t p2 = pk(px[2 * h], px[2 * h + 1]);
                const f2_t pt2 = h ? pk(p4.z, p4.w) : pk(p4.x, p4.y);
                const f2_t ft2 = h ? pk(f4.z, f4.w) : pk(f4.x, f4.y);
                const f2_t et2 = h ? pk(e4.z, e4.w) : pk(e4.x, e4.y);
                const f2_t d = fma2(ft2, mone, pk(lf[2 * h], lf[2 * h + 1]));
                const f2_t de = fma2(et2, mone, pk(eb[2 * h], eb[2 * h + 1]));
                kl = fma2(p2, add2(d, de), kl);
                tv = add2(tv, fma2(pt2, mone, p2) & 0x7fffffff7fffffffULL);
            }
        }
    };
    auto finish = [&](int64_t x) {
        float k0, k1, t0v, t1v;
        upk(kl, k0, k1);
        upk(tv, t0v, t1v);
        float skl = k0 + k1, stv = t0v + t1v;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            skl += __shfl_xor_sync(0xffffffffu, skl, o);
            stv += __shfl_xor_sync(0xffffffffu, stv, o);
        }
        skl *= kLn2;
        if (okl && skl < kExactBelow)   // warp-uniform: every lane holds the same sum
            skl = kl_row_exact(P, x, k_pad, nvec, tP, tL, tE, tab, lane);
        if (lane == 0) {
            if (okl) okl[x] = skl;
            if (otv) otv[x] = stv;
        }
        kl = tv = 0ULL;
    };
    // (row, chunk) items in order: row x = warp, warp + nwarps, ...
    auto advance = [&](int64_t &x, int64_t &ch) {
        if (++ch == nchunk) {
            ch = 0;
            x += nwarps;
        }
    };
    int64_t x = warp, ch = 0;     // item being computed
    int64_t xf = warp, chf = 0;   // next item to fetch
    if (x >= n_v) return;
    fetch(buf[0], xf, chf);
    advance(xf, chf);
    for (;;) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (xf < n_v) fetch(buf[s ^ 1], xf, chf);
            advance(xf, chf);
            if (ch < nfull)
                compute(buf[s], ch, std::true_type());
            else
                compute(buf[s], ch, std::false_type());
            if (ch == nchunk - 1) finish(x);
            advance(x, ch);
            if (x >= n_v) return;
        }
    }
}

// ------------------------------------------------------------------ many targets
// Tile shapes: TM rows x TN targets per CTA, 256 threads arranged as
// (TM/RM) row groups x (TN/CN) target groups, each thread an RM x CN micro-tile.
// b runs in chunks of BK = 32 staged through shared memory.  Wide target
// tiles suit many targets; tall row tiles waste less on few targets.
constexpr int kTileB = 32;

template <int TM, int TN, int RM, int CN>
struct TileShape {
    static constexpr int ROWG = TM / RM, COLG = TN / CN;
    static_assert(ROWG * COLG == 256, "256 threads");
    // transposed chunk arrays, the raw chunk buffer and the log table
    static constexpr size_t smem_bytes =
        (2 * kTileB * (TM + TN) + (kTileB + 4) * (TM + TN) + 2 * kLogTab) * sizeof(float);
};

// N consecutive floats from shared memory in 16-byte (or 8-byte) loads; src
// is aligned to 4 N bytes (N a multiple of 4) or 8 bytes (N = 2)
template <int N>
__device__ __forceinline__ void lds_vec(float (&dst)[N], const float *src) {
    if constexpr (N % 4 == 0) {
#pragma unroll
        for (int i = 0; i < N / 4; ++i) {
            const float4 v = reinterpret_cast<const float4 *>(src)[i];
            dst[4 * i] = v.x;
            dst[4 * i + 1] = v.y;
            dst[4 * i + 2] = v.z;
            dst[4 * i + 3] = v.w;
        }
    } else {
        static_assert(N == 2, "micro-tile widths 2, 4, 8");
        const float2 v = *reinterpret_cast<const float2 *>(src);
        dst[0] = v.x;
        dst[1] = v.y;
    }
}

// one output tile (rows x0.., targets a0..) of one problem; tsm holds the
// staging arrays.  KL / TV: which sums to form (a TV-only tile skips the
// logarithms).
//
// KL first pass: each P element's base-2 logarithm is formed once as one FP32
// number, fast_l2 = E + lg2 m (hardware mantissa log), so a term costs one
// subtraction and one multiply-add.  Against the exact split form a row's
// first-pass KL (in nats) errs by at most ln2 * DD_FAST_LOG_SPREAD (the
// varying part of the mantissa log's error; its constant part cancels) plus
// 2^-24 (2 ln k + 2 KL + 2): each logarithm rounds to half an ulp of its
// magnitude, sum_b P[x,b] |log P[x,b]| <= ln k, sum_b P[x,b] |log P[t,b]| =
// that entropy + KL, and the subtraction rounds relative to |log ratio|,
// whose P[x,b]-weighted sum is at most KL + 2.  Every (row, target) pair
// whose first-pass KL lies below kTileExactBelow -- the rows around each
// target, x = t among them -- is then recomputed by one warp with the table
// logarithm (fix_kl_rows_kernel), so every value keeps 1e-5
// relative accuracy.
//
// The target side's one-number log2 comes from the staged exponent and
// hardware mantissa log (sE, sF) when they are given -- bit for bit the value
// fast_l2 forms from the entry, and for an entry below FLT_MIN with a known
// logarithm (log2 P from dd_log_poisson_kernel) that logarithm instead of
// the clamp -- else from the staged entry itself (the multi-domain launch).
// Data movement (the arithmetic and its order are those of a plain loop over
// the columns in 64-column partial sums).  Each 32-column chunk of the row
// tile and of the target tile is
// fetched by cp.async into a raw buffer (rows of 32 floats at a pitch of 36,
// so that the transposing reads below hit different banks) while the
// previous chunk is being summed; after a barrier every thread transposes
// its share into [column][row] and [column][target] arrays, forming the
// logarithms on the way, and the tile is summed from there.  The transposed
// arrays are stored with an XOR swizzle of 4-element groups by column
// (group ^ (b / F) * (F / 4), F the elements per thread and chunk), so that
// the threads sharing a row or target write to different banks, while every
// 4-element group stays contiguous for the 16-byte reads of the sums.
constexpr int kRawPitch = kTileB + 4;

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
                 "r"(valid ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// position of element e (row or target) at chunk column b in a transposed
// array of N elements per column, F elements per thread and chunk
template <int N, int F>
__device__ __forceinline__ int swz(int e, int b) {
    constexpr int S = F / 4;                         // 0 for F = 2: no swizzle
    return ((((e >> 2) ^ ((b / F) * S)) & (N / 4 - 1)) << 2) | (e & 3);
}

template <int TM, int TN, int RM, int CN, bool KL = true, bool TV = true>
__device__ __forceinline__ void tile_body(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                          const float *__restrict__ sP, const float *__restrict__ sL,
                                          const float *__restrict__ sE, const float *__restrict__ sF, int32_t T,
                                          float *__restrict__ out_kl, float *__restrict__ out_tv, int64_t x0, int a0,
                                          float *tsm, const float *tab) {
    constexpr int COLG = TN / CN;
    constexpr int FR = TM * kTileB / 256;     // row floats per thread per chunk (multiple of 4)
    constexpr int FT = TN * kTileB / 256;     // target floats per thread per chunk (2, 4 or 8)
    static_assert(RM % 4 == 0 && FR % 4 == 0, "16-byte row groups");
    float *xP = tsm;                          // [kTileB][TM], swizzled
    float *xL = tsm + 1 * kTileB * TM;
    float *yP = tsm + 2 * kTileB * TM;        // [kTileB][TN], swizzled
    float *yL = tsm + 2 * kTileB * TM + 1 * kTileB * TN;
    float *rX = tsm + 2 * kTileB * (TM + TN);   // raw [TM][kRawPitch]
    float *rY = rX + TM * kRawPitch;            // raw [TN][kRawPitch]
    const int tid = threadIdx.x;
    const int tx = tid % COLG;        // target group: targets tx*CN ..
    const int ty = tid / COLG;        // row group: rows ty*RM ..
    (void)sL;

    // raw copies of the chunk at column b0: 8 threads per 128-byte row segment
    auto fetch = [&](int64_t b0) {
        for (int f = tid; f < TM * 8; f += 256) {
            const int r = f >> 3, c4 = f & 7;
            const int64_t x = x0 + r, b = b0 + 4 * c4;
            const bool ok = x < n_v && b < k_pad;
            cp_async16(rX + r * kRawPitch + 4 * c4, ok ? P + x * k_pad + b : P, ok);
        }
        for (int f = tid; f < TN * 8; f += 256) {
            const int a = f >> 3, c4 = f & 7;
            const int ag = a0 + a;
            const int64_t b = b0 + 4 * c4;
            const bool ok = ag < T && b < k_pad;
            cp_async16(rY + a * kRawPitch + 4 * c4, ok ? sP + (int64_t)ag * k_pad + b : sP, ok);
        }
        cp_async_commit();
    };

    // two-level summation: 64-term sums (two chunks), added into the totals
    // with a compensated (Kahan) sum for KL, whose terms partly cancel
    float kl[RM][CN], tv[RM][CN], klc[RM][CN];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < CN; ++c) kl[r][c] = tv[r][c] = klc[r][c] = 0.0f;

    // partial sums over two chunks (64 columns) between merges
    float ckl[RM][CN], ctv[RM][CN];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < CN; ++c) ckl[r][c] = ctv[r][c] = 0.0f;
    fetch(0);
    for (int64_t b0 = 0; b0 < k_pad; b0 += kTileB) {
        cp_async_wait_all();
        __syncthreads();        // the raw chunk has landed; the previous chunk's sums are done
        {
            // this thread's columns cb .. cb + FR - 1 share one swizzle: one base offset
            constexpr int TPR = kTileB / FR;
            const int r = tid / TPR, cb = (tid % TPR) * FR;
            float *bx = xP + cb * TM + swz<TM, FR>(r, cb);
            float *bl = xL + cb * TM + swz<TM, FR>(r, cb);
#pragma unroll
            for (int e = 0; e < FR; e += 4) {
                const float4 v4 = *reinterpret_cast<const float4 *>(rX + r * kRawPitch + cb + e);
                const float vals[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    bx[(e + q) * TM] = vals[q];
                    if (KL) bl[(e + q) * TM] = fast_l2(vals[q]);
                }
            }
        }
        {
            constexpr int TPT = kTileB / FT;
            const int a = tid / TPT, cb = (tid % TPT) * FT;
            const int ag = a0 + a;
            const int ot = cb * TN + swz<TN, FT>(a, cb);
#pragma unroll
            for (int e = 0; e < FT; e += 2) {
                const float2 p2 = *reinterpret_cast<const float2 *>(rY + a * kRawPitch + cb + e);
                const float pv[2] = {p2.x, p2.y};
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int b = cb + e + q, o = ot + (e + q) * TN;
                    yP[o] = pv[q];
                    if (KL) {
                        if (sF) {
                            // staged exponent and mantissa log2 (entries below FLT_MIN with a known log)
                            float ev = 12583039.0f, fv = 0.0f;
                            if (ag < T && b0 + b < k_pad) {
                                ev = __ldg(sE + (int64_t)ag * k_pad + b0 + b);
                                fv = __ldg(sF + (int64_t)ag * k_pad + b0 + b);
                            }
                            yL[o] = __fadd_rn(__fsub_rn(ev, 12583039.0f), fv);
                        } else {
                            yL[o] = fast_l2(fmaxf(pv[q], FLT_MIN));
                        }
                    }
                }
            }
        }
        __syncthreads();        // the chunk is transposed; the raw buffer is free
        if (b0 + kTileB < k_pad) fetch(b0 + kTileB);
        // columns in groups of G, inside which both swizzles are constant: the
        // swizzled offsets are formed once per group, the columns' addresses
        // are then fixed offsets from them
        constexpr int GR = FR >= kTileB ? kTileB : FR;                  // rows: constant over GR columns
        constexpr int GT = (FT < 4 || FT >= kTileB) ? kTileB : FT;     // targets (FT = 2: no swizzle)
        constexpr int G = GR < GT ? GR : GT;
#pragma unroll
        for (int bb = 0; bb < kTileB; bb += G) {
            int ro[RM / 4], co[CN % 4 == 0 ? CN / 4 : 1];
#pragma unroll
            for (int i = 0; i < RM / 4; ++i) ro[i] = bb * TM + swz<TM, FR>(ty * RM + 4 * i, bb);
            if constexpr (CN % 4 == 0) {
#pragma unroll
                for (int i = 0; i < CN / 4; ++i) co[i] = bb * TN + swz<TN, FT>(tx * CN + 4 * i, bb);
            } else {
                static_assert(CN == 2 && FT == 2, "micro-tile widths 2 (unswizzled), 4, 8");
                co[0] = bb * TN + tx * CN;
            }
#pragma unroll
            for (int j = 0; j < G; ++j) {
                float rP[RM], rL[RM], cP[CN], cL[CN];
#pragma unroll
                for (int i = 0; i < RM / 4; ++i) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(xP + ro[i] + j * TM);
                    rP[4 * i] = p4.x;
                    rP[4 * i + 1] = p4.y;
                    rP[4 * i + 2] = p4.z;
                    rP[4 * i + 3] = p4.w;
                    if (KL) {
                        const float4 l4 = *reinterpret_cast<const float4 *>(xL + ro[i] + j * TM);
                        rL[4 * i] = l4.x;
                        rL[4 * i + 1] = l4.y;
                        rL[4 * i + 2] = l4.z;
                        rL[4 * i + 3] = l4.w;
                    }
                }
                if constexpr (CN % 4 == 0) {
#pragma unroll
                    for (int i = 0; i < CN / 4; ++i) {
                        if (TV) {
                            const float4 p4 = *reinterpret_cast<const float4 *>(yP + co[i] + j * TN);
                            cP[4 * i] = p4.x;
                            cP[4 * i + 1] = p4.y;
                            cP[4 * i + 2] = p4.z;
                            cP[4 * i + 3] = p4.w;
                        }
                        if (KL) {
                            const float4 l4 = *reinterpret_cast<const float4 *>(yL + co[i] + j * TN);
                            cL[4 * i] = l4.x;
                            cL[4 * i + 1] = l4.y;
                            cL[4 * i + 2] = l4.z;
                            cL[4 * i + 3] = l4.w;
                        }
                    }
                } else {
                    if (TV) lds_vec(cP, yP + co[0] + j * TN);
                    if (KL) lds_vec(cL, yL + co[0] + j * TN);
                }
#pragma unroll
                for (int r = 0; r < RM; ++r)
#pragma unroll
                    for (int c = 0; c < CN; ++c) {
                        if (KL) ckl[r][c] = __fmaf_rn(rP[r], __fadd_rn(rL[r], -cL[c]), ckl[r][c]);
                        if (TV) ctv[r][c] = __fadd_rn(ctv[r][c], fabsf(__fadd_rn(rP[r], -cP[c])));
                    }
            }
        }
        if (((b0 / kTileB) & 1) || b0 + kTileB >= k_pad) {
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int c = 0; c < CN; ++c) {
                    const float y = __fsub_rn(ckl[r][c], klc[r][c]);
                    const float t = __fadd_rn(kl[r][c], y);
                    klc[r][c] = __fsub_rn(__fsub_rn(t, kl[r][c]), y);
                    kl[r][c] = t;
                    tv[r][c] = __fadd_rn(tv[r][c], ctv[r][c]);
                    ckl[r][c] = ctv[r][c] = 0.0f;
                }
        }
    }
    __syncthreads();            // the transposed arrays may be refilled by the next tile of this CTA
#pragma unroll
    for (int r = 0; r < RM; ++r) {
        const int64_t x = x0 + ty * RM + r;
        if (x >= n_v) continue;
#pragma unroll
        for (int c = 0; c < CN; ++c) {
            const int a = a0 + tx * CN + c;
            if (a >= T) continue;
            if (KL && out_kl) out_kl[(int64_t)a * n_v + x] = __fmul_rn(kl[r][c], kLn2);
            if (TV && out_tv) out_tv[(int64_t)a * n_v + x] = tv[r][c];
        }
    }
}

// ------------------------------------------------------------------ pipelined tile (tiled layout)
// The tile above spends a fifth of its time staging: every 32-column chunk is
// transposed through shared memory and its logarithms formed, between two
// barriers, while the FMA pipe waits.  The pipelined tile takes both out of
// the loop.  The mesh keeps a second copy of P in a tiled layout, [row tile
// of 64][column][row in tile], with the one-number log2 of every entry beside
// it in the same layout (formed once per mesh, by the same fast_l2); each
// call stages its targets the same way ([target tile of 64][column][target],
// P and log2).  A stage -- 64 columns of the CTA's two row tiles and of its
// target tile -- is then six contiguous 16 KB blocks, brought into shared
// memory by bulk async copies that complete on an mbarrier; two stages
// alternate, the CTA's warps release a stage on a second mbarrier and one
// thread refills it.  Every wait is bounded (error flag, no output).  With
// no staging phase left, the arithmetic is packed in FP32x2 over pairs of
// targets (the targets are staged negated, so each difference is one packed
// addition; the row operand is duplicated into both halves): a packed
// instruction occupies the FMA pipe as long as its two halves but takes one
// issue slot, and the slots it frees carry the shared-memory loads and the
// loop while the pipe is busy.  The sums are those of tile_body<64, 64, 4, 4>
// -- each half the same IEEE operation on the same operands, in the same
// order, partial sums merged after the same columns -- so the two kernels
// give bit-identical fields.
constexpr int kTiledRows = 64;      // rows (and targets) per tile of the tiled layout

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// P and fast_l2(P) of one row tile x 32 columns into the tiled layout (zero
// past n_v and k_pad; fast_l2(0) = -127 is finite)
__global__ void tiled_layout_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad, int64_t k32,
                                    float *__restrict__ PT, float *__restrict__ LT) {
    __shared__ float t[kTiledRows][33];
    const int64_t xt = blockIdx.x, b0 = (int64_t)blockIdx.y * 32;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int r = threadIdx.x / 8 + 32 * h, c4 = threadIdx.x % 8;
        const int64_t x = xt * kTiledRows + r, b = b0 + 4 * c4;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (x < n_v && b < k_pad) v = *reinterpret_cast<const float4 *>(P + x * k_pad + b);
        t[r][4 * c4] = v.x;
        t[r][4 * c4 + 1] = v.y;
        t[r][4 * c4 + 2] = v.z;
        t[r][4 * c4 + 3] = v.w;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = threadIdx.x + 256 * i;
        const int c = idx / kTiledRows, r = idx % kTiledRows;
        const float v = t[r][c];
        const int64_t o = (xt * k32 + b0 + c) * kTiledRows + r;
        PT[o] = v;
        LT[o] = fast_l2(v);
    }
}

// the staged targets (sP, and sE / sF when the staging holds logarithms of
// entries below FLT_MIN) into the tiled layout: -P[t,b] and -log2 P[t,b],
// the target-side log2 formed exactly as tile_body forms it
__device__ __forceinline__ void tiled_targets_block(const float *__restrict__ sP, const float *__restrict__ sE,
                                                    const float *__restrict__ sF, int32_t T, int64_t k_pad,
                                                    int64_t kt, float *__restrict__ TQ, float *__restrict__ TL,
                                                    int at, int64_t b0) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int idx = threadIdx.x + 256 * i;
        const int c = idx / kTiledRows, al = idx % kTiledRows;
        const int a = at * kTiledRows + al;
        const int64_t b = b0 + c;
        const bool ok = a < T && b < k_pad;
        const float q = ok ? sP[(int64_t)a * k_pad + b] : 0.0f;
        float lt;
        if (sF) {
            const float ev = ok ? sE[(int64_t)a * k_pad + b] : 12583039.0f;
            const float fv = ok ? sF[(int64_t)a * k_pad + b] : 0.0f;
            lt = __fadd_rn(__fsub_rn(ev, 12583039.0f), fv);
        } else {
            lt = fast_l2(fmaxf(q, FLT_MIN));
        }
        const int64_t o = ((int64_t)at * kt + b) * kTiledRows + al;
        TQ[o] = -q;
        TL[o] = -lt;
    }
}

__global__ void tiled_targets_kernel(const float *__restrict__ sP, const float *__restrict__ sE,
                                     const float *__restrict__ sF, int32_t T, int64_t k_pad, int64_t kt,
                                     float *__restrict__ TQ, float *__restrict__ TL) {
    tiled_targets_block(sP, sE, sF, T, k_pad, kt, TQ, TL, blockIdx.x, (int64_t)blockIdx.y * 32);
}

// One stage of the pipelined tile: PB columns of the CTA's rows and targets
// (cP / cL: this thread's 4 rows, cQ / cT: its 4 targets, column j at
// j * 64) summed into the 64-column partial sums.
template <bool KL, bool TV, int PB, int UNR>
__device__ __forceinline__ void pipe_stage(const float *cP, const float *cL, const float *cQ, const float *cT,
                                           float (&ckl)[4][4], float (&ctv)[4][4]) {
    constexpr int RM = 4;
#pragma unroll UNR
    for (int j = 0; j < PB; ++j) {
        float rP[RM], rL[RM], tQ[4], tL[4];
        {
            const float4 p4 = *reinterpret_cast<const float4 *>(cP + j * kTiledRows);
            rP[0] = p4.x, rP[1] = p4.y, rP[2] = p4.z, rP[3] = p4.w;
            if (KL) {
                const float4 l4 = *reinterpret_cast<const float4 *>(cL + j * kTiledRows);
                rL[0] = l4.x, rL[1] = l4.y, rL[2] = l4.z, rL[3] = l4.w;
                const float4 t4 = *reinterpret_cast<const float4 *>(cT + j * kTiledRows);
                tL[0] = t4.x, tL[1] = t4.y, tL[2] = t4.z, tL[3] = t4.w;
            }
            if (TV) {
                const float4 q4 = *reinterpret_cast<const float4 *>(cQ + j * kTiledRows);
                tQ[0] = q4.x, tQ[1] = q4.y, tQ[2] = q4.z, tQ[3] = q4.w;
            }
        }
        // packed over pairs of targets: the row operands duplicated into both
        // halves, the (negated) target values of a pair side by side
        const f2_t nl[2] = {pk(tL[0], tL[1]), pk(tL[2], tL[3])};
        const f2_t nq[2] = {pk(tQ[0], tQ[1]), pk(tQ[2], tQ[3])};
#pragma unroll
        for (int r = 0; r < RM; ++r) {
            const f2_t p2 = pk(rP[r], rP[r]);
            const f2_t l2 = pk(rL[r], rL[r]);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (KL) {
                    f2_t acc = pk(ckl[r][2 * h], ckl[r][2 * h + 1]);
                    acc = fma2(p2, add2(l2, nl[h]), acc);
                    upk(acc, ckl[r][2 * h], ckl[r][2 * h + 1]);
                }
                if (TV) {
                    float d0, d1;
                    upk(add2(p2, nq[h]), d0, d1);
                    ctv[r][2 * h] = __fadd_rn(ctv[r][2 * h], fabsf(d0));
                    ctv[r][2 * h + 1] = __fadd_rn(ctv[r][2 * h + 1], fabsf(d1));
                }
            }
        }
    }
}

// the 64-column partial sums into the totals (compensated for KL)
__device__ __forceinline__ void pipe_merge(float (&kl)[4][4], float (&klc)[4][4], float (&tv)[4][4],
                                           float (&ckl)[4][4], float (&ctv)[4][4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float y = __fsub_rn(ckl[r][q], klc[r][q]);
            const float t = __fadd_rn(kl[r][q], y);
            klc[r][q] = __fsub_rn(__fsub_rn(t, kl[r][q]), y);
            kl[r][q] = t;
            tv[r][q] = __fadd_rn(tv[r][q], ctv[r][q]);
            ckl[r][q] = ctv[r][q] = 0.0f;
        }
}

template <bool KL, bool TV>
__device__ __forceinline__ void pipe_store(const float (&kl)[4][4], const float (&tv)[4][4], int64_t xr, int ar,
                                           int64_t n_v, int32_t T, float *__restrict__ out_kl,
                                           float *__restrict__ out_tv) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t x = xr + r;
        if (x >= n_v) continue;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int a = ar + q;
            if (a >= T) continue;
            if (KL && out_kl) out_kl[(int64_t)a * n_v + x] = __fmul_rn(kl[r][q], kLn2);
            if (TV && out_tv) out_tv[(int64_t)a * n_v + x] = tv[r][q];
        }
    }
}

template <bool KL, bool TV, int H, int PB, int PS, int UNR>
__global__ void __launch_bounds__(256 * H, 2 / H) field_tile_pipe_kernel(const float *__restrict__ PT,
                                                                      const float *__restrict__ LT, int64_t n_v,
                                                                      int64_t kt, const float *__restrict__ TQ,
                                                                      const float *__restrict__ TL, int32_t T,
                                                                      float *__restrict__ out_kl,
                                                                      float *__restrict__ out_tv,
                                                                      int *__restrict__ err) {
    constexpr int RM = 4, CN = 4, NW = 8 * H;
    constexpr int TCH = PB * kTiledRows;            // floats per array, stage and 64-row (or target) tile
    constexpr int RCH = H * TCH;
    constexpr int SST = 2 * RCH + 2 * TCH;          // floats per stage
    extern __shared__ __align__(128) float psm[];   // [stage][P rows, log2 rows, P targets, log2 targets]
    __shared__ __align__(8) uint64_t full[PS], empty[PS];
    const int tid = threadIdx.x, lane = tid & 31;
    const int tx = tid % (kTiledRows / CN), ty = tid / (kTiledRows / CN);
    // target tiles vary fastest over the grid: the CTAs that read one pair of
    // row tiles run together and share it through L2
    const int64_t x0 = (int64_t)blockIdx.y * H * kTiledRows;
    const int a0 = blockIdx.x * kTiledRows;
    const float *gP = PT + (int64_t)blockIdx.y * H * kt * kTiledRows;
    const float *gL = LT + (int64_t)blockIdx.y * H * kt * kTiledRows;
    const float *gQ = TQ + (int64_t)blockIdx.x * kt * kTiledRows;
    const float *gT = TL + (int64_t)blockIdx.x * kt * kTiledRows;
    const int nch = (int)(kt / PB);
    constexpr uint32_t kArr = TCH * sizeof(float);
    constexpr uint32_t kStageBytes = kArr * (H * (KL ? 2 : 1) + (KL ? 1 : 0) + (TV ? 1 : 0));
    auto issue = [&](int c) {
        const int s = c % PS;
        float *st = psm + s * SST;
        const int64_t go = (int64_t)c * TCH;
        mbar_expect_tx(&full[s], kStageBytes);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            bulk_g2s(st + h * TCH, gP + (int64_t)h * kt * kTiledRows + go, kArr, &full[s]);
            if (KL) bulk_g2s(st + RCH + h * TCH, gL + (int64_t)h * kt * kTiledRows + go, kArr, &full[s]);
        }
        if (TV) bulk_g2s(st + 2 * RCH, gQ + go, kArr, &full[s]);
        if (KL) bulk_g2s(st + 2 * RCH + TCH, gT + go, kArr, &full[s]);
    };
    if (tid == 0) {
        for (int s = 0; s < PS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int issued = 0;
    if (tid == 0)
        for (; issued < PS && issued < nch; ++issued) issue(issued);

    float kl[RM][CN], tv[RM][CN], klc[RM][CN], ckl[RM][CN], ctv[RM][CN];
#pragma unroll
    for (int r = 0; r < RM; ++r)
#pragma unroll
        for (int c = 0; c < CN; ++c) kl[r][c] = tv[r][c] = klc[r][c] = ckl[r][c] = ctv[r][c] = 0.0f;
    // this thread's rows within the stage: 64-row half ty / 16, rows (ty % 16) * 4 ..
    const int roff = (ty / 16) * TCH + (ty % 16) * RM;
    bool ok = true;
    int c = 0;
    for (; c < nch; ++c) {
        const int s = c % PS;
        // refill the stage every warp released last with the chunk PS after it
        if (tid == 0 && c >= 1 && issued < nch) {
            const int cf = c - 1;
            if (!mbar_wait_suspend(&empty[cf % PS], (uint32_t)(cf / PS) & 1u, err)) {
                ok = false;
                break;
            }
            issue(issued++);
        }
        if (!mbar_wait_suspend(&full[s], (uint32_t)(c / PS) & 1u, err)) {
            ok = false;
            break;
        }
        const float *cP = psm + s * SST + roff;
        const float *cQ = psm + s * SST + 2 * RCH + tx * CN;
        pipe_stage<KL, TV, PB, UNR>(cP, cP + RCH, cQ, cQ + TCH, ckl, ctv);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        // 64-column partial sums, merged at the end of every 64 columns
        if (((c + 1) * PB) % 64 == 0 || c == nch - 1) pipe_merge(kl, klc, tv, ckl, ctv);
    }
    if (!ok) {
        // a wait gave up (the error flag is set): let this CTA's copies in flight land, waiting
        // again with a limit, and write nothing
        if (tid == 0)
            for (int cf = c; cf < issued; ++cf)
                if (!mbar_wait_suspend(&full[cf % PS], (uint32_t)(cf / PS) & 1u, err)) break;
        return;
    }
    pipe_store<KL, TV>(kl, tv, x0 + ty * RM, a0 + tx * CN, n_v, T, out_kl, out_tv);
}

// Many problems in one persistent launch, on the tiled layouts: one CTA of
// 512 threads per SM takes (problem, pair of row tiles, target tile) items
// from an atomic counter, largest first.  One thread streams the chunks of
// the items it takes, item after item, through the two stages, and records
// with each stage the item and chunk it holds; the CTA's warps start an item
// at its first chunk (the problem's sizes and outputs, zero sums) and write
// it out after its last, so the copies of one item's first chunks overlap
// the sums of the previous item's last.  The stage that follows the last item
// carries no copy and the item -1: the CTA ends there.  Every wait is bounded
// (error flag, no output from the CTA that gave up).
template <bool KL, bool TV>
__global__ void __launch_bounds__(512, 1) batch_pipe_kernel(const BatchProblem *__restrict__ probs,
                                                         const BatchItem *__restrict__ items, int32_t n_items,
                                                         int32_t *__restrict__ counter, int *__restrict__ err) {
    constexpr int H = 2, PB = 64, PS = 2, RM = 4, CN = 4, NW = 16;
    constexpr int TCH = PB * kTiledRows, RCH = H * TCH, SST = 2 * RCH + 2 * TCH;
    constexpr uint32_t kArr = TCH * sizeof(float);
    constexpr uint32_t kStageBytes = kArr * (H * (KL ? 2 : 1) + (KL ? 1 : 0) + (TV ? 1 : 0));
    extern __shared__ __align__(128) float psm[];
    __shared__ __align__(8) uint64_t full[PS], empty[PS];
    __shared__ int slot_item[PS], slot_chunk[PS];
    const int tid = threadIdx.x, lane = tid & 31;
    const int tx = tid % (kTiledRows / CN), ty = tid / (kTiledRows / CN);

    // producer state (thread 0)
    int p_item = -1, p_ch = 0, p_nch = 0, produced = 0;
    bool p_done = false;
    int64_t p_kt = 0;
    const float *gP = nullptr, *gL = nullptr, *gQ = nullptr, *gT = nullptr;
    auto produce = [&](int s) {
        if (p_ch >= p_nch) {
            const int it = atomicAdd(counter, 1);
            if (it >= n_items) {
                p_done = true;
                slot_item[s] = -1;
                slot_chunk[s] = 0;
                mbar_arrive(&full[s]);
                return;
            }
            const BatchItem w = items[it];
            const BatchProblem &q = probs[w.prob];
            p_item = it;
            p_ch = 0;
            p_kt = q.kt;
            p_nch = (int)(q.kt / PB);
            gP = q.PT + (int64_t)w.x_tile * H * q.kt * kTiledRows;
            gL = q.LT + (int64_t)w.x_tile * H * q.kt * kTiledRows;
            gQ = q.TQ + (int64_t)w.a_tile * q.kt * kTiledRows;
            gT = q.TL + (int64_t)w.a_tile * q.kt * kTiledRows;
        }
        slot_item[s] = p_item;
        slot_chunk[s] = p_ch;
        float *st = psm + s * SST;
        const int64_t go = (int64_t)p_ch * TCH;
        mbar_expect_tx(&full[s], kStageBytes);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            bulk_g2s(st + h * TCH, gP + (int64_t)h * p_kt * kTiledRows + go, kArr, &full[s]);
            if (KL) bulk_g2s(st + RCH + h * TCH, gL + (int64_t)h * p_kt * kTiledRows + go, kArr, &full[s]);
        }
        if (TV) bulk_g2s(st + 2 * RCH, gQ + go, kArr, &full[s]);
        if (KL) bulk_g2s(st + 2 * RCH + TCH, gT + go, kArr, &full[s]);
        ++p_ch;
        ++produced;
    };
    if (tid == 0) {
        for (int s = 0; s < PS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0)
        for (int s = 0; s < PS && !p_done; ++s) produce(s);

    float kl[RM][CN], tv[RM][CN], klc[RM][CN], ckl[RM][CN], ctv[RM][CN];
    int64_t n_v = 0, xr = 0;
    int32_t T = 0;
    int ar = 0, nch = 0;
    float *okl = nullptr, *otv = nullptr;
    const int roff = (ty / 16) * TCH + (ty % 16) * RM;
    bool ok = true;
    int c = 0;
    for (;; ++c) {
        const int s = c % PS;
        // refill the stage every warp released last with the next chunk of the stream
        if (tid == 0 && c >= 1 && !p_done) {
            const int cf = c - 1;
            if (!mbar_wait_suspend(&empty[cf % PS], (uint32_t)(cf / PS) & 1u, err)) {
                ok = false;
                break;
            }
            produce(cf % PS);
        }
        if (!mbar_wait_suspend(&full[s], (uint32_t)(c / PS) & 1u, err)) {
            ok = false;
            break;
        }
        const int it = slot_item[s], ch = slot_chunk[s];
        if (it < 0) break;
        if (ch == 0) {
            const BatchItem w = items[it];
            const BatchProblem &q = probs[w.prob];
            n_v = q.n_v;
            T = q.T;
            okl = q.out_kl;
            otv = q.out_tv;
            nch = (int)(q.kt / PB);
            xr = (int64_t)w.x_tile * H * kTiledRows + ty * RM;
            ar = w.a_tile * kTiledRows + tx * CN;
#pragma unroll
            for (int r = 0; r < RM; ++r)
#pragma unroll
                for (int q2 = 0; q2 < CN; ++q2) kl[r][q2] = tv[r][q2] = klc[r][q2] = ckl[r][q2] = ctv[r][q2] = 0.0f;
        }
        const float *cP = psm + s * SST + roff;
        const float *cQ = psm + s * SST + 2 * RCH + tx * CN;
        pipe_stage<KL, TV, PB, 16>(cP, cP + RCH, cQ, cQ + TCH, ckl, ctv);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        pipe_merge(kl, klc, tv, ckl, ctv);           // every stage is one 64-column block
        if (ch == nch - 1) pipe_store<KL, TV>(kl, tv, xr, ar, n_v, T, okl, otv);
    }
    if (!ok && tid == 0) {
        // a wait gave up (the error flag is set): let the copies in flight land, waiting again with a limit
        for (int cf = c; cf < produced; ++cf)
            if (!mbar_wait_suspend(&full[cf % PS], (uint32_t)(cf / PS) & 1u, err)) break;
    }
}

// the targets of every problem into the tiled layout: blockIdx.y a problem,
// blockIdx.x one (target tile, 32 columns) block of it
__global__ void batch_tiled_targets_kernel(const BatchProblem *__restrict__ probs) {
    const BatchProblem &q = probs[blockIdx.y];
    const int64_t cb = q.kt / 32, nt = (q.T + kTiledRows - 1) / kTiledRows;
    const int64_t i = blockIdx.x;
    if (i >= nt * cb) return;
    tiled_targets_block(q.sP, q.sE, nullptr, q.T, q.k_pad, q.kt, q.TQ, q.TL, (int)(i / cb), (i % cb) * 32);
}

// Exact recompute by row blocks (one domain).  One CTA takes 32 consecutive
// rows.  It scans their first-pass KL for every target (one 128-byte read per
// target) into a shared-memory mask of flagged rows per target, and lists the
// targets that flag any of its rows.  It then takes those targets in groups of
// 16: chunk by chunk (256 columns), the group's staged table logarithms
// (lm_t, E_t) go into shared memory, and each warp, for each of its rows
// that some target of the group flags, reads the row's 256 entries (8 per
// lane), forms their table logarithms once and sums the exact terms for every
// flagging target of the group (the same accumulate_kl operations as
// kl_row_exact; per lane 8 terms, a warp-shuffle sum, then the chunk sums in
// column order).  A row is read once per group, its logarithms formed once
// per group and chunk, and a target's arrays are read once per CTA that it
// flags -- against one row and one target read per flagged pair in
// a grid-wide scan with one warp per flagged pair (9.5 against 4.4 ms on
// grid450 with 1,024 targets), which was bound by those re-reads.
constexpr int kFixRB = 32;      // rows per CTA
constexpr int kFixTW = 1024;    // targets per scan window
constexpr int kFixG = 16;       // targets per staged group
constexpr int kFixCW = 256;     // columns per chunk: 8 per lane

struct FixSmem {
    float tab[2 * kLogTab];
    uint32_t rmask[kFixTW];          // per target of the window: bit r = row x0 + r flagged
    int ulist[kFixTW];               // the window's targets that flag any row of the block
    int nu;
    __align__(16) float gl[kFixG][kFixCW];
    __align__(16) float ge[kFixG][kFixCW];
    float acc[kFixRB][kFixG];
};

// rows x0 .. x0 + 31 of one problem (sh.tab built; called by all 256 threads).
// PF: each warp issues the loads of all its flagged rows of a chunk before
// it uses any (for launches of one wave, where nothing else hides their
// latency; the registers it takes cost occupancy on larger ones)
template <bool PF>
__device__ __forceinline__ void fix_rows(const float *__restrict__ P, int64_t n_v, int64_t k_pad, int32_t T,
                                         const float *__restrict__ sL, const float *__restrict__ sE,
                                         float *__restrict__ out_kl, int64_t x0, FixSmem &sh) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int w0 = 0; w0 < T; w0 += kFixTW) {
        const int tw = min(kFixTW, T - w0);
        __syncthreads();
        if (tid == 0) sh.nu = 0;
        __syncthreads();
        {
            // lane r reads row x0 + r of target a; eight targets per warp in flight
            const int64_t x = x0 + lane;
            for (int a0 = warp * 8; a0 < tw; a0 += 64) {
                bool low[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int a = a0 + i;
                    low[i] = a < tw && x < n_v && out_kl[(int64_t)(w0 + a) * n_v + x] < kTileExactBelow;
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const unsigned m = __ballot_sync(0xffffffffu, low[i]);
                    if (lane == 0 && a0 + i < tw) {
                        sh.rmask[a0 + i] = m;
                        if (m) sh.ulist[atomicAdd(&sh.nu, 1)] = a0 + i;
                    }
                }
            }
        }
        __syncthreads();
        const int n = sh.nu;
        for (int g0 = 0; g0 < n; g0 += kFixG) {
            const int ng = min(kFixG, n - g0);
            for (int i = tid; i < kFixRB * kFixG; i += 256) (&sh.acc[0][0])[i] = 0.0f;
            for (int64_t c0 = 0; c0 < k_pad; c0 += kFixCW) {
                __syncthreads();     // the previous chunk's staged logarithms are no longer read
                for (int i = tid; i < kFixG * (kFixCW / 4); i += 256) {
                    const int u = i / (kFixCW / 4), c4 = i % (kFixCW / 4);
                    float4 l = make_float4(0.f, 0.f, 0.f, 0.f), e = l;
                    if (u < ng && c0 + 4 * c4 < k_pad) {
                        const int64_t o = (int64_t)(w0 + sh.ulist[g0 + u]) * k_pad + c0 + 4 * c4;
                        l = *reinterpret_cast<const float4 *>(sL + o);
                        e = *reinterpret_cast<const float4 *>(sE + o);
                    }
                    *reinterpret_cast<float4 *>(&sh.gl[u][4 * c4]) = l;
                    *reinterpret_cast<float4 *>(&sh.ge[u][4 * c4]) = e;
                }
                __syncthreads();
                // this warp's rows warp, warp + 8, ..: the group's targets that flag
                // each (one bit per target), and the flagged rows' entries of the
                // chunk, all loads issued before any is used
                constexpr int RW = kFixRB / 8;
                constexpr int NB = PF ? RW : 1;       // rows whose entries are held at once
                unsigned gms[RW];
                float pxs[NB][8];
                auto load_row = [&](int i, float(&px)[8]) {
                    const int r = warp + 8 * i;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int64_t col = c0 + h * 128 + 4 * lane;
                        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (gms[i] && col < k_pad)
                            v = __ldcg(reinterpret_cast<const float4 *>(P + (x0 + r) * k_pad + col));
                        px[4 * h] = v.x, px[4 * h + 1] = v.y, px[4 * h + 2] = v.z, px[4 * h + 3] = v.w;
                    }
                };
#pragma unroll
                for (int i = 0; i < RW; ++i) {
                    const int r = warp + 8 * i;
                    const bool f = lane < ng && ((sh.rmask[sh.ulist[g0 + min(lane, ng - 1)]] >> r) & 1u);
                    gms[i] = __ballot_sync(0xffffffffu, f);
                    if (PF) load_row(i, pxs[PF ? i : 0]);
                }
#pragma unroll
                for (int i = 0; i < RW; ++i) {
                    const int r = warp + 8 * i;
                    unsigned gm = gms[i];
                    if (!gm) continue;
                    if (!PF) load_row(i, pxs[0]);
                    const float(&px)[8] = pxs[PF ? i : 0];
                    float lm[8], eb[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) split_log<false>(px[q], sh.tab, lm[q], eb[q]);
                    while (gm) {
                        const int u = __ffs(gm) - 1;
                        gm &= gm - 1;
                        float sum = 0.0f;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const float4 l4 = *reinterpret_cast<const float4 *>(&sh.gl[u][h * 128 + 4 * lane]);
                            const float4 e4 = *reinterpret_cast<const float4 *>(&sh.ge[u][h * 128 + 4 * lane]);
                            const float lt[4] = {l4.x, l4.y, l4.z, l4.w}, et[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                accumulate_kl(px[4 * h + q], lm[4 * h + q], eb[4 * h + q], lt[q], et[q], sum);
                        }
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
                        if (lane == 0) sh.acc[r][u] += sum;
                    }
                }
            }
            __syncthreads();
            for (int i = tid; i < kFixRB * ng; i += 256) {
                const int r = i / ng, u = i % ng;
                const int a = sh.ulist[g0 + u];
                if ((sh.rmask[a] >> r) & 1u) out_kl[(int64_t)(w0 + a) * n_v + x0 + r] = sh.acc[r][u];
            }
            __syncthreads();
        }
    }
}

template <bool PF>
__global__ void __launch_bounds__(256, PF ? 3 : 4) fix_kl_rows_kernel(const float *__restrict__ P, int64_t n_v,
                                                                     int64_t k_pad, int32_t T,
                                                                     const float *__restrict__ sL,
                                                                     const float *__restrict__ sE,
                                                                     float *__restrict__ out_kl) {
    __shared__ FixSmem sh;
    build_log_table(sh.tab);
    fix_rows<PF>(P, n_v, k_pad, T, sL, sE, out_kl, (int64_t)blockIdx.x * kFixRB, sh);
}

// Many problems: CTA g takes row block g of the problems' row blocks in
// order (problems without KL output have none); the CTA finds its problem by
// a block-wide prefix sum over the problems' row-block counts.
template <bool PF>
__global__ void __launch_bounds__(256, PF ? 3 : 4) fix_kl_rows_batch_kernel(const BatchProblem *__restrict__ probs,
                                                                           int32_t n_probs) {
    __shared__ FixSmem sh;
    __shared__ int64_t wsum[8];
    __shared__ int found_prob;
    __shared__ int64_t found_x0;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t g = blockIdx.x;
    if (tid == 0) found_prob = -1;
    build_log_table(sh.tab);
    int64_t base = 0;
    for (int c0 = 0; c0 < n_probs; c0 += 256) {
        const int i = c0 + tid;
        const int64_t nb = (i < n_probs && probs[i].out_kl) ? (probs[i].n_v + kFixRB - 1) / kFixRB : 0;
        int64_t incl = nb;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        int64_t before = base;
        for (int w = 0; w < warp; ++w) before += wsum[w];
        const int64_t lo = before + incl - nb;
        if (nb > 0 && g >= lo && g < lo + nb) {
            found_prob = i;
            found_x0 = (g - lo) * kFixRB;
        }
        for (int w = 0; w < 8; ++w) base += wsum[w];
        __syncthreads();
        if (found_prob >= 0) break;
    }
    if (found_prob < 0) return;
    const BatchProblem &q = probs[found_prob];
    fix_rows<PF>(q.P, q.n_v, q.k_pad, q.T, q.sL, q.sE, q.out_kl, found_x0, sh);
}

// the three shapes the autotuner chooses from
typedef TileShape<64, 64, 4, 4> TileA;
typedef TileShape<128, 32, 4, 4> TileB;
typedef TileShape<256, 16, 8, 2> TileC;

template <int TM, int TN, int RM, int CN, bool KL, bool TV>
__global__ void __launch_bounds__(256, 2) field_tile_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                                         const float *__restrict__ sP, const float *__restrict__ sL,
                                                         const float *__restrict__ sE, const float *__restrict__ sF,
                                                         int32_t T, float *__restrict__ out_kl,
                                                         float *__restrict__ out_tv) {
    extern __shared__ __align__(16) float tsm[];
    float *tab = tsm + 2 * kTileB * (TM + TN) + (kTileB + 4) * (TM + TN);
    build_log_table(tab);
    __syncthreads();
    tile_body<TM, TN, RM, CN, KL, TV>(P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv, (int64_t)blockIdx.x * TM,
                                      blockIdx.y * TN, tsm, tab);
}

template <class S, int TM, int TN, int RM, int CN>
void launch_tile(const float *P, int64_t n_v, int64_t k_pad, const float *sP, const float *sL, const float *sE,
                 const float *sF, int32_t T, float *out_kl, float *out_tv, cudaStream_t s) {
    const dim3 g((unsigned)((n_v + TM - 1) / TM), (unsigned)((T + TN - 1) / TN));
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem_bytes);
        KMark km_("field_tile_kernel", s);
        kern<<<g, 256, S::smem_bytes, s>>>(P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv);
    };
    if (out_kl && out_tv)
        go(field_tile_kernel<TM, TN, RM, CN, true, true>);
    else if (out_kl)
        go(field_tile_kernel<TM, TN, RM, CN, true, false>);
    else
        go(field_tile_kernel<TM, TN, RM, CN, false, true>);
}

int g_num_sms = 0;

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}
// the prefetching recompute when every row block is resident at once (three
// CTAs per SM at its register count), the other one beyond
bool fix_prefetch(int64_t blocks) { return blocks <= 3 * (int64_t)num_sms(); }


// ------------------------------------------------------------------ multi-problem persistent launch
// Work items are output tiles of several problems (domains); CTAs pull items
// from an atomic counter, largest rows first, and run the item's tile shape.
__global__ void __launch_bounds__(256, 2) batch_tile_kernel(const BatchProblem *__restrict__ probs,
                                                         const BatchItem *__restrict__ items, int32_t n_items,
                                                         int32_t *__restrict__ counter) {
    extern __shared__ __align__(16) float tsm[];
    __shared__ float tab[2 * kLogTab];
    __shared__ int cur;
    build_log_table(tab);
    __syncthreads();
    for (;;) {
        if (threadIdx.x == 0) cur = atomicAdd(counter, 1);
        __syncthreads();
        const int it = cur;
        __syncthreads();
        if (it >= n_items) break;
        const BatchItem w = items[it];
        const BatchProblem q = probs[w.prob];
        switch (q.variant) {
            case 0:
                tile_body<64, 64, 4, 4>(q.P, q.n_v, q.k_pad, q.sP, q.sL, q.sE, nullptr, q.T, q.out_kl, q.out_tv,
                                        (int64_t)w.x_tile * 64, w.a_tile * 64, tsm, tab);
                break;
            case 1:
                tile_body<128, 32, 4, 4>(q.P, q.n_v, q.k_pad, q.sP, q.sL, q.sE, nullptr, q.T, q.out_kl, q.out_tv,
                                         (int64_t)w.x_tile * 128, w.a_tile * 32, tsm, tab);
                break;
            default:
                tile_body<256, 16, 8, 2>(q.P, q.n_v, q.k_pad, q.sP, q.sL, q.sE, nullptr, q.T, q.out_kl, q.out_tv,
                                         (int64_t)w.x_tile * 256, w.a_tile * 16, tsm, tab);
                break;
        }
    }
}

// staging of the targets of several problems in one launch: blockIdx.y = global target
__global__ void batch_stage_kernel(const BatchProblem *__restrict__ probs, const int32_t *__restrict__ tprob,
                                   const int32_t *__restrict__ tlocal, const int32_t *__restrict__ targets,
                                   int64_t k_max) {
    __shared__ float tab[2 * kLogTab];
    build_log_table(tab);
    __syncthreads();
    const int g = blockIdx.y;
    const BatchProblem q = probs[tprob[g]];
    const int a = tlocal[g];
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < q.k_pad; b += (int64_t)gridDim.x * blockDim.x) {
        const float p = q.P[(int64_t)targets[g] * q.k_pad + b];
        float lm, E;
        split_log<true>(p, tab, lm, E);
        const int64_t o = (int64_t)a * q.k_pad + b;
        const_cast<float *>(q.sP)[o] = p;
        const_cast<float *>(q.sL)[o] = lm;
        const_cast<float *>(q.sE)[o] = E;
    }
    (void)k_max;
}

// (a 4 x 4 micro-tile in packed FP32x2 arithmetic, pairs along diagonals so
// that no operand needs a broadcast, was measured at 0.41 ms against 0.36 ms
// for shape 1 on 64 grid140 targets, and dropped: the inner loop is bound by
// shared-memory latency, not by FP32 issue)
constexpr int kNumShapes = 4;
const int kShapeRows[kNumShapes] = {64, 128, 256, 128}, kShapeTargets[kNumShapes] = {64, 32, 16, 64};
constexpr int kPipeShape = 3;      // the pipelined tile on the tiled layout (single-problem launches only)

// the pipelined tile: 128 rows x 64 targets per CTA of 512 threads (one CTA per
// SM), two stages of 64 columns (192 KB of shared memory); the column loop is
// unrolled 16 deep for KL+TV and 32 deep for one field
void launch_pipe(const TiledArgs &ta, int64_t n_v, int32_t T, float *out_kl, float *out_tv, int *err,
                 cudaStream_t s) {
    constexpr int H = 2, PB = 64, PS = 2;
    const dim3 g((unsigned)((T + kTiledRows - 1) / kTiledRows),
                 (unsigned)((n_v + H * kTiledRows - 1) / (H * kTiledRows)));
    auto go = [&](auto kern) {
        const size_t smem = (size_t)PS * (2 * H + 2) * PB * kTiledRows * sizeof(float);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        KMark km_("field_tile_kernel", s);
        kern<<<g, 256 * H, smem, s>>>(ta.PT, ta.LT, n_v, ta.kt, ta.TQ, ta.TL, T, out_kl, out_tv, err);
    };
    if (out_kl && out_tv)
        go(field_tile_pipe_kernel<true, true, H, PB, PS, 16>);
    else if (out_kl)
        go(field_tile_pipe_kernel<true, false, H, PB, PS, 32>);
    else
        go(field_tile_pipe_kernel<false, true, H, PB, PS, 32>);
}

void launch_variant(int v, const float *P, int64_t n_v, int64_t k_pad, const float *sP, const float *sL,
                    const float *sE, const float *sF, int32_t T, float *out_kl, float *out_tv, cudaStream_t s,
                    const TiledArgs *tiled = nullptr, int *err = nullptr) {
    if (v == kPipeShape && tiled && err) {
        launch_pipe(*tiled, n_v, T, out_kl, out_tv, err, s);
        return;
    }
    if (v == kPipeShape) v = 0;
    if (v == 0)
        launch_tile<TileA, 64, 64, 4, 4>(P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv, s);
    else if (v == 1)
        launch_tile<TileB, 128, 32, 4, 4>(P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv, s);
    else
        launch_tile<TileC, 256, 16, 8, 2>(P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv, s);
}

// ------------------------------------------------------------------ autotuner
// The first time a (rows, columns, targets) class is seen, every tile shape
// runs on the actual problem (three timed launches each, after a warm-up) and
// the fastest is kept for the class.  Classes: rows and k_pad in powers of
// two, targets in powers of two up to 256.
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int>, int> g_tune;

int ilog2_ceil(int64_t x) {
    int r = 0;
    while ((int64_t(1) << r) < x) ++r;
    return r;
}

std::tuple<int, int, int> tune_key(int64_t n_v, int64_t k_pad, int32_t T) {
    return std::make_tuple(ilog2_ceil(n_v), ilog2_ceil(k_pad), std::min(ilog2_ceil(T), 8));
}

int tune_variant(const float *P, int64_t n_v, int64_t k_pad, const float *sP, const float *sL, const float *sE,
                 const float *sF, int32_t T, float *out_kl, float *out_tv, cudaStream_t s,
                 const TiledArgs *tiled = nullptr, int *err = nullptr) {
    const bool pipe = tiled && err;
    // DD_TILE_SHAPE=0..3 pins the shape (tests run every shape through it)
    if (const char *pin = std::getenv("DD_TILE_SHAPE")) {
        const int v = std::atoi(pin);
        if (v >= 0 && v < kNumShapes && (v != kPipeShape || pipe)) return v;
    }
    // the classes of launches with and without the tiled layout are kept apart
    auto key = tune_key(n_v, k_pad, T);
    if (pipe) std::get<2>(key) += 100;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune.find(key);
        if (it != g_tune.end()) return it->second;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = 0;
    float best_ms = 1e30f;
    for (int v = 0; v < kNumShapes; ++v) {
        if (v == kPipeShape && !pipe) continue;
        launch_variant(v, P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv, s, tiled, err);   // warm-up
        cudaEventRecord(e0, s);
        for (int r = 0; r < 3; ++r)
            launch_variant(v, P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv, s, tiled, err);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[key] = best;
    return best;
}

}  // namespace

void launch_stage_targets(const float *P, int64_t n_v, int64_t k_pad, const int32_t *targets, int32_t T,
                          float4 *stage, cudaStream_t s, int *bad_id, const float *LP) {
    float *sP = reinterpret_cast<float *>(stage);
    float *sL = sP + (int64_t)T * k_pad;
    float *sE = sL + (int64_t)T * k_pad;
    float *sF = sE + (int64_t)T * k_pad;
    if (T <= 0) return;
    {
        KMark km_("stage_targets_kernel", s);
        stage_targets_kernel<<<(unsigned)T, 256, 0, s>>>(P, n_v, k_pad, targets, T, sP, sL, sE, sF, bad_id, LP);
    }
}

int64_t tiled_k32(int64_t k_pad) { return (k_pad + 63) / 64 * 64; }

size_t tiled_target_bytes(int64_t k_pad, int32_t T) {
    return 2 * (size_t)((T + kTiledRows - 1) / kTiledRows) * (size_t)tiled_k32(k_pad) * kTiledRows * sizeof(float);
}

dd_status prepare_tiled(DevMesh &m, cudaStream_t s, std::string &err) {
    if (m.pt_p) return DD_OK;
    // row tiles in pairs (a CTA of the wide shape takes two), columns to a multiple of 64
    const int64_t k32 = tiled_k32(m.k_pad), nt = (m.n_v + 2 * kTiledRows - 1) / (2 * kTiledRows) * 2;
    const size_t ne = (size_t)nt * k32 * kTiledRows;
    void *pp = nullptr, *pl = nullptr;
    if (cudaMalloc(&pp, ne * sizeof(float)) != cudaSuccess || cudaMalloc(&pl, ne * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        if (pp) cudaFree(pp);
        if (pl) cudaFree(pl);
        err = "allocation of the tiled copy of P failed";
        return DD_ENOMEM;
    }
    {
        KMark km_("tiled_layout_kernel", s);
        tiled_layout_kernel<<<dim3((unsigned)nt, (unsigned)(k32 / 32)), 256, 0, s>>>(m.P, m.n_v, m.k_pad, k32,
                                                                                    (float *)pp, (float *)pl);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(pp);
        cudaFree(pl);
        err = std::string("tiled layout launch failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    m.pt_p = (float *)pp;
    m.pt_l = (float *)pl;
    m.pt_kt = k32;
    m.owned.push_back(pp);
    m.owned.push_back(pl);
    m.bytes += (int64_t)(2 * ne * sizeof(float));
    return DD_OK;
}

void launch_fields_fp32(const float *P, int64_t n_v, int64_t k_pad, const float4 *stage, int32_t T, float *out_kl,
                        float *out_tv, int *err_flag, cudaStream_t s, int variant, bool staged_logs,
                        const TiledArgs *tiled, cudaEvent_t tile_done) {
    const float *sP = reinterpret_cast<const float *>(stage);
    const float *sL = sP + (int64_t)T * k_pad;
    const float *sE = sL + (int64_t)T * k_pad;
    const float *sF = sE + (int64_t)T * k_pad;
    // the tile kernel forms the target side's log2 from the staged entry itself
    // unless the staging holds logarithms of entries below FLT_MIN
    const float *tF = staged_logs ? sF : nullptr;
    const size_t smem = 4 * (size_t)k_pad * sizeof(float);
    if (T <= 2 && smem <= 200 * 1024) {
        // one target per grid row; loads run 8 float4 per lane ahead of the arithmetic
        auto kern = field_stream_kernel<8>;
        const int64_t row_blocks = (n_v + 7) / 8;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t grid_x = (int64_t)num_sms() * per_sm / T;
        if (grid_x < 1) grid_x = 1;
        if (grid_x > row_blocks) grid_x = row_blocks;
        {
            KMark km_("field_stream_kernel", s);
            kern<<<dim3((unsigned)grid_x, (unsigned)T), 256, smem, s>>>(P, n_v, k_pad, sP, sL, sE, sF, T, out_kl, out_tv,
                                                                       err_flag);
        }
        if (tile_done) cudaEventRecord(tile_done, s);
        return;
    }
    if (tiled) {
        // the staged targets in the tiled layout (P and the target-side log2)
        KMark km_("tiled_targets_kernel", s);
        tiled_targets_kernel<<<dim3((unsigned)((T + kTiledRows - 1) / kTiledRows), (unsigned)(tiled->kt / 32)), 256,
                               0, s>>>(sP, sE, tF, T, k_pad, tiled->kt, tiled->TQ, tiled->TL);
    }
    const int v = (variant >= 0 && variant < kNumShapes)
                      ? variant
                      : tune_variant(P, n_v, k_pad, sP, sL, sE, tF, T, out_kl, out_tv, s, tiled, err_flag);
    launch_variant(v, P, n_v, k_pad, sP, sL, sE, tF, T, out_kl, out_tv, s, tiled, err_flag);
    if (tile_done) cudaEventRecord(tile_done, s);
    if (out_kl) {
        KMark km_("fix_kl_kernel", s);        // the timing hook's name of the exact recompute
        const int64_t blocks = (n_v + kFixRB - 1) / kFixRB;
        if (fix_prefetch(blocks))
            fix_kl_rows_kernel<true><<<(unsigned)blocks, 256, 0, s>>>(P, n_v, k_pad, T, sL, sE, out_kl);
        else
            fix_kl_rows_kernel<false><<<(unsigned)blocks, 256, 0, s>>>(P, n_v, k_pad, T, sL, sE, out_kl);
    }
}


int tile_variant_for(const float *P, int64_t n_v, int64_t k_pad, const float *sP, const float *sL, const float *sE,
                     int32_t T, float *out_kl, float *out_tv, cudaStream_t s) {
    return tune_variant(P, n_v, k_pad, sP, sL, sE, nullptr, T, out_kl, out_tv, s);
}

int tile_rows(int variant) { return kShapeRows[variant]; }
int tile_targets(int variant) { return kShapeTargets[variant]; }

void launch_batch_stage(const BatchProblem *d_probs, const int32_t *d_tprob, const int32_t *d_tlocal,
                        const int32_t *d_targets, int32_t n_targets, int64_t k_max, cudaStream_t s) {
    if (n_targets <= 0) return;
    dim3 g((unsigned)std::max<int64_t>(1, std::min<int64_t>(8, (k_max + 255) / 256)), (unsigned)n_targets);
    {
        KMark km_("batch_stage_kernel", s);
        batch_stage_kernel<<<g, 256, 0, s>>>(d_probs, d_tprob, d_tlocal, d_targets, k_max);
    }
}

void launch_batch_fields(const BatchProblem *d_probs, int32_t n_probs, const BatchItem *d_items, int32_t n_items,
                         int32_t *d_counter, cudaStream_t s, int64_t fix_blocks) {
    if (n_items <= 0) return;
    const size_t smem = (size_t)(2 * kTileB + kTileB + 4) * (256 + 16) * sizeof(float);
    cudaFuncSetAttribute(batch_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_tile_kernel, 256, smem);
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)num_sms() * per_sm;
    if (grid > n_items) grid = n_items;
    cudaMemsetAsync(d_counter, 0, sizeof(int32_t), s);
    {
        KMark km_("batch_tile_kernel", s);
        batch_tile_kernel<<<(unsigned)grid, 256, smem, s>>>(d_probs, d_items, n_items, d_counter);
    }
    if (fix_blocks > 0) {
        KMark km_("fix_kl_batch_kernel", s);      // the timing hook's name of the exact recompute
        if (fix_prefetch(fix_blocks))
            fix_kl_rows_batch_kernel<true><<<(unsigned)fix_blocks, 256, 0, s>>>(d_probs, n_probs);
        else
            fix_kl_rows_batch_kernel<false><<<(unsigned)fix_blocks, 256, 0, s>>>(d_probs, n_probs);
    }
}

void launch_batch_fields_pipe(const BatchProblem *d_probs, int32_t n_probs, const BatchItem *d_items,
                              int32_t n_items, int32_t *d_counter, int *err, cudaStream_t s, int64_t fix_blocks,
                              int64_t max_tiles, bool f_kl, bool f_tv) {
    if (n_items <= 0) return;
    {
        KMark km_("tiled_targets_kernel", s);
        batch_tiled_targets_kernel<<<dim3((unsigned)max_tiles, (unsigned)n_probs), 256, 0, s>>>(d_probs);
    }
    constexpr size_t smem = (size_t)2 * 6 * 64 * kTiledRows * sizeof(float);
    cudaMemsetAsync(d_counter, 0, sizeof(int32_t), s);
    const unsigned grid = (unsigned)std::min<int64_t>(num_sms(), n_items);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        KMark km_("batch_tile_kernel", s);
        kern<<<grid, 512, smem, s>>>(d_probs, d_items, n_items, d_counter, err);
    };
    if (f_kl && f_tv)
        go(batch_pipe_kernel<true, true>);
    else if (f_kl)
        go(batch_pipe_kernel<true, false>);
    else
        go(batch_pipe_kernel<false, true>);
    if (fix_blocks > 0) {
        KMark km_("fix_kl_batch_kernel", s);
        if (fix_prefetch(fix_blocks))
            fix_kl_rows_batch_kernel<true><<<(unsigned)fix_blocks, 256, 0, s>>>(d_probs, n_probs);
        else
            fix_kl_rows_batch_kernel<false><<<(unsigned)fix_blocks, 256, 0, s>>>(d_probs, n_probs);
    }
}

int64_t fix_row_blocks(int64_t n_v) { return (n_v + kFixRB - 1) / kFixRB; }


// (fields asked for, log2 problems, log2 work) -> 0 staged / 1 pipelined
std::map<std::tuple<int, int, int>, int> g_batch_tune;

int batch_launch_choice(int32_t n_probs, int64_t work, uint32_t f_mask, const std::function<void()> &staged,
                        const std::function<void()> &pipelined, cudaStream_t s) {
    if (const char *pin = std::getenv("DD_BATCH_PIPE")) {
        if (pin[0] == '0') return 0;
        if (pin[0] == '1') return 1;
    }
    const auto key = std::make_tuple((int)f_mask, ilog2_ceil(n_probs), ilog2_ceil(work));
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_batch_tune.find(key);
        if (it != g_batch_tune.end()) return it->second;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    int best = 0;
    for (int v = 0; v < 2; ++v) {
        const std::function<void()> &f = v ? pipelined : staged;
        f();                                 // warm-up
        cudaEventRecord(e0, s);
        f();
        f();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best_ms) {
            best_ms = ms;
            best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_batch_tune[key] = best;
    return best;
}

std::string tuning_table() {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    std::string out;
    const char *names[kNumShapes] = {"64x64", "128x32", "256x16", "128x64 pipelined"};
    for (auto &kv : g_tune) {
        char buf[160];
        const int tk = std::get<2>(kv.first);
        std::snprintf(buf, sizeof buf, "rows<=2^%d k_pad<=2^%d T<=2^%d%s: %s\n", std::get<0>(kv.first),
                      std::get<1>(kv.first), tk % 100, tk >= 100 ? " (tiled copy of P)" : "", names[kv.second]);
        out += buf;
    }
    for (auto &kv : g_batch_tune) {
        char buf[160];
        const int fm = std::get<0>(kv.first);
        std::snprintf(buf, sizeof buf, "batch of problems<=2^%d n*k*T<=2^%d (%s): %s\n", std::get<1>(kv.first),
                      std::get<2>(kv.first), fm == 3 ? "KL+TV" : (fm == 1 ? "KL" : "TV"),
                      kv.second ? "pipelined persistent launch" : "staged persistent launch");
        out += buf;
    }
    return out;
}

// ------------------------------------------------------------------ fast-log self-check
namespace {
// per block: min and max of lg2_mant(m) - log2(m) over 256 consecutive mantissas
__global__ void fast_log_error_kernel(double *__restrict__ bmin, double *__restrict__ bmax) {
    __shared__ double smin[256], smax[256];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;           // mantissa bits, 0 .. 2^23 - 1
    const int bits = 0x3F800000 | j;
    const double e = (double)lg2_mant(bits) - log2((double)__int_as_float(bits));
    smin[threadIdx.x] = e;
    smax[threadIdx.x] = e;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + o]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bmin[blockIdx.x] = smin[0];
        bmax[blockIdx.x] = smax[0];
    }
}
}  // namespace

dd_status fast_log_spread(double *spread, std::string &err) {
    constexpr int kBlocks = (1 << 23) / 256;
    double *d = nullptr;
    if (cudaMalloc(&d, 2 * kBlocks * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        err = "fast-log check: device allocation failed";
        return DD_ENOMEM;
    }
    fast_log_error_kernel<<<kBlocks, 256>>>(d, d + kBlocks);
    std::vector<double> h(2 * kBlocks);
    cudaError_t e = cudaMemcpy(h.data(), d, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        err = std::string("fast-log check: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    double lo = h[0], hi = h[kBlocks];
    for (int b = 0; b < kBlocks; ++b) {
        lo = std::min(lo, h[b]);
        hi = std::max(hi, h[kBlocks + b]);
    }
    *spread = hi - lo;
    return DD_OK;
}
