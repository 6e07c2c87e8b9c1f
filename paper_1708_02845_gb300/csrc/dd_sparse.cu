// Sparse KL and TV fields, Section V: the Poisson kernel's small entries
// eliminated before the sums (threshold 1/sqrt(n) of each row's largest
// entry, about 90 % of the entries).  In Eq. (35) the weight row decides
// which terms remain (an eliminated weight drops its term) and the other row
// enters through its logarithm, taken from the full kernel:
//
//   KLT~_t(x) = sum_{b in S_t} P[t,b] log(P[t,b] / P[x,b])     target-weighted
//   KL~_t(x)  = sum_{b in S_x} P[x,b] log(P[x,b] / P[t,b])     field-weighted
//   TV~_t(x)  = sum_b |P~[x,b] - P~[t,b]|                      sparsified rows
//
// with S_y = {b : P[y,b] >= theta max_b' P[y,b'], P[y,b] > 0} (FP32 product)
// and P~ = P with the other entries set to 0.
//
// Layouts.  dd_sparsify stores the sparsified P as CSR (each row's kept
// entries in column order: FP32 values, 16-bit columns, 64-bit row offsets),
// about a sixth of the dense P at 84 % sparsity.  KL~ and TV~ read only that
// (csr_stream_kernel: one warp per row, the row's entries streamed into
// shared memory by bulk async copies with several chunks in flight per warp;
// the target row's thresholded values and logarithms staged in shared
// memory the same way and gathered by column).  KLT~ needs the field row at the target's kept columns, which
// the CSR row may not hold (an entry below the field row's own threshold is
// still non-zero), so it reads the dense P at the 4-column blocks holding
// S_t (sparse_field_kernel, the list built once per target by
// sparse_stage_kernel; S_t lies on a few arcs of the boundary, so the list
// is a few runs of consecutive blocks).
//
// Extension (not in the paper; DD_PREC_SPARSE_MERGED): S_t decides for both
// rows and every other column merges into one bin of mass
// M_y = sum_{b not in S_t} P[y,b]:
//
//   KL^_t(x)  = sum_{b in S_t} P[x,b] log(P[x,b] / P[t,b]) + M_x log(M_x / M_t)
//   KLT^_t(x) = sum_{b in S_t} P[t,b] log(P[t,b] / P[x,b]) + M_t log(M_t / M_x)
//   TV^_t(x)  = sum_{b in S_t} |P[x,b] - P[t,b]| + |M_x - M_t|
//
// M_x is the row's total (per mesh, exact 2^-62 fixed point) minus its S_t
// part, summed with compensation (Kahan) per lane and in FP64 across the warp
// once per row; M_t comes from the same routine in the same order on row t,
// so M_x = M_t bit for bit at x = t and the fields are exactly 0 there.
//
// Every KL sum takes the same two passes as the dense streaming kernel
// (exponents exact, hardware log2 of the mantissas, rows below
// DD_EXACT_BELOW recomputed with the table logarithm), and every field is
// exactly 0 at x = t.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "dd_bulk.cuh"
#include "dd_f32x2.cuh"
#include "dd_internal.h"
#include "dd_splitlog.cuh"

namespace {

constexpr float kLn2s = 0.693147180559945309f;
constexpr float kExactBelowS = (float)DD_EXACT_BELOW;

// p in units of 2^-62, from the bits: p = m 2^(e - 150) for the biased
// exponent e and the 24-bit significand m, so p 2^62 = m 2^(e - 88); values
// below 2^-39 are truncated, zero and subnormals give 0.  Exact for every
// p in [2^-39, 2): the sum of a row of P (about 1) stays below 2^63.
__device__ __forceinline__ long long fix62(float p) {
    const unsigned u = __float_as_uint(p);
    const int e = (int)((u >> 23) & 0xFFu);
    if (e == 0) return 0;
    const long long m = (long long)((u & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 88;
    return sh >= 0 ? (m << sh) : (sh > -24 ? (m >> -sh) : 0LL);
}

__device__ __forceinline__ double total62(long long q) { return __ll2double_rn(q) * 0x1p-62; }

// per row: fixed-point total of the stored FP32 row, and how many entries /
// 4-column blocks the row's own threshold keeps (the sparsity figure).  One
// warp per row.
__global__ void sparse_rows_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad, float theta,
                                   long long *__restrict__ rowsum, unsigned long long *__restrict__ counts,
                                   int32_t *__restrict__ row_kept, float *__restrict__ row_thr) {
    const int lane = threadIdx.x & 31;
    const int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (x >= n_v) return;
    const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
    const int nb = (int)(k_pad >> 2);
    float mx = 0.0f;
    long long s = 0;
    for (int j = lane; j < nb; j += 32) {
        const float4 v = __ldg(row + j);
        mx = fmaxf(mx, fmaxf(fmaxf(v.x, v.y), fmaxf(v.z, v.w)));
        s += fix62(v.x) + fix62(v.y) + fix62(v.z) + fix62(v.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        s += __shfl_xor_sync(0xffffffffu, s, o);
    }
    const float t = __fmul_rn(theta, mx);
    unsigned long long ne = 0, nbk = 0;
    for (int j = lane; j < nb; j += 32) {
        const float4 v = __ldg(row + j);
        const int c = (v.x >= t && v.x > 0.f) + (v.y >= t && v.y > 0.f) + (v.z >= t && v.z > 0.f) +
                      (v.w >= t && v.w > 0.f);
        ne += c;
        nbk += c > 0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ne += __shfl_xor_sync(0xffffffffu, ne, o);
        nbk += __shfl_xor_sync(0xffffffffu, nbk, o);
    }
    if (lane == 0) {
        rowsum[x] = s;
        row_kept[x] = (int32_t)ne;
        row_thr[x] = t;
        atomicAdd(counts, ne);
        atomicAdd(counts + 1, nbk);
    }
}

// CSR of the sparsified P: one warp per row writes the row's kept entries in
// column order from off[x] (a ballot compaction per 32 columns), the same
// decision as sparse_rows_kernel (P[x,b] >= row_thr[x] and P[x,b] > 0).
__global__ void csr_fill_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                const float *__restrict__ row_thr, const int64_t *__restrict__ off,
                                float *__restrict__ val, uint16_t *__restrict__ col) {
    const int lane = threadIdx.x & 31;
    const int64_t x = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (x >= n_v) return;
    const float *row = P + x * k_pad;
    const float t = row_thr[x];
    int64_t pos = off[x];
    for (int64_t b0 = 0; b0 < k_pad; b0 += 32) {
        const int64_t b = b0 + lane;
        const float v = b < k_pad ? __ldg(row + b) : 0.0f;
        const bool keep = v >= t && v > 0.0f;
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int64_t i = pos + __popc(ball & ((1u << lane) - 1u));
            val[i] = v;
            col[i] = (uint16_t)b;
        }
        pos += __popc(ball);
    }
}

// One listed block of a row against the staged target block: p4 (target
// entries, dropped ones 0), f4 / e4 (the dense target row's hardware mantissa
// log2 and biased exponent).  Accumulates, per pair of entries (0,1) and
// (2,3) in the halves of packed registers: kl += w d, kt += p_t d (KLT with
// the sign flipped), tv += |w - p_t|, and the mass w into the Kahan pair
// (s, c), where w = P[x,b] on kept columns and 0 on dropped ones and
// d = log2(P[x,b]/P[t,b]) from exact exponents and hardware mantissa logs.
template <bool KL, bool TV, bool KLT, bool MASS = true>
__device__ __forceinline__ void block_terms(const float4 &v, const float4 &p4, const float4 &f4, const float4 &e4,
                                            f2_t &kl, f2_t &tv, f2_t &kt, f2_t &s, f2_t &c) {
    const f2_t mone = pk(-1.0f, -1.0f);
    const float px[4] = {v.x, v.y, v.z, v.w}, pt[4] = {p4.x, p4.y, p4.z, p4.w};
    float w[4], lf[4], eb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        w[q] = pt[q] > 0.f ? px[q] : 0.f;
        if (KL || KLT) {
            const int bits = __float_as_int(fmaxf(px[q], FLT_MIN));
            lf[q] = lg2_mant(bits);
            eb[q] = __int_as_float((int)__funnelshift_r((unsigned)bits, (unsigned)kMagicHi, 23));
        }
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const f2_t w2 = pk(w[2 * h], w[2 * h + 1]);
        const f2_t pt2 = h ? pk(p4.z, p4.w) : pk(p4.x, p4.y);
        if (KL || KLT) {
            const f2_t ft2 = h ? pk(f4.z, f4.w) : pk(f4.x, f4.y);
            const f2_t et2 = h ? pk(e4.z, e4.w) : pk(e4.x, e4.y);
            const f2_t d = add2(fma2(ft2, mone, pk(lf[2 * h], lf[2 * h + 1])),
                                fma2(et2, mone, pk(eb[2 * h], eb[2 * h + 1])));
            if (KL) kl = fma2(w2, d, kl);
            if (KLT) kt = fma2(pt2, d, kt);
        }
        if (TV) tv = add2(tv, fma2(pt2, mone, w2) & 0x7fffffff7fffffffULL);
        if (MASS) {
            const f2_t y = fma2(c, mone, w2);             // Kahan: y = w - c
            const f2_t t = add2(s, y);
            c = fma2(y, mone, fma2(s, mone, t));          // c = (t - s) - y
            s = t;
        }
    }
}

// the lane's Kahan pair as one FP64 value, reduced over the warp (fixed order)
__device__ __forceinline__ double lane_mass_sum(f2_t s, f2_t c) {
    float s0, s1, c0, c1;
    upk(s, s0, s1);
    upk(c, c0, c1);
    double m = ((double)s0 - (double)c0) + ((double)s1 - (double)c1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    return m;
}

// S_t part of row x's mass for one warp: block_terms' additions in the field
// kernel's order (lane l takes list entries l, l + 32, ...)
__device__ __forceinline__ double kept_mass(const float *__restrict__ P, int64_t x, int64_t k_pad,
                                            const uint16_t *lst, int nl, const float4 *tP4, const float4 *tF4,
                                            const float4 *tE4, int lane) {
    const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
    f2_t kl = 0ULL, tv = 0ULL, kt = 0ULL, s = 0ULL, c = 0ULL;
    for (int i = lane; i < nl; i += 32) {
        const int j = lst[i];
        block_terms<false, false, false>(__ldcg(row + j), tP4[j], tF4[j], tE4[j], kl, tv, kt, s, c);
    }
    return lane_mass_sum(s, c);
}

// Per target (one CTA each), after stage_targets_kernel: zero the staged
// row's entries below theta x its maximum (the logs stay those of the dense
// row), list, in column order, the blocks holding a kept entry
// (list[a][0 .. count[a]), pitch lp), and compute M_t (mt_out[a]).
__global__ void sparse_stage_kernel(const float *__restrict__ P, float *__restrict__ sP, const float *__restrict__ sE,
                                    const float *__restrict__ sF, int64_t k_pad, float theta,
                                    uint16_t *__restrict__ list, int64_t lp, int32_t *__restrict__ count,
                                    const long long *__restrict__ rowsum, const int32_t *__restrict__ targets,
                                    double *__restrict__ mt_out) {
    __shared__ float red[32];
    __shared__ int wsum[32];
    const int a = blockIdx.x;
    float *row = sP + (int64_t)a * k_pad;
    uint16_t *L = list + (int64_t)a * lp;
    const int nb = (int)(k_pad >> 2);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float mx = 0.0f;
    for (int64_t b = threadIdx.x; b < k_pad; b += blockDim.x) mx = fmaxf(mx, row[b]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red[wid] = mx;
    __syncthreads();
    if (threadIdx.x < 32) {
        float m = threadIdx.x < nw ? red[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (threadIdx.x == 0) red[0] = m;
    }
    __syncthreads();
    const float t = __fmul_rn(theta, red[0]);
    // blocks in rounds of blockDim.x: threshold, then compact with a block-wide prefix
    int base = 0;
    for (int j0 = 0; j0 < nb; j0 += blockDim.x) {
        const int j = j0 + threadIdx.x;
        bool keep = false;
        if (j < nb) {
            float4 v = reinterpret_cast<float4 *>(row)[j];
            const bool kx = v.x >= t && v.x > 0.f, ky = v.y >= t && v.y > 0.f;
            const bool kz = v.z >= t && v.z > 0.f, kw = v.w >= t && v.w > 0.f;
            v.x = kx ? v.x : 0.f;
            v.y = ky ? v.y : 0.f;
            v.z = kz ? v.z : 0.f;
            v.w = kw ? v.w : 0.f;
            reinterpret_cast<float4 *>(row)[j] = v;
            keep = kx || ky || kz || kw;
        }
        const unsigned ball = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wsum[wid] = __popc(ball);
        __syncthreads();
        int before = base;
        for (int w = 0; w < wid; ++w) before += wsum[w];
        if (keep) L[before + __popc(ball & ((1u << lane) - 1u))] = (uint16_t)j;
        int total = 0;
        for (int w = 0; w < nw; ++w) total += wsum[w];
        base += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) count[a] = base;
    // the target's mass outside S_t, by the routine and lane order the field
    // kernel uses for every row (so that it reproduces this value at x = t)
    if (threadIdx.x < 32) {
        const double mt = total62(rowsum[targets[a]]) -
                          kept_mass(P, targets[a], k_pad, L, base, reinterpret_cast<const float4 *>(row),
                                    reinterpret_cast<const float4 *>(sF + (int64_t)a * k_pad),
                                    reinterpret_cast<const float4 *>(sE + (int64_t)a * k_pad), lane);
        if (lane == 0) mt_out[a] = mt;
    }
}

// exact (table) KL over the kept columns of one row, for one warp: the row
// weighted (TARGET_W false: sum P[x,b] log(P[x,b]/P[t,b])) or the target
// weighted (true: sum P[t,b] log(P[t,b]/P[x,b]), the row's log at >= FLT_MIN)
template <bool TARGET_W>
__device__ __forceinline__ float kept_kl_exact(const float *__restrict__ P, int64_t x, int64_t k_pad,
                                               const uint16_t *lst, int nl, const float4 *tP4, const float *tL,
                                               const float *tE, const float *tab, int lane) {
    const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
    float k0 = 0.0f, k1 = 0.0f;
    for (int i = lane; i < nl; i += 32) {
        const int j = lst[i];
        const float4 v = __ldcg(row + j);
        const float4 p4 = tP4[j];
        const float4 l4 = reinterpret_cast<const float4 *>(tL)[j];
        const float4 e4 = reinterpret_cast<const float4 *>(tE)[j];
        const float px[4] = {v.x, v.y, v.z, v.w}, pt[4] = {p4.x, p4.y, p4.z, p4.w};
        const float lt[4] = {l4.x, l4.y, l4.z, l4.w}, et[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!(pt[q] > 0.f)) continue;
            float lm, Eb;
            split_log<TARGET_W>(px[q], tab, lm, Eb);
            const float lr = __fmaf_rn(__fadd_rn(Eb, -et[q]), kLn2s, __fadd_rn(lm, -lt[q]));   // log(P_x/P_t)
            const float w = TARGET_W ? -pt[q] : px[q];
            if (q & 1)
                k1 = __fmaf_rn(w, lr, k1);
            else
                k0 = __fmaf_rn(w, lr, k0);
        }
    }
    float s = k0 + k1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// One target per grid row (blockIdx.y).  Dynamic smem: the thresholded target
// row, the dense row's table mantissa log, biased exponent and hardware
// mantissa log2 (k_pad floats each) and the block list (lp uint16); one bulk
// copy each.  Items are (row, group of 32 U listed blocks).  The row-side
// logarithms are taken at max(P[x,b], FLT_MIN): a zero entry contributes 0 to
// KL (weight 0) and a large finite term to KLT (the exact value is +inf).
template <int U, bool KL, bool TV, bool KLT, bool MERGED>
__global__ void __launch_bounds__(256, 3) sparse_field_kernel(
    const float *__restrict__ P, int64_t n_v, int64_t k_pad, const float *__restrict__ sP,
    const float *__restrict__ sL, const float *__restrict__ sE, const float *__restrict__ sF,
    const uint16_t *__restrict__ sList, int64_t lp, const int32_t *__restrict__ sCount,
    const double *__restrict__ sMt, const long long *__restrict__ rowsum, float *__restrict__ out_kl,
    float *__restrict__ out_tv, float *__restrict__ out_klt, int *__restrict__ err_flag) {
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ float tab[2 * kLogTab];
    float *tP = smem;
    float *tL = tP + k_pad;
    float *tE = tL + k_pad;
    float *tF = tE + k_pad;
    uint16_t *lst = reinterpret_cast<uint16_t *>(tF + k_pad);
    const int a = blockIdx.y;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t row_bytes = (uint32_t)(k_pad * sizeof(float));
        const uint32_t l_bytes = (uint32_t)(lp * sizeof(uint16_t));
        mbar_expect_tx(&bar, 4u * row_bytes + l_bytes);
        bulk_g2s(tP, sP + (int64_t)a * k_pad, row_bytes, &bar);
        bulk_g2s(tL, sL + (int64_t)a * k_pad, row_bytes, &bar);
        bulk_g2s(tE, sE + (int64_t)a * k_pad, row_bytes, &bar);
        bulk_g2s(tF, sF + (int64_t)a * k_pad, row_bytes, &bar);
        bulk_g2s(lst, sList + (int64_t)a * lp, l_bytes, &bar);
    }
    build_log_table(tab);
    __syncthreads();
    if (!mbar_wait(&bar, 0, err_flag)) {
        mbar_wait(&bar, 0, err_flag);     // copies may still land: wait once more (bounded) before exiting
        return;
    }
    const int nl = sCount[a];
    const int lane = threadIdx.x & 31;
    const float4 *tP4 = reinterpret_cast<const float4 *>(tP);
    const float4 *tF4 = reinterpret_cast<const float4 *>(tF);
    const float4 *tE4 = reinterpret_cast<const float4 *>(tE);
    const double Mt_d = sMt[a];
    const float Mt = (float)Mt_d;

    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int ngroups = nl > 0 ? (nl + 32 * U - 1) / (32 * U) : 1;
    float *okl = KL ? out_kl + (int64_t)a * n_v : nullptr;
    float *otv = TV ? out_tv + (int64_t)a * n_v : nullptr;
    float *okt = KLT ? out_klt + (int64_t)a * n_v : nullptr;

    float4 buf[2][U];
    int jb[2][U];                      // block index of each fetched block (-1: none)
    long long rsb[2];                  // the fetched row's total, loaded with its blocks
    f2_t kl = 0ULL, tv = 0ULL, kt = 0ULL, ms = 0ULL, mc = 0ULL;

    // S: which register buffer (a compile-time index, so the buffers stay in registers)
    auto fetch = [&](auto S_, int64_t x, int g) {
        constexpr int s = decltype(S_)::value;
        const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
        rsb[s] = MERGED ? rowsum[x] : 0LL;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int i = g * 32 * U + u * 32 + lane;
            jb[s][u] = i < nl ? (int)lst[i] : -1;
            buf[s][u] = jb[s][u] >= 0 ? __ldcs(row + jb[s][u]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto compute = [&](auto S_) {
        constexpr int s = decltype(S_)::value;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = jb[s][u];
            if (j < 0) break;
            block_terms<KL, TV, KLT, MERGED>(buf[s][u], tP4[j], tF4[j], tE4[j], kl, tv, kt, ms, mc);
        }
    };
    auto finish = [&](auto S_, int64_t x) {
        constexpr int s = decltype(S_)::value;
        float k0, k1, v0, v1, t0, t1;
        upk(kl, k0, k1);
        upk(tv, v0, v1);
        upk(kt, t0, t1);
        float skl = k0 + k1, stv = v0 + v1, skt = t0 + t1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            if (KL) skl += __shfl_xor_sync(0xffffffffu, skl, o);
            if (TV) stv += __shfl_xor_sync(0xffffffffu, stv, o);
            if (KLT) skt += __shfl_xor_sync(0xffffffffu, skt, o);
        }
        const double Mx_d = MERGED ? total62(rsb[s]) - lane_mass_sum(ms, mc) : 0.0;
        const float Mx = (float)Mx_d;
        if (KL) {
            const float merged = (MERGED && Mx > 0.f) ? Mx * logf(Mx / fmaxf(Mt, FLT_MIN)) : 0.f;
            skl = __fmaf_rn(skl, kLn2s, merged);
            if (skl < kExactBelowS)                      // warp-uniform
                skl = kept_kl_exact<false>(P, x, k_pad, lst, nl, tP4, tL, tE, tab, lane) + merged;
        }
        if (KLT) {
            const float merged = (MERGED && Mt > 0.f) ? Mt * logf(Mt / fmaxf(Mx, FLT_MIN)) : 0.f;
            skt = __fmaf_rn(-skt, kLn2s, merged);
            if (skt < kExactBelowS)
                skt = kept_kl_exact<true>(P, x, k_pad, lst, nl, tP4, tL, tE, tab, lane) + merged;
        }
        if (lane == 0) {
            if (KL) okl[x] = skl;
            if (TV) otv[x] = MERGED ? stv + (float)fabs(Mx_d - Mt_d) : stv;
            if (KLT) okt[x] = skt;
        }
        kl = tv = kt = ms = mc = 0ULL;
    };

    using B0 = std::integral_constant<int, 0>;
    using B1 = std::integral_constant<int, 1>;
    auto advance = [&](int64_t &xx, int &gg) {
        if (++gg == ngroups) {
            gg = 0;
            xx += nwarps;
        }
    };
    int64_t x = warp;
    int g = 0;
    if (x >= n_v) return;
    fetch(B0{}, x, g);
    for (;;) {
        int64_t xn = x;
        int gn = g;
        advance(xn, gn);
        if (xn < n_v) fetch(B1{}, xn, gn);
        compute(B0{});
        if (xn != x) finish(B0{}, x);
        if (xn >= n_v) break;
        x = xn;
        g = gn;
        advance(xn, gn);
        if (xn < n_v) fetch(B0{}, xn, gn);
        compute(B1{});
        if (xn != x) finish(B1{}, x);
        if (xn >= n_v) break;
        x = xn;
        g = gn;
    }
}

// exact (table) KL~ of one CSR row for one warp: sum over the row's entries
// of P[x,b] log(P[x,b] / P[t,b]), the target's table mantissa logs from its
// staged row in global memory, its biased exponents every es floats of tE
__device__ __forceinline__ float csr_kl_exact(const float *__restrict__ val, const uint16_t *__restrict__ col,
                                              int64_t o0, int64_t o1, const float *__restrict__ gL,
                                              const float *tE, int es, const float *tab, int lane) {
    float k0 = 0.0f, k1 = 0.0f;
    int q = 0;
    for (int64_t i = o0 + lane; i < o1; i += 32, ++q) {
        const float v = __ldcg(val + i);
        const int c = col[i];
        float lm, Eb;
        split_log<false>(v, tab, lm, Eb);
        const float lr = __fmaf_rn(__fadd_rn(Eb, -tE[es * c]), kLn2s, __fadd_rn(lm, -__ldg(gL + c)));
        if (q & 1)
            k1 = __fmaf_rn(v, lr, k1);
        else
            k0 = __fmaf_rn(v, lr, k0);
    }
    float s = k0 + k1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// the staged target mass over one CSR row's columns, sum_{b in S_x} P~[t,b],
// in the order csr_stream_kernel adds a row: lane l takes the pairs of
// entries i, i + 1 with i = a + 2 l (mod 64), a the row's first entry rounded
// down to a multiple of 8 (where its first chunk starts), in increasing
// order, then the fixed shuffle tree -- on row x = t it reproduces the
// target's total bit for bit
__device__ __forceinline__ float csr_target_mass(const uint16_t *__restrict__ col, int64_t o0, int64_t o1,
                                                 const float *tP, int lane) {
    float a = 0.0f;
    for (int64_t i = (o0 & ~(int64_t)7) + 2 * lane; i < o1; i += 64) {
        if (i >= o0) a = __fadd_rn(a, tP[col[i]]);
        if (i + 1 >= o0 && i + 1 < o1) a = __fadd_rn(a, tP[col[i + 1]]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = __fadd_rn(a, __shfl_xor_sync(0xffffffffu, a, o));
    return a;
}

// csr_stream_kernel's configurations: W warps, NS chunk buffers of C entries per warp
constexpr int kCsrW = 16, kCsrC = 512, kCsrNS = 3;

// KL~ and TV~ from the CSR rows, one target per grid row (blockIdx.y).
// Dynamic smem: the target's thresholded row P~[t,:] and its (hardware
// mantissa log2, biased exponent) pairs, staged by bulk copies; then, per
// warp, NS chunk buffers of C values and C columns.  One warp per row (rows
// strided by the grid's warp count).  A row is cut into chunks of at most C
// entries, from its first entry rounded down to a multiple of 8 to its last
// rounded up (so that both arrays start and end on 16-byte boundaries); each
// chunk is one pair of bulk copies completing on the warp's own mbarrier,
// NS chunks in flight per warp.  Lane 0 issues; the row offsets are read one
// row ahead.  Each lane takes two neighbouring entries per step (one 8-byte
// and one 4-byte shared load).  Per entry v = P[x,b] at column c (the
// rounded ends' entries of other rows skipped):
//   KL: v ((lg2 m_v - lg2 m_t[c]) + (E_v - E_t[c])), times ln2 at the end
//   TV: |v - P~[t,c]|, and the target mass the row covers, P~[t,c]
// so that TV~ = sum |v - P~[t,c]| + (M~_t - covered), M~_t the target's own
// total by the same additions (csr_target_mass on row t).  Rows with
// KL~ < DD_EXACT_BELOW are recomputed with the table logarithm, the target's
// table mantissa logs read from the staged array in global memory.
template <int W, int C, int NS, bool KL, bool TV>
__global__ void __launch_bounds__(W * 32, 1) csr_stream_kernel(
    const float *__restrict__ val, const uint16_t *__restrict__ col, const int64_t *__restrict__ off, int64_t n_v,
    int64_t k_pad, const float *__restrict__ sP, const float *__restrict__ sL, const float *__restrict__ sE,
    const float *__restrict__ sF, const int32_t *__restrict__ targets, float *__restrict__ out_kl,
    float *__restrict__ out_tv, int *__restrict__ err_flag) {
    static_assert(C % 64 == 0 && NS >= 2, "chunks of whole warp steps, at least double buffered");
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ __align__(8) uint64_t wbar[W][NS];
    __shared__ int64_t wdesc[W][NS][4];        // per chunk buffer: row (n_v: none), o0, o1, chunk start
    __shared__ float tab[2 * kLogTab];
    __shared__ float mt_sh;
    float *tP = smem;
    float2 *tEF = reinterpret_cast<float2 *>(smem + k_pad);              // (lg2 m_t, E_t) per column
    float *region = smem + 3 * k_pad;                                    // chunk buffers (first: E_t, lg2 m_t)
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *bv = region + (int64_t)wid * NS * C;
    uint16_t *bc = reinterpret_cast<uint16_t *>(region + (int64_t)W * NS * C) + (int64_t)wid * NS * C;
    uint64_t *wb = wbar[wid];
    int64_t(*wd)[4] = wdesc[wid];
    const int a_t = blockIdx.y;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        for (int w = 0; w < W; ++w)
            for (int s = 0; s < NS; ++s) mbar_init(&wbar[w][s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t row_bytes = (uint32_t)(k_pad * sizeof(float));
        mbar_expect_tx(&bar, 3u * row_bytes);
        bulk_g2s(tP, sP + (int64_t)a_t * k_pad, row_bytes, &bar);
        bulk_g2s(region, sE + (int64_t)a_t * k_pad, row_bytes, &bar);
        bulk_g2s(region + k_pad, sF + (int64_t)a_t * k_pad, row_bytes, &bar);
    }
    build_log_table(tab);
    // every thread waits (bounded); a CTA whose wait gave up waits once more
    // (also bounded) so that it does not exit while its copies may still land
    const bool ok = mbar_wait(&bar, 0, err_flag);
    if (!ok) mbar_wait(&bar, 0, err_flag);
    if (ok)
        for (int64_t c = threadIdx.x; c < k_pad; c += blockDim.x) tEF[c] = make_float2(region[k_pad + c], region[c]);
    __syncthreads();
    if (TV && threadIdx.x < 32) {
        const int64_t t = targets[a_t];
        const float m = ok ? csr_target_mass(col, off[t], off[t + 1], tP, lane) : 0.0f;
        if (lane == 0) mt_sh = m;
    }
    __syncthreads();
    if (!ok) return;
    const float Mt = TV ? mt_sh : 0.0f;
    const float *gL = sL + (int64_t)a_t * k_pad;
    float *okl = KL ? out_kl + (int64_t)a_t * n_v : nullptr;
    float *otv = TV ? out_tv + (int64_t)a_t * n_v : nullptr;
    const int64_t nw = (int64_t)gridDim.x * W;

    // issue state (meaningful in lane 0): row ix with entries [io0, io1),
    // next chunk start ia; the offsets of row ix + nw already requested
    int64_t ix = (int64_t)blockIdx.x * W + wid, io0 = 0, io1 = 0, ia = 0, po0 = 0, po1 = 0;
    if (lane == 0 && ix < n_v) {
        io0 = __ldg(off + ix);
        io1 = __ldg(off + ix + 1);
        ia = io0 & ~(int64_t)7;
        if (ix + nw < n_v) {
            po0 = __ldg(off + ix + nw);
            po1 = __ldg(off + ix + nw + 1);
        }
    }
    auto issue = [&](int s) {                  // lane 0: the next chunk into buffer s
        if (ix >= n_v) {
            wd[s][0] = n_v;
            return;
        }
        const int64_t end8 = (io1 + 7) & ~(int64_t)7;
        const int64_t e = ia + C < end8 ? ia + C : end8;
        const uint32_t ne = (uint32_t)(e - ia);
        wd[s][0] = ix;
        wd[s][1] = io0;
        wd[s][2] = io1;
        wd[s][3] = ia;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&wb[s], ne * 6u);       // 0 for an empty row: the phase completes at once
        if (ne) {
            bulk_g2s(bv + s * C, val + ia, ne * 4u, &wb[s]);
            bulk_g2s(bc + s * C, col + ia, ne * 2u, &wb[s]);
        }
        if (e < end8) {
            ia = e;
        } else {
            ix += nw;
            io0 = po0;
            io1 = po1;
            ia = io0 & ~(int64_t)7;
            if (ix + nw < n_v) {
                po0 = __ldg(off + ix + nw);
                po1 = __ldg(off + ix + nw + 1);
            }
        }
    };
    if (lane == 0)
        for (int s = 0; s < NS; ++s) issue(s);
    __syncwarp();

    float kl = 0.0f, tv = 0.0f, cov = 0.0f;
    auto entry = [&](float v, int c) {
        if (KL) {
            const int bits = __float_as_int(v);
            const float lf = lg2_mant(bits);
            const float eb = __int_as_float((int)__funnelshift_r((unsigned)bits, (unsigned)kMagicHi, 23));
            const float2 fe = tEF[c];
            kl = __fmaf_rn(v, __fadd_rn(__fadd_rn(lf, -fe.x), __fadd_rn(eb, -fe.y)), kl);
        }
        if (TV) {
            const float pt = tP[c];
            tv = __fadd_rn(tv, fabsf(__fadd_rn(v, -pt)));
            cov = __fadd_rn(cov, pt);
        }
    };
    int s = 0;
    uint32_t ph = 0;
    for (;;) {
        const int64_t x = wd[s][0];
        if (x >= n_v) break;
        const int64_t o0 = wd[s][1], o1 = wd[s][2], a = wd[s][3];
        if (!mbar_wait_suspend(&wb[s], ph, err_flag)) {
            // give up: wait (bounded) for this warp's other copies in flight, then leave
            for (int j = 1; j < NS; ++j) {
                const int sj = (s + j) % NS;
                if (wd[sj][0] < n_v) mbar_wait_suspend(&wb[sj], sj > s ? ph : ph ^ 1u, err_flag);
            }
            return;
        }
        const int64_t end8 = (o1 + 7) & ~(int64_t)7;
        const int ne = (int)((a + C < end8 ? a + C : end8) - a);
        const int lo = (int)(o0 > a ? o0 - a : 0);
        const int hi = (int)(o1 - a < ne ? o1 - a : ne);
        const float *cv = bv + s * C;
        const uint16_t *cc = bc + s * C;
#pragma unroll 2
        for (int q = 2 * lane; q < ne; q += 64) {
            const float2 v2 = *reinterpret_cast<const float2 *>(cv + q);
            const uint32_t c2 = *reinterpret_cast<const uint32_t *>(cc + q);
            if (q >= lo && q + 1 < hi) {       // both entries the row's (all but a row's two ends)
                entry(v2.x, (int)(c2 & 0xFFFFu));
                entry(v2.y, (int)(c2 >> 16));
            } else {
                if (q >= lo && q < hi) entry(v2.x, (int)(c2 & 0xFFFFu));
                if (q + 1 >= lo && q + 1 < hi) entry(v2.y, (int)(c2 >> 16));
            }
        }
        __syncwarp();                          // buffer s read by every lane
        if (lane == 0) issue(s);
        __syncwarp();                          // its descriptor visible
        if (a + C >= end8) {                   // the row's last chunk: reduce and store
            float skl = kl, stv = tv, sc = cov;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                if (KL) skl += __shfl_xor_sync(0xffffffffu, skl, o);
                if (TV) {
                    stv += __shfl_xor_sync(0xffffffffu, stv, o);
                    sc = __fadd_rn(sc, __shfl_xor_sync(0xffffffffu, sc, o));
                }
            }
            if (KL) {
                skl *= kLn2s;
                if (skl < kExactBelowS)              // warp-uniform
                    skl = csr_kl_exact(val, col, o0, o1, gL, reinterpret_cast<const float *>(tEF) + 1, 2, tab,
                                       lane);
            }
            if (lane == 0) {
                if (KL) okl[x] = skl;
                if (TV) otv[x] = __fadd_rn(stv, __fadd_rn(Mt, -sc));
            }
            kl = tv = cov = 0.0f;
        }
        if (++s == NS) {
            s = 0;
            ph ^= 1u;
        }
    }
}

int sms_now() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

}  // namespace

int64_t sparse_list_pitch(int64_t k_pad) { return (((k_pad >> 2) + 7) / 8) * 8; }

size_t sparse_field_smem(int64_t k_pad) {
    return 4 * (size_t)k_pad * sizeof(float) + (size_t)sparse_list_pitch(k_pad) * sizeof(uint16_t);
}

size_t sparse_count_bytes(int32_t T) { return ((size_t)T * sizeof(int32_t) + 15) / 16 * 16; }

// dynamic shared memory of csr_stream_kernel: the target's P~ row and
// (lg2 m, E) pairs, then W warps x NS chunk buffers of C FP32 values and C
// 16-bit columns (at least the two staged rows the pairs are built from); at
// most the 227 KB a CTA may hold less 4 KB for its static arrays
constexpr size_t kCsrSmemMax = 232448 - 4096;

size_t csr_stream_smem(int64_t k_pad, int W, int C, int NS) {
    const size_t bufs = (size_t)W * NS * C * (sizeof(float) + sizeof(uint16_t));
    return 3 * (size_t)k_pad * sizeof(float) + std::max(bufs, 2 * (size_t)k_pad * sizeof(float));
}

size_t sparse_stage_bytes(int64_t k_pad, int32_t T) {
    return 4 * (size_t)T * k_pad * sizeof(float) + (size_t)T * sparse_list_pitch(k_pad) * sizeof(uint16_t) +
           sparse_count_bytes(T) + (size_t)T * sizeof(double);
}

dd_status build_sparse_rows(DevMesh &m, double theta, cudaStream_t s, int64_t *kept_out, int64_t *bytes_out,
                            std::string &err) {
    if (m.k > 65536) {
        err = "sparse fields: more than 65,536 boundary columns (16-bit column ids)";
        return DD_EINVAL;
    }
    if (csr_stream_smem(m.k_pad, 8, 128, 2) > kCsrSmemMax || sparse_field_smem(m.k_pad) > kCsrSmemMax) {
        err = "sparse fields: the target's staged row does not fit in shared memory (k above about 13,500)";
        return DD_EINVAL;
    }
    long long *rowsum = nullptr;
    unsigned long long *counts = nullptr;
    int32_t *row_kept = nullptr;
    float *row_thr = nullptr;
    int64_t *off = nullptr;
    float *val = nullptr;
    uint16_t *col = nullptr;
    auto fail = [&](cudaError_t e) {
        for (void *p : {(void *)rowsum, (void *)counts, (void *)row_kept, (void *)row_thr, (void *)off, (void *)val,
                        (void *)col})
            if (p) cudaFree(p);
        cudaGetLastError();
        err = std::string("sparse fields: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? DD_ENOMEM : DD_ECUDA;
    };
    const int64_t n = m.n_v;
    cudaError_t e = cudaMalloc((void **)&rowsum, (size_t)n * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&counts, 2 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void **)&row_kept, (size_t)n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&row_thr, (size_t)n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&off, (size_t)(n + 1) * sizeof(int64_t));
    unsigned long long hc[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) {
        sparse_rows_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(m.P, n, m.k_pad, (float)theta, rowsum, counts,
                                                                   row_kept, row_thr);
        e = cudaGetLastError();
    }
    // row offsets: an exclusive scan of the per-row counts on the host (a one-off step)
    std::vector<int32_t> hk((size_t)n);
    std::vector<int64_t> ho((size_t)n + 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hc, counts, sizeof hc, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hk.data(), row_kept, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e);
    ho[0] = 0;
    for (int64_t x = 0; x < n; ++x) ho[x + 1] = ho[x] + hk[x];
    const int64_t nnz = ho[n];
    e = cudaMemcpyAsync(off, ho.data(), (size_t)(n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s);
    // both arrays padded (with zeros) to a multiple of 8 entries: the row
    // stream copies whole 16-byte pieces, up to the last row's end rounded up
    const int64_t nnz8 = (std::max<int64_t>(nnz, 1) + 7) / 8 * 8;
    if (e == cudaSuccess) e = cudaMalloc((void **)&val, (size_t)nnz8 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc((void **)&col, (size_t)nnz8 * sizeof(uint16_t));
    if (e == cudaSuccess) e = cudaMemsetAsync(val + nnz, 0, (size_t)(nnz8 - nnz) * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(col + nnz, 0, (size_t)(nnz8 - nnz) * sizeof(uint16_t), s);
    if (e == cudaSuccess) {
        csr_fill_kernel<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(m.P, n, m.k_pad, row_thr, off, val, col);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e);
    cudaFree(counts);
    cudaFree(row_kept);
    cudaFree(row_thr);
    m.sp_rowsum = rowsum;
    m.sp_off = off;
    m.sp_val = val;
    m.sp_col = col;
    m.sp_theta = (float)theta;
    m.sp_kept = (int64_t)hc[0];
    m.sp_bytes = (n + 1) * (int64_t)sizeof(int64_t) + nnz * (int64_t)(sizeof(float) + sizeof(uint16_t));
    for (void *p : {(void *)rowsum, (void *)off, (void *)val, (void *)col}) m.owned.push_back(p);
    m.bytes += n * (int64_t)sizeof(long long) + m.sp_bytes;
    if (kept_out) *kept_out = m.sp_kept;
    if (bytes_out) *bytes_out = m.sp_bytes;
    return DD_OK;
}

void launch_sparse_fields(const DevMesh &m, const int32_t *d_targets, float4 *stage, int32_t T, float *out_kl,
                          float *out_tv, float *out_klt, bool merged, int *err_flag, cudaStream_t s) {
    float *sP = reinterpret_cast<float *>(stage);
    const float *sL = sP + (int64_t)T * m.k_pad;
    const float *sE = sL + (int64_t)T * m.k_pad;
    const float *sF = sE + (int64_t)T * m.k_pad;
    const int64_t lp = sparse_list_pitch(m.k_pad);
    uint16_t *sList = reinterpret_cast<uint16_t *>(const_cast<float *>(sF) + (int64_t)T * m.k_pad);
    int32_t *sCount = reinterpret_cast<int32_t *>(sList + (int64_t)T * lp);
    double *sMt = reinterpret_cast<double *>(reinterpret_cast<char *>(sCount) + sparse_count_bytes(T));
    {
        KMark km_("sparse_stage_kernel", s);
        sparse_stage_kernel<<<(unsigned)T, 256, 0, s>>>(m.P, sP, sE, sF, m.k_pad, m.sp_theta, sList, lp, sCount,
                                                         m.sp_rowsum, d_targets, sMt);
    }
    const int64_t row_blocks = (m.n_v + 7) / 8;
    auto grid_x = [&](auto kern, size_t smem) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t gx = (int64_t)sms_now() * per_sm / T;
        if (gx < 1) gx = 1;
        if (gx > row_blocks) gx = row_blocks;
        return (unsigned)gx;
    };
    // the dense rows at the target's blocks: KLT~ (or the merged-bin fields)
    auto go = [&](auto kern) {
        const size_t smem = sparse_field_smem(m.k_pad);
        const unsigned gx = grid_x(kern, smem);
        KMark km_("sparse_field_kernel", s);
        kern<<<dim3(gx, (unsigned)T), 256, smem, s>>>(m.P, m.n_v, m.k_pad, sP, sL, sE, sF, sList, lp, sCount, sMt,
                                                       m.sp_rowsum, out_kl, out_tv, out_klt, err_flag);
    };
    // the CSR rows: KL~ and TV~.  The deepest pipeline whose buffers fit next
    // to the staged target row: 16 warps x 3 chunks of 512 entries (one CTA
    // per SM, 144 KB of chunk buffers), else fewer or shorter chunks.
    auto go_csr = [&](auto kern, int W, int C, int NS) {
        const size_t smem = csr_stream_smem(m.k_pad, W, C, NS);
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, W * 32, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t gx = (int64_t)sms_now() * per_sm / T;
        const int64_t row_groups = (m.n_v + W - 1) / W;
        if (gx < 1) gx = 1;
        if (gx > row_groups) gx = row_groups;
        KMark km_("csr_stream_kernel", s);
        kern<<<dim3((unsigned)gx, (unsigned)T), W * 32, smem, s>>>(m.sp_val, m.sp_col, m.sp_off, m.n_v, m.k_pad, sP,
                                                                    sL, sE, sF, d_targets, out_kl, out_tv, err_flag);
    };
    auto csr = [&](auto kl_, auto tv_) {
        constexpr bool KL = decltype(kl_)::value, TV = decltype(tv_)::value;
        if (csr_stream_smem(m.k_pad, kCsrW, kCsrC, kCsrNS) <= kCsrSmemMax)
            go_csr(csr_stream_kernel<kCsrW, kCsrC, kCsrNS, KL, TV>, kCsrW, kCsrC, kCsrNS);
        else if (csr_stream_smem(m.k_pad, 8, 512, 2) <= kCsrSmemMax)
            go_csr(csr_stream_kernel<8, 512, 2, KL, TV>, 8, 512, 2);
        else
            go_csr(csr_stream_kernel<8, 128, 2, KL, TV>, 8, 128, 2);
    };
    if (merged) {
        // two blocks per lane and item, three CTAs per SM (measured: U = 4 or 8 with
        // two CTAs per SM were slower; the pass is issue- and latency-bound)
        const int mask = (out_kl ? 1 : 0) | (out_tv ? 2 : 0) | (out_klt ? 4 : 0);
        switch (mask) {
            case 1: go(sparse_field_kernel<2, true, false, false, true>); break;
            case 2: go(sparse_field_kernel<2, false, true, false, true>); break;
            case 3: go(sparse_field_kernel<2, true, true, false, true>); break;
            case 4: go(sparse_field_kernel<2, false, false, true, true>); break;
            case 5: go(sparse_field_kernel<2, true, false, true, true>); break;
            case 6: go(sparse_field_kernel<2, false, true, true, true>); break;
            default: go(sparse_field_kernel<2, true, true, true, true>); break;
        }
        return;
    }
    using Yes = std::true_type;
    using No = std::false_type;
    if (out_kl && out_tv)
        csr(Yes{}, Yes{});
    else if (out_kl)
        csr(Yes{}, No{});
    else if (out_tv)
        csr(No{}, Yes{});
    if (out_klt) go(sparse_field_kernel<2, false, false, true, false>);
}
