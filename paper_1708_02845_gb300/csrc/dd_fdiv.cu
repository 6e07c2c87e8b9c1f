// Other f-divergence fields, Section VI: for a target t and every vertex x
//
//   d_f,t(x) = sum_b P[x,b] f(P[t,b] / P[x,b])
//
// with f in the form f(1) = f'(1) = 0 (adding c (u - 1) to f does not change
// a divergence between probability vectors), so that every term is
// non-negative and near the target no sum cancels:
//
//   chi2        (u - 1)^2                 term (P_t - P_x)^2 / P_x
//   hellinger   (sqrt u - 1)^2            term (P_t - P_x)^2 / (sqrt P_t + sqrt P_x)^2
//   power p     |1 - u|^p, p >= 1         term |P_t - P_x| (|P_t - P_x| / P_x)^(p-1)
//   alpha a     4/(1-a^2)(1 - u^((1+a)/2)) + 2/(1-a)(u - 1)
//               term P_x 2/(1-a) [expm1(L) - expm1(e L)/e], e = (1+a)/2, L = log(P_t/P_x)
//   kl_reverse  u log u                   term P_t log(P_t / P_x)
//
// L is formed from exact split logarithms (exponent difference exact, mantissa
// logs from the same table as the KL kernels), so x = t gives L = 0 and a
// zero term.  For |L| < 1/8 the alpha bracket is summed as its series
// sum_{n>=2} (1 - e^(n-1)) L^n / n! (six terms), which has no cancellation.
// A term with P[x,b] = 0 < P[t,b] is +inf for chi2, p > 1, alpha > 1 and
// kl_reverse; the kernels evaluate it with P[x,b] taken as FLT_MIN, which
// gives a finite value of order 1e30 or an FP32 overflow to +inf (for
// kl_reverse, P[t,b] (log P[t,b] - log FLT_MIN), as dd_distance does for KL).
//
// One warp per row, lanes along b, 16-byte loads of P four float4 per lane
// ahead; the target's P, log-mantissa and exponent rows staged in shared
// memory (the arrays of stage_targets_kernel); one target per grid row.
// The reverse KL and the alpha family with 0.1 <= |e| <= 2, |1 - e| >= 0.1
// take a first pass with hardware logarithms (and exp2) and recompute in the
// exact form above only the rows whose value is below DD_EXACT_BELOW
// (two_pass_kernel); the other families and parameters take the exact form
// throughout (fdiv_kernel).
#include <algorithm>
#include <cfloat>
#include <cmath>

#include "dd_f32x2.cuh"
#include "dd_internal.h"
#include "dd_splitlog.cuh"

namespace {

constexpr float kLn2f = 0.693147180559945309f;

struct FdParams {
    float p;         // power: p; alpha: e = (1 + a)/2
    float lin;       // alpha: 2 / (1 - a)
    int alpha_gt1;   // alpha: a > 1
    float inv_e;     // alpha: 1 / e
    float below;     // two-pass families: rows whose first-pass value is below this are recomputed
    float c[6];      // alpha exact form: (1 - e^(n-1)) / n!, n = 2 .. 7
};

// log(P_t / P_x) from the split logarithms (target side staged)
__device__ __forceinline__ float log_ratio(float px, float lmt, float Ebt, const float *tab) {
    float lm, Eb;
    split_log<true>(px, tab, lm, Eb);
    return __fmaf_rn(__fadd_rn(Ebt, -Eb), kLn2f, __fadd_rn(lmt, -lm));
}

// expm1(L) - expm1(e L) / e; for |L| < 1/8 its series sum_{n>=2} c_n L^n
// with c_n = (1 - e^(n-1)) / n! (FP64 on the host), which does not cancel
__device__ __forceinline__ float alpha_bracket(float L, const FdParams &q) {
    if (fabsf(L) < 0.125f) {
        float s = q.c[5];
#pragma unroll
        for (int i = 4; i >= 0; --i) s = __fmaf_rn(s, L, q.c[i]);
        return L * L * s;
    }
    return expm1f(L) - expm1f(q.p * L) * q.inv_e;
}

enum { kChi2 = DD_DIV_CHI2, kHell = DD_DIV_HELLINGER, kPow = DD_DIV_POWER, kAlpha = DD_DIV_ALPHA,
       kKlRev = DD_DIV_KL_REVERSE };

// Hardware approximations (one MUFU instruction each; relative errors of a
// few 2^-23, absolute error of lg2 a few 1e-7).  The chi2, Hellinger and power
// terms are non-negative, so the relative error of every term, and of the
// row's sum, stays at that level -- far inside the 1e-5 of the FP32 path.
__device__ __forceinline__ float rcp_hw(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_hw(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_hw(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float ex2_hw(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int FAM>
__device__ __forceinline__ float fterm(float px, float pt, float lmt, float Ebt, const FdParams &q, const float *tab) {
    if (FAM == kChi2) {
        const float d = pt - px;
        return d * d * rcp_hw(fmaxf(px, FLT_MIN));
    } else if (FAM == kHell) {
        const float d = pt - px, s = sqrt_hw(pt) + sqrt_hw(px);
        if (s == 0.0f) return 0.0f;
        const float r = d * rcp_hw(s);
        return r * r;
    } else if (FAM == kPow) {
        // |d| (|d| / P_x)^(p-1) = |d| 2^((p-1) log2(|d| / P_x))
        const float ad = fabsf(pt - px);
        if (ad == 0.0f || q.p == 1.0f) return ad;      // p = 1: TV's term, also where P_x = 0
        return ad * ex2_hw((q.p - 1.0f) * lg2_hw(ad * rcp_hw(fmaxf(px, FLT_MIN))));
    } else if (FAM == kAlpha) {
        if (px == 0.0f) return pt == 0.0f ? 0.0f : (q.alpha_gt1 ? INFINITY : q.lin * pt);
        return px * q.lin * alpha_bracket(log_ratio(px, lmt, Ebt, tab), q);
    } else {   // kKlRev
        if (pt == 0.0f) return 0.0f;
        return pt * log_ratio(px, lmt, Ebt, tab);
    }
}

// reverse KL term where P[x,b] is below FLT_MIN but its log2 lx is known:
// P_t (log P_t - log P_x) = P_t ((E_t - lx) ln2 + lm_t)
__device__ __forceinline__ float klrev_logp_term(float pt, float lmt, float Ebt, float lx) {
    if (pt == 0.0f) return 0.0f;
    return pt * __fmaf_rn(__fadd_rn(__fsub_rn(Ebt, 12583039.0f), -lx), kLn2f, lmt);
}

// First-pass alpha terms of four entries per lane, from L2 = log2(P_t / P_x)
// formed from exact exponents and hardware mantissa logs:
//   P_x lin [expm1(L) - expm1(e L)/e] = lin [(P_t - P_x) - P_x (2^(e L2) - 1)/e]
// with the hardware exp2.  Its error is absolute, not relative to the term:
// |lin| / |e| 2^-22 P_x 2^(e L2) from the exp2, whose sum over b is at most
// |lin| / |e| 2^-22 (sum_b P_t^e P_x^(1-e) <= 1 for 0 < e < 1, Hoelder; for
// e > 1 or e < 0 the value itself grows with that sum), plus the log's
// DD_FAST_LOG_SPREAD, whose effect vanishes to first order at u = 1.  So the
// rows whose first-pass value is below q.below = max(DD_EXACT_BELOW,
// 2e5 |lin| / |e| 2^-22) are recomputed in the exact form, and every other
// value is within 1e-5 / 2 of exact, relatively.  The entries with P_x = 0 or
// P_t = 0 take their limits by selection, evaluated only when a lane of the
// warp holds one; every lane of the warp must call it (padding entries pass
// P_x = P_t = 0 and give 0).
__device__ __forceinline__ void alpha_fast4(const float (&px)[4], const float (&pt)[4], const float (&ft)[4],
                                            const float (&et)[4], const FdParams &q, float (&t)[4]) {
    // the adds and multiplies two entries at a time in packed FP32x2 (each half
    // rounds exactly as the scalar operation: a product is fma(a, b, 0))
    const f2_t mone = pk(-1.0f, -1.0f), zero = pk(0.0f, 0.0f);
    const f2_t e2 = pk(q.p, q.p), nie2 = pk(-q.inv_e, -q.inv_e), lin2 = pk(q.lin, q.lin);
    bool special = false;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j0 = 2 * h, j1 = 2 * h + 1;
        // no clamp: P holds no subnormals, and a zero entry takes its limit below
        const int b0 = __float_as_int(px[j0]), b1 = __float_as_int(px[j1]);
        const f2_t lf = pk(lg2_mant(b0), lg2_mant(b1));
        const f2_t eb = pk(__int_as_float((int)__funnelshift_r((unsigned)b0, (unsigned)kMagicHi, 23)),
                           __int_as_float((int)__funnelshift_r((unsigned)b1, (unsigned)kMagicHi, 23)));
        const f2_t px2 = pk(px[j0], px[j1]), pt2 = pk(pt[j0], pt[j1]);
        // L2 = (lg2 m_t - lg2 m_x) + (E_t - E_x)
        const f2_t L2 = add2(fma2(lf, mone, pk(ft[j0], ft[j1])), fma2(eb, mone, pk(et[j0], et[j1])));
        float y0, y1;
        upk(fma2(L2, e2, zero), y0, y1);
        const f2_t um1 = add2(pk(ex2_hw(y0), ex2_hw(y1)), mone);                    // 2^(e L2) - 1
        const f2_t r = fma2(fma2(px2, nie2, zero), um1, fma2(px2, mone, pt2));      // (P_t - P_x) - P_x um1 / e
        upk(fma2(r, lin2, zero), t[j0], t[j1]);
        // a zero factor among P_x, P_t (a product that underflows only sends the
        // warp through the selection, which leaves every other entry as it is)
        float z0, z1;
        upk(fma2(px2, pt2, zero), z0, z1);
        special |= (z0 == 0.0f) | (z1 == 0.0f);
    }
    if (__any_sync(0xffffffffu, special)) {
        const float at_px0 = q.alpha_gt1 ? INFINITY : q.lin;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v = pt[j] == 0.0f ? px[j] * q.inv_e : t[j];                   // u = 0: lin P_x (1/e - 1) = P_x / e
            v = px[j] == 0.0f ? (pt[j] == 0.0f ? 0.0f : at_px0 * pt[j]) : v;    // P_x = 0: lin P_t, or +inf for a > 1
            t[j] = v;
        }
    }
}

// Rows x = warp, warp + nwarps, ... of P streamed by one warp in chunks of
// 32 U float4 (U per lane), with two register buffers: the loads of the next
// chunk (of this row or the next) are in flight while the current one is
// computed.  chunk(b, x, c0): the lane's U float4 b of row x, float4 columns
// c0 + u * 32 + lane (zero past the row's end); done(x): row x is complete.
template <int U, typename Chunk, typename Done>
__device__ __forceinline__ void stream_rows(const float *__restrict__ P, int64_t n_v, int64_t k_pad, int64_t warp,
                                            int64_t nwarps, int lane, Chunk chunk, Done done) {
    const int nvec = (int)(k_pad >> 2);
    const int nch = (nvec + 32 * U - 1) / (32 * U);
    float4 b0[U], b1[U];
    auto fetch = [&](float4(&b)[U], int64_t x, int ch) {
        const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = ch * 32 * U + u * 32 + lane;
            b[u] = c < nvec ? __ldcs(row + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto next = [&](int64_t &x, int &ch) {
        if (++ch == nch) {
            ch = 0;
            x += nwarps;
        }
    };
    int64_t x = warp;
    int ch = 0;
    if (x >= n_v) return;
    fetch(b0, x, 0);
    for (;;) {
        int64_t xn = x;
        int cn = ch;
        next(xn, cn);
        if (xn < n_v) fetch(b1, xn, cn);
        chunk(b0, x, ch * 32 * U);
        if (cn == 0) done(x);
        if (xn >= n_v) return;
        x = xn;
        ch = cn;
        next(xn, cn);
        if (xn < n_v) fetch(b0, xn, cn);
        chunk(b1, x, ch * 32 * U);
        if (cn == 0) done(x);
        if (xn >= n_v) return;
        x = xn;
        ch = cn;
    }
}

// floats per staged row of two_pass_kernel: k_pad rounded up to whole
// chunks of 32 lanes x 8 float4
__host__ __device__ constexpr int64_t two_pass_pitch(int64_t k_pad) { return (k_pad + 1023) / 1024 * 1024; }

// LP (reverse KL only, may be null): log2 P; an entry whose FP32 value is 0
// takes log P[x,b] from it instead of the clamp at FLT_MIN
template <int FAM>
__global__ void __launch_bounds__(256) fdiv_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                                   const float *__restrict__ sP, const float *__restrict__ sL,
                                                   const float *__restrict__ sE, FdParams q, float *__restrict__ out,
                                                   const float *__restrict__ LP) {
    extern __shared__ __align__(16) float fsm[];
    __shared__ float tab[2 * kLogTab];
    float *tP = fsm, *tL = fsm + k_pad, *tE = fsm + 2 * k_pad;
    const int a = blockIdx.y;
    for (int64_t b = threadIdx.x; b < k_pad; b += blockDim.x) {
        tP[b] = sP[(int64_t)a * k_pad + b];
        tL[b] = sL[(int64_t)a * k_pad + b];
        tE[b] = sE[(int64_t)a * k_pad + b];
    }
    build_log_table(tab);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nvec = (int)(k_pad >> 2);
    float s0 = 0.0f, s1 = 0.0f;
    auto chunk = [&](const float4(&v)[4], int64_t x, int c0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int c = c0 + u * 32 + lane;
            if (c >= nvec) break;
            const float4 p4 = reinterpret_cast<const float4 *>(tP)[c];
            const float4 l4 = reinterpret_cast<const float4 *>(tL)[c];
            const float4 e4 = reinterpret_cast<const float4 *>(tE)[c];
            if (FAM == kKlRev && LP &&
                ((v[u].x == 0.f && p4.x != 0.f) || (v[u].y == 0.f && p4.y != 0.f) ||
                 (v[u].z == 0.f && p4.z != 0.f) || (v[u].w == 0.f && p4.w != 0.f))) {
                const float4 lx = reinterpret_cast<const float4 *>(LP + x * k_pad)[c];
                const float px[4] = {v[u].x, v[u].y, v[u].z, v[u].w}, pt[4] = {p4.x, p4.y, p4.z, p4.w};
                const float lt[4] = {l4.x, l4.y, l4.z, l4.w}, et[4] = {e4.x, e4.y, e4.z, e4.w};
                const float l2[4] = {lx.x, lx.y, lx.z, lx.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float t = (px[e] == 0.f && l2[e] > -INFINITY) ? klrev_logp_term(pt[e], lt[e], et[e], l2[e])
                                                                       : fterm<FAM>(px[e], pt[e], lt[e], et[e], q, tab);
                    if (e & 1)
                        s1 += t;
                    else
                        s0 += t;
                }
                continue;
            }
            s0 += fterm<FAM>(v[u].x, p4.x, l4.x, e4.x, q, tab);
            s1 += fterm<FAM>(v[u].y, p4.y, l4.y, e4.y, q, tab);
            s0 += fterm<FAM>(v[u].z, p4.z, l4.z, e4.z, q, tab);
            s1 += fterm<FAM>(v[u].w, p4.w, l4.w, e4.w, q, tab);
        }
    };
    auto done = [&](int64_t x) {
        float sum = s0 + s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (lane == 0) out[(int64_t)a * n_v + x] = sum;
        s0 = s1 = 0.0f;
    };
    stream_rows<4>(P, n_v, k_pad, warp, nwarps, lane, chunk, done);
}

// The reverse KL (the target-weighted KL of dd_distance's DD_F_KLT) and the
// alpha family in two passes, as the streaming KL kernel.  A first pass per
// element with exact exponents and hardware mantissa logs:
//   reverse KL: P_t ((lg2 m_t - lg2 m_x) + (E_t - E_x))   (times ln2 at the end),
//     within ln2 DD_FAST_LOG_SPREAD sum_b P[t,b] = 3.5e-7 of the exact form
//     (the constant part of the mantissa log's error cancels between the two
//     sides);
//   alpha: alpha_fast_term, within a few 1e-6 of the exact term relatively;
// then every row whose first-pass value is below DD_EXACT_BELOW -- the rows
// around the target, x = t among them -- recomputed by its warp with the
// table logarithm (fterm), so every value keeps 1e-5 relative accuracy.  A
// row entry P[x,b] = 0 is taken at FLT_MIN on both passes (reverse KL).
// Shared memory: the target's P, table mantissa log, biased exponent and
// hardware mantissa log2.
template <int FAM>
__global__ void __launch_bounds__(256) two_pass_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                                       const float *__restrict__ sP, const float *__restrict__ sL,
                                                       const float *__restrict__ sE, const float *__restrict__ sF,
                                                       FdParams q, float *__restrict__ out) {
    constexpr int U = 8;       // float4 per lane and buffer: 2 x 4 KB per warp in flight
    extern __shared__ __align__(16) float fsm[];
    __shared__ float tab[2 * kLogTab];
    // alpha: the staged rows zero-padded to whole chunks (two_pass_pitch), so
    // that every lane of a chunk reads its target entries without a test
    const int64_t kp = FAM == kAlpha ? two_pass_pitch(k_pad) : k_pad;
    float *tP = fsm, *tL = fsm + kp, *tE = fsm + 2 * kp, *tF = fsm + 3 * kp;
    const int a = blockIdx.y;
    for (int64_t b = threadIdx.x; b < kp; b += blockDim.x) {
        const bool in = b < k_pad;
        tP[b] = in ? sP[(int64_t)a * k_pad + b] : 0.0f;
        tL[b] = in ? sL[(int64_t)a * k_pad + b] : 0.0f;
        tE[b] = in ? sE[(int64_t)a * k_pad + b] : 0.0f;
        tF[b] = in ? sF[(int64_t)a * k_pad + b] : 0.0f;
    }
    build_log_table(tab);
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nvec = (int)(k_pad >> 2);
    float s0 = 0.0f, s1 = 0.0f;
    auto chunk = [&](const float4(&v)[U], int64_t, int c0) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int c = c0 + u * 32 + lane;
            if (FAM == kAlpha) {
                // every lane takes part (the first pass votes per group of four
                // entries); past the row's end P and the padded target row are 0
                const float4 p4 = reinterpret_cast<const float4 *>(tP)[c];
                const float4 f4 = reinterpret_cast<const float4 *>(tF)[c];
                const float4 e4 = reinterpret_cast<const float4 *>(tE)[c];
                const float px[4] = {v[u].x, v[u].y, v[u].z, v[u].w}, pt[4] = {p4.x, p4.y, p4.z, p4.w};
                const float ft[4] = {f4.x, f4.y, f4.z, f4.w}, et[4] = {e4.x, e4.y, e4.z, e4.w};
                float t[4];
                alpha_fast4(px, pt, ft, et, q, t);
                s0 += t[0];
                s1 += t[1];
                s0 += t[2];
                s1 += t[3];
                continue;
            }
            if (c >= nvec) break;
            const float4 p4 = reinterpret_cast<const float4 *>(tP)[c];
            const float4 f4 = reinterpret_cast<const float4 *>(tF)[c];
            const float4 e4 = reinterpret_cast<const float4 *>(tE)[c];
            const float px[4] = {v[u].x, v[u].y, v[u].z, v[u].w}, pt[4] = {p4.x, p4.y, p4.z, p4.w};
            const float ft[4] = {f4.x, f4.y, f4.z, f4.w}, et[4] = {e4.x, e4.y, e4.z, e4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int bits = __float_as_int(fmaxf(px[e], FLT_MIN));
                const float lf = lg2_mant(bits);
                const float eb = __int_as_float((int)__funnelshift_r((unsigned)bits, (unsigned)kMagicHi, 23));
                const float t = pt[e] * __fadd_rn(__fadd_rn(ft[e], -lf), __fadd_rn(et[e], -eb));
                if (e & 1)
                    s1 += t;
                else
                    s0 += t;
            }
        }
    };
    auto done = [&](int64_t x) {
        float sum = s0 + s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        if (FAM == kKlRev) sum *= kLn2f;
        if (sum < q.below) {                    // warp-uniform: the exact (table) form
            const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
            float r0 = 0.0f, r1 = 0.0f;
            for (int c = lane; c < nvec; c += 32) {
                const float4 vx = __ldcg(row + c);
                const float4 p4 = reinterpret_cast<const float4 *>(tP)[c];
                const float4 l4 = reinterpret_cast<const float4 *>(tL)[c];
                const float4 e4 = reinterpret_cast<const float4 *>(tE)[c];
                r0 += fterm<FAM>(vx.x, p4.x, l4.x, e4.x, q, tab);
                r1 += fterm<FAM>(vx.y, p4.y, l4.y, e4.y, q, tab);
                r0 += fterm<FAM>(vx.z, p4.z, l4.z, e4.z, q, tab);
                r1 += fterm<FAM>(vx.w, p4.w, l4.w, e4.w, q, tab);
            }
            sum = r0 + r1;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        }
        if (lane == 0) out[(int64_t)a * n_v + x] = sum;
        s0 = s1 = 0.0f;
    };
    stream_rows<U>(P, n_v, k_pad, warp, nwarps, lane, chunk, done);
}

}  // namespace

dd_status launch_fdiv(const float *P, int64_t n_v, int64_t k_pad, const float4 *stage, int32_t T, int32_t family,
                      double param, float *out, cudaStream_t s, std::string &err, const float *LP) {
    const float *sP = reinterpret_cast<const float *>(stage);
    const float *sL = sP + (int64_t)T * k_pad;
    const float *sE = sL + (int64_t)T * k_pad;
    const size_t smem = 3 * (size_t)k_pad * sizeof(float);
    if (smem > 200 * 1024) {
        err = "divergence fields: k_pad too large for the staged target row";
        return DD_EINVAL;
    }
    FdParams q{};
    q.p = (float)param;
    q.lin = 0.0f;
    q.alpha_gt1 = 0;
    q.below = (float)DD_EXACT_BELOW;
    bool alpha_fast = false;
    if (family == DD_DIV_ALPHA) {
        const double e = (1.0 + param) / 2.0, lin = 2.0 / (1.0 - param);
        q.p = (float)e;
        q.lin = (float)lin;
        q.alpha_gt1 = param > 1.0;
        q.inv_e = (float)(1.0 / e);
        double en = e, fact = 1.0;                         // e^(n-1), n!
        for (int n = 2; n <= 7; ++n) {
            fact *= n;
            q.c[n - 2] = (float)((1.0 - en) / fact);
            en *= e;
        }
        q.below = (float)std::max((double)DD_EXACT_BELOW, 2e5 * std::fabs(lin / e) * std::ldexp(1.0, -22));
        alpha_fast = std::fabs(e) >= 0.1 && std::fabs(e) <= 2.0 && std::fabs(1.0 - e) >= 0.1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    auto go = [&](auto kern) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t gx = (int64_t)sms * per_sm / (T > 0 ? T : 1);
        const int64_t rows_blocks = (n_v + 7) / 8;
        if (gx < 1) gx = 1;
        if (gx > rows_blocks) gx = rows_blocks;
        {
            KMark km_("fdiv_kernel", s);
            kern<<<dim3((unsigned)gx, (unsigned)T), 256, smem, s>>>(P, n_v, k_pad, sP, sL, sE, q, out,
                                                                   family == DD_DIV_KL_REVERSE ? LP : nullptr);
        }
    };
    if ((family == DD_DIV_KL_REVERSE && !LP) || alpha_fast) {
        // two passes (hardware mantissa logs, then the table form near the target)
        const float *sF = sE + (int64_t)T * k_pad;
        const size_t smem4 =
            4 * (size_t)(family == DD_DIV_ALPHA ? two_pass_pitch(k_pad) : k_pad) * sizeof(float);
        if (smem4 <= 200 * 1024) {
            auto kern = family == DD_DIV_ALPHA ? two_pass_kernel<kAlpha> : two_pass_kernel<kKlRev>;
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4);
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem4);
            if (per_sm < 1) per_sm = 1;
            int64_t gx = (int64_t)sms * per_sm / (T > 0 ? T : 1);
            const int64_t rows_blocks = (n_v + 7) / 8;
            if (gx < 1) gx = 1;
            if (gx > rows_blocks) gx = rows_blocks;
            KMark km_("two_pass_kernel", s);
            kern<<<dim3((unsigned)gx, (unsigned)T), 256, smem4, s>>>(P, n_v, k_pad, sP, sL, sE, sF, q, out);
            return DD_OK;
        }
    }
    switch (family) {
        case DD_DIV_CHI2: go(fdiv_kernel<kChi2>); break;
        case DD_DIV_HELLINGER: go(fdiv_kernel<kHell>); break;
        case DD_DIV_POWER: go(fdiv_kernel<kPow>); break;
        case DD_DIV_ALPHA: go(fdiv_kernel<kAlpha>); break;
        case DD_DIV_KL_REVERSE: go(fdiv_kernel<kKlRev>); break;
        default:
            err = "unknown divergence family";
            return DD_EINVAL;
    }
    return DD_OK;
}
