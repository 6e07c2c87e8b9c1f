// TV and KL divergence fields in FP32, Section IV Eq. (34)-(35).
//
//   TV_t(x) = sum_b |P[x,b] - P[t,b]|
//   KL_t(x) = sum_b P[x,b] (log P[x,b] - log P[t,b])      (Eq. 17, z = x, w = t)
//
// Near the target the two logarithms agree to many digits and KL is a small
// sum of nearly-cancelling terms, so each log is kept as an exact split
//   log p = E ln2 + lm,   E integer,  lm = log(m) for the mantissa m in [1/sqrt2, sqrt2)
// and the difference is formed as (lm_x - lm_t) + (E_x - E_t) ln2: the mantissa
// logs carry relative (not absolute) error, the exponent difference is exact,
// and x = t gives exactly 0 (the same code runs on both operands).  lm uses
// the series log m = 2 atanh(s) = 2 (s + s^3/3 + s^5/5 + s^7/7 + s^9/9),
// s = (m - 1)/(m + 1), |s| <= 0.1716, truncation error below 2e-9 relative.
// Every step uses explicit round-to-nearest intrinsics so all call sites
// produce bit-identical values.  Arguments below FLT_MIN (including the
// 0 log 0 terms, whose weight P[x,b] is 0) are evaluated at FLT_MIN.
//
// Two kernels:
//  * field_stream (few targets): one warp per row, lanes along b, 16-byte
//    loads of P, the target rows staged in shared memory by a bulk async
//    copy completing on an mbarrier, warp-shuffle reductions.  HBM-bound.
//  * field_tile (many targets): 64 rows x 64 targets per CTA, b in chunks of
//    32 staged through shared memory, 4 x 4 register micro-tiles.  Each P
//    element's logarithm is computed once per CTA and reused for 64 targets.
#include <cfloat>
#include <cstdint>

#include "dd_internal.h"

namespace {

constexpr float kLn2 = 0.693147180559945309f;

// ---- packed FP32x2 helpers (two IEEE round-to-nearest operations per instruction)
typedef unsigned long long f2_t;

__device__ __forceinline__ f2_t pk(float a, float b) {
    f2_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2_t r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ f2_t add2(f2_t a, f2_t b) {
    f2_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t mul2(f2_t a, f2_t b) {
    f2_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2_t fma2(f2_t a, f2_t b, f2_t c) {
    f2_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

constexpr float kC3 = 2.0f / 3.0f, kC5 = 2.0f / 5.0f, kC7 = 2.0f / 7.0f, kC9 = 2.0f / 9.0f;
constexpr int kMagicE = 0x4B400000;              // float 12582912 = 1.5 * 2^23: + e keeps e exact
constexpr float kMagicEf = 12582912.0f;

// split logarithm of max(p, FLT_MIN): log = E ln2 + lm.  The reciprocal is a
// hardware approximation refined by one Newton step; every other step is an
// IEEE round-to-nearest operation, and split_log2 below performs the same
// operations lane by lane, so both give bit-identical results.
__device__ __forceinline__ void split_log(float p, float &lm, float &E) {
    p = fmaxf(p, FLT_MIN);
    const int i = __float_as_int(p);
    const int e = (i - 0x3f3504f3) >> 23;            // m = p 2^-e in [1/sqrt2, sqrt2)
    const float m = __int_as_float(i - (e << 23));
    E = __fadd_rn(__int_as_float(e + kMagicE), -kMagicEf);
    const float u = __fadd_rn(m, -1.0f);              // exact (Sterbenz)
    const float v = __fadd_rn(m, 1.0f);
    float r = rcp_approx(v);
    const float er = __fmaf_rn(__fmaf_rn(m, -1.0f, -1.0f), r, 1.0f);
    r = __fmaf_rn(r, er, r);
    const float s = __fmul_rn(u, r);
    const float z = __fmul_rn(s, s);
    float q = __fmaf_rn(z, kC9, kC7);
    q = __fmaf_rn(q, z, kC5);
    q = __fmaf_rn(q, z, kC3);
    lm = __fmaf_rn(__fmul_rn(s, z), q, __fadd_rn(s, s));
}

// the same for two values at once (packed lanes)
__device__ __forceinline__ void split_log2(float p0, float p1, f2_t &lm, f2_t &E) {
    p0 = fmaxf(p0, FLT_MIN);
    p1 = fmaxf(p1, FLT_MIN);
    const int i0 = __float_as_int(p0), i1 = __float_as_int(p1);
    const int e0 = (i0 - 0x3f3504f3) >> 23, e1 = (i1 - 0x3f3504f3) >> 23;
    const f2_t m = pk(__int_as_float(i0 - (e0 << 23)), __int_as_float(i1 - (e1 << 23)));
    const f2_t one = pk(1.0f, 1.0f), mone = pk(-1.0f, -1.0f);
    E = add2(pk(__int_as_float(e0 + kMagicE), __int_as_float(e1 + kMagicE)), pk(-kMagicEf, -kMagicEf));
    const f2_t u = add2(m, mone);
    const f2_t v = add2(m, one);
    float v0, v1;
    upk(v, v0, v1);
    f2_t r = pk(rcp_approx(v0), rcp_approx(v1));
    const f2_t er = fma2(fma2(m, mone, mone), r, one);
    r = fma2(r, er, r);
    const f2_t sv = mul2(u, r);
    const f2_t z = mul2(sv, sv);
    f2_t q = fma2(z, pk(kC9, kC9), pk(kC7, kC7));
    q = fma2(q, z, pk(kC5, kC5));
    q = fma2(q, z, pk(kC3, kC3));
    lm = fma2(mul2(sv, z), q, add2(sv, sv));
}

// one term of each sum; accumulators updated in place
__device__ __forceinline__ void accumulate(float px, float lmx, float ex, float pt, float lmt, float et,
                                           float &kl, float &tv) {
    const float d = __fadd_rn(lmx, -lmt);
    const float de = __fadd_rn(ex, -et);
    const float lr = __fmaf_rn(de, kLn2, d);          // log(P_x / P_t)
    kl = __fmaf_rn(px, lr, kl);
    tv = __fadd_rn(tv, fabsf(__fadd_rn(px, -pt)));
}

// packed: two (x, b) terms against the matching target entries
__device__ __forceinline__ void accumulate2(f2_t px, f2_t lmx, f2_t ex, f2_t pt, f2_t lmt, f2_t et, f2_t &kl,
                                            f2_t &tv) {
    const f2_t mone = pk(-1.0f, -1.0f);
    const f2_t d = fma2(lmt, mone, lmx);
    const f2_t de = fma2(et, mone, ex);
    const f2_t lr = fma2(de, pk(kLn2, kLn2), d);
    kl = fma2(px, lr, kl);
    const f2_t dp = fma2(pt, mone, px);
    tv = add2(tv, dp & 0x7fffffff7fffffffULL);
}

// stage_P / stage_L / stage_E: [T][k_pad] target row, its mantissa log and exponent
__global__ void stage_targets_kernel(const float *__restrict__ P, int64_t k_pad, const int32_t *__restrict__ targets,
                                     int32_t T, float *__restrict__ sP, float *__restrict__ sL,
                                     float *__restrict__ sE) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (b >= k_pad || a >= T) return;
    const float p = P[(int64_t)targets[a] * k_pad + b];
    float lm, E;
    split_log(p, lm, E);
    sP[(int64_t)a * k_pad + b] = p;
    sL[(int64_t)a * k_pad + b] = lm;
    sE[(int64_t)a * k_pad + b] = E;
}

// ------------------------------------------------------------------ mbarrier helpers
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}

// bulk global -> shared copy (no tensor map, no multicast); size multiple of 16
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

constexpr uint32_t kMaxWaitIters = 1u << 26;   // bounded spin; then the error flag is set

// ------------------------------------------------------------------ few targets
// smem: for each of TT targets, three k_pad float arrays (P, lm, E); grid.y walks target groups.
template <int TT>
__global__ void __launch_bounds__(256) field_stream_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                                           const float *__restrict__ sP, const float *__restrict__ sL,
                                                           const float *__restrict__ sE, int32_t T,
                                                           float *__restrict__ out_kl, float *__restrict__ out_tv,
                                                           int *__restrict__ err_flag) {
    extern __shared__ __align__(16) float smem[];
    __shared__ __align__(8) uint64_t bar;
    const int a0 = blockIdx.y * TT;
    const int nt = (T - a0) < TT ? (T - a0) : TT;
    float *tP = smem;                          // [TT][k_pad]
    float *tL = smem + TT * k_pad;
    float *tE = smem + 2 * TT * k_pad;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t row_bytes = (uint32_t)(k_pad * sizeof(float));
        mbar_expect_tx(&bar, 3u * nt * row_bytes);
        for (int j = 0; j < nt; ++j) {
            bulk_g2s(tP + j * k_pad, sP + (int64_t)(a0 + j) * k_pad, row_bytes, &bar);
            bulk_g2s(tL + j * k_pad, sL + (int64_t)(a0 + j) * k_pad, row_bytes, &bar);
            bulk_g2s(tE + j * k_pad, sE + (int64_t)(a0 + j) * k_pad, row_bytes, &bar);
        }
    }
    uint32_t it = 0;
    while (!mbar_try_wait(&bar, 0)) {
        if (++it == kMaxWaitIters) {
            atomicExch(err_flag, 1);
            break;
        }
    }
    // a CTA whose wait gave up must not return while its copies may still land;
    // wait once more (also bounded) before touching the data or exiting
    if (it == kMaxWaitIters) {
        uint32_t it2 = 0;
        while (!mbar_try_wait(&bar, 0) && ++it2 < kMaxWaitIters) {
        }
        return;
    }

    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nvec = k_pad >> 2;                       // float4 per row
    constexpr int U = 4;                                   // float4 per lane per chunk
    const int64_t nchunk = (nvec + 32 * U - 1) / (32 * U);
    // software pipeline over (row, chunk): the loads of the next chunk are in
    // flight while the current one is computed
    float4 nxt[U];
    auto fetch = [&](int64_t x, int64_t ch) {
        const float4 *row = reinterpret_cast<const float4 *>(P + x * k_pad);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = ch * 32 * U + u * 32 + lane;
            nxt[u] = c < nvec ? __ldcs(row + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    int64_t x = warp, ch = 0;
    if (x < n_v) fetch(x, 0);
    f2_t kl[TT], tv[TT];
#pragma unroll
    for (int j = 0; j < TT; ++j) kl[j] = tv[j] = 0ULL;
    while (x < n_v) {
        float4 cur[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cur[u] = nxt[u];
        int64_t xn = x, chn = ch + 1;
        if (chn == nchunk) {
            chn = 0;
            xn += nwarps;
        }
        if (xn < n_v) fetch(xn, chn);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t c = ch * 32 * U + u * 32 + lane;
            if (c >= nvec) continue;
            f2_t lm01, e01, lm23, e23;
            split_log2(cur[u].x, cur[u].y, lm01, e01);
            split_log2(cur[u].z, cur[u].w, lm23, e23);
            const f2_t p01 = pk(cur[u].x, cur[u].y), p23 = pk(cur[u].z, cur[u].w);
#pragma unroll
            for (int j = 0; j < TT; ++j) {
                if (j >= nt) break;
                const float4 p4 = reinterpret_cast<const float4 *>(tP + j * k_pad)[c];
                const float4 l4 = reinterpret_cast<const float4 *>(tL + j * k_pad)[c];
                const float4 e4 = reinterpret_cast<const float4 *>(tE + j * k_pad)[c];
                accumulate2(p01, lm01, e01, pk(p4.x, p4.y), pk(l4.x, l4.y), pk(e4.x, e4.y), kl[j], tv[j]);
                accumulate2(p23, lm23, e23, pk(p4.z, p4.w), pk(l4.z, l4.w), pk(e4.z, e4.w), kl[j], tv[j]);
            }
        }
        if (ch == nchunk - 1) {
#pragma unroll
            for (int j = 0; j < TT; ++j) {
                float k0, k1, t0v, t1v;
                upk(kl[j], k0, k1);
                upk(tv[j], t0v, t1v);
                float skl = k0 + k1, stv = t0v + t1v;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    skl += __shfl_xor_sync(0xffffffffu, skl, o);
                    stv += __shfl_xor_sync(0xffffffffu, stv, o);
                }
                if (lane == 0 && j < nt) {
                    if (out_kl) out_kl[(int64_t)(a0 + j) * n_v + x] = skl;
                    if (out_tv) out_tv[(int64_t)(a0 + j) * n_v + x] = stv;
                }
                kl[j] = tv[j] = 0ULL;
            }
        }
        x = xn;
        ch = chn;
    }
}

// ------------------------------------------------------------------ many targets
constexpr int kTileRows = 64, kTileTargets = 64, kTileB = 32;

__global__ void __launch_bounds__(256, 2) field_tile_kernel(const float *__restrict__ P, int64_t n_v, int64_t k_pad,
                                                         const float *__restrict__ sP, const float *__restrict__ sL,
                                                         const float *__restrict__ sE, int32_t T,
                                                         float *__restrict__ out_kl, float *__restrict__ out_tv) {
    __shared__ __align__(16) float xP[kTileB][kTileRows];
    __shared__ __align__(16) float xL[kTileB][kTileRows];
    __shared__ __align__(16) float xE[kTileB][kTileRows];
    __shared__ __align__(16) float yP[kTileB][kTileTargets];
    __shared__ __align__(16) float yL[kTileB][kTileTargets];
    __shared__ __align__(16) float yE[kTileB][kTileTargets];

    const int tid = threadIdx.x;
    const int tx = tid & 15;          // target group: targets tx*4 .. tx*4+3
    const int ty = tid >> 4;          // row group: rows ty*4 .. ty*4+3
    const int64_t x0 = (int64_t)blockIdx.x * kTileRows;
    const int a0 = blockIdx.y * kTileTargets;

    // two-level summation: 32-term chunk sums, added into the totals with a
    // compensated (Kahan) sum for KL, whose terms cancel near the target
    float kl[4][4], tv[4][4], klc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) kl[r][c] = tv[r][c] = klc[r][c] = 0.0f;

    for (int64_t b0 = 0; b0 < k_pad; b0 += kTileB) {
        float ckl[4][4], ctv[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) ckl[r][c] = ctv[r][c] = 0.0f;
        // rows: 64 x 32 floats, 256 threads x two float4 (8 consecutive b of one row)
        {
            const int r = tid >> 2, cb = (tid & 3) * 8;
            const int64_t x = x0 + r;
            float vals[8];
#pragma unroll
            for (int e = 0; e < 8; e += 4) {
                float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (x < n_v && b0 + cb + e < k_pad)
                    v4 = __ldg(reinterpret_cast<const float4 *>(P + x * k_pad + b0 + cb + e));
                vals[e] = v4.x;
                vals[e + 1] = v4.y;
                vals[e + 2] = v4.z;
                vals[e + 3] = v4.w;
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                float lm, E;
                split_log(vals[e], lm, E);
                xP[cb + e][r] = vals[e];
                xL[cb + e][r] = lm;
                xE[cb + e][r] = E;
            }
        }
        // targets: 64 x 32 floats of each staged array
        {
            const int a = tid >> 2, cb = (tid & 3) * 8;
            const int ag = a0 + a;
#pragma unroll
            for (int e = 0; e < 8; e += 4) {
                float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f), l4 = p4, e4 = p4;
                if (ag < T && b0 + cb + e < k_pad) {
                    const int64_t off = (int64_t)ag * k_pad + b0 + cb + e;
                    p4 = __ldg(reinterpret_cast<const float4 *>(sP + off));
                    l4 = __ldg(reinterpret_cast<const float4 *>(sL + off));
                    e4 = __ldg(reinterpret_cast<const float4 *>(sE + off));
                }
                yP[cb + e][a] = p4.x; yP[cb + e + 1][a] = p4.y; yP[cb + e + 2][a] = p4.z; yP[cb + e + 3][a] = p4.w;
                yL[cb + e][a] = l4.x; yL[cb + e + 1][a] = l4.y; yL[cb + e + 2][a] = l4.z; yL[cb + e + 3][a] = l4.w;
                yE[cb + e][a] = e4.x; yE[cb + e + 1][a] = e4.y; yE[cb + e + 2][a] = e4.z; yE[cb + e + 3][a] = e4.w;
            }
        }
        __syncthreads();
#pragma unroll 4
        for (int b = 0; b < kTileB; ++b) {
            const float4 rp = *reinterpret_cast<const float4 *>(&xP[b][ty * 4]);
            const float4 rl = *reinterpret_cast<const float4 *>(&xL[b][ty * 4]);
            const float4 re = *reinterpret_cast<const float4 *>(&xE[b][ty * 4]);
            const float4 cp = *reinterpret_cast<const float4 *>(&yP[b][tx * 4]);
            const float4 cl = *reinterpret_cast<const float4 *>(&yL[b][tx * 4]);
            const float4 ce = *reinterpret_cast<const float4 *>(&yE[b][tx * 4]);
            const float rP[4] = {rp.x, rp.y, rp.z, rp.w}, rL[4] = {rl.x, rl.y, rl.z, rl.w},
                        rE[4] = {re.x, re.y, re.z, re.w};
            const float cP[4] = {cp.x, cp.y, cp.z, cp.w}, cL[4] = {cl.x, cl.y, cl.z, cl.w},
                        cE[4] = {ce.x, ce.y, ce.z, ce.w};
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c)
                    accumulate(rP[r], rL[r], rE[r], cP[c], cL[c], cE[c], ckl[r][c], ctv[r][c]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float y = __fsub_rn(ckl[r][c], klc[r][c]);
                const float t = __fadd_rn(kl[r][c], y);
                klc[r][c] = __fsub_rn(__fsub_rn(t, kl[r][c]), y);
                kl[r][c] = t;
                tv[r][c] = __fadd_rn(tv[r][c], ctv[r][c]);
            }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t x = x0 + ty * 4 + r;
        if (x >= n_v) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int a = a0 + tx * 4 + c;
            if (a >= T) continue;
            if (out_kl) out_kl[(int64_t)a * n_v + x] = kl[r][c];
            if (out_tv) out_tv[(int64_t)a * n_v + x] = tv[r][c];
        }
    }
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

}  // namespace

void launch_stage_targets(const float *P, int64_t k_pad, int64_t /*k*/, const int32_t *targets, int32_t T,
                          float4 *stage, cudaStream_t s) {
    float *sP = reinterpret_cast<float *>(stage);
    float *sL = sP + (int64_t)T * k_pad;
    float *sE = sL + (int64_t)T * k_pad;
    dim3 g((unsigned)((k_pad + 255) / 256), (unsigned)T);
    stage_targets_kernel<<<g, 256, 0, s>>>(P, k_pad, targets, T, sP, sL, sE);
}

void launch_fields_fp32(const float *P, int64_t n_v, int64_t k_pad, const float4 *stage, int32_t T, float *out_kl,
                        float *out_tv, int *err_flag, cudaStream_t s) {
    const float *sP = reinterpret_cast<const float *>(stage);
    const float *sL = sP + (int64_t)T * k_pad;
    const float *sE = sL + (int64_t)T * k_pad;
    if (T <= 2) {
        constexpr int TT = 1;
        const size_t smem = 3 * TT * (size_t)k_pad * sizeof(float);
        cudaFuncSetAttribute(field_stream_kernel<TT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, field_stream_kernel<TT>, 256, smem);
        if (per_sm < 1) per_sm = 1;
        int64_t rows_blocks = (n_v + 7) / 8;
        int64_t grid_x = (int64_t)num_sms() * per_sm / T;
        if (grid_x < 1) grid_x = 1;
        if (grid_x > rows_blocks) grid_x = rows_blocks;
        dim3 g((unsigned)grid_x, (unsigned)T);
        field_stream_kernel<TT><<<g, 256, smem, s>>>(P, n_v, k_pad, sP, sL, sE, T, out_kl, out_tv, err_flag);
        return;
    }
    dim3 g((unsigned)((n_v + kTileRows - 1) / kTileRows), (unsigned)((T + kTileTargets - 1) / kTileTargets));
    field_tile_kernel<<<g, 256, 0, s>>>(P, n_v, k_pad, sP, sL, sE, T, out_kl, out_tv);
}

size_t field_smem_limit_ok(int64_t k_pad) { return 3 * (size_t)k_pad * sizeof(float); }
