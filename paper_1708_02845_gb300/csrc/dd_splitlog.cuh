// Split logarithm shared by the field kernels: log p = E ln2 + lm, p = m 2^E,
// m in [1, 2), lm table driven (Tang, "Table-driven implementation of the
// logarithm function in IEEE floating-point arithmetic", ACM TOMS 1990).
// Every kernel that compares logarithms of two values takes both from these
// functions, so equal arguments give bit-identical results.
#pragma once

#include <cfloat>
#include <cmath>
#include <cstdint>

namespace {

constexpr int kLogTab = 128;                     // entries over [1, 2)
constexpr int kMagicHi = 0x4B400000 >> 9;        // funnel-shift high word: 0x4B400000 | (bits >> 23)

// Entry j covers the mantissas m in [1 + j/128, 1 + (j+1)/128): r_j = 1/c_j
// rounded (c_j the midpoint) at tab[j], L_j = -log r_j at tab[kLogTab + j],
// both computed in FP64.
__device__ __forceinline__ void build_log_table(float *tab) {
    for (int j = threadIdx.x; j < kLogTab; j += blockDim.x) {
        const double c = 1.0 + (j + 0.5) / kLogTab;
        const float r = (float)(1.0 / c);
        tab[j] = r;
        tab[kLogTab + j] = (float)(-log((double)r));
    }
}

// Split logarithm: log p = E ln2 + lm, p = m 2^E with m in [1, 2).
// split_log_parts: the integer steps.  The exponent comes back biased, as the
// float 12582912 + 127 + E (exact), so that a difference of two is the exact
// exponent difference; one funnel shift forms it from the bit pattern.  Only
// positive normal arguments give the logarithm; for +0 and -0 (and
// subnormals) the result is finite and meaningless, which is harmless where
// the argument is also the term's weight (the row side, P[x,b]) and is why
// CLAMP (max with FLT_MIN, used for the target side) exists.  The library's
// P holds no subnormals or -0.  split_log_tail: the floating-point steps from
// the table entry (r, L).  Every caller runs exactly these operations, so
// equal arguments give bit-identical results at every call site.
template <bool CLAMP>
__device__ __forceinline__ void split_log_parts(float p, int &mb, float &Eb, int &j) {
    if (CLAMP) p = fmaxf(p, FLT_MIN);
    const int i = __float_as_int(p);
    Eb = __int_as_float((int)__funnelshift_r((unsigned)i, (unsigned)kMagicHi, 23));
    mb = (i & 0x007FFFFF) | 0x3F800000;
    j = (i >> 16) & (kLogTab - 1);
}

__device__ __forceinline__ float split_log_tail(int mb, float r, float L) {
    const float u = __fmaf_rn(__int_as_float(mb), r, -1.0f);            // m/c - 1, one rounding
    const float w = __fmaf_rn(u, 1.0f / 3.0f, -0.5f);
    return __fadd_rn(L, __fmaf_rn(__fmul_rn(u, u), w, u));              // log c + log(1 + u)
}

// table with one copy (stride 1)
template <bool CLAMP>
__device__ __forceinline__ void split_log(float p, const float *tab, float &lm, float &Eb) {
    int mb, j;
    split_log_parts<CLAMP>(p, mb, Eb, j);
    lm = split_log_tail(mb, tab[j], tab[kLogTab + j]);
}

// Hardware base-2 logarithm (lg2.approx) of the mantissa m in [1, 2) of a
// float bit pattern i; the result lies in [0, 1].  Its error over all 2^23
// mantissas spans at most DD_FAST_LOG_SPREAD (measured by dd_check_fast_log).
__device__ __forceinline__ float lg2_mant(int i) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(__int_as_float((i & 0x007FFFFF) | 0x3F800000)));
    return y;
}

// Base-2 logarithm as one FP32 number: the exponent E (exact, from the bit
// pattern: 2^23 + biased E as a float, minus 2^23 + 127) plus the hardware
// mantissa log, rounded once to half an ulp of the result.  Positive normal
// arguments only; +0 gives -127 (finite), harmless where the argument is
// also the term's weight.
__device__ __forceinline__ float fast_l2(float p) {
    const int i = __float_as_int(p);
    const float E = __fsub_rn(__int_as_float(0x4B000000 | (int)((unsigned)i >> 23)), 8388735.0f);
    return __fadd_rn(E, lg2_mant(i));
}

}  // namespace
