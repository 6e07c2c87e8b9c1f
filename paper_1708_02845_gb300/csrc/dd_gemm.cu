// KL cross term as a tensor-core GEMM (split BF16), for many targets at once.
//
// Eq. (35) with the field row x as the weight (Eq. 17, z = x) splits into
//   KL_t(x) = e_x - C[x, t],   e_x = sum_b P[x,b] log P[x,b],
//   C[x, t] = sum_b P[x,b] log P[t,b]
// and C is a dense contraction over the boundary (M = n rows, N = T targets,
// K = k columns).  Each FP32 operand is split into BF16 hi + lo parts and
// C = Phi.Lhi + Phi.Llo + Plo.Lhi is accumulated in FP32 (the lo.lo product,
// about 2^-16 relative, is dropped), so the error is about 2^-15 of
// S_x = sum_b P[x,b] |log P[t,b]|.  e_x is computed once per mesh in FP64.
//
// sm_103a kernel, persistent: one CTA per SM walks the 128-row x 256-target
// output tiles (tile i of a CTA = blockIdx.x + i gridDim.x; consecutive tiles
// share their row tile, so the CTAs working at one time read each A tile once
// from HBM).  Warp 0 loads A (P hi/lo) and B (log P_t hi/lo) tiles with TMA
// (128-byte swizzle, K-major, two stages on mbarriers, one ring across all
// tiles, so the next tile's loads start while the current one finishes);
// warp 1 issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulator in TMEM,
// 128 x 256 x 16 per instruction) into one of two 256-column TMEM
// accumulators; warps 2-5 read the other accumulator with tcgen05.ld and
// write KL = e_x - C, then hand it back, so the epilogue of one tile overlaps
// the main loop of the next.  Every mbarrier wait is bounded and also gives up
// when another role has given up (a flag in shared memory); the kernel then
// sets an error flag, drains its own copies, frees TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "dd_internal.h"

namespace {

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 2;
constexpr int A_BYTES = BM * BK * 2;                         // 16 KB
constexpr int B_BYTES = BN * BK * 2;                         // 32 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;       // 96 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;   // + alignment slack, barriers, TMEM slot, abort flag
constexpr uint32_t TMEM_COLS = 512;                          // two 256-column accumulators
constexpr uint32_t kWaitLimit = 1u << 25;                    // bounded spins (non-suspending test_wait)

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, N = 256, M = 128
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(saddr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: true when the phase completed; false (error flag set, abort
// raised for the other roles) when the limit expired or another role aborted
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, volatile int *abort) {
    for (uint32_t i = 0; i < kWaitLimit; ++i) {
        if (mbar_test(bar, parity)) return true;
        if (*abort) return false;
    }
    atomicExch(err, 2);
    *abort = 1;
    return false;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            saddr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(saddr(bar))
        : "memory");
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFF) >> 4);          // start address
    d |= (uint64_t)1 << 16;                           // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
    d |= (uint64_t)1 << 46;                           // descriptor version
    d |= (uint64_t)2 << 61;                           // 128-byte swizzle
    return d;
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

struct GemmArgs {
    const float *ex;    // [n_v]
    float *out;         // [T][n_v]
    int64_t n_v;
    int32_t T;
    int32_t kblocks;
    int *err;
};

__global__ void __launch_bounds__(192, 1) kl_gemm_kernel(const __grid_constant__ CUtensorMap tAhi,
                                                         const __grid_constant__ CUtensorMap tAlo,
                                                         const __grid_constant__ CUtensorMap tBhi,
                                                         const __grid_constant__ CUtensorMap tBlo, const GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
    uint64_t *empty = full + STAGES;
    uint64_t *accf = empty + STAGES;     // [2] accumulator written (MMA commit)
    uint64_t *acce = accf + 2;           // [2] accumulator read out (4 epilogue warps)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntn = (g.T + BN - 1) / BN;
    const int ntiles = ntn * (int)((g.n_v + BM - 1) / BM);

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], 4);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: one ring of stages across all of this CTA's tiles
            int issued = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
                const int m0 = (t / ntn) * BM, n0 = (t % ntn) * BN;
                for (int kb = 0; kb < g.kblocks; ++kb, ++issued) {
                    const int s = issued % STAGES, round = issued / STAGES;
                    if (round > 0 && !mbar_wait(&empty[s], (round - 1) & 1, g.err, abort)) break;
                    uint8_t *st = smem + s * STAGE_BYTES;
                    mbar_expect_tx(&full[s], STAGE_BYTES);
                    tma_load_2d(st, &tAhi, &full[s], kb * BK, m0);
                    tma_load_2d(st + A_BYTES, &tAlo, &full[s], kb * BK, m0);
                    tma_load_2d(st + 2 * A_BYTES, &tBhi, &full[s], kb * BK, n0);
                    tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tBlo, &full[s], kb * BK, n0);
                }
            }
            // drain: every issued stage must have landed before the CTA may exit
            volatile int never = 0;
            for (int q = issued - STAGES < 0 ? 0 : issued - STAGES; q < issued; ++q)
                mbar_wait(&full[q % STAGES], (q / STAGES) & 1, g.err, &never);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: tile i into accumulator i & 1
            int consumed = 0, i = 0, last_buf = -1, last_par = 0;
            for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++i) {
                const int buf = i & 1, use = i >> 1;
                if (use > 0 && !mbar_wait(&acce[buf], (use - 1) & 1, g.err, abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(buf * BN);
                bool ok = true;
                for (int kb = 0; kb < g.kblocks; ++kb, ++consumed) {
                    const int s = consumed % STAGES, round = consumed / STAGES;
                    if (!mbar_wait(&full[s], round & 1, g.err, abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t st = saddr(smem + s * STAGE_BYTES);
                    const uint64_t ahi = smem_desc(st), alo = smem_desc(st + A_BYTES);
                    const uint64_t bhi = smem_desc(st + 2 * A_BYTES), blo = smem_desc(st + 2 * A_BYTES + B_BYTES);
#pragma unroll
                    for (int kk = 0; kk < BK / 16; ++kk) {
                        const uint64_t off = (uint64_t)((kk * 32) >> 4);   // 16 BF16 = 32 bytes along K
                        mma_bf16(acc, ahi + off, bhi + off, (kb > 0 || kk > 0) ? 1u : 0u);
                        mma_bf16(acc, ahi + off, blo + off, 1u);
                        mma_bf16(acc, alo + off, bhi + off, 1u);
                    }
                    mma_commit(&empty[s]);      // the stage is free once these MMAs complete
                }
                mma_commit(&accf[buf]);         // accumulator ready (also after an early stop)
                last_buf = buf;
                last_par = use & 1;
                if (!ok) break;
            }
            // every MMA issued here has completed before TMEM may be freed
            volatile int never = 0;
            if (last_buf >= 0) mbar_wait(&accf[last_buf], (uint32_t)last_par, g.err, &never);
        }
    } else {
        // ---------------- epilogue: warps 2..5 read TMEM lanes 32*(warp % 4) .. +31
        const int q = warp & 3;
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int buf = i & 1, use = i >> 1;
            const bool ok = __all_sync(0xffffffffu, mbar_wait(&accf[buf], use & 1, g.err, abort));
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m0 = (t / ntn) * BM, n0 = (t % ntn) * BN;
            const int64_t row = (int64_t)m0 + q * 32 + lane;
            const float e = row < g.n_v ? g.ex[row] : 0.0f;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN + c0);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                      "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                      "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < g.n_v) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int a = n0 + c0 + j;
                        if (a < g.T) g.out[(int64_t)a * g.n_v + row] = e - __uint_as_float(r[j]);
                    }
                }
            }
            // hand the accumulator back to the MMA warp
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&acce[buf]);
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// P (FP32, pitch k_pad) -> BF16 hi/lo (pitch kb, zero padding) and e_x in FP64
__global__ void split_p_kernel(const float *__restrict__ P, int64_t n_v, int64_t k, int64_t k_pad, int64_t kb,
                               __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v * kb) return;
    const int64_t x = i / kb, b = i % kb;
    const float p = b < k ? P[x * k_pad + b] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(p);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(p - __bfloat162float(h));
}

__global__ void row_entropy_kernel(const float *__restrict__ P, int64_t n_v, int64_t k, int64_t k_pad,
                                   float *__restrict__ ex) {
    const int64_t x = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (x >= n_v) return;
    double s = 0.0;
    for (int64_t b = lane; b < k; b += 32) {
        const double p = (double)P[x * k_pad + b];
        if (p > 0.0) s += p * log(p);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) ex[x] = (float)s;
}

// log P_t split into BF16 hi/lo, [T][kb]; log taken at max(P, FLT_MIN) as in the FP32 path
__global__ void split_targets_kernel(const float *__restrict__ P, int64_t k, int64_t k_pad, int64_t kb,
                                     const int32_t *__restrict__ targets, int32_t T, __nv_bfloat16 *__restrict__ hi,
                                     __nv_bfloat16 *__restrict__ lo) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int a = blockIdx.y;
    if (b >= kb || a >= T) return;
    float L = 0.0f;
    if (b < k) {
        const float p = fmaxf(P[(int64_t)targets[a] * k_pad + b], FLT_MIN);
        L = logf(p);
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(L);
    hi[(int64_t)a * kb + b] = h;
    lo[(int64_t)a * kb + b] = __float2bfloat16_rn(L - __bfloat162float(h));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    });
    return fn;
}

// 2-D BF16 K-major map: rows x kb, box 64 x box_rows, 128-byte swizzle
bool make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t kb, uint32_t box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)kb, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)kb * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

int64_t gemm_kb(int64_t k) { return (k + 63) / 64 * 64; }

dd_status prepare_bf16(DevMesh &m, cudaStream_t s, std::string &err) {
    if (m.p_hi) return DD_OK;
    const int64_t kb = gemm_kb(m.k);
    const size_t ne = (size_t)m.n_v * kb;
    void *hi = nullptr, *lo = nullptr, *ex = nullptr;
    if (cudaMalloc(&hi, ne * 2) != cudaSuccess || cudaMalloc(&lo, ne * 2) != cudaSuccess ||
        cudaMalloc(&ex, (size_t)m.n_v * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        if (hi) cudaFree(hi);
        if (lo) cudaFree(lo);
        if (ex) cudaFree(ex);
        err = "allocation of the BF16 split of P failed";
        return DD_ENOMEM;
    }
    split_p_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(m.P, m.n_v, m.k, m.k_pad, kb,
                                                                 (__nv_bfloat16 *)hi, (__nv_bfloat16 *)lo);
    row_entropy_kernel<<<(unsigned)((m.n_v + 7) / 8), 256, 0, s>>>(m.P, m.n_v, m.k, m.k_pad, (float *)ex);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        cudaFree(hi);
        cudaFree(lo);
        cudaFree(ex);
        err = std::string("BF16 split launch failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    m.p_hi = hi;
    m.p_lo = lo;
    m.ex = (float *)ex;
    m.kb = kb;
    m.owned.push_back(hi);
    m.owned.push_back(lo);
    m.owned.push_back(ex);
    m.bytes += (int64_t)(ne * 4 + m.n_v * sizeof(float));
    return DD_OK;
}

size_t gemm_target_scratch_bytes(const DevMesh &m, int32_t T) { return (size_t)T * gemm_kb(m.k) * 2 * 2; }

dd_status launch_kl_gemm(const DevMesh &m, const int32_t *d_targets, int32_t T, void *scratch, float *out_kl,
                         int *err_flag, cudaStream_t s, std::string &err) {
    const int64_t kb = m.kb;
    __nv_bfloat16 *bhi = reinterpret_cast<__nv_bfloat16 *>(scratch);
    __nv_bfloat16 *blo = bhi + (size_t)T * kb;
    dim3 gs((unsigned)((kb + 255) / 256), (unsigned)T);
    {
        KMark km_("split_targets_kernel", s);
        split_targets_kernel<<<gs, 256, 0, s>>>(m.P, m.k, m.k_pad, kb, d_targets, T, bhi, blo);
    }
    CUtensorMap tAhi, tAlo, tBhi, tBlo;
    if (!make_map(&tAhi, m.p_hi, m.n_v, kb, BM) || !make_map(&tAlo, m.p_lo, m.n_v, kb, BM) ||
        !make_map(&tBhi, bhi, T, kb, BN) || !make_map(&tBlo, blo, T, kb, BN)) {
        err = "tensor map encoding failed";
        return DD_ECUDA;
    }
    static std::once_flag attr_once;
    std::call_once(attr_once,
                   [] { cudaFuncSetAttribute(kl_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES); });
    GemmArgs g;
    g.ex = m.ex;
    g.out = out_kl;
    g.n_v = m.n_v;
    g.T = T;
    g.kblocks = (int32_t)(kb / BK);
    g.err = err_flag;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t ntiles = (int64_t)((T + BN - 1) / BN) * ((m.n_v + BM - 1) / BM);
    dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ntiles, sms > 0 ? sms : 1)));   // one CTA per SM
    {
        KMark km_("kl_gemm_kernel", s);
        kl_gemm_kernel<<<grid, 192, SMEM_BYTES, s>>>(tAhi, tAlo, tBhi, tBlo, g);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("KL GEMM launch failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    return DD_OK;
}
