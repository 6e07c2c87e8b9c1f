// dd_distance_noalloc: the FP32 divergence fields for callers that must not
// allocate device memory.
//
// Who needs this: code that runs where a cudaMalloc is not allowed or not
// wanted -- a robot's real-time control loop that may only allocate during
// start-up (an allocation can stall the device and break the loop's timing
// budget), or a plugin whose host framework owns every device byte through
// its own pool.  Such a caller already holds the Poisson kernel, the target
// ids and the output in memory it obtained elsewhere; this entry point needs
// nothing more.
//
// The per-target staging rows that dd_distance keeps in context scratch live
// here in one file-scope device array of fixed size, shared by every call on
// a device and kept until the process exits.  Its device address is looked
// up once per device (cudaGetSymbolAddress, with that device current) on the
// first call there; host code never passes the symbol itself to a kernel.
//
// Nothing here times or tunes: for more than two targets the tile shape is a
// fixed function of T (the autotuner behind dd_distance would run timed
// launches and synchronise the first time it meets a size class), and every
// tile shape gives bit-identical fields, so the result equals dd_distance's.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dd_internal.h"

namespace {

constexpr int64_t kNoallocStageFloats = 4LL * (1LL << 20);   // 4 arrays x T*k_pad <= 2^20 floats (16 MiB)
constexpr int kMaxDevices = 64;

__device__ __align__(256) float g_noalloc_stage[kNoallocStageFloats];
__device__ __align__(256) int g_noalloc_flag[64];    // [0]: a bounded wait gave up, [1]: a target id out of range

std::mutex g_noalloc_mutex;
float *g_stage_ptr[kMaxDevices] = {};
int *g_flag_ptr[kMaxDevices] = {};

// device addresses of the static scratch for the current device (looked up once)
dd_status noalloc_setup(int dev, float **stage, int **flag) {
    if (dev < 0 || dev >= kMaxDevices) return DD_EINVAL;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_stage_ptr[dev]) {
        void *s = nullptr, *f = nullptr;
        if (cudaGetSymbolAddress(&s, g_noalloc_stage) != cudaSuccess ||
            cudaGetSymbolAddress(&f, g_noalloc_flag) != cudaSuccess) {
            cudaGetLastError();
            return DD_ECUDA;
        }
        g_stage_ptr[dev] = static_cast<float *>(s);
        g_flag_ptr[dev] = static_cast<int *>(f);
    }
    *stage = g_stage_ptr[dev];
    *flag = g_flag_ptr[dev];
    return DD_OK;
}

// the tile shape for T targets: narrow target tiles for few targets, wide for many
int fixed_tile_shape(int32_t T) { return T <= 16 ? 2 : (T <= 32 ? 1 : 0); }

}  // namespace

extern "C" dd_status dd_distance_noalloc(const float *P, int64_t n_v, int64_t k_pad, const int32_t *targets,
                                         int32_t T, uint32_t f_mask, float *out, void *cuda_stream) {
    if (!P || !targets || !out) return DD_EINVAL;
    if (n_v < 1 || T < 1 || k_pad < 4 || (k_pad % 4) != 0) return DD_EINVAL;
    // 16-byte loads of P, 4-byte accesses of the ids and the output
    if ((reinterpret_cast<uintptr_t>(P) & 15) || (reinterpret_cast<uintptr_t>(targets) & 3) ||
        (reinterpret_cast<uintptr_t>(out) & 3))
        return DD_EINVAL;
    if (f_mask == 0 || (f_mask & ~(uint32_t)(DD_F_KL | DD_F_TV))) return DD_EINVAL;
    if ((int64_t)T * k_pad > kNoallocStageFloats / 4) return DD_EINVAL;   // beyond the fixed scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return DD_ECUDA;
    }
    float *stage = nullptr;
    int *flag = nullptr;
    dd_status st = noalloc_setup(dev, &stage, &flag);
    if (st != DD_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    // the flags keep the previous call's values: clear them first
    if (cudaMemsetAsync(flag, 0, 2 * sizeof(int), s) != cudaSuccess) {
        cudaGetLastError();
        return DD_ECUDA;
    }
    float *kl = (f_mask & DD_F_KL) ? out : nullptr;
    float *tv = (f_mask & DD_F_TV) ? out + ((f_mask & DD_F_KL) ? (int64_t)T * n_v : 0) : nullptr;
    // an id outside [0, n_v) is never used as a row index: the staging kernel
    // zero-fills its rows and raises flag[1]
    launch_stage_targets(P, n_v, k_pad, targets, T, reinterpret_cast<float4 *>(stage), s, flag + 1);
    launch_fields_fp32(P, n_v, k_pad, reinterpret_cast<const float4 *>(stage), T, kl, tv, flag, s,
                       fixed_tile_shape(T));
    if (cudaGetLastError() != cudaSuccess) return DD_ECUDA;
    int h[2] = {0, 0};
    if (cudaMemcpyAsync(h, flag, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return DD_ECUDA;
    }
    if (h[1]) return DD_EINVAL;
    return h[0] ? DD_ETIMEOUT : DD_OK;
}
