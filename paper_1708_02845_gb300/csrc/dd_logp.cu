// The Poisson kernel to full relative precision in every entry, and log P,
// for domains whose kernel spans hundreds of orders of magnitude (Section V,
// Precision: maze-like domains, where the paper turns to computing log P).
//
// The block CG of dd_pcg.cu resolves an entry only relative to the largest
// entries of its column (a residual norm cannot see an entry of 1e-40), and
// FP32 flushes everything below 1.2e-38 to zero, where the logarithm of
// Eq. (35) then has to be clamped.  This refinement keeps P's accurate part
// and recomputes the rest by the fixed-point form of Eq. (32),
//
//   P[i,b] = ( sum_{j in I} w_ij P[j,b] + w_ib ) / d_i,   d_i = sum_j w_ij
//
// (Jacobi sweeps in FP64 over all columns of a chunk at once).  With
// non-negative edge weights every sweep adds non-negative terms only, so an
// entry carries a relative error of a few units of rounding however small
// it is, and the sweeps converge to every entry's own precision: starting
// from the CG values where they are large (>= 2^-30) and from 0 elsewhere,
// the error at an entry falls once the walk conditioned to end at column b
// has left the region that started wrong -- after a number of sweeps of the
// order of the corridor length, not of the global mixing time.  The
// stored FP32 P takes the refined values (flushed below FLT_MIN as before)
// and a second array holds log2 P in FP32 for every entry (-inf where P is
// exactly 0), which the field kernels consult where the FP32 entry is 0.
// Limit: FP64; an entry below about 1e-300 underflows.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "dd_internal.h"

namespace {

constexpr int kRelaxCols = 128;     // columns (threads) of one CTA

// X[r][c] = P[I[r]][c0 + c] where it is at least tau (the CG value), else 0
__global__ void relax_init_kernel(int64_t m, int64_t ncols, int64_t ld, int64_t c0, int64_t k_pad,
                                  const int32_t *__restrict__ interior, const float *__restrict__ P, double tau,
                                  double *__restrict__ X, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kRelaxCols + threadIdx.x;
    if (c >= ld) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    for (int64_t r = r0; r < r1; ++r) {
        double v = 0.0;
        if (c < ncols) {
            const double p = (double)P[(int64_t)interior[r] * k_pad + c0 + c];
            v = p >= tau ? p : 0.0;
        }
        X[r * ld + c] = v;
    }
}

// F[r][c] = w_{I[r], B[c0 + c]} (the boundary weights of row r)
__global__ void relax_rhs_kernel(int64_t n_rb, const int32_t *__restrict__ rb_row, const int32_t *__restrict__ rb_col,
                                 const double *__restrict__ rb_val, int64_t c0, int64_t ncols, int64_t ld,
                                 double *__restrict__ F) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rb) return;
    const int64_t c = (int64_t)rb_col[i] - c0;
    if (c < 0 || c >= ncols) return;
    F[(int64_t)rb_row[i] * ld + c] += rb_val[i];   // one edge per (row, column): no race
}

// One sweep: Y = (F + W X) / d with W the off-diagonal magnitudes of
// -L_II (its CSR holds -w_ij off the diagonal and d_i on it); every term
// non-negative.  With CHECK, the largest relative change |Y - X| / Y over
// the block (a new non-zero counts as 1) goes into *maxchg (bits of a
// non-negative double).
template <bool CHECK>
__global__ void relax_sweep_kernel(int64_t m, int64_t ld, const int64_t *__restrict__ a_off,
                                   const int32_t *__restrict__ a_col, const double *__restrict__ a_val,
                                   const double *__restrict__ a_diag, const double *__restrict__ F,
                                   const double *__restrict__ X, double *__restrict__ Y,
                                   unsigned long long *__restrict__ maxchg, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kRelaxCols + threadIdx.x;
    double chg = 0.0;
    if (c < ld) {
        const int64_t r0 = (int64_t)blockIdx.x * rpb;
        const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
        for (int64_t r = r0; r < r1; ++r) {
            double s = F[r * ld + c];
            for (int64_t q = a_off[r]; q < a_off[r + 1]; ++q) {
                const int32_t j = a_col[q];
                if (j != r) s += -a_val[q] * X[(int64_t)j * ld + c];
            }
            const double y = s / a_diag[r];
            Y[r * ld + c] = y;
            if (CHECK && y > 0.0) chg = fmax(chg, fabs(y - X[r * ld + c]) / y);
        }
    }
    if (CHECK) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) chg = fmax(chg, __shfl_xor_sync(0xffffffffu, chg, o));
        if ((threadIdx.x & 31) == 0 && chg > 0.0) atomicMax(maxchg, (unsigned long long)__double_as_longlong(chg));
    }
}

// P[I[r]][c0 + c] = X as FP32 (flushed below FLT_MIN), LP = log2 X in FP32 (-inf for 0)
__global__ void relax_store_kernel(int64_t m, int64_t ncols, int64_t ld, int64_t c0, int64_t k_pad,
                                   const int32_t *__restrict__ interior, const double *__restrict__ X,
                                   float *__restrict__ P, float *__restrict__ LP, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kRelaxCols + threadIdx.x;
    if (c >= ncols) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    for (int64_t r = r0; r < r1; ++r) {
        const double v = X[r * ld + c];
        const int64_t o = (int64_t)interior[r] * k_pad + c0 + c;
        P[o] = v < (double)FLT_MIN ? 0.0f : (float)v;
        LP[o] = v > 0.0 ? (float)log2(v) : -INFINITY;
    }
}

__global__ void fill_kernel(float *__restrict__ a, int64_t n, float v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// boundary rows of LP: log2 1 = 0 on the row's own column
__global__ void lp_boundary_kernel(int64_t k, int64_t k_pad, const int32_t *__restrict__ boundary,
                                   float *__restrict__ LP) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) LP[(int64_t)boundary[j] * k_pad + j] = 0.0f;
}

int relax_rows_per_block(int64_t rows, int64_t ld) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    const int64_t colblocks = (ld + kRelaxCols - 1) / kRelaxCols;
    const int64_t want = rows * colblocks / (16LL * sms);
    int rpb = 64;
    while (rpb > 1 && rpb > want) rpb >>= 1;
    return rpb;
}

}  // namespace

dd_status refine_log_poisson(DevMesh &M, double tol, int32_t max_sweeps, cudaStream_t s, int32_t *sweeps_out,
                             double *change_out, std::string &err) {
    const int64_t m = M.m, k = M.k;
    const size_t lp_bytes = (size_t)M.n_v * M.k_pad * sizeof(float);
    if (!M.LP) {
        DD_CUDA_TRY(cudaMalloc((void **)&M.LP, lp_bytes), err);
        M.owned.push_back(M.LP);
        M.bytes += (int64_t)lp_bytes;
    }
    const int64_t nlp = M.n_v * M.k_pad;
    fill_kernel<<<(unsigned)((nlp + 255) / 256), 256, 0, s>>>(M.LP, nlp, -INFINITY);
    if (k > 0) lp_boundary_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(k, M.k_pad, M.boundary, M.LP);
    int32_t sweeps_max = 0;
    double chg_max = 0.0;
    if (m == 0 || k == 0) {
        DD_CUDA_TRY(cudaStreamSynchronize(s), err);
        if (sweeps_out) *sweeps_out = 0;
        if (change_out) *change_out = 0.0;
        return DD_OK;
    }
    // chunk width: three FP64 [m][kc] blocks within a 24 GB workspace budget
    int64_t kc = (int64_t)(24e9 / (3.0 * 8.0 * (double)m));
    kc = kc / kRelaxCols * kRelaxCols;
    if (kc < kRelaxCols) kc = kRelaxCols;
    if (kc > k) kc = k;
    const size_t vec = (size_t)m * kc;
    double *X = nullptr, *Y = nullptr, *F = nullptr;
    unsigned long long *chg = nullptr;
    cudaError_t ce = cudaMalloc((void **)&X, vec * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc((void **)&Y, vec * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc((void **)&F, vec * sizeof(double));
    if (ce == cudaSuccess) ce = cudaMalloc((void **)&chg, sizeof(unsigned long long));
    auto release = [&]() {
        for (void *p : {(void *)X, (void *)Y, (void *)F, (void *)chg})
            if (p) cudaFree(p);
    };
    if (ce != cudaSuccess) {
        release();
        cudaGetLastError();
        err = std::string("log-P workspace allocation failed: ") + cudaGetErrorString(ce);
        return DD_ENOMEM;
    }
    const int rpb = relax_rows_per_block(m, kc);
    const dim3 g((unsigned)((m + rpb - 1) / rpb), (unsigned)((kc + kRelaxCols - 1) / kRelaxCols));
    const int check_every = 32;
    const double tau = std::ldexp(1.0, -30);
    dd_status st = DD_OK;
    for (int64_t c0 = 0; c0 < k && st == DD_OK; c0 += kc) {
        const int64_t ncols = (k - c0) < kc ? (k - c0) : kc;
        relax_init_kernel<<<g, kRelaxCols, 0, s>>>(m, ncols, kc, c0, M.k_pad, M.interior, M.P, tau, X, rpb);
        cudaMemsetAsync(F, 0, vec * sizeof(double), s);
        if (M.n_rb > 0)
            relax_rhs_kernel<<<(unsigned)((M.n_rb + 255) / 256), 256, 0, s>>>(M.n_rb, M.rb_row, M.rb_col, M.rb_val,
                                                                              c0, ncols, kc, F);
        int32_t it = 0;
        double change = 1.0;
        for (it = 1; it <= max_sweeps; ++it) {
            const bool check = (it % check_every == 0) || it == max_sweeps;
            if (check) {
                cudaMemsetAsync(chg, 0, sizeof(unsigned long long), s);
                relax_sweep_kernel<true><<<g, kRelaxCols, 0, s>>>(m, kc, M.a_off, M.a_col, M.a_val, M.a_diag, F, X,
                                                                   Y, chg, rpb);
            } else {
                relax_sweep_kernel<false><<<g, kRelaxCols, 0, s>>>(m, kc, M.a_off, M.a_col, M.a_val, M.a_diag, F,
                                                                    X, Y, chg, rpb);
            }
            std::swap(X, Y);
            if (check) {
                unsigned long long bits = 0;
                cudaError_t e1 = cudaMemcpyAsync(&bits, chg, sizeof bits, cudaMemcpyDeviceToHost, s);
                cudaError_t e2 = cudaStreamSynchronize(s);
                if (e1 != cudaSuccess || e2 != cudaSuccess) {
                    err = std::string("log-P sweep failed: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2);
                    st = DD_ECUDA;
                    break;
                }
                std::memcpy(&change, &bits, sizeof change);
                if (change <= tol) break;
            }
        }
        if (st != DD_OK) break;
        if (it > max_sweeps) it = max_sweeps;
        if (it > sweeps_max) sweeps_max = it;
        if (change > chg_max) chg_max = change;
        relax_store_kernel<<<dim3(g.x, (unsigned)((ncols + kRelaxCols - 1) / kRelaxCols)), kRelaxCols, 0, s>>>(
            m, ncols, kc, c0, M.k_pad, M.interior, X, M.P, M.LP, rpb);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    release();
    if (st != DD_OK) return st;
    if (e != cudaSuccess) {
        err = std::string("log-P refinement failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    if (sweeps_out) *sweeps_out = sweeps_max;
    if (change_out) *change_out = chg_max;
    if (!(chg_max <= tol)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "log-P refinement stopped at %d sweeps with relative change %.3e > %.3e",
                      sweeps_max, chg_max, tol);
        err = buf;
        return DD_ENOTCONV;
    }
    return DD_OK;
}
