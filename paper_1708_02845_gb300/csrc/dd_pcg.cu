// Poisson-kernel preprocessing, Section IV Eq. (32)-(33), in FP64 on the GPU.
//
// Solves (-L_II) X = L_IB for all k boundary columns at once: one
// preconditioned conjugate-gradient recurrence per column, run in lock-step
// over a block of columns so that every sparse product streams the whole
// row-major [m][kc] block.  The preconditioner is a smoothed-aggregation
// multigrid V-cycle (dd_amg.cpp builds the hierarchy on the host); the
// diagonal (Jacobi) preconditioner remains for tiny meshes and as the
// fallback when no hierarchy can be built.  -L_II is a symmetric positive-definite
// M-matrix, so CG converges; its iterates are kept in FP64 because the
// small entries of P (shadowed boundary parts) need many correct digits for
// the logarithms of Eq. (35).  The block stops when every column's residual
// satisfies ||r|| <= rtol ||b||; only columns with b = 0 (no interior
// support) are skipped.  Columns are processed in chunks that fit a
// workspace budget; the result is written as FP32 P (row pitch k_pad).
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <functional>

#include "dd_amg.h"
#include "dd_internal.h"

namespace {

constexpr int kColsPerBlock = 128;   // columns (threads) of one CTA

struct Work {
    int64_t m = 0, kc = 0, nrb = 0;
    double *X = nullptr, *R = nullptr, *Pd = nullptr, *AP = nullptr;
    double *part0 = nullptr, *part1 = nullptr;   // [nrb][kc] partial column sums
    double *alpha = nullptr, *beta = nullptr, *rz = nullptr, *bnorm = nullptr, *dinv = nullptr;
    int *done = nullptr;
    unsigned long long *maxres = nullptr;        // bits of a non-negative double
};

// AP = A Pd over one row block; partial column sums of Pd . AP
__global__ void spmm_dot_kernel(int64_t m, int64_t kc, const int64_t *__restrict__ a_off,
                                const int32_t *__restrict__ a_col, const double *__restrict__ a_val,
                                const double *__restrict__ Pd, double *__restrict__ AP,
                                double *__restrict__ part, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        double s = 0.0;
        for (int64_t q = a_off[r]; q < a_off[r + 1]; ++q) s += a_val[q] * Pd[(int64_t)a_col[q] * kc + c];
        AP[r * kc + c] = s;
        acc += Pd[r * kc + c] * s;
    }
    part[(int64_t)blockIdx.x * kc + c] = acc;
}

// X += alpha Pd, R -= alpha AP; partial sums of R.Z (Z = D^-1 R) and R.R
__global__ void update_xr_kernel(int64_t m, int64_t kc, const double *__restrict__ alpha,
                                 const double *__restrict__ dinv, double *__restrict__ X,
                                 double *__restrict__ R, const double *__restrict__ Pd,
                                 const double *__restrict__ AP, double *__restrict__ part_rz,
                                 double *__restrict__ part_rr, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    const double a = alpha[c];
    double srz = 0.0, srr = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * kc + c;
        double rr = R[i];
        if (a != 0.0) {
            X[i] += a * Pd[i];
            rr -= a * AP[i];
            R[i] = rr;
        }
        srz += rr * rr * dinv[r];
        srr += rr * rr;
    }
    part_rz[(int64_t)blockIdx.x * kc + c] = srz;
    part_rr[(int64_t)blockIdx.x * kc + c] = srr;
}

// Pd = D^-1 R + beta Pd
__global__ void update_p_kernel(int64_t m, int64_t kc, const double *__restrict__ beta,
                                const double *__restrict__ dinv, const double *__restrict__ R,
                                double *__restrict__ Pd, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    const double b = beta[c];
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * kc + c;
        Pd[i] = R[i] * dinv[r] + b * Pd[i];
    }
}

// Sum the [nrb][kc] partials of each column: blockDim (32, 8)
__device__ __forceinline__ double column_sum(const double *part, int64_t nrb, int64_t kc, int64_t c,
                                             double (*sh)[33]) {
    double s = 0.0;
    if (c < kc)
        for (int64_t b = threadIdx.y; b < nrb; b += blockDim.y) s += part[b * kc + c];
    sh[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0) {
        for (int y = 1; y < (int)blockDim.y; ++y) s += sh[y][threadIdx.x];
    }
    __syncthreads();
    return s;   // valid in threadIdx.y == 0
}

__global__ void alpha_kernel(int64_t nrb, int64_t kc, const double *__restrict__ part,
                             const double *__restrict__ rz, const int *__restrict__ done,
                             double *__restrict__ alpha) {
    __shared__ double sh[8][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    double pAp = column_sum(part, nrb, kc, c, sh);
    if (threadIdx.y == 0 && c < kc) alpha[c] = (!done[c] && pAp > 0.0) ? rz[c] / pAp : 0.0;
}

__global__ void beta_kernel(int64_t nrb, int64_t kc, const double *__restrict__ part_rz,
                            const double *__restrict__ part_rr, const double *__restrict__ bnorm,
                            double *__restrict__ rz, const int *__restrict__ done,
                            double *__restrict__ beta, unsigned long long *__restrict__ maxres) {
    __shared__ double sh[8][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    double rz_new = column_sum(part_rz, nrb, kc, c, sh);
    double rr = column_sum(part_rr, nrb, kc, c, sh);
    if (threadIdx.y == 0 && c < kc) {
        double res = bnorm[c] > 0.0 ? sqrt(rr) / bnorm[c] : 0.0;
        // columns are not frozen at rtol: every column keeps iterating until the
        // slowest one converges, which drives the small entries of P (shadowed
        // boundary parts, whose logarithms enter Eq. 35) far below rtol
        const int d = done[c];
        beta[c] = (!d && rz[c] > 0.0) ? rz_new / rz[c] : 0.0;
        rz[c] = rz_new;
        atomicMax(maxres, (unsigned long long)__double_as_longlong(res));
    }
}

// R = L_IB[:, c0:c0+kc] (scatter of the edge weights to boundary columns)
__global__ void scatter_rhs_kernel(int64_t n_rb, const int32_t *__restrict__ rb_row,
                                   const int32_t *__restrict__ rb_col, const double *__restrict__ rb_val,
                                   int64_t c0, int64_t ncols, int64_t ld, double *__restrict__ R) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_rb) return;
    int64_t c = (int64_t)rb_col[i] - c0;
    if (c < 0 || c >= ncols) return;
    R[(int64_t)rb_row[i] * ld + c] += rb_val[i];   // one edge per (row, column): no race
}

__global__ void dinv_kernel(int64_t m, const double *__restrict__ diag, double *__restrict__ dinv) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) dinv[i] = 1.0 / diag[i];
}

// initial Pd = Z = D^-1 R and per-column partials of R.Z and R.R
__global__ void init_p_kernel(int64_t m, int64_t kc, const double *__restrict__ dinv,
                              const double *__restrict__ R, double *__restrict__ Pd,
                              double *__restrict__ part_rz, double *__restrict__ part_rr, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    double srz = 0.0, srr = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * kc + c;
        double rr = R[i], z = rr * dinv[r];
        Pd[i] = z;
        srz += rr * z;
        srr += rr * rr;
    }
    part_rz[(int64_t)blockIdx.x * kc + c] = srz;
    part_rr[(int64_t)blockIdx.x * kc + c] = srr;
}

__global__ void init_scalars_kernel(int64_t nrb, int64_t kc, const double *__restrict__ part_rz,
                                    const double *__restrict__ part_rr, double *__restrict__ rz,
                                    double *__restrict__ bnorm, int *__restrict__ done) {
    __shared__ double sh[8][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    double s_rz = column_sum(part_rz, nrb, kc, c, sh);
    double s_rr = column_sum(part_rr, nrb, kc, c, sh);
    if (threadIdx.y == 0 && c < kc) {
        rz[c] = s_rz;
        bnorm[c] = sqrt(s_rr);
        done[c] = s_rr > 0.0 ? 0 : 1;   // a column with no interior support is exactly zero
    }
}

// P[I[r], c0 + c] = X[r, c] as FP32, negatives clamped to 0 and values below FLT_MIN flushed
__global__ void pack_chunk_kernel(int64_t m, int64_t ncols, int64_t ld, int64_t c0, int64_t k_pad,
                                  const int32_t *__restrict__ interior, const double *__restrict__ X,
                                  float *__restrict__ P, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= ncols) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    for (int64_t r = r0; r < r1; ++r) {
        double v = X[r * ld + c];
        float f = v < (double)FLT_MIN ? 0.0f : (float)v;
        P[(int64_t)interior[r] * k_pad + c0 + c] = f;
    }
}

__global__ void boundary_identity_kernel(int64_t k, int64_t k_pad, const int32_t *__restrict__ boundary,
                                         float *__restrict__ P) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < k) P[(int64_t)boundary[j] * k_pad + j] = 1.0f;
}

__global__ void store_host_p_kernel(int64_t n_v, int64_t k, int64_t k_pad, const double *__restrict__ src,
                                    float *__restrict__ P) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_v * k) return;
    int64_t v = i / k, c = i % k;
    double x = src[i];
    P[v * k_pad + c] = x < (double)FLT_MIN ? 0.0f : (float)x;
}

// ---------------------------------------------------------------- multigrid V-cycle kernels
// Row-major [rows][kc] FP64 blocks, one thread per column, CTAs over row blocks.
enum { kSpmmSet = 0, kSpmmResidual = 1, kSpmmAdd = 2 };

// MODE kSpmmSet: Y = M X;  kSpmmResidual: Y = B - M X;  kSpmmAdd: Y += M X
template <int MODE>
__global__ void csr_spmm_kernel(int64_t rows, int64_t kc, const int64_t *__restrict__ off,
                                const int32_t *__restrict__ col, const double *__restrict__ val,
                                const double *__restrict__ X, const double *__restrict__ B, double *__restrict__ Y,
                                int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < rows ? r0 + rpb : rows;
    for (int64_t r = r0; r < r1; ++r) {
        double s = 0.0;
        for (int64_t q = off[r]; q < off[r + 1]; ++q) s += val[q] * X[(int64_t)col[q] * kc + c];
        const int64_t i = r * kc + c;
        if (MODE == kSpmmSet) Y[i] = s;
        if (MODE == kSpmmResidual) Y[i] = B[i] - s;
        if (MODE == kSpmmAdd) Y[i] += s;
    }
}

// X = omega D^-1 B (one Jacobi sweep from zero)
__global__ void jacobi0_kernel(int64_t rows, int64_t kc, double omega, const double *__restrict__ dinv,
                               const double *__restrict__ B, double *__restrict__ X, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < rows ? r0 + rpb : rows;
    for (int64_t r = r0; r < r1; ++r) X[r * kc + c] = omega * dinv[r] * B[r * kc + c];
}

// X += omega D^-1 Res; with DOT, also partial column sums of Rp . X (the
// preconditioned residual's inner product, on the fine level)
template <bool DOT>
__global__ void jacobi_add_kernel(int64_t rows, int64_t kc, double omega, const double *__restrict__ dinv,
                                  const double *__restrict__ Res, double *__restrict__ X,
                                  const double *__restrict__ Rp, double *__restrict__ part, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < rows ? r0 + rpb : rows;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * kc + c;
        const double x = X[i] + omega * dinv[r] * Res[i];
        X[i] = x;
        if (DOT) acc += Rp[i] * x;
    }
    if (DOT) part[(int64_t)blockIdx.x * kc + c] = acc;
}

// X = Ainv B on the coarsest level (Ainv dense n x n, row-major)
__global__ void coarse_solve_kernel(int64_t n, int64_t kc, const double *__restrict__ ainv,
                                    const double *__restrict__ B, double *__restrict__ X) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i = blockIdx.y;
    if (c >= kc || i >= n) return;
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) s += ainv[i * n + j] * B[j * kc + c];
    X[i * kc + c] = s;
}

// X += alpha Pd, R -= alpha AP; partial column sums of R.R
__global__ void update_xr_plain_kernel(int64_t m, int64_t kc, const double *__restrict__ alpha,
                                       double *__restrict__ X, double *__restrict__ R,
                                       const double *__restrict__ Pd, const double *__restrict__ AP,
                                       double *__restrict__ part_rr, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    const double a = alpha[c];
    double srr = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * kc + c;
        double rr = R[i];
        if (a != 0.0) {
            X[i] += a * Pd[i];
            rr -= a * AP[i];
            R[i] = rr;
        }
        srr += rr * rr;
    }
    part_rr[(int64_t)blockIdx.x * kc + c] = srr;
}

// partial column sums of R.R
__global__ void dot_rr_kernel(int64_t m, int64_t kc, const double *__restrict__ R, double *__restrict__ part,
                              int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    double acc = 0.0;
    for (int64_t r = r0; r < r1; ++r) acc += R[r * kc + c] * R[r * kc + c];
    part[(int64_t)blockIdx.x * kc + c] = acc;
}

// Pd = Z + beta Pd (beta = 0 on the first iteration)
__global__ void update_p_z_kernel(int64_t m, int64_t kc, const double *__restrict__ beta,
                                  const double *__restrict__ Z, double *__restrict__ Pd, int first, int rpb) {
    const int64_t c = (int64_t)blockIdx.y * kColsPerBlock + threadIdx.x;
    if (c >= kc) return;
    const int64_t r0 = (int64_t)blockIdx.x * rpb;
    const int64_t r1 = r0 + rpb < m ? r0 + rpb : m;
    const double b = first ? 0.0 : beta[c];
    for (int64_t r = r0; r < r1; ++r) {
        const int64_t i = r * kc + c;
        Pd[i] = first ? Z[i] : Z[i] + b * Pd[i];
    }
}

// rz = column sums of part_rz, bnorm from part_rr, done flags (first iteration)
__global__ void amg_init_scalars_kernel(int64_t nrb, int64_t kc, const double *__restrict__ part_rz,
                                        const double *__restrict__ part_rr, double *__restrict__ rz,
                                        double *__restrict__ bnorm, int *__restrict__ done) {
    __shared__ double sh[8][33];
    const int64_t c = (int64_t)blockIdx.x * 32 + threadIdx.x;
    double s_rz = column_sum(part_rz, nrb, kc, c, sh);
    double s_rr = column_sum(part_rr, nrb, kc, c, sh);
    if (threadIdx.y == 0 && c < kc) {
        rz[c] = s_rz;
        bnorm[c] = sqrt(s_rr);
        done[c] = s_rr > 0.0 ? 0 : 1;   // a column with no interior support is exactly zero
    }
}

template <typename T>
cudaError_t alloc(T **p, size_t count) {
    return cudaMalloc((void **)p, count * sizeof(T));
}

// rows per CTA for a [rows][kc] block: enough CTAs (about 16 per SM), at most 256 rows
int rows_per_block(int64_t rows, int64_t kc) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    const int64_t colblocks = (kc + kColsPerBlock - 1) / kColsPerBlock;
    const int64_t want = rows * colblocks / (16LL * sms);
    int rpb = 256;
    while (rpb > 4 && rpb > want) rpb >>= 1;
    return rpb;
}

struct DevCsr {
    int64_t rows = 0;
    int64_t *off = nullptr;
    int32_t *col = nullptr;
    double *val = nullptr;
};

// Block CG with the smoothed-aggregation V-cycle as preconditioner (one
// Jacobi pre- and post-sweep per level, exact coarsest solve): symmetric and
// positive definite, so CG applies.  Returns DD_ENOTCONV with *fallback set
// when the hierarchy cannot be built (the caller then uses Jacobi).
dd_status run_pcg_amg(DevMesh &M, double rtol, int32_t max_iter, cudaStream_t s, int32_t *iters_out,
                      double *resid_out, std::string &err, bool *fallback) {
    *fallback = false;
    const int64_t m = M.m, k = M.k;
    // host copy of A = -L_II and the hierarchy
    AmgCsr A0;
    A0.rows = A0.cols = m;
    A0.off.resize(m + 1);
    DD_CUDA_TRY(cudaMemcpy(A0.off.data(), M.a_off, (m + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost), err);
    const int64_t nnz = A0.off[m];
    A0.col.resize(nnz);
    A0.val.resize(nnz);
    DD_CUDA_TRY(cudaMemcpy(A0.col.data(), M.a_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost), err);
    DD_CUDA_TRY(cudaMemcpy(A0.val.data(), M.a_val, nnz * sizeof(double), cudaMemcpyDeviceToHost), err);
    AmgHierarchy H;
    std::string why;
    if (!build_amg(A0, H, why)) {
        *fallback = true;
        err = why;
        return DD_ENOTCONV;
    }
    const int nl = (int)H.levels.size();

    std::vector<void *> tmp;
    cudaError_t ce = cudaSuccess;
    auto dalloc = [&](void **p, size_t bytes) {
        if (ce != cudaSuccess) return;
        ce = cudaMalloc(p, bytes > 0 ? bytes : 8);
        if (ce == cudaSuccess) tmp.push_back(*p);
    };
    auto upload = [&](void *dst, const void *src, size_t bytes) {
        if (ce == cudaSuccess && bytes > 0) ce = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s);
    };
    auto up_csr = [&](const AmgCsr &h, DevCsr &d) {
        d.rows = h.rows;
        dalloc((void **)&d.off, h.off.size() * sizeof(int64_t));
        dalloc((void **)&d.col, h.col.size() * sizeof(int32_t));
        dalloc((void **)&d.val, h.val.size() * sizeof(double));
        upload(d.off, h.off.data(), h.off.size() * sizeof(int64_t));
        upload(d.col, h.col.data(), h.col.size() * sizeof(int32_t));
        upload(d.val, h.val.data(), h.val.size() * sizeof(double));
    };
    std::vector<DevCsr> dA(nl), dP(nl), dR(nl);
    std::vector<double *> dinv(nl, nullptr);
    for (int l = 0; l < nl; ++l) {
        const AmgLevel &L = H.levels[l];
        if (l == 0) {
            dA[0].rows = m;
            dA[0].off = M.a_off;
            dA[0].col = M.a_col;
            dA[0].val = M.a_val;
        } else {
            up_csr(L.A, dA[l]);
        }
        dalloc((void **)&dinv[l], L.dinv.size() * sizeof(double));
        upload(dinv[l], L.dinv.data(), L.dinv.size() * sizeof(double));
        if (l + 1 < nl) {
            up_csr(L.P, dP[l]);
            up_csr(L.R, dR[l]);
        }
    }
    double *ainv = nullptr;
    dalloc((void **)&ainv, H.coarse_inv.size() * sizeof(double));
    upload(ainv, H.coarse_inv.data(), H.coarse_inv.size() * sizeof(double));

    // chunk width: six FP64 [m][kc] vectors on the fine level, three per coarser
    // level, within a 24 GB workspace budget
    double per_col = 6.0 * 8.0 * (double)m;
    for (int l = 1; l < nl; ++l) per_col += 3.0 * 8.0 * (double)H.levels[l].A.rows;
    int64_t kc = (int64_t)(24e9 / per_col);
    kc = kc / 128 * 128;
    if (kc < 128) kc = 128;
    if (kc > ((k + 3) / 4) * 4) kc = ((k + 3) / 4) * 4;
    const int rpb0 = rows_per_block(m, kc);
    const int64_t nrb = (m + rpb0 - 1) / rpb0;
    std::vector<int> rpb(nl);
    for (int l = 0; l < nl; ++l) rpb[l] = rows_per_block(H.levels[l].A.rows, kc);
    const size_t vec = (size_t)m * kc * sizeof(double);
    double *X = nullptr, *R = nullptr, *Z = nullptr, *Pd = nullptr, *AP = nullptr;
    double *part0 = nullptr, *part1 = nullptr, *alpha = nullptr, *beta = nullptr, *rz = nullptr, *bnorm = nullptr;
    int *done = nullptr;
    unsigned long long *maxres = nullptr;
    dalloc((void **)&X, vec);
    dalloc((void **)&R, vec);
    dalloc((void **)&Z, vec);
    dalloc((void **)&Pd, vec);
    dalloc((void **)&AP, vec);
    std::vector<double *> lb(nl, nullptr), lx(nl, nullptr), lr(nl, nullptr);
    for (int l = 0; l < nl; ++l) {
        const size_t lv = (size_t)H.levels[l].A.rows * kc * sizeof(double);
        dalloc((void **)&lr[l], lv);
        if (l > 0) {
            dalloc((void **)&lb[l], lv);
            dalloc((void **)&lx[l], lv);
        }
    }
    dalloc((void **)&part0, (size_t)nrb * kc * sizeof(double));
    dalloc((void **)&part1, (size_t)nrb * kc * sizeof(double));
    dalloc((void **)&alpha, kc * sizeof(double));
    dalloc((void **)&beta, kc * sizeof(double));
    dalloc((void **)&rz, kc * sizeof(double));
    dalloc((void **)&bnorm, kc * sizeof(double));
    dalloc((void **)&done, kc * sizeof(int));
    dalloc((void **)&maxres, sizeof(unsigned long long));
    auto release = [&]() {
        cudaStreamSynchronize(s);
        for (void *p : tmp) cudaFree(p);
        tmp.clear();
    };
    if (ce != cudaSuccess) {
        release();
        cudaGetLastError();
        *fallback = true;
        err = std::string("multigrid workspace allocation failed: ") + cudaGetErrorString(ce);
        return DD_ENOMEM;
    }

    auto grid = [&](int64_t rows, int rb) {
        return dim3((unsigned)((rows + rb - 1) / rb), (unsigned)((kc + kColsPerBlock - 1) / kColsPerBlock));
    };
    // z = V(b) on level l (x must not alias b); dot: partial sums of b.x into part0 (fine level)
    std::function<void(int, const double *, double *, bool)> vcycle = [&](int l, const double *b, double *x,
                                                                          bool dot) {
        const int64_t n = H.levels[l].A.rows;
        if (l == nl - 1) {   // coarsest level (never the fine one here: nl >= 2)
            coarse_solve_kernel<<<dim3((unsigned)((kc + 127) / 128), (unsigned)n), 128, 0, s>>>(n, kc, ainv, b, x);
            return;
        }
        const double w = H.levels[l].omega;
        const dim3 g = grid(n, rpb[l]);
        const int64_t nc = H.levels[l + 1].A.rows;
        jacobi0_kernel<<<g, kColsPerBlock, 0, s>>>(n, kc, w, dinv[l], b, x, rpb[l]);
        csr_spmm_kernel<kSpmmResidual><<<g, kColsPerBlock, 0, s>>>(n, kc, dA[l].off, dA[l].col, dA[l].val, x, b,
                                                                    lr[l], rpb[l]);
        csr_spmm_kernel<kSpmmSet><<<grid(nc, rpb[l + 1]), kColsPerBlock, 0, s>>>(
            nc, kc, dR[l].off, dR[l].col, dR[l].val, lr[l], nullptr, lb[l + 1], rpb[l + 1]);
        vcycle(l + 1, lb[l + 1], lx[l + 1], false);
        csr_spmm_kernel<kSpmmAdd><<<g, kColsPerBlock, 0, s>>>(n, kc, dP[l].off, dP[l].col, dP[l].val, lx[l + 1],
                                                               nullptr, x, rpb[l]);
        csr_spmm_kernel<kSpmmResidual><<<g, kColsPerBlock, 0, s>>>(n, kc, dA[l].off, dA[l].col, dA[l].val, x, b,
                                                                    lr[l], rpb[l]);
        if (dot)
            jacobi_add_kernel<true><<<g, kColsPerBlock, 0, s>>>(n, kc, w, dinv[l], lr[l], x, b, part0, rpb[l]);
        else
            jacobi_add_kernel<false><<<g, kColsPerBlock, 0, s>>>(n, kc, w, dinv[l], lr[l], x, nullptr, nullptr,
                                                                  rpb[l]);
    };

    dd_status st = DD_OK;
    int32_t iters_max = 0;
    double res_max = 0.0;
    const int check_every = 4;
    const dim3 g0 = grid(m, rpb0), gc((unsigned)((kc + 31) / 32)), bc(32, 8);
    for (int64_t c0 = 0; c0 < k && st == DD_OK; c0 += kc) {
        const int64_t kcur = (k - c0) < kc ? (k - c0) : kc;
        cudaMemsetAsync(X, 0, vec, s);
        cudaMemsetAsync(R, 0, vec, s);
        if (M.n_rb > 0)
            scatter_rhs_kernel<<<(unsigned)((M.n_rb + 255) / 256), 256, 0, s>>>(M.n_rb, M.rb_row, M.rb_col, M.rb_val,
                                                                                c0, kcur, kc, R);
        if (nl == 1) {   // the whole problem is the coarsest level: one exact solve
            coarse_solve_kernel<<<dim3((unsigned)((kc + 127) / 128), (unsigned)m), 128, 0, s>>>(m, kc, ainv, R, X);
            pack_chunk_kernel<<<dim3((unsigned)nrb, (unsigned)((kcur + kColsPerBlock - 1) / kColsPerBlock)),
                                kColsPerBlock, 0, s>>>(m, kcur, kc, c0, M.k_pad, M.interior, X, M.P, rpb0);
            iters_max = std::max(iters_max, 1);
            continue;
        }
        vcycle(0, R, Z, true);
        dot_rr_kernel<<<g0, kColsPerBlock, 0, s>>>(m, kc, R, part1, rpb0);
        amg_init_scalars_kernel<<<gc, bc, 0, s>>>(nrb, kc, part0, part1, rz, bnorm, done);
        update_p_z_kernel<<<g0, kColsPerBlock, 0, s>>>(m, kc, beta, Z, Pd, 1, rpb0);
        int32_t it = 0;
        double res = 1.0;
        for (it = 1; it <= max_iter; ++it) {
            spmm_dot_kernel<<<g0, kColsPerBlock, 0, s>>>(m, kc, M.a_off, M.a_col, M.a_val, Pd, AP, part0, rpb0);
            alpha_kernel<<<gc, bc, 0, s>>>(nrb, kc, part0, rz, done, alpha);
            update_xr_plain_kernel<<<g0, kColsPerBlock, 0, s>>>(m, kc, alpha, X, R, Pd, AP, part1, rpb0);
            vcycle(0, R, Z, true);
            cudaMemsetAsync(maxres, 0, sizeof(unsigned long long), s);
            beta_kernel<<<gc, bc, 0, s>>>(nrb, kc, part0, part1, bnorm, rz, done, beta, maxres);
            update_p_z_kernel<<<g0, kColsPerBlock, 0, s>>>(m, kc, beta, Z, Pd, 0, rpb0);
            if (it % check_every == 0 || it == max_iter) {
                unsigned long long bits = 0;
                cudaError_t e1 = cudaMemcpyAsync(&bits, maxres, sizeof bits, cudaMemcpyDeviceToHost, s);
                cudaError_t e2 = cudaStreamSynchronize(s);
                if (e1 != cudaSuccess || e2 != cudaSuccess) {
                    err = std::string("PCG iteration failed: ") + cudaGetErrorString(e1 != cudaSuccess ? e1 : e2);
                    st = DD_ECUDA;
                    break;
                }
                std::memcpy(&res, &bits, sizeof res);
                if (res <= rtol) break;
            }
        }
        if (st != DD_OK) break;
        if (it > max_iter) it = max_iter;
        iters_max = std::max(iters_max, it);
        res_max = std::max(res_max, res);
        pack_chunk_kernel<<<dim3((unsigned)nrb, (unsigned)((kcur + kColsPerBlock - 1) / kColsPerBlock)),
                            kColsPerBlock, 0, s>>>(m, kcur, kc, c0, M.k_pad, M.interior, X, M.P, rpb0);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaGetLastError();
    release();
    if (st != DD_OK) return st;
    if (e != cudaSuccess) {
        err = std::string("PCG failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    if (iters_out) *iters_out = iters_max;
    if (resid_out) *resid_out = res_max;
    M.has_P = true;
    if (!(res_max <= rtol)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "PCG stopped at %d iterations with relative residual %.3e > %.3e",
                      iters_max, res_max, rtol);
        err = buf;
        return DD_ENOTCONV;
    }
    return DD_OK;
}

bool use_multigrid(int64_t m) {
    static int mode = -1;
    if (mode < 0) {
        const char *e = getenv("DD_PCG_PRECOND");
        mode = (e && !strcmp(e, "jacobi")) ? 0 : 1;
    }
    return mode == 1 && m >= 256;
}

}  // namespace

dd_status run_pcg(DevMesh &M, double rtol, int32_t max_iter, cudaStream_t s, int32_t *iters_out,
                  double *resid_out, std::string &err) {
    const int64_t m = M.m, k = M.k;
    if (!M.P) {
        DD_CUDA_TRY(cudaMalloc((void **)&M.P, (size_t)M.n_v * M.k_pad * sizeof(float)), err);
        M.owned.push_back(M.P);
        M.bytes += (int64_t)M.n_v * M.k_pad * sizeof(float);
    }
    DD_CUDA_TRY(cudaMemsetAsync(M.P, 0, (size_t)M.n_v * M.k_pad * sizeof(float), s), err);
    if (k > 0)
        boundary_identity_kernel<<<(unsigned)((k + 255) / 256), 256, 0, s>>>(k, M.k_pad, M.boundary, M.P);
    int32_t iters_max = 0;
    double res_max = 0.0;
    if (m == 0) {
        M.has_P = true;
        if (iters_out) *iters_out = 0;
        if (resid_out) *resid_out = 0.0;
        return DD_OK;
    }

    if (use_multigrid(m)) {
        bool fallback = false;
        const dd_status sa = run_pcg_amg(M, rtol, max_iter, s, iters_out, resid_out, err, &fallback);
        if (!fallback) return sa;
        err.clear();   // the hierarchy could not be built: the diagonal preconditioner below
    }

    // chunk width: four FP64 [m][kc] vectors within a 24 GB workspace budget
    const double budget = 24e9;
    int64_t kc = (int64_t)(budget / (4.0 * 8.0 * (double)m));
    kc = kc / 128 * 128;
    if (kc < 128) kc = 128;
    if (kc > ((k + 3) / 4) * 4) kc = ((k + 3) / 4) * 4;

    Work w;
    w.m = m;
    w.kc = kc;
    // rows per CTA: enough CTAs (about 16 per SM) for small meshes, 256 rows for large ones
    int rpb = 256;
    {
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
        const int64_t colblocks = (kc + kColsPerBlock - 1) / kColsPerBlock;
        const int64_t want = m * colblocks / (16LL * sms);
        while (rpb > 8 && rpb > want) rpb >>= 1;
    }
    w.nrb = (m + rpb - 1) / rpb;
    std::vector<void *> tmp;
    cudaError_t ce = cudaSuccess;
    size_t vec = (size_t)m * kc;
    if ((ce = alloc(&w.X, vec)) == cudaSuccess) tmp.push_back(w.X);
    if (ce == cudaSuccess && (ce = alloc(&w.R, vec)) == cudaSuccess) tmp.push_back(w.R);
    if (ce == cudaSuccess && (ce = alloc(&w.Pd, vec)) == cudaSuccess) tmp.push_back(w.Pd);
    if (ce == cudaSuccess && (ce = alloc(&w.AP, vec)) == cudaSuccess) tmp.push_back(w.AP);
    if (ce == cudaSuccess && (ce = alloc(&w.part0, (size_t)w.nrb * kc)) == cudaSuccess) tmp.push_back(w.part0);
    if (ce == cudaSuccess && (ce = alloc(&w.part1, (size_t)w.nrb * kc)) == cudaSuccess) tmp.push_back(w.part1);
    if (ce == cudaSuccess && (ce = alloc(&w.alpha, (size_t)kc)) == cudaSuccess) tmp.push_back(w.alpha);
    if (ce == cudaSuccess && (ce = alloc(&w.beta, (size_t)kc)) == cudaSuccess) tmp.push_back(w.beta);
    if (ce == cudaSuccess && (ce = alloc(&w.rz, (size_t)kc)) == cudaSuccess) tmp.push_back(w.rz);
    if (ce == cudaSuccess && (ce = alloc(&w.bnorm, (size_t)kc)) == cudaSuccess) tmp.push_back(w.bnorm);
    if (ce == cudaSuccess && (ce = alloc(&w.dinv, (size_t)m)) == cudaSuccess) tmp.push_back(w.dinv);
    if (ce == cudaSuccess && (ce = alloc(&w.done, (size_t)kc)) == cudaSuccess) tmp.push_back(w.done);
    if (ce == cudaSuccess && (ce = alloc(&w.maxres, 1)) == cudaSuccess) tmp.push_back(w.maxres);
    auto release = [&]() {
        for (void *p : tmp) cudaFree(p);
        tmp.clear();
    };
    if (ce != cudaSuccess) {
        release();
        cudaGetLastError();
        err = std::string("PCG workspace allocation failed: ") + cudaGetErrorString(ce);
        return DD_ENOMEM;
    }

    dd_status st = DD_OK;
    const int check_every = 16;
    dinv_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, M.a_diag, w.dinv);
    for (int64_t c0 = 0; c0 < k && st == DD_OK; c0 += kc) {
        const int64_t kcur = (k - c0) < kc ? (k - c0) : kc;   // columns in this chunk
        // vectors keep pitch kc; columns beyond kcur stay zero and converge at once
        dim3 g2((unsigned)w.nrb, (unsigned)((kc + kColsPerBlock - 1) / kColsPerBlock));
        dim3 gc((unsigned)((kc + 31) / 32));
        dim3 bc(32, 8);
        cudaMemsetAsync(w.X, 0, vec * sizeof(double), s);
        cudaMemsetAsync(w.R, 0, vec * sizeof(double), s);
        if (M.n_rb > 0)
            scatter_rhs_kernel<<<(unsigned)((M.n_rb + 255) / 256), 256, 0, s>>>(M.n_rb, M.rb_row, M.rb_col,
                                                                                M.rb_val, c0, kcur, kc, w.R);
        init_p_kernel<<<g2, kColsPerBlock, 0, s>>>(m, kc, w.dinv, w.R, w.Pd, w.part0, w.part1, rpb);
        init_scalars_kernel<<<gc, bc, 0, s>>>(w.nrb, kc, w.part0, w.part1, w.rz, w.bnorm, w.done);
        int32_t it = 0;
        double res = 1.0;
        for (it = 1; it <= max_iter; ++it) {
            spmm_dot_kernel<<<g2, kColsPerBlock, 0, s>>>(m, kc, M.a_off, M.a_col, M.a_val, w.Pd, w.AP, w.part0, rpb);
            alpha_kernel<<<gc, bc, 0, s>>>(w.nrb, kc, w.part0, w.rz, w.done, w.alpha);
            update_xr_kernel<<<g2, kColsPerBlock, 0, s>>>(m, kc, w.alpha, w.dinv, w.X, w.R, w.Pd, w.AP, w.part0,
                                                          w.part1, rpb);
            cudaMemsetAsync(w.maxres, 0, sizeof(unsigned long long), s);
            beta_kernel<<<gc, bc, 0, s>>>(w.nrb, kc, w.part0, w.part1, w.bnorm, w.rz, w.done, w.beta,
                                          w.maxres);
            update_p_kernel<<<g2, kColsPerBlock, 0, s>>>(m, kc, w.beta, w.dinv, w.R, w.Pd, rpb);
            if (it % check_every == 0 || it == max_iter) {
                unsigned long long bits = 0;
                cudaError_t e1 = cudaMemcpyAsync(&bits, w.maxres, sizeof bits, cudaMemcpyDeviceToHost, s);
                cudaError_t e2 = cudaStreamSynchronize(s);
                if (e1 != cudaSuccess || e2 != cudaSuccess) {
                    err = std::string("PCG iteration failed: ") +
                          cudaGetErrorString(e1 != cudaSuccess ? e1 : e2);
                    st = DD_ECUDA;
                    break;
                }
                double r;
                static_assert(sizeof(r) == sizeof(bits), "size");
                std::memcpy(&r, &bits, sizeof r);
                res = r;
                if (res <= rtol) break;
            }
        }
        if (st != DD_OK) break;
        if (it > max_iter) it = max_iter;
        if (it > iters_max) iters_max = it;
        if (res > res_max) res_max = res;
        pack_chunk_kernel<<<dim3((unsigned)w.nrb, (unsigned)((kcur + kColsPerBlock - 1) / kColsPerBlock)),
                            kColsPerBlock, 0, s>>>(m, kcur, kc, c0, M.k_pad, M.interior, w.X, M.P, rpb);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    release();
    if (st != DD_OK) return st;
    if (e != cudaSuccess) {
        err = std::string("PCG failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("PCG launch failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    M.has_P = true;
    if (iters_out) *iters_out = iters_max;
    if (resid_out) *resid_out = res_max;
    if (!(res_max <= rtol)) {
        char buf[160];
        std::snprintf(buf, sizeof buf, "PCG stopped at %d iterations with relative residual %.3e > %.3e",
                      iters_max, res_max, rtol);
        err = buf;
        return DD_ENOTCONV;
    }
    return DD_OK;
}

dd_status store_poisson(DevMesh &M, const double *P, cudaStream_t s, std::string &err) {
    if (!M.P) {
        DD_CUDA_TRY(cudaMalloc((void **)&M.P, (size_t)M.n_v * M.k_pad * sizeof(float)), err);
        M.owned.push_back(M.P);
        M.bytes += (int64_t)M.n_v * M.k_pad * sizeof(float);
    }
    const size_t n = (size_t)M.n_v * M.k;
    double *d = nullptr;
    if (cudaMalloc((void **)&d, n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        err = "staging allocation for the Poisson kernel failed";
        return DD_ENOMEM;
    }
    cudaError_t e = cudaMemcpyAsync(d, P, n * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(M.P, 0, (size_t)M.n_v * M.k_pad * sizeof(float), s);
    if (e == cudaSuccess) {
        store_host_p_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(M.n_v, M.k, M.k_pad, d, M.P);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) {
        err = std::string("storing the Poisson kernel failed: ") + cudaGetErrorString(e);
        return DD_ECUDA;
    }
    M.has_P = true;
    return DD_OK;
}
