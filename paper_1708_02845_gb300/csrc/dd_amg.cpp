// Smoothed-aggregation algebraic multigrid hierarchy for A = -L_II, built on
// the host once per Poisson-kernel solve.  The V-cycle (dd_pcg.cu) serves as
// the preconditioner of the block conjugate-gradient iteration of Eq. (32):
// with it the iteration count no longer grows with the mesh size the way the
// diagonal (Jacobi) preconditioner's does.
//
// Construction (Vanek, Mandel and Brezina, "Algebraic multigrid by smoothed
// aggregation for second and fourth order elliptic problems", Computing 1996),
// written here:
//  * strength: j is a strong neighbour of i when |a_ij| >= theta sqrt(a_ii a_jj);
//  * aggregation in three passes: a node whose strong neighbours are all free
//    starts an aggregate with them; a free node joins the first-pass aggregate
//    of its strongest aggregated neighbour; what is left forms aggregates of
//    itself and its free strong neighbours;
//  * tentative prolongator T: one column per aggregate, 1 on its nodes
//    (the constant vector is the near-null space of the Laplacian);
//  * smoothed prolongator P = (I - w D^-1 A) T with w = 4 / (3 rho(D^-1 A)),
//    rho from a power iteration;
//  * Galerkin coarse operator A_c = P^T A P, recursively, down to at most
//    kCoarsest unknowns, whose dense inverse is formed by Cholesky in FP64.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "dd_amg.h"

namespace {

constexpr double kTheta = 0.08;
constexpr int64_t kCoarsest = 64;
constexpr int kMaxLevels = 16;

// C = A B (Gustavson: one dense accumulator row with a touched list)
AmgCsr spgemm(const AmgCsr &A, const AmgCsr &B) {
    AmgCsr C;
    C.rows = A.rows;
    C.cols = B.cols;
    C.off.assign(A.rows + 1, 0);
    std::vector<double> acc(B.cols, 0.0);
    std::vector<int32_t> mark(B.cols, -1), touched;
    for (int64_t i = 0; i < A.rows; ++i) {
        touched.clear();
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p) {
            const int32_t k = A.col[p];
            const double a = A.val[p];
            for (int64_t q = B.off[k]; q < B.off[k + 1]; ++q) {
                const int32_t j = B.col[q];
                if (mark[j] != (int32_t)i) {
                    mark[j] = (int32_t)i;
                    acc[j] = 0.0;
                    touched.push_back(j);
                }
                acc[j] += a * B.val[q];
            }
        }
        std::sort(touched.begin(), touched.end());
        for (int32_t j : touched) {
            C.col.push_back(j);
            C.val.push_back(acc[j]);
        }
        C.off[i + 1] = (int64_t)C.col.size();
    }
    return C;
}

AmgCsr transpose(const AmgCsr &A) {
    AmgCsr T;
    T.rows = A.cols;
    T.cols = A.rows;
    T.off.assign(A.cols + 1, 0);
    for (int32_t j : A.col) ++T.off[j + 1];
    for (int64_t j = 0; j < A.cols; ++j) T.off[j + 1] += T.off[j];
    T.col.resize(A.col.size());
    T.val.resize(A.val.size());
    std::vector<int64_t> pos(T.off.begin(), T.off.end() - 1);
    for (int64_t i = 0; i < A.rows; ++i)
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p) {
            const int64_t q = pos[A.col[p]]++;
            T.col[q] = (int32_t)i;
            T.val[q] = A.val[p];
        }
    return T;
}

std::vector<double> diagonal(const AmgCsr &A) {
    std::vector<double> d(A.rows, 0.0);
    for (int64_t i = 0; i < A.rows; ++i)
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p)
            if (A.col[p] == (int32_t)i) d[i] = A.val[p];
    return d;
}

// largest eigenvalue of D^-1 A by a power iteration from a fixed start
double spectral_radius(const AmgCsr &A, const std::vector<double> &d) {
    const int64_t n = A.rows;
    std::vector<double> x(n), y(n);
    for (int64_t i = 0; i < n; ++i) x[i] = 1.0 + 0.5 * std::sin(0.7 * (double)i);
    double lam = 1.0;
    for (int it = 0; it < 24; ++it) {
        double nrm = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p) s += A.val[p] * x[A.col[p]];
            y[i] = s / d[i];
            nrm += y[i] * y[i];
        }
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0)) break;
        double xn = 0.0;
        for (int64_t i = 0; i < n; ++i) xn += x[i] * x[i];
        lam = nrm / std::sqrt(xn);
        for (int64_t i = 0; i < n; ++i) x[i] = y[i] / nrm;
    }
    return lam;
}

// aggregate id of every node; returns the number of aggregates
int64_t aggregate(const AmgCsr &A, const std::vector<double> &d, std::vector<int64_t> &agg) {
    const int64_t n = A.rows;
    auto strong = [&](int64_t i, int64_t p) {
        const int32_t j = A.col[p];
        return j != (int32_t)i && std::fabs(A.val[p]) >= kTheta * std::sqrt(d[i] * d[j]);
    };
    agg.assign(n, -1);
    int64_t na = 0;
    // pass 1: nodes whose strong neighbourhood is entirely free
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        bool free_nb = true;
        for (int64_t p = A.off[i]; p < A.off[i + 1] && free_nb; ++p)
            if (strong(i, p) && agg[A.col[p]] >= 0) free_nb = false;
        if (!free_nb) continue;
        agg[i] = na;
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p)
            if (strong(i, p)) agg[A.col[p]] = na;
        ++na;
    }
    // pass 2: join the first-pass aggregate of the strongest aggregated neighbour
    const std::vector<int64_t> first(agg);
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        double best = -1.0;
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p)
            if (strong(i, p) && first[A.col[p]] >= 0 && std::fabs(A.val[p]) > best) {
                best = std::fabs(A.val[p]);
                agg[i] = first[A.col[p]];
            }
    }
    // pass 3: the rest, with their free strong neighbours
    for (int64_t i = 0; i < n; ++i) {
        if (agg[i] >= 0) continue;
        agg[i] = na;
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p)
            if (strong(i, p) && agg[A.col[p]] < 0) agg[A.col[p]] = na;
        ++na;
    }
    return na;
}

// P = (I - w D^-1 A) T for the aggregation `agg` (na aggregates)
AmgCsr smoothed_prolongator(const AmgCsr &A, const std::vector<double> &d, const std::vector<int64_t> &agg,
                            int64_t na, double w) {
    AmgCsr P;
    P.rows = A.rows;
    P.cols = na;
    P.off.assign(A.rows + 1, 0);
    std::vector<double> acc(na, 0.0);
    std::vector<int32_t> mark(na, -1), touched;
    for (int64_t i = 0; i < A.rows; ++i) {
        touched.clear();
        auto add = [&](int64_t g, double v) {
            if (mark[g] != (int32_t)i) {
                mark[g] = (int32_t)i;
                acc[g] = 0.0;
                touched.push_back((int32_t)g);
            }
            acc[g] += v;
        };
        add(agg[i], 1.0);
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p) add(agg[A.col[p]], -w * A.val[p] / d[i]);
        std::sort(touched.begin(), touched.end());
        for (int32_t g : touched) {
            if (acc[g] == 0.0) continue;
            P.col.push_back(g);
            P.val.push_back(acc[g]);
        }
        P.off[i + 1] = (int64_t)P.col.size();
    }
    return P;
}

// dense inverse of an SPD matrix by Cholesky; false if not positive definite
bool dense_spd_inverse(const AmgCsr &A, std::vector<double> &inv) {
    const int64_t n = A.rows;
    std::vector<double> L(n * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p) L[i * n + A.col[p]] = A.val[p];
    for (int64_t j = 0; j < n; ++j) {
        double s = L[j * n + j];
        for (int64_t k = 0; k < j; ++k) s -= L[j * n + k] * L[j * n + k];
        if (!(s > 0.0)) return false;
        const double ljj = std::sqrt(s);
        L[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; ++i) {
            double t = L[i * n + j];
            for (int64_t k = 0; k < j; ++k) t -= L[i * n + k] * L[j * n + k];
            L[i * n + j] = t / ljj;
        }
        for (int64_t i = 0; i < j; ++i) L[i * n + j] = 0.0;
    }
    inv.assign(n * n, 0.0);
    std::vector<double> y(n);
    for (int64_t c = 0; c < n; ++c) {
        for (int64_t i = 0; i < n; ++i) {              // L y = e_c
            double t = (i == c) ? 1.0 : 0.0;
            for (int64_t k = 0; k < i; ++k) t -= L[i * n + k] * y[k];
            y[i] = t / L[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; --i) {         // L^T x = y
            double t = y[i];
            for (int64_t k = i + 1; k < n; ++k) t -= L[k * n + i] * inv[k * n + c];
            inv[i * n + c] = t / L[i * n + i];
        }
    }
    return true;
}

}  // namespace

bool build_amg(const AmgCsr &A0, AmgHierarchy &H, std::string &err) {
    H = AmgHierarchy();
    AmgCsr A = A0;
    for (int lev = 0; lev < kMaxLevels; ++lev) {
        const std::vector<double> d = diagonal(A);
        for (double v : d)
            if (!(v > 0.0)) {
                err = "multigrid setup: non-positive diagonal";
                return false;
            }
        AmgLevel L;
        L.dinv.resize(A.rows);
        for (int64_t i = 0; i < A.rows; ++i) L.dinv[i] = 1.0 / d[i];
        if (A.rows <= kCoarsest) {
            if (!dense_spd_inverse(A, H.coarse_inv)) {
                err = "multigrid setup: coarsest operator not positive definite";
                return false;
            }
            H.coarse_n = A.rows;
            L.A = std::move(A);
            L.omega = 0.0;
            H.levels.push_back(std::move(L));
            return true;
        }
        const double rho = spectral_radius(A, d);
        L.omega = 4.0 / (3.0 * rho);
        std::vector<int64_t> agg;
        const int64_t na = aggregate(A, d, agg);
        if (na < 1 || na > A.rows * 9 / 10) {
            // coarsening stalled: make this the coarsest level if it is small enough
            if (A.rows <= 8 * kCoarsest && dense_spd_inverse(A, H.coarse_inv)) {
                H.coarse_n = A.rows;
                L.A = std::move(A);
                L.omega = 0.0;
                H.levels.push_back(std::move(L));
                return true;
            }
            err = "multigrid setup: aggregation did not coarsen";
            return false;
        }
        L.P = smoothed_prolongator(A, d, agg, na, L.omega);
        L.R = transpose(L.P);
        AmgCsr Ac = spgemm(L.R, spgemm(A, L.P));
        L.A = std::move(A);
        H.levels.push_back(std::move(L));
        A = std::move(Ac);
    }
    err = "multigrid setup: too many levels";
    return false;
}

// ---------------------------------------------------------------- host check
namespace {

void csr_apply(const AmgCsr &A, const std::vector<double> &x, std::vector<double> &y) {
    y.assign(A.rows, 0.0);
    for (int64_t i = 0; i < A.rows; ++i) {
        double s = 0.0;
        for (int64_t p = A.off[i]; p < A.off[i + 1]; ++p) s += A.val[p] * x[A.col[p]];
        y[i] = s;
    }
}

// the V-cycle of the device solver, on the host: x = V(b) on level l
void host_vcycle(const AmgHierarchy &H, size_t l, const std::vector<double> &b, std::vector<double> &x) {
    const AmgLevel &L = H.levels[l];
    const int64_t n = L.A.rows;
    x.assign(n, 0.0);
    if (l + 1 == H.levels.size()) {
        for (int64_t i = 0; i < n; ++i) {
            double s = 0.0;
            for (int64_t j = 0; j < n; ++j) s += H.coarse_inv[i * n + j] * b[j];
            x[i] = s;
        }
        return;
    }
    for (int64_t i = 0; i < n; ++i) x[i] = L.omega * L.dinv[i] * b[i];
    std::vector<double> t, r(n), bc, xc;
    csr_apply(L.A, x, t);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - t[i];
    csr_apply(L.R, r, bc);
    host_vcycle(H, l + 1, bc, xc);
    csr_apply(L.P, xc, t);
    for (int64_t i = 0; i < n; ++i) x[i] += t[i];
    csr_apply(L.A, x, t);
    for (int64_t i = 0; i < n; ++i) x[i] += L.omega * L.dinv[i] * (b[i] - t[i]);
}

}  // namespace

bool amg_host_solve(const AmgCsr &A, const std::vector<double> &b, std::vector<double> &x, double rtol,
                    int32_t max_iter, int32_t *iters, int32_t *levels, std::string &err) {
    AmgHierarchy H;
    if (!build_amg(A, H, err)) return false;
    *levels = (int32_t)H.levels.size();
    const int64_t n = A.rows;
    std::vector<double> r(b), z, p, Ap;
    x.assign(n, 0.0);
    double bn = 0.0;
    for (double v : b) bn += v * v;
    bn = std::sqrt(bn);
    *iters = 0;
    if (!(bn > 0.0)) return true;
    host_vcycle(H, 0, r, z);
    p = z;
    double rz = 0.0;
    for (int64_t i = 0; i < n; ++i) rz += r[i] * z[i];
    for (int32_t it = 1; it <= max_iter; ++it) {
        csr_apply(A, p, Ap);
        double pAp = 0.0;
        for (int64_t i = 0; i < n; ++i) pAp += p[i] * Ap[i];
        const double a = rz / pAp;
        double rr = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            x[i] += a * p[i];
            r[i] -= a * Ap[i];
            rr += r[i] * r[i];
        }
        *iters = it;
        if (std::sqrt(rr) <= rtol * bn) return true;
        host_vcycle(H, 0, r, z);
        double rz2 = 0.0;
        for (int64_t i = 0; i < n; ++i) rz2 += r[i] * z[i];
        const double beta = rz2 / rz;
        rz = rz2;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    err = "host multigrid PCG did not converge";
    return false;
}
