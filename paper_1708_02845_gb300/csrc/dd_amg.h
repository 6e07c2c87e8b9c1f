// Smoothed-aggregation multigrid hierarchy (host side), used as the
// preconditioner of the Poisson-kernel solve.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

// CSR matrix with FP64 values (rows ascending, columns ascending in a row)
struct AmgCsr {
    int64_t rows = 0, cols = 0;
    std::vector<int64_t> off;
    std::vector<int32_t> col;
    std::vector<double> val;
};

// One level: its operator A, the inverse diagonal, the Jacobi weight omega
// (also the prolongator-smoothing weight) and, except on the coarsest level,
// the prolongator P to it from the next coarser level and R = P^T.
struct AmgLevel {
    AmgCsr A, P, R;
    std::vector<double> dinv;
    double omega = 0.0;
};

struct AmgHierarchy {
    std::vector<AmgLevel> levels;      // levels[0] is the fine operator
    std::vector<double> coarse_inv;    // dense inverse of the coarsest operator, row-major
    int64_t coarse_n = 0;
};

// Build the hierarchy for the SPD matrix A0; false (with a message) when a
// step fails.
bool build_amg(const AmgCsr &A0, AmgHierarchy &H, std::string &err);

// The device solver's multigrid-preconditioned CG for one right-hand side, on
// the host (a check of the hierarchy and the V-cycle without a GPU): solves
// A x = b to ||r|| <= rtol ||b||.  *levels: hierarchy depth.
bool amg_host_solve(const AmgCsr &A, const std::vector<double> &b, std::vector<double> &x, double rtol,
                    int32_t max_iter, int32_t *iters, int32_t *levels, std::string &err);
