"""Poisson kernel with every entry to full relative precision, and log P
(oracle, FP64 CPU).

Test infrastructure only: imported by tests/ and bench.py's CPU legs, never
by the library.

Section V (Precision): on maze-like domains the Poisson-kernel vectors, like
the Dirichlet Green's function, take values many orders of magnitude apart,
and an ordinary solve resolves the small ones only relative to the large
ones; the paper points to computing log P instead (the method of Wray et
al.).  Here the same goal -- every entry of P, however small, to a few units
of rounding relative to itself -- is reached by an elimination that never
subtracts: Eq. 32, (-L_II) P_IB = L_IB, has an M-matrix on the left
(positive diagonal, off-diagonals -w_ij <= 0, each row's diagonal equal to
the sum of its off-diagonal magnitudes plus the row's boundary weights s_i)
and a non-negative right-hand side.  Gaussian elimination of such a system
can be carried out on the magnitudes alone (the Grassmann-Taksar-Heyman
form of elimination for Markov chains):

* off-diagonal magnitudes grow by |a_ik| |a_kj| / a_kk when column k is
  eliminated (a sum of non-negative numbers);
* each row's slack grows by |a_ik| s_k / a_kk, and the pivot a_kk is formed
  as s_k plus the row's remaining off-diagonal magnitudes, never as a
  difference (the diagonal update a_ii - a_ik a_ki / a_kk is the one
  subtraction of plain elimination, and the one this form avoids);
* the right-hand side grows by |a_ik| b_k / a_kk, and back substitution adds
  non-negative terms.

Every quantity is then a sum of products of non-negative rounded numbers,
so each entry of P carries a relative error of a small multiple of the unit
roundoff times the number of operations, whatever its size.  Requires
non-negative edge weights (every grid and Delaunay mesh here).  Limit: FP64
itself; entries below about 1e-300 would underflow, and the synthetic mazes
are sized to stay above that (the tests check it).  Dense O(m^3): meant for
the small maze-like meshes of the tests.
"""

import numpy as np

from .laplacian import cotan_laplacian
from .topology import split_boundary


def poisson_subtraction_free(xy, tri, loops) -> np.ndarray:
    """P (n x k, Eq. 33) by subtraction-free elimination: entries to full relative precision."""
    n = xy.shape[0]
    B, I = split_boundary(n, tri, loops)
    B, I = np.asarray(B), np.asarray(I)
    k, m = len(B), len(I)
    Lc = cotan_laplacian(xy, tri).tocsr()
    W = Lc[I][:, I].toarray()
    np.fill_diagonal(W, 0.0)                  # w_ij >= 0 between interior vertices
    F = Lc[I][:, B].toarray()                 # L_IB: w_ib >= 0
    if (W < 0).any() or (F < 0).any():
        raise ValueError("subtraction-free elimination needs non-negative edge weights")
    s = F.sum(axis=1)                         # row slack: the boundary weights of each interior row
    piv = np.zeros(m)
    for c in range(m):
        d = s[c] + W[c, c + 1:].sum()         # the pivot a_cc as a sum of non-negative numbers
        piv[c] = d
        f = W[c + 1:, c] / d                  # |a_ic| / a_cc
        W[c + 1:, c + 1:] += f[:, None] * W[c, c + 1:][None, :]
        s[c + 1:] += f * s[c]
        F[c + 1:] += f[:, None] * F[c][None, :]
    X = np.zeros((m, k))
    for c in range(m - 1, -1, -1):            # x_c = (b_c + sum_{j > c} |a_cj| x_j) / a_cc
        X[c] = (F[c] + W[c, c + 1:] @ X[c + 1:]) / piv[c]
    P = np.zeros((n, k))
    P[I] = X
    P[B, np.arange(k)] = 1.0
    return P


def log_poisson(xy, tri, loops) -> np.ndarray:
    """Natural log of P (-inf where P is exactly 0: off-diagonal boundary
    entries and columns with no interior support)."""
    P = poisson_subtraction_free(xy, tri, loops)
    with np.errstate(divide="ignore"):
        return np.log(P)
