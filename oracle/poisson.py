"""Discrete Poisson kernel, Section IV Eq. (32)-(33) (oracle, FP64 CPU).

P is the n x k matrix whose column b is the discrete harmonic function with
boundary values the indicator of boundary vertex b:
    (L_II  L_IB) [P_IB; I] = 0   =>   P_IB = -L_II^-1 L_IB,   P_BB = I.
The paper notes (Section IV) that L, L^c and L^n give the same P; L^c is used
because it is symmetric.

The solve is a direct sparse LU of the M-matrix -L_II (SuperLU, symmetric
ordering, diagonal pivots), a library primitive used as one step.  Rows of P
are kept in original vertex order; columns follow the boundary loop order.

For large meshes, single rows are available without forming P: because L^c is
symmetric, row x of P_IB is -(L_II^-1 e_x)^T L_IB, one solve per sampled row
(the discrete form of Eq. (11)/(14): P is the boundary normal derivative of
the Green's function with pole x).
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .laplacian import cotan_laplacian
from .topology import split_boundary


class PoissonOracle:
    """Factorises -L_II once; returns full P or selected rows."""

    def __init__(self, xy, tri, loops, L=None):
        self.n = xy.shape[0]
        self.B, self.I = split_boundary(self.n, tri, loops)
        self.k = len(self.B)
        self.m = len(self.I)
        self.L = cotan_laplacian(xy, tri) if L is None else L
        Lcsc = self.L.tocsc()
        self.L_II = Lcsc[self.I][:, self.I].tocsc()
        self.L_IB = Lcsc[self.I][:, self.B].tocsc()
        self.pos_in_I = -np.ones(self.n, dtype=np.int64)
        self.pos_in_I[self.I] = np.arange(self.m)
        self.col_of = -np.ones(self.n, dtype=np.int64)
        self.col_of[self.B] = np.arange(self.k)
        self._lu = None

    @property
    def lu(self):
        if self._lu is None:
            self._lu = spla.splu((-self.L_II).tocsc(), permc_spec="MMD_AT_PLUS_A",
                                 diag_pivot_thresh=0.0,
                                 options={"SymmetricMode": True})
        return self._lu

    def full(self) -> np.ndarray:
        """Dense P (n x k), Eq. (33)."""
        P = np.zeros((self.n, self.k))
        rhs = self.L_IB.toarray()                 # -L_II X = L_IB  <=>  X = -L_II^-1 L_IB
        P_IB = self.lu.solve(rhs) if self.m else np.zeros((0, self.k))
        P[self.I] = P_IB
        P[self.B, np.arange(self.k)] = 1.0
        return P

    def rows(self, xs) -> np.ndarray:
        """Rows P[x, :] for the given vertex ids (Green's-row form for interior x)."""
        xs = np.asarray(xs, dtype=np.int64)
        out = np.zeros((len(xs), self.k))
        interior = [a for a, x in enumerate(xs) if self.pos_in_I[x] >= 0]
        if interior:
            E = np.zeros((self.m, len(interior)))
            for c, a in enumerate(interior):
                E[self.pos_in_I[xs[a]], c] = 1.0
            G = self.lu.solve(E)                  # G = (-L_II)^-1 e_x  (symmetric)
            rowsIB = (self.L_IB.T @ G).T          # = -(L_II^-1 e_x)^T L_IB
            for c, a in enumerate(interior):
                out[a] = rowsIB[c]
        for a, x in enumerate(xs):
            if self.col_of[x] >= 0:
                out[a, self.col_of[x]] = 1.0
        return out
