"""Dirichlet Green's function column, Section IV Eq. (19)-(21) (oracle, FP64 CPU).

For an interior pole p: L_II D_Ip = e_p, D_B = 0.  With L^c negative definite
on the interior, D_Ip <= 0 has its minimum at p and vanishes on the boundary,
so gradient descent on D_Ip runs to p; the path-agreement check (Theorem A6)
compares divergence-distance paths with paths traced on this field.
"""

import numpy as np


def dirichlet_green_column(po, p: int) -> np.ndarray:
    """Field over all n vertices: D_Ip on I, 0 on B.  `po` is a PoissonOracle."""
    e = np.zeros(po.m)
    e[po.pos_in_I[p]] = 1.0
    d_I = -po.lu.solve(e)             # (-L_II)^-1 e_p = -D_Ip
    out = np.zeros(po.n)
    out[po.I] = d_I
    return out
