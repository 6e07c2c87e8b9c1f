"""Cotangent Laplacian of Section IV (oracle, FP64 CPU).

L^c_ij = (cot alpha_ij + cot beta_ij) / 2 for an edge (i, j), alpha and beta the
angles opposite the edge (one of them only on a boundary edge), and
L^c_ii = -sum_j L^c_ij.  Also the area-weighted L = A^-1 L^c, a_i a third of
the areas of the triangles around vertex i, and the normalised L^n = Z^-1 L^c,
Z = diag(L^c).
"""

import numpy as np
import scipy.sparse as sp


def cot_weights(xy: np.ndarray, tri: np.ndarray):
    """Per-edge weight dict {(i, j), i < j: w_ij} summed over incident triangles."""
    w = {}
    for t in tri:
        for c in range(3):
            k = int(t[c])
            i, j = int(t[(c + 1) % 3]), int(t[(c + 2) % 3])
            u = xy[i] - xy[k]
            v = xy[j] - xy[k]
            dot = u[0] * v[0] + u[1] * v[1]
            cross = abs(u[0] * v[1] - u[1] * v[0])
            key = (i, j) if i < j else (j, i)
            w[key] = w.get(key, 0.0) + 0.5 * dot / cross
    return w


def cotan_laplacian(xy: np.ndarray, tri: np.ndarray) -> sp.csr_matrix:
    """Symmetric sparse L^c (n x n), off-diagonals w_ij, diagonal -row sum."""
    n = xy.shape[0]
    w = cot_weights(xy, tri)
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    for (i, j), v in w.items():
        rows += [i, j]
        cols += [j, i]
        vals += [v, v]
        diag[i] -= v
        diag[j] -= v
    rows += list(range(n))
    cols += list(range(n))
    vals += list(diag)
    return sp.csr_matrix((np.asarray(vals), (np.asarray(rows), np.asarray(cols))), shape=(n, n))


def vertex_areas(xy: np.ndarray, tri: np.ndarray) -> np.ndarray:
    a = np.zeros(xy.shape[0])
    for t in tri:
        p0, p1, p2 = xy[t[0]], xy[t[1]], xy[t[2]]
        area = 0.5 * abs((p1[0] - p0[0]) * (p2[1] - p0[1]) - (p1[1] - p0[1]) * (p2[0] - p0[0]))
        for v in t:
            a[int(v)] += area / 3.0
    return a


def area_laplacian(xy, tri) -> sp.csr_matrix:
    """L = A^-1 L^c."""
    Lc = cotan_laplacian(xy, tri)
    return sp.diags(1.0 / vertex_areas(xy, tri)) @ Lc


def normalised_laplacian(xy, tri) -> sp.csr_matrix:
    """L^n = Z^-1 L^c, Z = diag(L^c) (unit diagonal)."""
    Lc = cotan_laplacian(xy, tri)
    return sp.diags(1.0 / Lc.diagonal()) @ Lc
