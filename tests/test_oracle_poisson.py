"""Pins for the oracle's discrete Poisson kernel (Eq. 32-33) -- CPU only.

Pinned by: exact rational brute force on tiny grids (an independent Gaussian
elimination over Fractions), the unit-sum and non-negativity invariants
(Eq. 13), linear precision of harmonic interpolation, the disk closed form
Eq. (15) with its convergence under refinement, and the Section IV remark
that L, L^c and L^n give the same P.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle.laplacian import area_laplacian, normalised_laplacian
from oracle.poisson import PoissonOracle
from oracle.topology import split_boundary
from synthetic.meshes import disk_rings, grid_obstacles
from synthetic import workloads
from tests._meshes import hexagon, plain_grid


def exact_poisson_grid(mesh):
    """P by exact rational elimination on a grid mesh (integer coordinates).

    Cot weights from integer vectors: dot / |cross| as Fractions.
    """
    N = mesh.meta["N"]
    ixy = np.rint(mesh.xy * N).astype(np.int64)
    n = mesh.n_v
    W = {}
    for t in mesh.tri:
        for c in range(3):
            k, i, j = int(t[c]), int(t[(c + 1) % 3]), int(t[(c + 2) % 3])
            u = ixy[i] - ixy[k]
            v = ixy[j] - ixy[k]
            dot = int(u[0] * v[0] + u[1] * v[1])
            cross = abs(int(u[0] * v[1] - u[1] * v[0]))
            key = (min(i, j), max(i, j))
            W[key] = W.get(key, Fraction(0)) + Fraction(dot, 2 * cross)
    B, I = split_boundary(n, mesh.tri, mesh.loops)
    pos = {int(v): a for a, v in enumerate(I)}
    col = {int(v): a for a, v in enumerate(B)}
    m, k = len(I), len(B)
    # A = -L_II (diag = sum of weights), rhs = L_IB
    A = [[Fraction(0)] * m for _ in range(m)]
    R = [[Fraction(0)] * k for _ in range(m)]
    for (i, j), w in W.items():
        for a, b in ((i, j), (j, i)):
            if a in pos:
                A[pos[a]][pos[a]] += w
                if b in pos:
                    A[pos[a]][pos[b]] -= w
                else:
                    R[pos[a]][col[b]] += w
    # Gauss-Jordan
    for p in range(m):
        piv = A[p][p]
        for q in range(m):
            if q != p and A[q][p] != 0:
                f = A[q][p] / piv
                A[q] = [x - f * y for x, y in zip(A[q], A[p])]
                R[q] = [x - f * y for x, y in zip(R[q], R[p])]
    P = [[Fraction(0)] * k for _ in range(n)]
    for v, a in pos.items():
        P[v] = [x / A[a][a] for x in R[a]]
    for v, b in col.items():
        P[v][b] = Fraction(1)
    return P


def test_three_by_three_centre_row():
    m = plain_grid(2)
    P = PoissonOracle(m.xy, m.tri, m.loops).full()
    ids = m.meta["ids"]
    c = ids[1, 1]
    B, _ = split_boundary(m.n_v, m.tri, m.loops)
    row = dict(zip(B.tolist(), P[c]))
    for v in (ids[0, 1], ids[1, 0], ids[1, 2], ids[2, 1]):
        assert row[v] == pytest.approx(0.25, abs=1e-15)
    for v in (ids[0, 0], ids[0, 2], ids[2, 0], ids[2, 2]):
        assert abs(row[v]) < 1e-15


@pytest.mark.parametrize("mesh", [plain_grid(3), plain_grid(4), grid_obstacles(5, [(2, 2, 1, 1)]),
                                  grid_obstacles(6, [(1, 1, 2, 1), (4, 3, 1, 2)])])
def test_exact_rational_brute_force(mesh):
    exact = exact_poisson_grid(mesh)
    P = PoissonOracle(mesh.xy, mesh.tri, mesh.loops).full()
    E = np.asarray([[float(x) for x in row] for row in exact])
    assert np.abs(P - E).max() < 1e-14


def test_hexagon_centre_is_uniform():
    m = hexagon()
    P = PoissonOracle(m.xy, m.tri, m.loops).full()
    assert np.allclose(P[0], 1.0 / 6.0, atol=1e-15)


@pytest.mark.parametrize("mesh", [disk_rings(16, 128), workloads.small_grid(40, 3).mesh])
def test_unit_rows_nonneg_linear_precision(mesh):
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    P = po.full()
    assert np.abs(P.sum(axis=1) - 1.0).max() < 1e-12           # Eq. (13)
    assert P.min() > -1e-15                                     # harmonic measure >= 0
    recon = P @ mesh.xy[po.B]                                   # harmonic interpolation of x, y
    assert np.abs(recon - mesh.xy).max() < 1e-12
    assert np.allclose(P[po.B], np.eye(po.k))                   # P_BB = I


def test_same_kernel_for_all_three_laplacians():
    m = disk_rings(6, 24)
    P_c = PoissonOracle(m.xy, m.tri, m.loops).full()
    for L in (area_laplacian(m.xy, m.tri), normalised_laplacian(m.xy, m.tri)):
        po = PoissonOracle(m.xy, m.tri, m.loops, L=L)
        A = (-po.L_II).toarray()
        X = np.linalg.solve(A, po.L_IB.toarray())
        assert np.abs(X - P_c[po.I]).max() < 1e-13


def test_green_rows_match_full():
    m = workloads.small_grid(30, 3).mesh
    po = PoissonOracle(m.xy, m.tri, m.loops)
    P = po.full()
    xs = [0, 5, int(po.I[3]), int(po.I[-1]), int(po.B[2])]
    assert np.abs(po.rows(xs) - P[xs]).max() < 1e-13


def _disk_error(R, S):
    m = disk_rings(R, S)
    po = PoissonOracle(m.xy, m.tri, m.loops)
    P = po.full()
    z = m.xy[:, 0] + 1j * m.xy[:, 1]
    s = z[po.B] / np.abs(z[po.B])
    r = np.abs(z)
    sel = r <= 0.8
    # Eq. (15): density (1 - |z|^2) / (2 pi |s - z|^2) times arc length 2 pi / S
    Pc = (1 - r[sel, None] ** 2) / np.abs(z[sel, None] - s[None, :]) ** 2 / S
    return np.abs(P[sel] - Pc).max() / Pc.max()


def test_disk_closed_form_converges():
    e16 = _disk_error(16, 128)
    e32 = _disk_error(32, 256)
    assert e16 < 3e-2
    assert e32 < e16 / 2.5
