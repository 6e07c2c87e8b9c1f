"""Pins for the oracle's cotangent Laplacian (Section IV) -- CPU only."""
import math

import numpy as np
import pytest

from oracle.laplacian import cot_weights, cotan_laplacian, area_laplacian, normalised_laplacian
from oracle.topology import split_boundary, TopologyError
from synthetic.meshes import disk_rings, grid_obstacles
from tests._meshes import hexagon, plain_grid


def test_grid_weights_are_axis_one_diagonal_zero():
    # right isosceles triangles: axis edges see two 45-degree angles, the
    # diagonal sees two right angles (cot 45 = 1, cot 90 = 0)
    m = plain_grid(4)
    w = cot_weights(m.xy, m.tri)
    ids = m.meta["ids"]
    assert w[tuple(sorted((ids[1, 1], ids[1, 2])))] == pytest.approx(1.0, abs=1e-14)
    assert w[tuple(sorted((ids[1, 1], ids[2, 1])))] == pytest.approx(1.0, abs=1e-14)
    assert abs(w[tuple(sorted((ids[1, 1], ids[2, 2])))]) < 1e-14
    # boundary axis edge has one triangle: cot 45 / 2
    assert w[tuple(sorted((ids[0, 0], ids[0, 1])))] == pytest.approx(0.5, abs=1e-14)


def test_equilateral_weights():
    m = hexagon()
    w = cot_weights(m.xy, m.tri)
    for i in range(1, 7):
        assert w[(0, i)] == pytest.approx(1.0 / math.sqrt(3.0), rel=1e-13)   # two 60-degree angles
    assert w[(1, 2)] == pytest.approx(0.5 / math.sqrt(3.0), rel=1e-13)       # boundary edge


def test_rows_sum_to_zero_and_symmetric():
    m = disk_rings(6, 24)
    L = cotan_laplacian(m.xy, m.tri).toarray()
    assert np.abs(L.sum(axis=1)).max() < 1e-12
    assert np.abs(L - L.T).max() < 1e-14
    assert (np.diag(L) < 0).all()


@pytest.mark.parametrize("mesh", [disk_rings(8, 32), grid_obstacles(12, [(3, 3, 3, 2)]), hexagon()])
def test_linear_precision(mesh):
    # the planar cotangent Laplacian annihilates linear functions at interior
    # vertices: L_II x_I + L_IB x_B = 0 for both coordinates
    L = cotan_laplacian(mesh.xy, mesh.tri).toarray()
    B, I = split_boundary(mesh.n_v, mesh.tri, mesh.loops)
    for c in range(2):
        r = L[I] @ mesh.xy[:, c]
        assert np.abs(r).max() < 1e-12


def test_variants_share_harmonic_functions():
    # L = A^-1 L^c and L^n = Z^-1 L^c scale rows only, so they share null rows
    m = disk_rings(5, 20)
    Lc = cotan_laplacian(m.xy, m.tri).toarray()
    La = area_laplacian(m.xy, m.tri).toarray()
    Ln = normalised_laplacian(m.xy, m.tri).toarray()
    assert np.allclose(np.diag(Ln), 1.0)
    ratio_a = La / np.where(Lc != 0, Lc, 1.0)
    for i in range(m.n_v):
        nz = Lc[i] != 0
        assert np.allclose(ratio_a[i, nz], ratio_a[i, nz][0])


def test_topology_rejects_bad_loops():
    m = plain_grid(3)
    loops = [m.loops[0][:-1]]
    with pytest.raises(TopologyError):
        split_boundary(m.n_v, m.tri, loops)
    bad = [m.loops[0][::-1].copy()]
    bad[0][[0, 1]] = bad[0][[1, 0]]
    with pytest.raises(TopologyError):
        split_boundary(m.n_v, m.tri, bad)
