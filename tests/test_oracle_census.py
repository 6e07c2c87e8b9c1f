"""Pins for the oracle's local-minimum census and edge-following paths
(Sections IV-V) -- CPU only.

Pinned by: the discrete maximum principle (the Dirichlet Green's function,
an M-matrix solve, has no interior minimum but its pole), planted wells
whose minima are known by construction, and the defining properties of an
edge-following path (every move is to a mesh neighbour with a smaller value,
so the values strictly decrease; it stops exactly at the target or at a
planted well).
"""
import numpy as np
import pytest

from oracle import census
from oracle.greens import dirichlet_green_column
from oracle.poisson import PoissonOracle
from oracle.topology import vertex_neighbours
from synthetic.meshes import disk_rings, grid_obstacles

MESHES = [lambda: disk_rings(8, 48), lambda: grid_obstacles(18, [(4, 4, 3, 3), (10, 9, 4, 2)])]


def interior_mask(po, n_v):
    m = np.zeros(n_v, dtype=bool)
    m[po.I] = True
    return m


@pytest.mark.parametrize("make", MESHES)
def test_green_function_has_no_spurious_minimum(make):
    mesh = make()
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    mask = interior_mask(po, mesh.n_v)
    for p in (int(po.I[3]), int(po.I[len(po.I) // 2]), int(po.I[-5])):
        d = dirichlet_green_column(po, p)
        assert census.local_minima(d, mesh.tri, mask, p).size == 0
        # and the pole itself is the one minimum when it is not excluded
        assert list(census.local_minima(d, mesh.tri, mask, -1)) == [p]


@pytest.mark.parametrize("make", MESHES)
def test_planted_wells(make):
    mesh = make()
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    mask = interior_mask(po, mesh.n_v)
    centres = [int(po.I[i]) for i in (2, len(po.I) // 3, 2 * len(po.I) // 3)]
    d2 = np.min([np.sum((mesh.xy - mesh.xy[c]) ** 2, axis=1) for c in centres], axis=0)
    t = centres[0]
    assert list(census.local_minima(d2, mesh.tri, mask, t)) == sorted(centres[1:])
    # an edge path started next to the second well stops there
    nb = vertex_neighbours(mesh.n_v, mesh.tri)
    q = next(u for u in nb[centres[1]] if mask[u] and u not in centres)
    pts, st = census.edge_path(d2, mesh.tri, mesh.xy, q, t)
    assert st == census.STUCK and np.allclose(pts[-1], mesh.xy[centres[1]])


@pytest.mark.parametrize("make", MESHES)
def test_edge_paths_descend_to_the_target(make):
    mesh = make()
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    nb = vertex_neighbours(mesh.n_v, mesh.tri)
    p = int(po.I[len(po.I) // 2])
    d = dirichlet_green_column(po, p)
    index = {tuple(np.round(xy, 12)): i for i, xy in enumerate(mesh.xy)}
    for q in (int(po.I[0]), int(po.I[-1]), int(po.I[len(po.I) // 5])):
        pts, st = census.edge_path(d, mesh.tri, mesh.xy, q, p)
        assert st == census.OK
        ids = [index[tuple(np.round(x, 12))] for x in pts]
        assert ids[0] == q and ids[-1] == p
        for a, b in zip(ids, ids[1:]):
            assert b in nb[a] and d[b] < d[a]
            # the move takes the lowest neighbour
            assert d[b] == min(d[u] for u in nb[a])
    pts, st = census.edge_path(d, mesh.tri, mesh.xy, int(po.I[0]), p, max_pts=2)
    assert st == census.TRUNCATED and len(pts) == 2


@pytest.mark.parametrize("n_goal,seed", [(175, 1), (175, 3), (500, 2)])
def test_convex_holes_mesh_and_maximum_principle(n_goal, seed):
    """The low-resolution convex-holes meshes are valid inputs (loops are the
    topological boundary, every edge touching the interior has a
    non-negative cotangent weight: Delaunay), so P is a stochastic matrix and
    the Dirichlet Green's function of every interior target has no spurious
    minimum."""
    from oracle.laplacian import cotan_laplacian
    from oracle.topology import split_boundary
    from synthetic.meshes import convex_holes

    mesh = convex_holes(n_goal, seed=seed)
    split_boundary(mesh.n_v, mesh.tri, mesh.loops)
    assert abs(mesh.n_v - n_goal) < 0.2 * n_goal
    bf = mesh.boundary_flags()
    L = cotan_laplacian(mesh.xy, mesh.tri).tocoo()
    touch = (L.row != L.col) & ~(bf[L.row] & bf[L.col])
    assert np.all(L.data[touch] > 0.0)             # off-diagonal = +w_ij here, w_ij > 0
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    P = po.full()
    assert P.min() >= -1e-14 and np.allclose(P.sum(axis=1), 1.0, atol=1e-12)
    mask = interior_mask(po, mesh.n_v)
    for t in po.I[::3]:
        assert census.local_minima(dirichlet_green_column(po, int(t)), mesh.tri, mask, int(t)).size == 0
