"""Host-side mesh validation of libdd (no GPU): counts agree with the oracle's
topology and malformed meshes are rejected with DD_EINVAL."""
import numpy as np
import pytest

from oracle.topology import split_boundary, edge_triangle_counts
from synthetic import workloads
from synthetic.meshes import convex_holes, disk_rings, grid_obstacles


@pytest.fixture(scope="module")
def dd():
    from paper_1708_02845_gb300.build import build
    build()
    from paper_1708_02845_gb300 import dd as mod
    return mod


@pytest.mark.parametrize("mesh", [disk_rings(16, 128), workloads.grid140(T=1, S=0).mesh,
                                  grid_obstacles(7, [(2, 2, 2, 3)]), convex_holes(500, 4, 2),
                                  convex_holes(2000, 2, 3)])
def test_counts_match_oracle(dd, mesh):
    idx, off = mesh.loop_arrays()
    n_v, k, m, ne = dd.dd_check_mesh(mesh.xy, mesh.tri, idx, off)
    B, I = split_boundary(mesh.n_v, mesh.tri, mesh.loops)
    assert (n_v, k, m, ne) == (mesh.n_v, len(B), len(I), len(edge_triangle_counts(mesh.tri)))


def test_rejects_malformed(dd):
    mesh = grid_obstacles(6, [(2, 2, 2, 2)])
    idx, off = mesh.loop_arrays()
    cw = mesh.tri[:, [0, 2, 1]].copy()
    with pytest.raises(dd.DDError, match="counter-clockwise"):
        dd.dd_check_mesh(mesh.xy, cw, idx, off)
    with pytest.raises(dd.DDError, match="boundary"):
        dd.dd_check_mesh(mesh.xy, mesh.tri, idx[:-4], np.array([0, off[1], off[2] - 4]))
    swapped = idx.copy()
    swapped[[1, 2]] = swapped[[2, 1]]
    with pytest.raises(dd.DDError, match="not a boundary edge"):
        dd.dd_check_mesh(mesh.xy, mesh.tri, swapped, off)
    bad = mesh.tri.copy()
    bad[0, 0] = mesh.n_v + 5
    with pytest.raises(dd.DDError, match="out of range"):
        dd.dd_check_mesh(mesh.xy, bad, idx, off)
    xy = mesh.xy.copy()
    xy[3, 0] = np.nan
    with pytest.raises(dd.DDError, match="non-finite"):
        dd.dd_check_mesh(xy, mesh.tri, idx, off)
    extra = np.vstack([mesh.xy, [[0.5, 0.5]]])
    with pytest.raises(dd.DDError):
        dd.dd_check_mesh(extra, mesh.tri, idx, off)
