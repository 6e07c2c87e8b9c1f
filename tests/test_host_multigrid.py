"""Host-side check of the Poisson-kernel solver's multigrid preconditioner
(no GPU): the library's hierarchy and V-cycle, driving conjugate gradients on
the interior cotangent Laplacian of the synthetic meshes, reproduce a direct
sparse solve, and the iteration count stays flat as the mesh grows (the
point of the multigrid preconditioner, whose diagonal counterpart needs
hundreds to thousands of iterations on these meshes)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.laplacian import cotan_laplacian
from oracle.topology import split_boundary
from synthetic import workloads
from synthetic.meshes import convex_holes, disk_rings, grid_obstacles


@pytest.fixture(scope="module")
def dd():
    from paper_1708_02845_gb300.build import build
    build()
    from paper_1708_02845_gb300 import dd as mod
    return mod


def interior_system(mesh):
    L = cotan_laplacian(mesh.xy, mesh.tri).tocsr()
    B, I = split_boundary(mesh.n_v, mesh.tri, mesh.loops)
    A = (-L[I][:, I]).tocsr()
    A.sort_indices()
    rhs = L[I][:, B].tocsc()          # Eq. 32: (-L_II) P_IB = L_IB
    return A, rhs, len(I)


MESHES = {
    "disk16": lambda: disk_rings(16, 128),
    "grid37": lambda: workloads.small_grid(37, 3, T=1, S=0).mesh,
    "grid140": lambda: workloads.grid140(T=1, S=0).mesh,
    "holes10k": lambda: convex_holes(10000, 4, 1),          # unstructured Delaunay, five boundary loops
}


@pytest.mark.parametrize("name", list(MESHES))
def test_multigrid_cg_matches_direct_solve(dd, name):
    A, rhs, m = interior_system(MESHES[name]())
    lu = spla.splu(A.tocsc())
    iters = []
    for j in (0, rhs.shape[1] // 2, rhs.shape[1] - 1):
        b = np.asarray(rhs[:, j].todense()).ravel()
        if not np.any(b):
            continue
        x, it, levels = dd.dd_multigrid_check(A.indptr, A.indices, A.data, b, rtol=1e-13, max_iter=200)
        ref = lu.solve(b)
        assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()
        assert np.linalg.norm(b - A @ x) <= 1e-13 * np.linalg.norm(b) * 1.0001
        iters.append(it)
        assert levels >= 2
    assert iters and max(iters) <= 40, iters


def test_iterations_do_not_grow_with_the_mesh(dd):
    counts = {}
    for name in ("grid37", "grid140"):
        A, rhs, m = interior_system(MESHES[name]())
        # one boundary column (the sum of all of them is the constant vector,
        # which the coarse space represents exactly)
        j = int(np.argmax(np.asarray(abs(rhs).sum(axis=0)).ravel()))
        b = np.asarray(rhs[:, j].todense()).ravel()
        _, it, _ = dd.dd_multigrid_check(A.indptr, A.indices, A.data, b, rtol=1e-15, max_iter=200)
        counts[name] = (m, it)
    (m_small, it_small), (m_big, it_big) = counts["grid37"], counts["grid140"]
    assert m_big > 10 * m_small
    assert it_big <= it_small + 8, counts


def test_rejects_bad_input(dd):
    A = sp.identity(4, format="csr")
    with pytest.raises(dd.DDError):
        dd.dd_multigrid_check(A.indptr, np.array([0, 1, 2, 7], np.int32), A.data, np.ones(4))
