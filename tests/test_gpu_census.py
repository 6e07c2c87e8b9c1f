"""GPU parity of the spurious-local-minimum census and the edge-following
paths (Sections IV-V), through the C ABI.  Both only compare the given FP32
field values, so they must agree exactly with the oracle's rule applied to
the same values: identical minimum flags and counts, identical vertex
sequences and statuses.
"""
import numpy as np
import pytest

from oracle import census
from oracle.divergence import kl_field, tv_field
from oracle.fdiv import field
from oracle.greens import dirichlet_green_column
from oracle.poisson import PoissonOracle
from oracle.topology import vertex_neighbours
from synthetic import workloads
from synthetic.meshes import convex_holes, disk_rings, grid_obstacles
from tests._gpu import ctx_and_lib, load

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    yield dd, ctx
    dd.dd_destroy(ctx)


MESHES = {
    "disk_coarse": lambda: disk_rings(6, 32),
    "grid_coarse": lambda: grid_obstacles(14, [(3, 3, 2, 2), (8, 7, 3, 2)]),
    "grid140": lambda: workloads.grid140(T=1, S=1).mesh,
}


def _fields(dd, ctx, mesh, targets):
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    out = torch.empty((2, len(targets), mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, out)
    dd.dd_sync(ctx)
    return mid, out


@pytest.mark.parametrize("name", list(MESHES))
def test_census_matches_oracle_rule(env, name):
    dd, ctx = env
    mesh = MESHES[name]()
    interior = ~mesh.boundary_flags()
    ids = np.nonzero(interior)[0]
    targets = [int(ids[i]) for i in np.linspace(0, len(ids) - 1, 6).astype(int)]
    mid, out = _fields(dd, ctx, mesh, targets)
    for fi in range(2):
        f = out[fi].contiguous()
        flags = torch.zeros((len(targets), mesh.n_v), dtype=torch.uint8, device="cuda")
        counts = dd.dd_local_minima(ctx, mid, f, targets, flags)
        host_flags = np.zeros((len(targets), mesh.n_v), dtype=np.uint8)
        counts_h = dd.dd_local_minima(ctx, mid, f, targets, host_flags)
        fh = f.cpu().numpy().astype(np.float64)
        for a, t in enumerate(targets):
            ref = census.local_minima(fh[a], mesh.tri, interior, t)
            got = np.nonzero(flags[a].cpu().numpy())[0]
            assert np.array_equal(got, ref)
            assert np.array_equal(np.nonzero(host_flags[a])[0], ref)
            assert counts[a] == counts_h[a] == len(ref)
    dd.dd_unload_mesh(ctx, mid)


@pytest.mark.parametrize("name", list(MESHES))
def test_edge_paths_match_oracle_rule(env, name):
    dd, ctx = env
    mesh = MESHES[name]()
    interior = ~mesh.boundary_flags()
    ids = np.nonzero(interior)[0]
    targets = [int(ids[len(ids) // 3]), int(ids[2 * len(ids) // 3])]
    S = 12
    sources = np.array([[int(ids[(a * 7919 + s * 104729) % len(ids)]) for s in range(S)] for a in range(2)], np.int32)
    mid, out = _fields(dd, ctx, mesh, targets)
    mp = 4096
    for fi in range(2):
        f = out[fi].contiguous()
        xy = torch.empty((2 * S, mp, 2), dtype=torch.float32, device="cuda")
        ln = torch.empty(2 * S, dtype=torch.int32, device="cuda")
        st = torch.empty(2 * S, dtype=torch.int32, device="cuda")
        dd.dd_trace_edges(ctx, mid, f, targets, sources, mp, xy, ln, st)
        dd.dd_sync(ctx)
        xy, ln, st = xy.cpu().numpy(), ln.cpu().numpy(), st.cpu().numpy()
        fh = f.cpu().numpy().astype(np.float64)
        for a, t in enumerate(targets):
            for s in range(S):
                pts, status = census.edge_path(fh[a], mesh.tri, mesh.xy, int(sources[a, s]), t, max_pts=mp)
                i = a * S + s
                assert st[i] == status
                assert ln[i] == len(pts)
                assert np.allclose(xy[i, :ln[i]], pts.astype(np.float32), atol=0, rtol=0)
    dd.dd_unload_mesh(ctx, mid)


def _margin(f, nb, v):
    return min(f[u] for u in nb[v]) - f[v]


@pytest.mark.parametrize("n_goal,seed", [(175, 2), (500, 4)])
def test_census_on_fp64_fields(env, n_goal, seed):
    """Census of the FP32 fields (TV, KL, target-weighted KL) on the oracle's
    kernel against the census of the FP64 oracle fields, all interior targets
    of a low-resolution convex-holes mesh.  A vertex may be classified
    differently only where the FP64 field's gap to its lowest neighbour is
    within the two fields' FP32 error bounds (2 x 1e-5 relative, floor 1e-2)."""
    dd, ctx = env
    mesh = convex_holes(n_goal, seed=seed)
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    P = po.full()
    interior = ~mesh.boundary_flags()
    nb = vertex_neighbours(mesh.n_v, mesh.tri)
    targets = [int(t) for t in np.nonzero(interior)[0]]
    T = len(targets)
    mid = load(dd, ctx, mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    tk = torch.empty((2, T, mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, tk)
    rev = torch.empty((T, mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_divergence(ctx, mid, targets, dd.DD_DIV_KL_REVERSE, 0.0, rev)
    dd.dd_sync(ctx)
    fams = [("kl", tk[0], kl_field), ("tv", tk[1], tv_field),
            ("kl_target_weighted", rev, lambda P_, Pt: field(P_, Pt, "kl_reverse"))]
    for name, g, ref_fn in fams:
        flags = torch.zeros((T, mesh.n_v), dtype=torch.uint8, device="cuda")
        counts = dd.dd_local_minima(ctx, mid, g.contiguous(), targets, flags)
        fl = flags.cpu().numpy()
        for a, t in enumerate(targets):
            r = ref_fn(P, P[t])
            ref = set(census.local_minima(r, mesh.tri, interior, t).tolist())
            got = set(np.nonzero(fl[a])[0].tolist())
            assert counts[a] == len(got)
            for v in got ^ ref:
                tol = 2e-5 * max(abs(r[v]), 1e-2)
                assert abs(_margin(r, nb, v)) <= tol, (name, t, v, _margin(r, nb, v))
    # the Green's-function check of the maximum principle: none at all
    assert all(census.local_minima(dirichlet_green_column(po, t), mesh.tri, interior, t).size == 0
               for t in targets[::7])
    dd.dd_unload_mesh(ctx, mid)
