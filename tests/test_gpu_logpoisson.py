"""GPU parity of the full-precision Poisson kernel and log P on a maze
(Section V, Precision), through the C ABI.

A serpentine corridor of 6 x 4 x 40 cells: its kernel spans 1 .. 1e-76, a
quarter of the entries lie below FP32's smallest normal (1.2e-38, flushed to
0 in the stored P), and entries below ~1e-16 of their column's largest are
beyond what the block CG's residual can resolve.  Against the oracle's
subtraction-free kernel (every entry to full relative precision):

* before dd_log_poisson_kernel the FP32 path's KL fields are far off for
  targets whose kernel row has such entries (shown, as the contrast);
* after it, log2 P matches the oracle's to FP32 rounding of the logarithm,
  the stored P matches where it is a normal float (0 below), and KL, TV and
  the target-weighted KL of targets deep in the maze meet the FP32 path's
  tolerance |g - r| / max(|r|, 1e-2) <= 1e-5, through both field kernels
  (one or two targets, and more), with exact zeros at the targets; paths
  traced on the KL fields agree with the oracle's tracer on the oracle's
  fields (status, Hausdorff within half a mean edge).
"""
import numpy as np
import pytest

from oracle.divergence import kl_field_fast, tv_field
from oracle.fdiv import kl_reverse_field
from oracle.hausdorff import hausdorff
from oracle.logpoisson import poisson_subtraction_free
from oracle.trace import Tracer
from synthetic.meshes import serpentine
from synthetic.rng import SplitMix64
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load, mean_edge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TINY = float(np.finfo(np.float32).tiny)


@pytest.fixture(scope="module")
def maze():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    mesh = serpentine(6, 4, 40)
    P = poisson_subtraction_free(mesh.xy, mesh.tri, mesh.loops)
    yield dd, ctx, mesh, P
    dd.dd_destroy(ctx)


def _targets(mesh, P, count):
    """Interior targets, spread over the maze, whose kernel rows reach below FLT_MIN."""
    interior = np.nonzero(~mesh.boundary_flags())[0]
    deep = [int(t) for t in interior if 0 < np.min(P[t][P[t] > 0]) < TINY]
    pick = np.linspace(0, len(deep) - 1, count).astype(int)
    return [deep[i] for i in pick]


def _fields(dd, ctx, mid, n, targets, mask=None):
    mask = mask or (dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT)
    nf = bin(mask).count("1")
    out = torch.empty((nf, len(targets), n), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, mask, dd.DD_PREC_FP32, out)
    dd.dd_sync(ctx)
    return out.cpu().numpy()


def test_log_poisson_and_fields(maze):
    dd, ctx, mesh, P = maze
    n = mesh.n_v
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    targets = _targets(mesh, P, 8)
    refs = [(kl_field_fast(P, P[t]), tv_field(P, P[t]), kl_reverse_field(P, P[t])) for t in targets]
    # the contrast: the solver's FP32 kernel with log P[t,b] evaluated at FLT_MIN
    old = _fields(dd, ctx, mid, n, targets)
    assert max(field_error(old[0, a], refs[a][0]) for a in range(len(targets))) > 1e-3

    sweeps, change = dd.dd_log_poisson_kernel(ctx, mid, 1e-14, 200000)
    assert change <= 1e-14 and sweeps > 0
    k = P.shape[1]
    LP = np.empty((n, k), np.float32)
    dd.dd_get_log_poisson_kernel(ctx, mid, LP)
    P32 = np.empty((n, k), np.float32)
    dd.dd_get_poisson_kernel(ctx, mid, P32)
    pos = P > 0
    with np.errstate(divide="ignore"):
        L = np.log2(P)
    assert np.array_equal(np.isfinite(LP), pos)
    assert np.max(np.abs(LP[pos] - L[pos]) / np.maximum(1.0, np.abs(L[pos]))) < 2.4e-7
    normal = P >= TINY
    assert np.max(np.abs(P32[normal] - P[normal]) / P[normal]) < 1.2e-7
    assert np.all(P32[~normal] == 0.0)

    for sel in (targets[:1], targets[:2], targets):
        got = _fields(dd, ctx, mid, n, sel)
        for a, t in enumerate(sel):
            r = refs[targets.index(t)]
            for f, lo in ((0, 80.0), (1, None), (2, 50.0)):
                assert field_error(got[f, a], r[f]) <= TOL_FP32, (len(sel), t, f, field_error(got[f, a], r[f]))
                assert got[f, a, t] == 0.0
                inf = ~np.isfinite(r[f])
                if lo is not None and inf.any():
                    assert np.all(got[f, a][inf] >= lo)
    dd.dd_unload_mesh(ctx, mid)


def test_paths_on_the_maze(maze):
    dd, ctx, mesh, P = maze
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    dd.dd_log_poisson_kernel(ctx, mid, 1e-14, 200000)
    targets = _targets(mesh, P, 2)
    interior = np.nonzero(~mesh.boundary_flags())[0]
    rng = SplitMix64(170802845 + 903)
    src = np.array([[int(interior[rng.choice(len(interior))]) for _ in range(16)] for _ in targets], np.int32)
    for a, t in enumerate(targets):
        src[a][src[a] == t] = int(interior[0])
    T, S, mp = len(targets), src.shape[1], 4096
    xy = np.zeros((T * S, mp, 2), np.float32)
    ln = np.zeros(T * S, np.int32)
    st = np.zeros(T * S, np.int32)
    f = np.zeros((2, T, mesh.n_v), np.float32)
    dd.dd_query(ctx, mid, targets, src, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, dd.DD_F_KL, mp, f, xy, ln, st)
    tr = Tracer(mesh.xy, mesh.tri)
    h = mean_edge(mesh)
    for a, t in enumerate(targets):
        kl = kl_field_fast(P, P[t])
        for s in range(S):
            i = a * S + s
            path, status = tr.trace(kl, int(src[a, s]), t, max_pts=mp)
            assert st[i] == status, (t, int(src[a, s]), st[i], status)
            assert hausdorff(xy[i, :ln[i]], path, h / 10) <= 0.5 * h
    dd.dd_unload_mesh(ctx, mid)
