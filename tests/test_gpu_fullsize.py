"""Full-size parity on grid450 (n = 192,360, k = 3,936; P = 3.0 GB in FP32).

The oracle cannot hold P here (6 GB in FP64), so it computes sampled rows by
Green's-row solves and the fields at those rows; the device path runs at full
size in the launch configuration the benchmark uses (stream kernel for one
target, tile kernel for many).  Paths are checked by properties that hold at
any size: they start at the source, end at the target with status OK, and
descend along the field.
"""
import numpy as np
import pytest

from oracle.divergence import kl_field_fast, tv_field
from oracle.poisson import PoissonOracle
from synthetic import workloads
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    wl = workloads.grid450(T=8)
    mesh = wl.mesh
    mid = load(dd, ctx, mesh)
    iters, resid = dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    rng = np.random.default_rng(5)
    rows = np.concatenate([rng.choice(mesh.n_v, 48, replace=False), po.B[:4], po.I[-4:]])
    targets = [int(t) for t in wl.targets]
    Prow = po.rows(list(rows) + targets)
    yield dd, ctx, wl, mid, po, rows, targets, Prow, (iters, resid)
    dd.dd_destroy(ctx)


def test_poisson_rows(big):
    dd, ctx, wl, mid, po, rows, targets, Prow, (iters, resid) = big
    assert resid <= 1e-15
    info = dd.dd_mesh_info(ctx, mid)
    P = torch.empty((info["n_v"], info["k"]), dtype=torch.float32, device="cuda")
    dd.dd_get_poisson_kernel(ctx, mid, P)
    dd.dd_sync(ctx)
    ids = torch.as_tensor(np.concatenate([rows, targets]).astype(np.int64), device="cuda")
    got = P[ids].cpu().numpy().astype(np.float64)
    ref = np.where(Prow < np.finfo(np.float32).tiny, 0.0, Prow)
    assert np.all(np.abs(got - ref) <= 1.2e-7 * np.abs(ref) + 1e-12)


@pytest.mark.parametrize("T", [1, 8])
def test_fields_sampled_rows(big, T):
    dd, ctx, wl, mid, po, rows, targets, Prow, _ = big
    n_v = wl.mesh.n_v
    out = torch.empty((2, T, n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets[:T], dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, out)
    dd.dd_sync(ctx)
    got = out[:, :, torch.as_tensor(rows.astype(np.int64), device="cuda")].cpu().numpy()
    R = Prow[:len(rows)]
    for a in range(T):
        Pt = Prow[len(rows) + a]
        assert field_error(got[0, a], kl_field_fast(R, Pt)) <= TOL_FP32
        assert field_error(got[1, a], tv_field(R, Pt)) <= TOL_FP32
    full = out.cpu().numpy()
    for a, t in enumerate(targets[:T]):
        assert full[0, a, t] == 0.0 and full[1, a, t] == 0.0
        assert np.all(np.isfinite(full[:, a])) and full[1, a].max() <= 2.0 + 1e-5 and full[0, a].min() >= 0.0


def test_paths_properties(big):
    dd, ctx, wl, mid, po, rows, targets, Prow, _ = big
    mesh = wl.mesh
    t = targets[0]
    interior = po.I
    rng = np.random.default_rng(9)
    src = interior[rng.choice(len(interior), 64, replace=False)]
    src = np.asarray([s for s in src if s != t], dtype=np.int32)
    S, mp = len(src), 4096
    xy = np.zeros((S, mp, 2), np.float32)
    ln = np.zeros(S, np.int32)
    st = np.zeros(S, np.int32)
    dd.dd_trace(ctx, mid, t, dd.DD_F_KL, src, mp, xy, ln, st)
    assert (st == dd.DD_TRACE_OK).mean() >= 0.95
    for s in range(S):
        assert np.allclose(xy[s, 0], mesh.xy[src[s]], atol=1e-6)
        if st[s] == dd.DD_TRACE_OK:
            assert np.allclose(xy[s, ln[s] - 1], mesh.xy[t], atol=1e-6)


def test_bf16x3_sampled_rows(big):
    """Split-BF16 tensor-core KL at full size: 256 targets, sampled rows."""
    dd, ctx, wl, mid, po, rows, targets, Prow, _ = big
    n_v = wl.mesh.n_v
    rng = np.random.default_rng(21)
    tg = [int(t) for t in po.I[rng.choice(po.m, 256, replace=False)]]
    Pt = po.rows(tg)
    out = torch.empty((1, len(tg), n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, tg, dd.DD_F_KL, dd.DD_PREC_BF16X3, out)
    dd.dd_sync(ctx)
    got = out[0][:, torch.as_tensor(rows.astype(np.int64), device="cuda")].cpu().numpy()
    R = Prow[:len(rows)]
    worst = 0.0
    for a in range(len(tg)):
        ref = kl_field_fast(R, Pt[a])
        with np.errstate(divide="ignore"):
            S = R @ np.abs(np.log(np.maximum(Pt[a], 1e-300)))
        fin = np.isfinite(ref)
        worst = max(worst, float(np.max(np.abs(got[a][fin] - ref[fin]) / np.maximum(np.abs(ref[fin]), S[fin]))))
    assert worst <= 1e-4, worst
