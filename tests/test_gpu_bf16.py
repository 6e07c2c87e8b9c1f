"""Split-BF16 tensor-core KL (DD_PREC_BF16X3) against the FP64 oracle.

The cross term C[x,t] = sum_b P[x,b] log P[t,b] runs as a tcgen05 GEMM of BF16
hi/lo operands with FP32 accumulation; its error scales with
S_x = sum_b P[x,b] |log P[t,b]|, so the bound is |g - r| <= 1e-4 max(|r|, S_x).
TV requested with this precision is the FP32 path and must match it exactly.
"""
import numpy as np
import pytest

from oracle.divergence import kl_field_fast
from oracle.poisson import PoissonOracle
from synthetic import workloads
from tests._gpu import ctx_and_lib, load

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TOL_BF16 = 1e-4


def scale(P, Pt):
    with np.errstate(divide="ignore"):
        L = np.abs(np.log(np.maximum(Pt, 1e-300)))
    return P @ L


def bf16_error(got, ref, S):
    fin = np.isfinite(ref)
    return float(np.max(np.abs(got[fin] - ref[fin]) / np.maximum(np.maximum(np.abs(ref[fin]), S[fin]), 1e-30)))


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    yield dd, ctx
    dd.dd_destroy(ctx)


@pytest.mark.parametrize("name,T", [("disk", 1), ("grid37", 70), ("grid37", 300), ("grid140", 64)])
def test_bf16x3_kl(env, name, T):
    dd, ctx = env
    wl = {"disk": lambda: workloads.disk(), "grid37": lambda: workloads.small_grid(37, 3, T=4, S=1, seed=777),
          "grid140": lambda: workloads.grid140(T=64, S=1)}[name]()
    mesh = wl.mesh
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    P = po.full()
    targets = [int(po.I[(i * 7919 + 13) % po.m]) for i in range(T)]
    mid = load(dd, ctx, mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    n_v = mesh.n_v
    got = torch.empty((2, T, n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_BF16X3, got)
    ref32 = torch.empty((1, T, n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_TV, dd.DD_PREC_FP32, ref32)
    dd.dd_sync(ctx)
    g = got.cpu().numpy()
    assert np.array_equal(g[1], ref32.cpu().numpy()[0])
    worst = 0.0
    for a, t in enumerate(targets):
        r = kl_field_fast(P, P[t])
        S = scale(P, P[t])
        e = bf16_error(g[0, a], r, S)
        worst = max(worst, e)
        assert np.all(np.isfinite(g[0, a]))
    assert worst <= TOL_BF16, worst
    dd.dd_unload_mesh(ctx, mid)
