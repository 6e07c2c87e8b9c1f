"""GPU parity of the other f-divergence fields (Section VI) against the FP64
oracle, through the C ABI (dd_divergence).

Tolerance as for KL/TV: |g - r| / max(|r|, 1e-2) <= 1e-5 where the oracle is
finite, d(t,t) = 0 exactly; where the oracle is +inf (boundary rows meeting
P[x,b] = 0 < P[t,b]) the result is >= 1e30 (chi2, p > 1, alpha > 1) or >= 50
(reverse KL, log argument taken at FLT_MIN).
"""
import math

import numpy as np
import pytest

from oracle import fdiv
from oracle.poisson import PoissonOracle
from synthetic import workloads
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = {
    "disk": lambda: workloads.disk(),
    "grid37": lambda: workloads.small_grid(37, 3, T=6, S=2, seed=777),
    "grid140": lambda: workloads.grid140(T=3, S=2),
}
_cache = {}


def case(name):
    if name not in _cache:
        wl = CASES[name]()
        po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
        _cache[name] = (wl, po, po.full())
    return _cache[name]


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    yield dd, ctx
    dd.dd_destroy(ctx)


FAMILIES = [("chi2", "DD_DIV_CHI2", 0.0), ("hellinger", "DD_DIV_HELLINGER", 0.0), ("power", "DD_DIV_POWER", 1.0),
            ("power", "DD_DIV_POWER", 2.5), ("alpha", "DD_DIV_ALPHA", 0.5), ("alpha", "DD_DIV_ALPHA", -0.7),
            ("alpha", "DD_DIV_ALPHA", 3.0), ("alpha", "DD_DIV_ALPHA", 0.8), ("alpha", "DD_DIV_ALPHA", -5.0),
            ("alpha", "DD_DIV_ALPHA", 0.95), ("alpha", "DD_DIV_ALPHA", 4.5), ("kl_reverse", "DD_DIV_KL_REVERSE", 0.0)]
# alpha: 0.5, -0.7, 3.0, 0.8 and -5.0 take the two-pass form (first pass with
# hardware logarithms and exp2), 0.95 and 4.5 the exact form throughout


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("fam,const,prm", FAMILIES)
def test_fdiv_on_oracle_kernel(env, name, fam, const, prm):
    dd, ctx = env
    wl, po, P = case(name)
    targets = [int(t) for t in wl.targets[:3]]
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    out = torch.empty((len(targets), wl.mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_divergence(ctx, mid, targets, getattr(dd, const), prm, out)
    dd.dd_sync(ctx)
    got = out.cpu().numpy()
    for a, t in enumerate(targets):
        ref = fdiv.field(P, P[t], fam, prm)
        assert field_error(got[a], ref) <= TOL_FP32, (fam, prm, field_error(got[a], ref))
        assert got[a, t] == 0.0
        inf = ~np.isfinite(ref)
        if inf.any():
            lo = 50.0 if fam == "kl_reverse" else 1e30
            assert np.all(got[a][inf] >= lo)
    dd.dd_unload_mesh(ctx, mid)


def test_fdiv_host_buffers_and_errors(env):
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    t = [int(wl.targets[0])]
    host = np.empty((1, wl.mesh.n_v), dtype=np.float32)
    dd.dd_divergence(ctx, mid, t, dd.DD_DIV_HELLINGER, 0.0, host)
    dev = torch.empty((1, wl.mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_divergence(ctx, mid, t, dd.DD_DIV_HELLINGER, 0.0, dev)
    dd.dd_sync(ctx)
    assert np.array_equal(host, dev.cpu().numpy())
    for fam, prm in ((dd.DD_DIV_POWER, 0.5), (dd.DD_DIV_ALPHA, 1.0), (dd.DD_DIV_ALPHA, -1.0), (99, 0.0)):
        with pytest.raises(dd.DDError):
            dd.dd_divergence(ctx, mid, t, fam, prm, host)
    dd.dd_unload_mesh(ctx, mid)


def test_fdiv_end_to_end_grid140(env):
    """Device PCG, then the divergence fields, against the oracle."""
    dd, ctx = env
    wl, po, P = case("grid140")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    t = [int(wl.targets[1])]
    host = np.empty((1, wl.mesh.n_v), dtype=np.float32)
    for fam, const, prm in (("chi2", dd.DD_DIV_CHI2, 0.0), ("alpha", dd.DD_DIV_ALPHA, 0.5)):
        dd.dd_divergence(ctx, mid, t, const, prm, host)
        assert field_error(host[0], fdiv.field(P, P[t[0]], fam, prm)) <= TOL_FP32
    dd.dd_unload_mesh(ctx, mid)
