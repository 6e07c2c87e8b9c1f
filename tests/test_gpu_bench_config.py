"""Parity at exactly the configurations bench.py times, through the C ABI (GPU).

* grid450 (the headline): one dd_query over the benchmark's first batch --
  1,024 targets, KL+TV on the FP32 path with the autotuned tile shape, 1,024 x
  16 paths on the KL fields, max_pts 4,096.  The oracle cannot hold P here
  (6 GB in FP64), so every one of the 1,024 fields is checked on 128 sampled
  rows (Green's-row solves) at the FP32 tolerance, with exact zeros at the
  targets; every path by the properties that hold at any size (it starts at
  its source and, with status OK, ends at its target).
* grid450 tracer unit: the walk on caller-supplied fields of full size --
  the oracle's Dirichlet Green's functions of four targets (no spurious
  minima by the maximum principle), rounded to FP32 -- against the oracle's
  tracer on the same values, path by path: identical status, Hausdorff within
  half a mean edge.
* grid140 (a side measurement): one dd_query with 64 targets x 256 sources,
  KL+TV FP32, max_pts 1,024; all 64 fields against the oracle's full kernel,
  and a seeded sample of 1,024 paths, 16 of every target, against the
  oracle's tracer on the oracle's FP64 KL fields: identical status,
  Hausdorff within half a mean edge.
"""
import numpy as np
import pytest

from oracle.divergence import kl_field_fast, tv_field
from oracle.greens import dirichlet_green_column
from oracle.hausdorff import hausdorff
from oracle.poisson import PoissonOracle
from oracle.trace import Tracer
from synthetic import workloads
from synthetic.rng import SplitMix64
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load, mean_edge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    yield dd, ctx
    dd.dd_destroy(ctx)


@pytest.fixture(scope="module")
def g450(env):
    dd, ctx = env
    wl = workloads.grid450(T=1024, S=16)
    mid = load(dd, ctx, wl.mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
    po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
    yield wl, mid, po
    dd.dd_unload_mesh(ctx, mid)


def test_grid450_step_all_targets(env, g450):
    dd, ctx = env
    wl, mid, po = g450
    mesh = wl.mesh
    T, S, mp = 1024, 16, 4096
    fields = torch.empty((2, T, mesh.n_v), dtype=torch.float32, device="cuda")
    xy = torch.empty((T * S, mp, 2), dtype=torch.float32, device="cuda")
    ln = torch.empty(T * S, dtype=torch.int32, device="cuda")
    st = torch.empty(T * S, dtype=torch.int32, device="cuda")
    dd.dd_query(ctx, mid, wl.targets, wl.sources, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, dd.DD_F_KL, mp,
                fields, xy, ln, st)
    dd.dd_sync(ctx)
    rng = SplitMix64(170802845 + 901)
    rows = np.array(sorted({int(po.I[rng.choice(po.m)]) for _ in range(128)}), np.int64)
    R = po.rows(list(rows) + [int(t) for t in wl.targets])
    Px, Pt = R[:len(rows)], R[len(rows):]
    got = fields[:, :, torch.as_tensor(rows, device="cuda")].cpu().numpy()
    at_t = fields[:, torch.arange(T, device="cuda"), torch.as_tensor(wl.targets.astype(np.int64), device="cuda")]
    assert bool((at_t == 0).all())
    worst = [0.0, 0.0]
    for a in range(T):
        worst[0] = max(worst[0], field_error(got[0, a], kl_field_fast(Px, Pt[a])))
        worst[1] = max(worst[1], field_error(got[1, a], tv_field(Px, Pt[a])))
    assert worst[0] <= TOL_FP32 and worst[1] <= TOL_FP32, worst
    stn, lnn = st.cpu().numpy(), ln.cpu().numpy()
    assert np.mean(stn == dd.DD_TRACE_OK) >= 0.98
    first = xy[:, 0].cpu().numpy()
    assert np.allclose(first, mesh.xy[wl.sources.reshape(-1)], atol=1e-6)
    last = xy[torch.arange(T * S, device="cuda"), (ln.long() - 1).clamp(min=0)].cpu().numpy()
    ok = stn == dd.DD_TRACE_OK
    assert np.allclose(last[ok], mesh.xy[np.repeat(wl.targets, S)][ok], atol=1e-6)
    assert lnn.max() < mp


def test_grid450_tracer_unit(env, g450):
    dd, ctx = env
    wl, mid, po = g450
    mesh = wl.mesh
    tr = Tracer(mesh.xy, mesh.tri)
    h = mean_edge(mesh)
    targets = [int(t) for t in wl.targets[:4]]
    F = np.stack([dirichlet_green_column(po, t) for t in targets]).astype(np.float32)
    src = np.asarray(wl.sources)[:4, :8]
    T, S, mp = len(targets), src.shape[1], 4096
    xy = np.zeros((T * S, mp, 2), np.float32)
    ln = np.zeros(T * S, np.int32)
    st = np.zeros(T * S, np.int32)
    fd = torch.as_tensor(F, device="cuda")
    dd.dd_trace_fields(ctx, mid, fd, targets, src, mp, xy, ln, st)
    for a, t in enumerate(targets):
        f64 = F[a].astype(np.float64)
        for s in range(S):
            i = a * S + s
            path, status = tr.trace(f64, int(src[a, s]), t, max_pts=mp)
            assert st[i] == status == 0, (t, int(src[a, s]), st[i], status)
            assert hausdorff(xy[i, :ln[i]], path, h / 10) <= 0.5 * h


def test_grid140_step_fields_and_sampled_paths(env):
    dd, ctx = env
    wl = workloads.grid140(T=64, S=256)
    mesh = wl.mesh
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    P = PoissonOracle(mesh.xy, mesh.tri, mesh.loops).full()
    T, S, mp = 64, 256, 1024
    fields = torch.empty((2, T, mesh.n_v), dtype=torch.float32, device="cuda")
    xy = torch.empty((T * S, mp, 2), dtype=torch.float32, device="cuda")
    ln = torch.empty(T * S, dtype=torch.int32, device="cuda")
    st = torch.empty(T * S, dtype=torch.int32, device="cuda")
    dd.dd_query(ctx, mid, wl.targets, wl.sources, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, dd.DD_F_KL, mp,
                fields, xy, ln, st)
    dd.dd_sync(ctx)
    g = fields.cpu().numpy()
    stn, lnn = st.cpu().numpy(), ln.cpu().numpy()
    tr = Tracer(mesh.xy, mesh.tri)
    h = mean_edge(mesh)
    rng = SplitMix64(170802845 + 902)
    for a, t in enumerate(wl.targets):
        t = int(t)
        kl = kl_field_fast(P, P[t])
        assert field_error(g[0, a], kl) <= TOL_FP32
        assert field_error(g[1, a], tv_field(P, P[t])) <= TOL_FP32
        assert g[0, a, t] == 0.0 and g[1, a, t] == 0.0
        picks = set()
        while len(picks) < 16:
            picks.add(rng.choice(S))
        for s in sorted(picks):
            i = a * S + s
            q = int(wl.sources[a, s])
            path, status = tr.trace(kl, q, t, max_pts=mp)
            assert stn[i] == status, (t, q, stn[i], status)
            p = xy[i, :lnn[i]].cpu().numpy()
            assert hausdorff(p, path, h / 10) <= 0.5 * h
    dd.dd_unload_mesh(ctx, mid)
