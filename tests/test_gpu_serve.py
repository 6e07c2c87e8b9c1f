"""Query server (continuous batching): every query's paths are the same served
in a mixed batch as computed alone, within the path tolerance (identical
status, Hausdorff <= half a mean edge length); oversized queries are refused."""
import numpy as np
import pytest

from oracle.hausdorff import hausdorff
from synthetic import workloads
from synthetic.rng import SplitMix64
from tests._gpu import ctx_and_lib, load, mean_edge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_served_equals_alone():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    sv = None
    try:
        wls = [workloads.disk(n_rings=10, n_seg=64, n_sources=2),
               workloads.small_grid(40, 3, T=2, S=2, seed=11),
               workloads.small_grid(64, 5, T=2, S=2, seed=12)]
        mids = []
        for wl in wls:
            mid = load(dd, ctx, wl.mesh)
            dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
            mids.append(mid)
        dd.dd_sync(ctx)
        mp = 2048
        sv = dd.dd_server_create(ctx, 1 << 30, n_slots=3, max_batch=8, max_pts=mp)
        rng = SplitMix64(2024)
        queries = []
        for qid in range(48):
            d = rng.choice(len(wls))
            m = wls[d].mesh
            interior = np.nonzero(~m.boundary_flags())[0]
            t = int(interior[rng.choice(len(interior))])
            S = 1 + rng.choice(24)
            src = [int(interior[rng.choice(len(interior))]) for _ in range(S)]
            assert dd.dd_server_submit(sv, qid, mids[d], t, src) == dd.DD_OK
            queries.append((qid, d, t, np.asarray(src, np.int32)))
        assert dd.dd_server_submit(sv, 999, mids[0], int(queries[0][2]), np.zeros(200000, np.int32)) == dd.DD_EBUDGET
        dd.dd_server_wait_idle(sv, 120.0)
        ids, sts, lat = dd.dd_server_poll(sv)
        assert sorted(ids.tolist()) == list(range(48)) and np.all(sts == 0) and np.all(lat > 0)
        for qid, d, t, src in queries:
            S = len(src)
            xy, ln, st = dd.dd_server_take(sv, qid, S, mp)
            axy = np.zeros((S, mp, 2), np.float32)
            aln = np.zeros(S, np.int32)
            ast = np.zeros(S, np.int32)
            dd.dd_trace(ctx, mids[d], t, dd.DD_F_KL, src, mp, axy, aln, ast)
            h = mean_edge(wls[d].mesh)
            for s in range(S):
                assert st[s] == ast[s]
                assert hausdorff(xy[s, :ln[s]], axy[s, :aln[s]], h / 10) <= 0.5 * h
    finally:
        if sv is not None:
            dd.dd_server_destroy(sv)
        dd.dd_destroy(ctx)


def test_arrivals_join_while_batches_run():
    """Queries submitted while earlier batches are on the device (some of the
    first wave done, others not yet) are served, and each result equals the
    query computed alone."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import time
    dd, ctx = ctx_and_lib()
    sv = None
    try:
        wl = workloads.grid140(T=1, S=1)
        mid = load(dd, ctx, wl.mesh)
        dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
        dd.dd_sync(ctx)
        mp = 2048
        sv = dd.dd_server_create(ctx, 2 << 30, n_slots=2, max_batch=4, max_pts=mp)
        interior = np.nonzero(~wl.mesh.boundary_flags())[0]
        rng = SplitMix64(4096)

        def draw(qid):
            t = int(interior[rng.choice(len(interior))])
            src = np.asarray([int(interior[rng.choice(len(interior))]) for _ in range(1 + rng.choice(32))], np.int32)
            return qid, t, src

        wave1 = [draw(q) for q in range(64)]
        for qid, t, src in wave1:
            assert dd.dd_server_submit(sv, qid, mid, t, src) == dd.DD_OK
        done = {}
        t0 = time.perf_counter()
        while not done and time.perf_counter() - t0 < 60.0:
            ids, sts, _ = dd.dd_server_poll(sv)
            done.update(zip(ids.tolist(), sts.tolist()))
        assert 0 < len(done) < len(wave1)          # the first wave is partly served, partly in flight
        wave2 = [draw(q) for q in range(100, 124)]
        for qid, t, src in wave2:
            assert dd.dd_server_submit(sv, qid, mid, t, src) == dd.DD_OK
        dd.dd_server_wait_idle(sv, 120.0)
        ids, sts, _ = dd.dd_server_poll(sv)
        done.update(zip(ids.tolist(), sts.tolist()))
        assert sorted(done) == sorted(q for q, _, _ in wave1 + wave2) and all(v == 0 for v in done.values())
        h = mean_edge(wl.mesh)
        for qid, t, src in wave1 + wave2:
            S = len(src)
            xy, ln, st = dd.dd_server_take(sv, qid, S, mp)
            axy = np.zeros((S, mp, 2), np.float32)
            aln = np.zeros(S, np.int32)
            ast = np.zeros(S, np.int32)
            dd.dd_trace(ctx, mid, t, dd.DD_F_KL, src, mp, axy, aln, ast)
            for s in range(S):
                assert st[s] == ast[s]
                assert hausdorff(xy[s, :ln[s]], axy[s, :aln[s]], h / 10) <= 0.5 * h
    finally:
        if sv is not None:
            dd.dd_server_destroy(sv)
        dd.dd_destroy(ctx)
