"""Batched multi-domain query (one persistent field launch with autotuned tile
shapes, one tracer launch) against the single-domain path and the oracle;
the staged and the pipelined persistent launches give the same fields."""
import numpy as np
import pytest

from oracle.divergence import kl_field_fast, tv_field
from oracle.hausdorff import hausdorff
from oracle.poisson import PoissonOracle
from synthetic import workloads
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load, mean_edge

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_batch_matches_single_and_oracle(monkeypatch):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    try:
        wls = [workloads.disk(n_rings=8, n_seg=64, n_sources=4),
               workloads.small_grid(24, 2, T=5, S=4),
               workloads.small_grid(37, 3, T=70, S=4, seed=777),
               workloads.small_grid(50, 4, T=17, S=4, seed=901),
               workloads.small_grid(30, 0, T=33, S=4, seed=55)]
        S, mp = 4, 2048
        mids, Ts, tg, sr, Ps = [], [], [], [], []
        for wl in wls:
            m = wl.mesh
            mid = load(dd, ctx, m)
            dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
            po = PoissonOracle(m.xy, m.tri, m.loops)
            P = po.full()
            T = len(wl.targets)
            mids.append(mid)
            Ts.append(T)
            tg.append(np.asarray(wl.targets, np.int32))
            s = wl.sources[:, :S] if wl.sources.shape[1] >= S else np.resize(wl.sources, (T, S))
            sr.append(np.asarray(s, np.int32))
            Ps.append(P)
        n_f = sum(2 * T * wl.mesh.n_v for T, wl in zip(Ts, wls))
        nT = sum(Ts)
        out = torch.full((n_f,), float("nan"), dtype=torch.float32, device="cuda")
        xy = torch.zeros((nT * S, mp, 2), dtype=torch.float32, device="cuda")
        ln = torch.zeros(nT * S, dtype=torch.int32, device="cuda")
        st = torch.zeros(nT * S, dtype=torch.int32, device="cuda")
        runs = []
        for pipe in ("0", "1"):
            monkeypatch.setenv("DD_BATCH_PIPE", pipe)
            out.fill_(float("nan"))
            dd.dd_query_batch(ctx, mids, Ts, np.concatenate(tg), np.concatenate([x.reshape(-1) for x in sr]), S,
                              3, 1, mp, out, xy, ln, st)
            dd.dd_sync(ctx)
            runs.append((out.cpu().numpy(), xy.cpu().numpy(), ln.cpu().numpy(), st.cpu().numpy()))
        monkeypatch.delenv("DD_BATCH_PIPE")
        # the staged and the pipelined launch: the same sums in the same order
        assert np.array_equal(runs[0][0], runs[1][0])
        assert np.array_equal(runs[0][2], runs[1][2]) and np.array_equal(runs[0][3], runs[1][3])
        fo, to = 0, 0
        outn, xyn, lnn, stn = runs[1]
        for i, wl in enumerate(wls):
            n_v, T, P = wl.mesh.n_v, Ts[i], Ps[i]
            blk = outn[fo:fo + 2 * T * n_v].reshape(2, T, n_v)
            single = torch.empty((2, T, n_v), dtype=torch.float32, device="cuda")
            sxy = torch.zeros((T * S, mp, 2), dtype=torch.float32, device="cuda")
            sln = torch.zeros(T * S, dtype=torch.int32, device="cuda")
            sst = torch.zeros(T * S, dtype=torch.int32, device="cuda")
            dd.dd_query(ctx, mids[i], tg[i], sr[i], 3, 0, 1, mp, single, sxy, sln, sst)
            dd.dd_sync(ctx)
            sn = single.cpu().numpy()
            h = mean_edge(wl.mesh)
            for a, t in enumerate(tg[i]):
                assert field_error(blk[0, a], kl_field_fast(P, P[t])) <= TOL_FP32
                assert field_error(blk[1, a], tv_field(P, P[t])) <= TOL_FP32
                assert blk[0, a, t] == 0.0 and blk[1, a, t] == 0.0
                assert np.abs(blk[:, a] - sn[:, a]).max() <= 1e-5 * max(1.0, np.abs(sn[:, a]).max())
            sstn, slnn, sxyn = sst.cpu().numpy(), sln.cpu().numpy(), sxy.cpu().numpy()
            for q in range(T * S):
                g = to * S + q
                assert stn[g] == sstn[q]
                assert hausdorff(xyn[g, :lnn[g]], sxyn[q, :slnn[q]], h / 10) <= 0.5 * h
            fo += 2 * T * n_v
            to += T
        assert "k_pad" in dd.dd_tuning_table()
    finally:
        dd.dd_destroy(ctx)
