"""The query check of __graft_entry__.smoke() on the CPU, with a stand-in for
the library that writes the oracle's fields (and, for a planted mistake,
wrong ones), so that the check's own indexing and thresholds are tested
without a GPU."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import __graft_entry__ as entry  # noqa: E402
from oracle.divergence import kl_field_fast, tv_field  # noqa: E402
from oracle.poisson import PoissonOracle  # noqa: E402
from synthetic import workloads  # noqa: E402


class _FakeDD:
    DD_F_KL, DD_F_TV, DD_PREC_FP32 = 1, 2, 0

    def __init__(self, P, scale=1.0):
        self.P, self.scale, self.calls = P, scale, []

    def dd_query(self, ctx, mid, targets, sources, f_mask, prec, trace_f, max_pts, f, xy, ln, st):
        self.calls.append((list(targets), np.asarray(sources).shape, f_mask, prec, trace_f, max_pts))
        for a, t in enumerate(targets):
            kl = kl_field_fast(self.P, self.P[t])
            f[0, a] = torch.from_numpy(np.where(np.isfinite(kl), kl * self.scale, 87.0).astype(np.float32))
            f[1, a] = torch.from_numpy(tv_field(self.P, self.P[t]).astype(np.float32))
        ln.fill_(2)
        st.zero_()

    def dd_sync(self, ctx):
        pass


def _case():
    wl = workloads.disk(n_rings=8, n_seg=64, n_sources=8)
    po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
    P = po.full()
    t = int(wl.targets[0])
    src = np.asarray(wl.sources[0], dtype=np.int32)
    targets = entry._query_targets(po.I, t, src)
    assert all(bool(~wl.mesh.boundary_flags()[v]) for v in targets)
    return P, targets, np.tile(src, (4, 1))


def test_query_check_accepts_the_oracle_and_rejects_a_planted_error():
    P, targets, sources = _case()
    assert len(set(targets)) == 4 and not np.any(sources == np.asarray(targets)[:, None])
    fake = _FakeDD(P)
    err = entry._query_check(fake, None, 0, P, targets, sources, "cpu")
    assert err < 1e-6
    assert fake.calls == [(targets, (4, 8), 3, 0, 1, 256)]
    with pytest.raises(AssertionError):
        entry._query_check(_FakeDD(P, scale=1.0 + 1e-4), None, 0, P, targets, sources, "cpu")


def _fake_library(P, mesh):
    from oracle.trace import Tracer
    import types
    m = types.ModuleType("paper_1708_02845_gb300.dd")
    m.DD_F_KL, m.DD_F_TV, m.DD_PREC_FP32, m.DD_TRACE_OK = 1, 2, 0, 0
    m.dd_create = lambda dev, stream=0: object()
    m.dd_destroy = lambda ctx: None
    m.dd_sync = lambda ctx: None
    m.dd_load_mesh = lambda ctx, xy, tri, idx, off: 0
    m.dd_poisson_kernel = lambda ctx, mid, rtol, it: (30, 1e-16)
    tracer = Tracer(mesh.xy, mesh.tri)

    def fields(targets, out):
        for a, t in enumerate(targets):
            kl = kl_field_fast(P, P[t])
            out[0, a] = torch.from_numpy(np.where(np.isfinite(kl), kl, 87.0).astype(np.float32))
            out[1, a] = torch.from_numpy(tv_field(P, P[t]).astype(np.float32))

    def paths(t, sources, max_pts, xy, ln, st, base=0):
        kl = kl_field_fast(P, P[t])
        for s, q in enumerate(sources):
            path, status = tracer.trace(kl, int(q), int(t), max_pts=max_pts)
            xy[base + s, :len(path)] = torch.from_numpy(np.asarray(path, dtype=np.float32))
            ln[base + s] = len(path)
            st[base + s] = status

    m.dd_distance = lambda ctx, mid, targets, f, prec, out: fields(targets, out)
    m.dd_trace = lambda ctx, mid, t, f, sources, max_pts, xy, ln, st: paths(t, sources, max_pts, xy, ln, st)

    def query(ctx, mid, targets, sources, f, prec, tf, max_pts, out, xy, ln, st):
        fields(targets, out)
        S = np.asarray(sources).shape[1]
        for a, t in enumerate(targets):
            paths(t, np.asarray(sources)[a], max_pts, xy, ln, st, base=a * S)

    m.dd_query = query
    return m


def test_smoke_runs_end_to_end_with_a_stand_in_library(monkeypatch, capsys):
    """The whole of smoke() on the CPU: the stand-in returns the oracle's own
    fields and paths, so every check in smoke() must pass and it must report
    both the one-target and the four-target errors."""
    import paper_1708_02845_gb300 as pkg
    wl = workloads.disk(n_rings=8, n_seg=64, n_sources=8)
    po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
    fake = _fake_library(po.full(), wl.mesh)
    monkeypatch.setitem(sys.modules, "paper_1708_02845_gb300.dd", fake)
    monkeypatch.setattr(pkg, "dd", fake, raising=False)
    real_empty = torch.empty
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **kw: real_empty(*a, **kw))
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: type("S", (), {"cuda_stream": 0})())
    entry.smoke()
    out = capsys.readouterr().out
    assert "smoke ok" in out and "query4=" in out
