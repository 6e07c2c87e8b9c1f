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
