"""Pins for the oracle's triangle-walking tracer (Section IV) -- CPU only.

Pinned by: the hyperbolic geodesics of the unit disk (Appendix 2.2: the
path between q and t is the image under the inverse Moebius map of the radial
segment), the Equivalence Theorem A6 (KL paths agree with paths of the
Dirichlet Green's function on a simply-connected domain), radial lines for a
centred target (Theorem A5), and hand-built fields that force each status.
The paper's CPU scheme (Table I: divergences evaluated only at the vertices
the path needs) traces the same paths as the full field, evaluating a small
share of the vertices.
"""
import math

import numpy as np
import pytest

from oracle.divergence import kl_field_fast, tv_field
from oracle.greens import dirichlet_green_column
from oracle.hausdorff import hausdorff
from oracle.poisson import PoissonOracle
from oracle.trace import OK, STEP_LIMIT, STUCK_LOCAL_MIN, TRUNCATED, PathOnlyField, Tracer
from synthetic import workloads
from synthetic.meshes import disk_rings, grid_obstacles


def mean_edge(mesh):
    E = set()
    for t in mesh.tri:
        for e in range(3):
            a, b = int(t[e]), int(t[(e + 1) % 3])
            E.add((min(a, b), max(a, b)))
    return float(np.mean([np.hypot(*(mesh.xy[a] - mesh.xy[b])) for a, b in E]))


def geodesic(q, t, n=400):
    q = complex(*q)
    t = complex(*t)
    cq = (q - t) / (1 - np.conj(t) * q)
    u = cq * (1 - np.linspace(0, 1, n))
    z = (u + t) / (1 + np.conj(t) * u)
    return np.stack([z.real, z.imag], 1)


@pytest.fixture(scope="module")
def disk_setup():
    wl = workloads.disk()
    m = wl.mesh
    po = PoissonOracle(m.xy, m.tri, m.loops)
    P = po.full()
    t = int(wl.targets[0])
    return wl, po, P, t, Tracer(m.xy, m.tri), mean_edge(m)


def test_disk_paths_are_hyperbolic_geodesics(disk_setup):
    wl, po, P, t, tr, h = disk_setup
    kl = kl_field_fast(P, P[t])
    tv = tv_field(P, P[t])
    for q in wl.sources[0]:
        for f in (kl, tv):
            path, st = tr.trace(f, int(q), t)
            assert st == OK
            assert np.allclose(path[0], wl.mesh.xy[q]) and np.allclose(path[-1], wl.mesh.xy[t])
            assert hausdorff(path, geodesic(wl.mesh.xy[q], wl.mesh.xy[t]), h / 20) <= 0.5 * h


def test_path_only_scheme_traces_the_same_paths(disk_setup):
    wl, po, P, t, tr, h = disk_setup
    for kind, full in (("kl", kl_field_fast(P, P[t])), ("tv", tv_field(P, P[t]))):
        for q in wl.sources[0][:8]:
            lazy = PathOnlyField(P, t, kind)
            p1, s1 = tr.trace(full, int(q), t)
            p2, s2 = tr.trace(lazy, int(q), t)
            assert s1 == s2 == OK
            assert p1.shape == p2.shape and np.allclose(p1, p2, rtol=0, atol=1e-12)
            ids = np.fromiter(lazy.cache.keys(), dtype=np.int64)
            vals = np.fromiter(lazy.cache.values(), dtype=np.float64)
            assert np.allclose(vals, full[ids], rtol=1e-12, atol=1e-14)
            assert 0 < lazy.evaluated < wl.mesh.n_v // 4


def test_equivalence_with_green_paths(disk_setup):
    wl, po, P, t, tr, h = disk_setup
    kl = kl_field_fast(P, P[t])
    D = dirichlet_green_column(po, t)
    for q in wl.sources[0]:
        p1, s1 = tr.trace(kl, int(q), t)
        p2, s2 = tr.trace(D, int(q), t)
        assert s1 == OK and s2 == OK
        assert hausdorff(p1, p2, h / 20) <= h


def test_path_descends_and_centre_target_is_radial():
    m = disk_rings(16, 128)
    po = PoissonOracle(m.xy, m.tri, m.loops)
    P = po.full()
    t = 0                                                  # the centre vertex
    kl = kl_field_fast(P, P[t])
    tr = Tracer(m.xy, m.tri)
    h = mean_edge(m)
    for q in (200, 777, 1500):
        path, st = tr.trace(kl, q, t)
        assert st == OK
        # radial: every point within a fraction of an edge of the segment q -> 0
        d = np.abs(path[:, 0] * m.xy[q, 1] - path[:, 1] * m.xy[q, 0]) / np.hypot(*m.xy[q])
        assert d.max() < 0.25 * h


def test_status_codes():
    m = grid_obstacles(8, [])
    tr = Tracer(m.xy, m.tri)
    ids = m.meta["ids"]
    # bowl centred at vertex (2,2) plus a deeper one at the target (6,6):
    # a source near (2,2) gets stuck
    X, Y = m.xy[:, 0], m.xy[:, 1]
    f = np.minimum((X - 0.25) ** 2 + (Y - 0.25) ** 2 + 0.01, (X - 0.75) ** 2 + (Y - 0.75) ** 2)
    path, st = tr.trace(f, int(ids[1, 2]), int(ids[6, 6]))
    assert st == STUCK_LOCAL_MIN
    g = (X - 0.75) ** 2 + (Y - 0.75) ** 2
    path, st = tr.trace(g, int(ids[1, 1]), int(ids[6, 6]))
    assert st == OK
    assert np.all(np.diff([_interp(m, tr, g, p) for p in path]) <= 1e-12)
    path, st = tr.trace(g, int(ids[1, 1]), int(ids[6, 6]), max_pts=3)
    assert st == TRUNCATED and len(path) == 3
    path, st = tr.trace(g, int(ids[1, 1]), int(ids[6, 6]), max_steps=2)
    assert st == STEP_LIMIT


def _interp(m, tr, f, p):
    # value of the piecewise-linear field at point p (brute force over triangles)
    for ti, t in enumerate(m.tri):
        a, b, c = m.xy[t[0]], m.xy[t[1]], m.xy[t[2]]
        M = np.array([[b[0] - a[0], c[0] - a[0]], [b[1] - a[1], c[1] - a[1]]])
        l1, l2 = np.linalg.solve(M, np.asarray(p) - a)
        if l1 >= -1e-9 and l2 >= -1e-9 and l1 + l2 <= 1 + 1e-9:
            return (1 - l1 - l2) * f[t[0]] + l1 * f[t[1]] + l2 * f[t[2]]
    raise AssertionError("point outside mesh")
