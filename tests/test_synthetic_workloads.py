"""The input recipe: the seeded synthetic workloads have the sizes, seeds and
draw rules the benchmark and the parity tests state for them -- CPU only.

Checks determinism (two builds are identical), the vertex and boundary
counts quoted in the benchmark's workload strings, the k/n ratios within the
paper's range (2.5 % to 33 %, Section V), and the draw rules: targets
interior, sources interior and never the target, the disk's sources inside
r <= 0.95 (up to the snap to the nearest vertex), the batch's and the
server's size ranges.
"""
import numpy as np

from synthetic import workloads
from synthetic.rng import SplitMix64


def _interior(mesh):
    return ~mesh.boundary_flags()


def _same(a, b):
    return (np.array_equal(a.mesh.xy, b.mesh.xy) and np.array_equal(a.mesh.tri, b.mesh.tri)
            and np.array_equal(a.targets, b.targets) and np.array_equal(a.sources, b.sources))


def test_disk_recipe():
    a, b = workloads.disk(), workloads.disk()
    assert _same(a, b)
    m = a.mesh
    assert (m.n_v, int(m.boundary_flags().sum())) == (2049, 128)
    t = int(a.targets[0])
    assert np.argmin(np.hypot(m.xy[:, 0] - 0.3, m.xy[:, 1] - 0.2)) == t
    src = a.sources[0]
    assert len(src) == 32 and np.all(src != t) and np.all(_interior(m)[src])
    r = np.hypot(m.xy[src, 0], m.xy[src, 1])
    h = 1.0 / 16
    assert np.all(r <= 0.95 + h)


def test_grid140_recipe():
    a = workloads.grid140()
    b = workloads.grid140()
    assert _same(a, b)
    m = a.mesh
    k = int(m.boundary_flags().sum())
    assert (m.n_v, k) == (18174, 1028)
    assert a.targets.shape == (64,) and a.sources.shape == (64, 256)
    inner = _interior(m)
    assert np.all(inner[a.targets]) and np.all(inner[a.sources])
    assert np.all(a.sources != a.targets[:, None])
    assert 0.025 <= k / m.n_v <= 0.33
    assert a.meta["N"] == 140 and len(a.meta["blocks"]) == 8


def test_grid450_recipe():
    a = workloads.grid450(T=16)
    m = a.mesh
    k = int(m.boundary_flags().sum())
    assert (m.n_v, k) == (192360, 3936)
    assert 0.02 <= k / m.n_v <= 0.33
    assert np.all(_interior(m)[a.targets])
    # the first draws do not depend on how many targets are asked for
    assert np.array_equal(workloads.grid450(T=4).targets, a.targets[:4])


def test_batch64_and_serving_ranges():
    doms = workloads.batch64(n_domains=8)
    for d in doms:
        assert 4000 <= d.mesh.n_v <= 110000
        assert 16 <= len(d.targets) <= 256 and d.sources.shape == (len(d.targets), 64)
        assert len(d.meta["blocks"]) <= 16
    again = workloads.batch64(n_domains=8)
    assert all(_same(x, y) for x, y in zip(doms, again))
    sd = workloads.serving_domains(n_domains=2)
    q = workloads.serving_queries(sd, rate_qps=200.0, duration_s=1.0)
    assert 100 <= len(q) <= 300                               # Poisson(200)
    times = [x[0] for x in q]
    assert times == sorted(times) and times[-1] < 1.0
    for _, d, t, src in q:
        inner = _interior(sd[d].mesh)
        assert inner[t] and 1 <= len(src) <= 1024 and np.all(src != t) and np.all(inner[src])


def test_seeds_follow_the_base():
    assert workloads.BASE_SEED == 170802845
    r1, r2 = SplitMix64(workloads.BASE_SEED + 1), SplitMix64(workloads.BASE_SEED + 1)
    assert [r1.next_u64() for _ in range(4)] == [r2.next_u64() for _ in range(4)]
    assert SplitMix64(workloads.BASE_SEED).next_u64() != SplitMix64(workloads.BASE_SEED + 1).next_u64()
