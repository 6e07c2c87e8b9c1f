"""Pins for the oracle's TV/KL fields (Eq. 34-35) -- CPU only.

Pinned by: the divergence axioms (DV >= 0, DV(t,t) = 0, TV in [0, 2];
Section III), brute force over exact rational Poisson kernels of tiny grids,
and the unit-disk closed forms KL = -log(1 - |C|^2) (Eq. A6) and
TV = (4/pi) asin|C| (Eq. A8), carried to any target by the Moebius map (A10)
and conformal invariance (Theorem A2), converging under refinement.
"""
import math

import numpy as np
import pytest

from oracle.divergence import kl_field, kl_field_fast, tv_field
from oracle.poisson import PoissonOracle
from synthetic import workloads
from synthetic.meshes import disk_rings, grid_obstacles
from tests.test_oracle_poisson import exact_poisson_grid


def test_axioms_on_obstacle_grid():
    wl = workloads.small_grid(32, 3, T=6)
    po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
    P = po.full()
    interior = np.ones(P.shape[0], bool)
    interior[po.B] = False
    for t in wl.targets:
        kl = kl_field_fast(P, P[t])
        tv = tv_field(P, P[t])
        assert kl[t] == 0.0 and tv[t] == 0.0
        assert (kl[interior] > 0).sum() == interior.sum() - 1
        assert (kl[np.isfinite(kl)] >= 0).all()
        assert tv.min() >= 0 and tv.max() <= 2 + 1e-12
        assert np.allclose(kl_field(P[interior][:50], P[t]), kl[interior][:50], rtol=1e-13, atol=1e-15)


def test_tv_symmetric_kl_not():
    m = workloads.small_grid(20, 2).mesh
    P = PoissonOracle(m.xy, m.tri, m.loops).full()
    a, b = 50, 200
    assert tv_field(P, P[a])[b] == pytest.approx(tv_field(P, P[b])[a], rel=1e-13)
    # the field point weights the sum (Eq. 17 with z = x): KL_t(x) = KL(P_x || P_t)
    kl_ab = kl_field_fast(P, P[a])[b]
    nz = P[b] > 0
    assert kl_ab == pytest.approx(float(np.sum(P[b][nz] * np.log(P[b][nz] / P[a][nz]))), rel=1e-13)


@pytest.mark.parametrize("mesh", [grid_obstacles(4, []), grid_obstacles(5, [(2, 2, 1, 1)])])
def test_brute_force_exact_kernel(mesh):
    exact = exact_poisson_grid(mesh)
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    P = po.full()
    n = mesh.n_v
    for t in po.I:
        pt = exact[t]
        for x in range(n):
            px = exact[x]
            tv = float(sum(abs(a - b) for a, b in zip(px, pt)))
            kl = 0.0
            for a, b in zip(px, pt):
                if a > 0:
                    kl += float(a) * (math.log(a.numerator) - math.log(a.denominator)
                                      - math.log(b.numerator) + math.log(b.denominator)) if b > 0 else math.inf
            assert tv_field(P[x:x + 1], P[t])[0] == pytest.approx(tv, abs=1e-14)
            got = kl_field(P[x:x + 1], P[t])[0]
            if math.isinf(kl):
                assert math.isinf(got)
            else:
                assert got == pytest.approx(kl, abs=1e-13)


def _disk_field_errors(R, S):
    m = disk_rings(R, S)
    po = PoissonOracle(m.xy, m.tri, m.loops)
    P = po.full()
    z = m.xy[:, 0] + 1j * m.xy[:, 1]
    t = int(np.argmin(np.abs(z - (0.3 + 0.2j))))
    C = (z - z[t]) / (1 - np.conj(z[t]) * z)            # Eq. (A10)
    kl = kl_field_fast(P, P[t])
    tv = tv_field(P, P[t])
    sel = np.abs(z) <= 0.8
    ekl = np.abs(kl + np.log(1 - np.abs(C) ** 2))[sel].max()         # Eq. (A6)
    etv = np.abs(tv - 4 / math.pi * np.arcsin(np.abs(C)))[sel].max()  # Eq. (A8)
    return ekl, etv


def test_disk_closed_forms_converge():
    k16, t16 = _disk_field_errors(16, 128)
    k32, t32 = _disk_field_errors(32, 256)
    assert k16 < 2e-3 and t16 < 1.2e-3
    assert k32 < k16 / 2.5 and t32 < t16 / 2.5


def test_zero_column_gives_infinite_boundary_kl():
    # a boundary vertex joined to interior vertices only through zero-weight
    # diagonals has an all-zero column, hence KL = +inf at that boundary row
    m = grid_obstacles(6, [])
    po = PoissonOracle(m.xy, m.tri, m.loops)
    P = po.full()
    corner = m.meta["ids"][0, 0]
    t = int(po.I[0])
    assert P[po.I][:, po.col_of[corner]].max() == 0.0
    kl = kl_field_fast(P, P[t])
    assert math.isinf(kl[corner])
    assert tv_field(P, P[t])[corner] == pytest.approx(2.0)
