"""Pins for the oracle's sparse KL/TV fields (Section V, P thresholded at
1/sqrt(n) relative to each row's largest entry) -- CPU only.

Pinned by: a hand-worked row (which entries a threshold keeps, and the two
sums written out), the dense fields as the theta -> 0 limit, the bounds on
what dropping entries can change (each term removed from the KL sum is
P[x,b] log(P[x,b]/P[t,b]); the triangle inequality for TV), exact zeros at
the target, nested kept sets as theta grows, and the disk's centre row,
whose entries are all equal by the mesh's rotational symmetry, so that no
threshold below 1 drops any of them.
"""
import math

import numpy as np
import pytest

from oracle import sparse
from oracle.divergence import kl_field_fast, tv_field
from oracle.poisson import PoissonOracle
from synthetic import workloads
from synthetic.meshes import disk_rings


def test_hand_row():
    # rows sum to 1; theta = 0.01 keeps entries >= 0.01 * row max
    P = np.array([[0.5, 0.004, 0.496, 0.0],
                  [0.25, 0.25, 0.25, 0.25],
                  [0.9, 0.0089, 0.0911, 0.0]])
    keep = sparse.keep_mask(P, 0.01)
    assert keep.tolist() == [[True, False, True, False], [True] * 4, [True, False, True, False]]
    # KL~ of row 0 against target row 1: 0.5 log(0.5/0.25) + 0.496 log(0.496/0.25)
    kl = sparse.sparse_kl_field(P, 1, 0.01)
    assert kl[0] == pytest.approx(0.5 * math.log(2.0) + 0.496 * math.log(0.496 / 0.25), rel=1e-15)
    assert kl[1] == 0.0
    # TV~ of row 2 against target row 0: |0.9 - 0.5| + |0 - 0| + |0.0911 - 0.496| + 0
    tv = sparse.sparse_tv_field(P, 0, 0.01)
    assert tv[2] == pytest.approx(0.4 + 0.4049, rel=1e-14)
    assert tv[0] == 0.0
    # dropped mass: 0.004 from row 0, 0.0089 from row 2
    assert sparse.dropped_mass(P, 0.01) == pytest.approx([0.004, 0.0, 0.0089], abs=1e-17)


def test_threshold_decided_in_fp32():
    # 0.01 * 0.5 rounds in FP32; an entry equal to the FP32 product is kept,
    # the next FP32 value below it is not
    thr = np.float32(0.01) * np.float32(0.5)
    below = np.nextafter(thr, np.float32(0.0))
    P = np.array([[0.5, float(thr), float(below), 0.5 - float(thr) - float(below)]])
    assert sparse.keep_mask(P, 0.01).tolist() == [[True, True, False, True]]


def _cases():
    wl = workloads.small_grid(37, 3, T=4, seed=777)
    disk = workloads.disk()
    return [(wl.mesh, [int(t) for t in wl.targets]), (disk.mesh, [int(disk.targets[0])])]


@pytest.mark.parametrize("idx", [0, 1])
def test_dense_limit_bounds_and_zeros(idx):
    mesh, targets = _cases()[idx]
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    P = po.full()
    theta = sparse.default_theta(mesh.n_v)
    keep = sparse.keep_mask(P, theta)
    drop_mass = sparse.dropped_mass(P, theta)
    for t in targets:
        kl, tv = kl_field_fast(P, P[t]), tv_field(P, P[t])
        # theta -> 0: every positive entry kept, the dense fields
        k0 = sparse.sparse_kl_field(P, t, 1e-30)
        fin = np.isfinite(kl)
        assert np.allclose(k0[fin], kl[fin], rtol=1e-12, atol=1e-14)
        assert np.allclose(sparse.sparse_tv_field(P, t, 1e-30), tv, rtol=1e-12, atol=1e-14)
        ks, ts = sparse.sparse_kl_field(P, t, theta), sparse.sparse_tv_field(P, t, theta)
        assert ks[t] == 0.0 and ts[t] == 0.0
        for x in po.I:
            dropped = ~keep[x] & (P[x] > 0)
            bound = float(np.sum(P[x][dropped] * np.abs(np.log(P[x][dropped] / P[t][dropped]))))
            assert abs(ks[x] - kl[x]) <= bound * (1 + 1e-9) + 1e-13
            assert abs(ts[x] - tv[x]) <= (drop_mass[x] + drop_mass[t]) * (1 + 1e-9) + 1e-13


def test_nested_and_disk_centre():
    mesh = disk_rings(8, 48)
    po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
    P = po.full()
    prev = None
    for theta in (1e-4, 1e-3, 1e-2, 0.1, 0.5):
        k = sparse.keep_mask(P[po.I], theta)
        if prev is not None:
            assert not np.any(k & ~prev)          # a larger theta keeps a subset
        prev = k
    # vertex 0 is the centre: all 48 entries equal up to the solve's rounding
    assert np.ptp(P[0]) < 1e-12
    assert sparse.keep_mask(P[:1], 0.999).all()
    assert sparse.sparsity(P[:1], sparse.default_theta(mesh.n_v)) == 0.0
