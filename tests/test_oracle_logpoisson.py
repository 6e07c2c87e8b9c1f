"""Pins for the oracle's subtraction-free Poisson kernel and log P (Section V,
Precision) -- CPU only.

Pinned by: the discrete decay rate along a straight corridor, a closed form
(separable harmonic functions of the five-point stencil, which the split
grid's cot weights are: axis edges 1, diagonals 0): far from both ends the
kernel of the far end-cap vertex falls by exp(-lambda) per cell along the
centre line, cosh(lambda) = 2 - cos(pi / w) for a corridor w cells wide,
checked where the entries lie between 1e-10 and 1e-59 (far below FP32's
smallest normal); exact rational elimination on small maze-like and
obstacle grids; agreement with the direct sparse solve on the entries it
resolves; unit row sums, linear precision and positivity on a serpentine
maze whose smallest entries lie near 1e-76.
"""
import math

import numpy as np
import pytest

from oracle.logpoisson import log_poisson, poisson_subtraction_free
from oracle.poisson import PoissonOracle
from oracle.topology import split_boundary
from synthetic.meshes import grid_obstacles, serpentine, strip
from tests.test_oracle_poisson import exact_poisson_grid


def test_corridor_decay_closed_form():
    w, L = 4, 200
    m = strip(w, L)
    lp = log_poisson(m.xy, m.tri, m.loops)
    ids = m.meta["ids"]                        # ids[j, i]: vertex at column i, row j
    B, _ = split_boundary(m.n_v, m.tri, m.loops)
    b = int(np.nonzero(np.asarray(B) == ids[w // 2, L])[0][0])    # middle of the far end cap
    lam = math.acosh(2.0 - math.cos(math.pi / w))
    row = np.array([lp[ids[w // 2, i], b] for i in range(L + 1)])
    steps = row[21:171] - row[20:170]
    assert np.max(np.abs(steps - lam)) < 1e-9
    assert row[20] < math.log(1e-55) and row[170] > math.log(1e-11)


@pytest.mark.parametrize("mesh", [serpentine(3, 2, 5), serpentine(2, 3, 6), grid_obstacles(6, [(1, 1, 2, 1)])])
def test_exact_rational(mesh):
    exact = exact_poisson_grid(mesh)
    E = np.asarray([[float(x) for x in row] for row in exact])
    P = poisson_subtraction_free(mesh.xy, mesh.tri, mesh.loops)
    pos = E > 0
    assert np.array_equal(P > 0, pos)
    assert np.max(np.abs(P[pos] - E[pos]) / E[pos]) < 1e-13


def test_serpentine_invariants_and_direct_solve():
    m = serpentine(6, 4, 40)
    P = poisson_subtraction_free(m.xy, m.tri, m.loops)
    B, I = split_boundary(m.n_v, m.tri, m.loops)
    Q = PoissonOracle(m.xy, m.tri, m.loops).full()
    big = Q > 1e-8
    assert np.max(np.abs(P[big] - Q[big]) / Q[big]) < 1e-12
    assert np.max(np.abs(P.sum(axis=1) - 1.0)) < 1e-14
    xyB = m.xy[np.asarray(B)]
    assert np.max(np.abs(P[I] @ xyB - m.xy[I])) < 1e-14                # linear precision
    # every column with interior support (grid corners have none: zero cot weights) is positive on
    # every interior row of the connected domain
    sup = P[I].max(axis=0) > 0
    PI = P[I][:, sup]
    assert np.all(PI > 0) and sup.mean() > 0.8
    assert 1e-300 < PI.min() < 1e-70                                    # far below FP32, inside FP64
    assert np.mean(PI < np.finfo(np.float32).tiny) > 0.2
