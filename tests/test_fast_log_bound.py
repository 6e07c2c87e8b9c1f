"""The error bound of the tile kernel's first KL pass, checked on the CPU by
emulating its arithmetic in float32 (no GPU, no library code).

The first pass forms each base-2 logarithm as one FP32 number,
L = fl(E + g(m)) with E the exponent and g the hardware mantissa log, whose
error against log2 m lies in an interval of width DD_FAST_LOG_SPREAD; a term
is P[x,b] * fl(L_x - L_t).  The documented bound on the resulting KL (in
nats, before the summation's own rounding) is

    ln2 * DD_FAST_LOG_SPREAD + 2^-24 (2 ln k + 2 KL + 2).

Here g is emulated as the correctly rounded log2 m plus a deterministic
pseudo-random offset spread over that interval (both ends reached), every
rounding of the kernel is applied in float32, and the terms are summed
exactly in float64 so that only the logarithms' errors remain.  The rows
come from the oracle's Poisson kernel of a small obstacle grid and of the
ring disk, targets drawn from the interior.
"""
import math

import numpy as np
import pytest

from oracle.poisson import PoissonOracle
from synthetic import workloads

SPREAD = 5.0e-7          # DD_FAST_LOG_SPREAD of include/dd.h
FLT_MIN = np.float32(1.1754944e-38)


def _emulated_l2(p32, offset):
    """fl(E + fl(log2 m + offset(m))) for positive float32 p (and 0 -> -127)."""
    bits = p32.view(np.uint32)
    e = ((bits >> 23) & 0xFF).astype(np.int64) - 127
    m = ((bits & 0x007FFFFF) | 0x3F800000).view(np.float32).astype(np.float64)
    j = (bits & 0x007FFFFF).astype(np.int64)
    g = np.float32(np.log2(m) + offset(j))              # hardware mantissa log, rounded once
    return np.float32(e.astype(np.float32) + g)          # one rounding of E + g


def _offset_factory(c0):
    # deterministic pseudo-random offset in [c0, c0 + SPREAD] per mantissa
    def off(j):
        h = (j * 2654435761) % 4294967296
        return c0 + SPREAD * (h / 4294967295.0)
    return off


@pytest.mark.parametrize("case", ["grid", "disk"])
@pytest.mark.parametrize("c0", [-SPREAD, -SPREAD / 2, 0.0])
def test_first_pass_within_documented_bound(case, c0):
    wl = workloads.small_grid(37, 3, T=12, seed=777) if case == "grid" else workloads.disk()
    po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
    P = po.full()
    k = P.shape[1]
    off = _offset_factory(c0)
    P32 = P.astype(np.float32)
    Lrow = _emulated_l2(P32, off)
    rng = np.random.default_rng(5)
    targets = rng.choice(po.I, size=6, replace=False)
    worst = 0.0
    for t in targets:
        pt32 = np.maximum(P32[t], FLT_MIN)
        Lt = _emulated_l2(pt32, off)
        d32 = np.float32(Lrow - Lt[None, :])                     # one rounding per term
        fast = (P32.astype(np.float64) * d32.astype(np.float64)).sum(axis=1) * math.log(2.0)
        px = P32.astype(np.float64)
        ptd = pt32.astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            terms = np.where(px > 0, px * np.log(np.where(px > 0, px, 1.0) / ptd[None, :]), 0.0)
        exact = terms.sum(axis=1)
        bound = math.log(2.0) * SPREAD + 2.0 ** -24 * (2 * math.log(k) + 2 * np.abs(exact) + 2)
        err = np.abs(fast - exact)
        assert np.all(err <= bound), (t, float((err / bound).max()))
        worst = max(worst, float((err / bound).max()))
    assert worst > 0.0


def test_threshold_keeps_relative_accuracy():
    """Above DD_TILE_EXACT_BELOW = 0.25 the bound stays below 6.5e-6
    relative for k up to 8,192 boundary columns (5.3e-6 at k = 1,028), the
    rest of 1e-5 left for the summation, and below 1e-5 up to 2^20 columns."""
    for k, limit in ((128, 6.5e-6), (1028, 5.3e-6), (3930, 6.5e-6), (8192, 6.5e-6), (1 << 20, 1e-5)):
        for kl in (0.25, 1.0, 10.0, 100.0):
            b = math.log(2.0) * SPREAD + 2.0 ** -24 * (2 * math.log(k) + 2 * kl + 2)
            assert b / kl < limit, (k, kl, b / kl)
