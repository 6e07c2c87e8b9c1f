"""Pins for the oracle's other f-divergence fields (Section VI) -- CPU only.

Pinned by: the unit-disk closed forms of the appendix's comparison table
(chi2: 2|C|^2 / (1 - |C|^2), the table's (1 + x^2)/(1 - x^2) less the constant
that f(u) = u^2 - 1 and (u - 1)^2 differ by; KL in either direction:
-log(1 - |C|^2); TV = p = 1: (4/pi) asin|C|) carried to any target by the
Moebius map (A10); numerical quadrature of the continuous integral on the
disk for Hellinger and alpha; the family identities alpha = 0 -> 2 Hellinger,
alpha = 3 -> chi2 / 2, p = 2 -> chi2, alpha -> -1 -> KL and alpha -> 1 ->
reverse KL; and the divergence axioms.
"""
import math

import numpy as np
import pytest
from scipy.integrate import quad

from oracle.divergence import kl_field_fast, tv_field
from oracle.fdiv import alpha_field, chi2_field, hellinger_field, kl_reverse_field, power_field
from oracle.poisson import PoissonOracle
from synthetic.meshes import disk_rings, grid_obstacles

_cache = {}


def disk(R, S):
    if (R, S) not in _cache:
        m = disk_rings(R, S)
        po = PoissonOracle(m.xy, m.tri, m.loops)
        P = po.full()
        z = m.xy[:, 0] + 1j * m.xy[:, 1]
        t = int(np.argmin(np.abs(z - (0.3 + 0.2j))))
        _cache[(R, S)] = (m, P, z, t)
    return _cache[(R, S)]


def _closed_form_errors(R, S):
    m, P, z, t = disk(R, S)
    sel = np.abs(z) <= 0.8
    C = np.abs((z - z[t]) / (1 - np.conj(z[t]) * z))[sel]     # Eq. (A10)
    Ps = P[sel]
    e_chi2 = np.abs(chi2_field(Ps, P[t]) - 2 * C ** 2 / (1 - C ** 2)).max()
    e_klr = np.abs(kl_reverse_field(Ps, P[t]) + np.log(1 - C ** 2)).max()
    e_p1 = np.abs(power_field(Ps, P[t], 1.0) - 4 / math.pi * np.arcsin(C)).max()
    return e_chi2, e_klr, e_p1


def test_disk_closed_forms_converge():
    a16 = _closed_form_errors(16, 128)
    a32 = _closed_form_errors(32, 256)
    assert max(a16) < 5e-3, a16
    for e16, e32 in zip(a16, a32):
        assert e32 < e16 / 2.5, (a16, a32)


def _disk_integral(f, z, w):
    """oint P(s, z) f(P(s, w) / P(s, z)) ds on the unit circle (continuous)."""
    def P(s, q):
        return (1 - abs(q) ** 2) / (2 * math.pi * abs(q - complex(math.cos(s), math.sin(s))) ** 2)
    val, _ = quad(lambda s: P(s, z) * f(P(s, w) / P(s, z)), 0.0, 2 * math.pi, limit=400, epsabs=1e-13)
    return val


FAMILIES = [
    ("hellinger", lambda P, Pt: hellinger_field(P, Pt), lambda u: (math.sqrt(u) - 1) ** 2),
    ("alpha0.5", lambda P, Pt: alpha_field(P, Pt, 0.5),
     lambda u: 4 / 0.75 * (1 - u ** 0.75) + 4 * (u - 1)),
    ("alpha-0.5", lambda P, Pt: alpha_field(P, Pt, -0.5),
     lambda u: 4 / 0.75 * (1 - u ** 0.25) + (4 / 3) * (u - 1)),
    ("power3", lambda P, Pt: power_field(P, Pt, 3.0), lambda u: abs(1 - u) ** 3),
]


@pytest.mark.parametrize("name,fn,f", FAMILIES)
def test_disk_quadrature_converges(name, fn, f):
    errs = []
    for R, S in ((16, 128), (32, 256)):
        m, P, z, t = disk(R, S)
        got = fn(P, P[t])
        # a few vertices at radius <= 0.7, chosen by position (the same points on both meshes)
        picks = [int(np.argmin(np.abs(z - q))) for q in (0.0, 0.5j, -0.4 + 0.1j, 0.6 - 0.2j)]
        errs.append(max(abs(got[x] - _disk_integral(f, z[x], z[t])) for x in picks))
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 2.5, errs


def _grid():
    m = grid_obstacles(20, [(5, 5, 3, 4), (12, 10, 4, 3)])
    po = PoissonOracle(m.xy, m.tri, m.loops)
    return m, po, po.full()


def test_family_identities():
    m, po, P = _grid()
    t = int(po.I[len(po.I) // 3])
    Pt = P[t]
    inter = po.I
    chi2 = chi2_field(P, Pt)
    hel = hellinger_field(P, Pt)
    np.testing.assert_allclose(alpha_field(P, Pt, 0.0)[inter], 2 * hel[inter], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(alpha_field(P, Pt, 3.0)[inter], chi2[inter] / 2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(power_field(P, Pt, 2.0)[inter], chi2[inter], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(power_field(P, Pt, 1.0), tv_field(P, Pt), rtol=1e-12, atol=1e-15)
    kl = kl_field_fast(P, Pt)
    klr = kl_reverse_field(P, Pt)
    for eps in (1e-3, 1e-4):
        a_lo = alpha_field(P, Pt, -1 + eps)[inter]
        a_hi = alpha_field(P, Pt, 1 - eps)[inter]
        assert np.abs(a_lo - kl[inter]).max() <= 4 * eps * (1 + kl[inter].max())
        assert np.abs(a_hi - klr[inter]).max() <= 4 * eps * (1 + klr[inter].max())


def test_axioms():
    m, po, P = _grid()
    for t in (int(po.I[7]), int(po.I[-9])):
        Pt = P[t]
        for d in (chi2_field(P, Pt), hellinger_field(P, Pt), power_field(P, Pt, 2.5), alpha_field(P, Pt, 0.3),
                  alpha_field(P, Pt, -2.0), kl_reverse_field(P, Pt)):
            assert d[t] == pytest.approx(0.0, abs=1e-14)
            fin = np.isfinite(d)
            assert (d[fin] >= -1e-14).all()
            assert fin[po.I].all()                      # interior rows: P[x,b] > 0 for every b
    # a boundary row meets P[x,b] = 0 < P[t,b]: +inf for chi2, finite Hellinger
    b = int(po.B[0])
    t = int(po.I[7])
    assert math.isinf(chi2_field(P[b:b + 1], P[t])[0])
    assert math.isfinite(hellinger_field(P[b:b + 1], P[t])[0])
