"""Other f-divergence fields, Section VI (oracle, FP64 CPU).

Test infrastructure only: imported by tests/, __graft_entry__.smoke() and the
CPU baseline of bench.py, never by the library.

The paper's family (Section VI, and the appendix's comparison table) is

    d_f(z, w) = oint P(t, z) f(P(t, w) / P(t, z)) dt,   f convex, f(1) = 0,

read on the mesh with z = x (the field vertex) and w = t (the target), as for
KL (Eq. 17):

    d_f,t(x) = sum_b P[x,b] f(P[t,b] / P[x,b]).

Adding c (u - 1) to f changes nothing between probability vectors
(sum_b P[x,b] = sum_b P[t,b] = 1; the paper notes the same for -log x and
x log x, which both give KL), so each f is taken in the form with
f(1) = f'(1) = 0, whose terms are non-negative:

    chi2        f(u) = (u - 1)^2                       (the paper's x^2 - 1)
    hellinger   f(u) = (sqrt(u) - 1)^2
    power p     f(u) = |1 - u|^p, p >= 1               (p = 1: TV, p = 2: chi2)
    alpha a     f(u) = 4/(1 - a^2) (1 - u^((1+a)/2)) + 2/(1 - a) (u - 1),  a != +-1
    kl_reverse  f(u) = u log u, i.e. sum_b P[t,b] log(P[t,b] / P[x,b])

(KL itself, f(u) = -log u, and TV are in divergence.py.)  A term with
P[x,b] = 0 takes its limit P[t,b] lim_{u->inf} f(u)/u (0 when P[t,b] = 0),
which is +inf for chi2, power p > 1, kl_reverse and alpha > 1.
"""

import math

import numpy as np


def _ratio_terms(P, Pt, f, slope_inf):
    """sum_b P[x,b] f(Pt[b] / P[x,b]) with the P[x,b] = 0 limit slope_inf * Pt[b]."""
    P = np.asarray(P, dtype=np.float64)
    Pt = np.asarray(Pt, dtype=np.float64)
    out = np.zeros(P.shape[0])
    for x in range(P.shape[0]):
        px = P[x]
        pos = px > 0.0
        s = float(np.sum(px[pos] * f(Pt[pos] / px[pos])))
        zero = ~pos & (Pt > 0.0)
        if np.any(zero):
            s += slope_inf * float(np.sum(Pt[zero]))
        out[x] = s
    return out


def chi2_field(P, Pt):
    return _ratio_terms(P, Pt, lambda u: (u - 1.0) ** 2, math.inf)


def hellinger_field(P, Pt):
    return _ratio_terms(P, Pt, lambda u: (np.sqrt(u) - 1.0) ** 2, 1.0)


def power_field(P, Pt, p: float):
    if p < 1.0:
        raise ValueError("p >= 1")
    return _ratio_terms(P, Pt, lambda u: np.abs(1.0 - u) ** p, 1.0 if p == 1.0 else math.inf)


def alpha_field(P, Pt, a: float):
    if abs(abs(a) - 1.0) < 1e-12:
        raise ValueError("alpha != +-1")
    c = 4.0 / (1.0 - a * a)
    e = (1.0 + a) / 2.0
    lin = 2.0 / (1.0 - a)

    def f(u):
        with np.errstate(divide="ignore"):          # u = 0 with e < 0: f = +inf, the exact value
            return c * (1.0 - u ** e) + lin * (u - 1.0)

    # lim f(u)/u: u^e/u -> 0 for a < 1, so the limit is lin; for a > 1 it is +inf
    return _ratio_terms(P, Pt, f, lin if a < 1.0 else math.inf)


def kl_reverse_field(P, Pt):
    """sum_b P[t,b] log(P[t,b] / P[x,b]) (f(u) = u log u); 0 log 0 = 0."""
    return _ratio_terms(P, Pt, lambda u: np.where(u > 0.0, u * np.log(np.where(u > 0.0, u, 1.0)), 0.0), math.inf)


FAMILIES = {
    "chi2": lambda P, Pt, prm: chi2_field(P, Pt),
    "hellinger": lambda P, Pt, prm: hellinger_field(P, Pt),
    "power": lambda P, Pt, prm: power_field(P, Pt, prm),
    "alpha": lambda P, Pt, prm: alpha_field(P, Pt, prm),
    "kl_reverse": lambda P, Pt, prm: kl_reverse_field(P, Pt),
}


def field(P, Pt, family: str, param: float = 0.0):
    return FAMILIES[family](P, Pt, param)
