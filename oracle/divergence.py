"""TV and KL divergence fields, Section IV Eq. (34)-(35) (oracle, FP64 CPU).

For a target vertex t and every vertex x:
    TV_t(x) = sum_b |P[x,b] - P[t,b]|                        (Eq. 34; range [0, 2], Eq. 16)
    KL_t(x) = sum_b P[x,b] * log(P[x,b] / P[t,b])            (Eq. 35 read with Eq. 17)
KL is weighted by the field point's harmonic measure: Eq. (17) integrates
P(s, z) log(P(s, z) / P(s, w)), and the field is evaluated at z = x for the
fixed target w = t.  Terms with P[x,b] = 0 contribute 0 (the limit of
p log p), which happens on boundary rows (P_BB = I).
"""

import numpy as np


def tv_field(P: np.ndarray, Pt: np.ndarray) -> np.ndarray:
    """TV between every row of P and the target row Pt."""
    return np.abs(P - Pt[None, :]).sum(axis=1)


def kl_field(P: np.ndarray, Pt: np.ndarray) -> np.ndarray:
    """KL(row x || target row), 0 log 0 = 0."""
    out = np.zeros(P.shape[0])
    for x in range(P.shape[0]):
        px = P[x]
        nz = px > 0.0
        with np.errstate(divide="ignore"):
            out[x] = np.sum(px[nz] * np.log(px[nz] / Pt[nz]))
    return out


def kl_field_fast(P: np.ndarray, Pt: np.ndarray) -> np.ndarray:
    """Same sum as kl_field, vectorised over rows (used for large sampled sets)."""
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = np.where(P > 0.0, P * np.log(np.where(P > 0.0, P, 1.0) / Pt[None, :]), 0.0)
    return terms.sum(axis=1)
