"""Sparse KL and TV fields: the Poisson kernel with its small entries dropped
(Section V: P is sparsified by eliminating entries below a threshold of
1/sqrt(n), about 90 % sparsity, before the KL sum; the sum it names, Eq. 36,
is not printed) (oracle, FP64 CPU).

Test infrastructure only: imported by tests/ and the CPU baseline of
bench.py, never by the library.

The paper gives the threshold's value but not what it is relative to.
Reading: relative to the row's largest entry.  A field row x keeps

    P[x,b]  if  P[x,b] >= theta * max_b' P[x,b'],   theta = 1/sqrt(n) (n = vertices),

and drops the rest to 0 (no renormalisation): P~[x,:].  (An absolute 1/sqrt(n)
would drop nearly every entry of the disk's rows, where the paper reports 0 %
sparsity; relative to the row maximum the disk stays the least sparse domain.)
Whether an entry is kept is decided in FP32, as the device decides it on its
FP32 copy of P: float32(P[x,b]) >= float32(theta) * float32(row max), the
product rounded to FP32.

    KL~_t(x) = sum_b P~[x,b] log(P~[x,b] / P[t,b])     (target row dense)
    TV~_t(x) = sum_b |P~[x,b] - P~[t,b]|

The target row stays dense inside the logarithm: a dropped target entry under
a kept field entry would make the term infinite.  Both fields are exactly 0
at x = t (the kept entries of row t meet themselves).  Against the dense
fields of divergence.py:

    |KL~ - KL| <= sum_{b dropped from row x} P[x,b] |log(P[x,b] / P[t,b])|
    |TV~ - TV| <= (mass dropped from row x) + (mass dropped from row t).
"""

import math

import numpy as np


def default_theta(n_v: int) -> float:
    return 1.0 / math.sqrt(n_v)


def keep_mask(P, theta: float) -> np.ndarray:
    """Boolean [rows][k]: the entries a row keeps, decided in FP32."""
    p32 = np.asarray(P).astype(np.float32)
    thr = np.float32(theta) * p32.max(axis=1, keepdims=True)      # FP32 product, round to nearest
    return (p32 >= thr) & (p32 > 0.0)


def thresholded(P, theta: float) -> np.ndarray:
    P = np.asarray(P, dtype=np.float64)
    return np.where(keep_mask(P, theta), P, 0.0)


def sparse_kl_field(P, t: int, theta: float) -> np.ndarray:
    """KL~_t(x) for every row x of P (0 log 0 = 0; +inf where a kept P[x,b]
    meets P[t,b] = 0)."""
    P = np.asarray(P, dtype=np.float64)
    Pk = thresholded(P, theta)
    Pt = P[t]
    out = np.zeros(P.shape[0])
    for x in range(P.shape[0]):
        keep = Pk[x] > 0.0
        px = Pk[x][keep]
        pt = Pt[keep]
        if np.any(pt == 0.0):
            out[x] = math.inf
            continue
        out[x] = float(np.sum(px * np.log(px / pt)))
    return out


def sparse_tv_field(P, t: int, theta: float) -> np.ndarray:
    """TV~_t(x) = sum_b |P~[x,b] - P~[t,b]| for every row x."""
    Pk = thresholded(P, theta)
    return np.abs(Pk - Pk[t][None, :]).sum(axis=1)


def dropped_mass(P, theta: float) -> np.ndarray:
    """Per row: the mass the threshold removes, sum_b (P - P~)[x,b]."""
    P = np.asarray(P, dtype=np.float64)
    return (P - thresholded(P, theta)).sum(axis=1)


def sparsity(P, theta: float) -> float:
    """Fraction of the entries of the given rows that are not kept."""
    return 1.0 - float(np.mean(keep_mask(P, theta)))
