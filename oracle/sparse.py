"""Sparse KL and TV fields: the target's Poisson kernel row with its small
entries eliminated (Section V: P is sparsified by eliminating entries below a
threshold of 1/sqrt(n), about 90 % sparsity, before the KL sum; the sum it
names, Eq. 36, is not printed) (oracle, FP64 CPU).

Test infrastructure only: imported by tests/ and the CPU baseline of
bench.py, never by the library.

Readings (the paper gives the threshold's value and nothing else):
* relative to the row's largest entry: row y keeps P[y,b] >= theta * max_b' P[y,b'],
  theta = 1/sqrt(n) (n = vertices).  An absolute 1/sqrt(n) would drop nearly
  every entry of the disk's rows, where the paper reports 0 % sparsity.
  The decision is taken in FP32, as the device takes it on its FP32 copy of
  P: float32(P[y,b]) >= float32(theta) * float32(row max), product rounded.
* the kept entries of the TARGET row t decide which columns take part,
  S_t = {b kept in row t}; every other column is merged into one bin, for
  the target and for the field row alike.  The fields are then the same
  divergences between the two coarse-grained harmonic measures
  (P[y,b] for b in S_t, and M_y = sum_{b not in S_t} P[y,b]):

    KL~_t(x)  = sum_{b in S_t} P[x,b] log(P[x,b] / P[t,b]) + M_x log(M_x / M_t)
    KLT~_t(x) = sum_{b in S_t} P[t,b] log(P[t,b] / P[x,b]) + M_t log(M_t / M_x)
    TV~_t(x)  = sum_{b in S_t} |P[x,b] - P[t,b]| + |M_x - M_t|

  (0 log 0 = 0; KLT is the KL weighted by the target's row, Eq. 35 with p
  the target, whose dropped terms are the small ones).  Since every field row meets the same column set, the
  field is as smooth in x as the dense one; a threshold applied to each
  field row instead makes neighbouring rows keep different columns, and
  the fields jump (measured: spurious minima for most targets).  Merging
  columns can only lose information, so 0 <= KL~ <= KL and 0 <= TV~ <= TV
  and 0 <= KLT~ <= KLT (the data-processing inequality), all are exactly 0
  at x = t, and TV - TV~ <= 2 M_t.
"""

import math

import numpy as np


def default_theta(n_v: int) -> float:
    return 1.0 / math.sqrt(n_v)


def keep_mask(P, theta: float) -> np.ndarray:
    """Boolean [rows][k]: the entries a row keeps, decided in FP32."""
    p32 = np.atleast_2d(np.asarray(P)).astype(np.float32)
    thr = np.float32(theta) * p32.max(axis=1, keepdims=True)      # FP32 product, round to nearest
    return (p32 >= thr) & (p32 > 0.0)


def support(P, t: int, theta: float) -> np.ndarray:
    """S_t: boolean [k], the columns the target row keeps."""
    return keep_mask(np.asarray(P)[t], theta)[0]


def _xlogy_ratio(a, b):
    """a log(a / b) elementwise with 0 log 0 = 0 and a log(a/0) = +inf for a > 0."""
    a, b = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64))
    out = np.zeros(a.shape)
    pos = a > 0.0
    with np.errstate(divide="ignore"):
        out[pos] = a[pos] * np.log(a[pos] / b[pos])
    return out


def sparse_kl_field(P, t: int, theta: float) -> np.ndarray:
    """KL~_t(x) for every row x of P."""
    P = np.asarray(P, dtype=np.float64)
    S = support(P, t, theta)
    Mx = P[:, ~S].sum(axis=1)
    Mt = float(Mx[t])                      # the same sum, so that x = t gives exactly 0
    return _xlogy_ratio(P[:, S], P[t, S][None, :]).sum(axis=1) + _xlogy_ratio(Mx, Mt)


def sparse_klt_field(P, t: int, theta: float) -> np.ndarray:
    """KLT~_t(x) for every row x of P (+inf where a kept P[t,b] meets
    P[x,b] = 0, e.g. every boundary row)."""
    P = np.asarray(P, dtype=np.float64)
    S = support(P, t, theta)
    Mx = P[:, ~S].sum(axis=1)
    Mt = float(Mx[t])
    return _xlogy_ratio(P[t, S][None, :], P[:, S]).sum(axis=1) + _xlogy_ratio(Mt, Mx)


def sparse_tv_field(P, t: int, theta: float) -> np.ndarray:
    """TV~_t(x) for every row x of P."""
    P = np.asarray(P, dtype=np.float64)
    S = support(P, t, theta)
    Mx = P[:, ~S].sum(axis=1)
    Mt = float(Mx[t])
    return np.abs(P[:, S] - P[t, S][None, :]).sum(axis=1) + np.abs(Mx - Mt)


def merged_mass(P, t: int, theta: float) -> float:
    """M_t: the target's mass outside its kept columns."""
    P = np.asarray(P, dtype=np.float64)
    return float(P[t, ~support(P, t, theta)].sum())


def sparsity(P, theta: float) -> float:
    """Fraction of the entries of the given rows that the threshold drops."""
    return 1.0 - float(np.mean(keep_mask(P, theta)))
