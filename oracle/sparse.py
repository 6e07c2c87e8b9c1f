"""Sparse KL and TV fields, Section V (oracle, FP64 CPU).

Test infrastructure only: imported by tests/ and the CPU baseline of
bench.py, never by the library.

Section V: the Poisson kernel matrix P is sparsified by eliminating its very
small entries, those below a threshold of 1/sqrt(n) (n = vertices; about 90 %
of the entries go), and the KL sum is then taken over what is left, with the
kernel's logarithms (the "vectors log P") at hand for every entry.

Readings (the paper gives the threshold's value and nothing else):
* The threshold is relative to the row's largest entry: row y keeps
  P[y,b] >= theta * max_b' P[y,b'] (and P[y,b] > 0), theta = 1/sqrt(n),
  decided here in FP64 on the FP64 kernel.  An absolute 1/sqrt(n) would
  drop nearly every entry of the disk's rows, where Table I prints 0 %
  sparsity.
* In Eq. 35 one row is the weight of every term and the other appears only
  inside the logarithm.  Eliminating a small entry of the weight row drops
  its term (0 log 0 = 0), so the sum runs over the weight row's kept
  entries; the other row enters through its logarithm, taken from the full
  kernel (a zero there would make the term infinite).  So:

    KLT~_t(x) = sum_{b in S_t} P[t,b] log(P[t,b] / P[x,b])     (Eq. 35, p = t)
    KL~_t(x)  = sum_{b in S_x} P[x,b] log(P[x,b] / P[t,b])     (Eq. 35, p = x)

  with S_y the columns row y keeps.  KLT~ is the primary sparse field: its
  weight is the target's row, so one set S_t serves the whole field and the
  dropped terms are small wherever P[x,b] is not much smaller than P[t,b].
* TV (Eq. 34) has no weight row; its sparse form is the TV between the two
  sparsified rows: TV~_t(x) = sum_b |P~[x,b] - P~[t,b]|, P~ = P with every
  row's eliminated entries set to 0.

All three are exactly 0 at x = t.  They are approximations, not divergences:
KL~ and KLT~ can be negative (a restricted sum), and they are bounded below
by the log-sum inequality, sum_{b in S} a_b log(a_b / c_b) >= A log(A / C)
with A, C the sums of a, c over S.

Extension (not in the paper): the merged-bin fields, in which the target
row's kept columns S_t are kept and every other column of both rows is
merged into one bin of mass M_y = sum_{b not in S_t} P[y,b].  They are the
divergences between the two coarse-grained harmonic measures, so
0 <= KL^ <= KL, 0 <= KLT^ <= KLT and 0 <= TV^ <= TV (data processing):

    KL^_t(x)  = sum_{b in S_t} P[x,b] log(P[x,b] / P[t,b]) + M_x log(M_x / M_t)
    KLT^_t(x) = sum_{b in S_t} P[t,b] log(P[t,b] / P[x,b]) + M_t log(M_t / M_x)
    TV^_t(x)  = sum_{b in S_t} |P[x,b] - P[t,b]| + |M_x - M_t|
"""

import math

import numpy as np


def default_theta(n_v: int) -> float:
    """The paper's threshold 1/sqrt(n)."""
    return 1.0 / math.sqrt(n_v)


def keep_mask(P, theta: float) -> np.ndarray:
    """Boolean [rows][k]: the entries a row keeps, P >= theta * (row max) and P > 0."""
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    return (P >= theta * P.max(axis=1, keepdims=True)) & (P > 0.0)


def sparsify(P, theta: float) -> np.ndarray:
    """P~: every row with its eliminated entries set to 0."""
    P = np.atleast_2d(np.asarray(P, dtype=np.float64))
    return np.where(keep_mask(P, theta), P, 0.0)


def support(P, t: int, theta: float) -> np.ndarray:
    """S_t: boolean [k], the columns the target row keeps."""
    return keep_mask(np.asarray(P, dtype=np.float64)[t], theta)[0]


def _xlogy_ratio(a, b):
    """a log(a / b) elementwise with 0 log 0 = 0 and a log(a/0) = +inf for a > 0."""
    a, b = np.broadcast_arrays(np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64))
    out = np.zeros(a.shape)
    pos = a > 0.0
    with np.errstate(divide="ignore"):
        out[pos] = a[pos] * np.log(a[pos] / b[pos])
    return out


# ---------------------------------------------------------------- Section V's reading
def sparse_klt_field(P, t: int, theta: float) -> np.ndarray:
    """KLT~_t(x) = sum over the target's kept columns of P[t,b] log(P[t,b]/P[x,b])
    for every row x (+inf where a kept column meets P[x,b] = 0, e.g. on
    boundary rows)."""
    P = np.asarray(P, dtype=np.float64)
    S = support(P, t, theta)
    return _xlogy_ratio(P[t, S][None, :], P[:, S]).sum(axis=1)


def sparse_kl_field(P, t: int, theta: float) -> np.ndarray:
    """KL~_t(x) = sum over row x's own kept entries of P[x,b] log(P[x,b]/P[t,b])
    (+inf where a kept entry meets P[t,b] = 0)."""
    P = np.asarray(P, dtype=np.float64)
    return _xlogy_ratio(sparsify(P, theta), P[t][None, :]).sum(axis=1)


def sparse_tv_field(P, t: int, theta: float) -> np.ndarray:
    """TV~_t(x) = sum_b |P~[x,b] - P~[t,b]| between the sparsified rows."""
    Ps = sparsify(P, theta)
    return np.abs(Ps - Ps[t][None, :]).sum(axis=1)


def sparsity(P, theta: float) -> float:
    """Fraction of the entries of the given rows that the threshold drops."""
    return 1.0 - float(np.mean(keep_mask(P, theta)))


# ---------------------------------------------------------------- merged-bin extension
def merged_mass(P, t: int, theta: float) -> float:
    """M_t: the target's mass outside its kept columns."""
    P = np.asarray(P, dtype=np.float64)
    return float(P[t, ~support(P, t, theta)].sum())


def merged_kl_field(P, t: int, theta: float) -> np.ndarray:
    """KL^_t(x) for every row x of P."""
    P = np.asarray(P, dtype=np.float64)
    S = support(P, t, theta)
    Mx = P[:, ~S].sum(axis=1)
    Mt = float(Mx[t])                      # the same sum, so that x = t gives exactly 0
    return _xlogy_ratio(P[:, S], P[t, S][None, :]).sum(axis=1) + _xlogy_ratio(Mx, Mt)


def merged_klt_field(P, t: int, theta: float) -> np.ndarray:
    """KLT^_t(x) for every row x of P (+inf where a kept P[t,b] meets P[x,b] = 0)."""
    P = np.asarray(P, dtype=np.float64)
    S = support(P, t, theta)
    Mx = P[:, ~S].sum(axis=1)
    Mt = float(Mx[t])
    return _xlogy_ratio(P[t, S][None, :], P[:, S]).sum(axis=1) + _xlogy_ratio(Mt, Mx)


def merged_tv_field(P, t: int, theta: float) -> np.ndarray:
    """TV^_t(x) for every row x of P."""
    P = np.asarray(P, dtype=np.float64)
    S = support(P, t, theta)
    Mx = P[:, ~S].sum(axis=1)
    Mt = float(Mx[t])
    return np.abs(P[:, S] - P[t, S][None, :]).sum(axis=1) + np.abs(Mx - Mt)
