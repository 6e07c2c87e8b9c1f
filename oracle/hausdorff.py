"""Hausdorff distance between two polylines (oracle, FP64 CPU).

Each polyline is sampled at spacing at most `step` (its vertices included);
the directed distance is the largest, over the samples of one polyline, of
the exact point-to-segment distance to the other polyline.  The result is the
larger of the two directed distances.
"""

import numpy as np


def _samples(P: np.ndarray, step: float) -> np.ndarray:
    pts = [P[:1]]
    for a, b in zip(P[:-1], P[1:]):
        L = float(np.hypot(*(b - a)))
        n = max(1, int(np.ceil(L / step)))
        s = (np.arange(1, n + 1) / n)[:, None]
        pts.append(a[None, :] * (1 - s) + b[None, :] * s)
    return np.concatenate(pts, axis=0)


def _point_to_polyline(X: np.ndarray, P: np.ndarray) -> np.ndarray:
    if len(P) == 1:
        return np.hypot(X[:, 0] - P[0, 0], X[:, 1] - P[0, 1])
    A = P[:-1][None, :, :]
    D = (P[1:] - P[:-1])[None, :, :]
    Xe = X[:, None, :]
    dd = (D ** 2).sum(-1)
    s = np.where(dd > 0, ((Xe - A) * D).sum(-1) / np.where(dd > 0, dd, 1.0), 0.0)
    s = np.clip(s, 0.0, 1.0)
    C = A + s[..., None] * D
    dist = np.hypot(Xe[..., 0] - C[..., 0], Xe[..., 1] - C[..., 1])
    return dist.min(axis=1)


def hausdorff(P: np.ndarray, Q: np.ndarray, step: float) -> float:
    P = np.asarray(P, dtype=np.float64).reshape(-1, 2)
    Q = np.asarray(Q, dtype=np.float64).reshape(-1, 2)
    out = 0.0
    for A, B in ((P, Q), (Q, P)):
        X = _samples(A, step)
        for lo in range(0, len(X), 2048):
            out = max(out, float(_point_to_polyline(X[lo:lo + 2048], B).max()))
    return out
