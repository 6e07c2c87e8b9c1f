"""Spurious local minima and edge-following paths, Section V ("Low resolution
discretizations") and Section IV ("Gradient-descent path generation") (oracle,
FP64 CPU).

Test infrastructure only: imported by tests/ and the CPU baseline of bench.py,
never by the library.

* A spurious local minimum of a distance field f with target t is an interior
  vertex v != t none of whose mesh neighbours has a smaller value:
  f[v] <= f[u] for every neighbour u.  Gradient descent can stop at such a
  vertex; the discrete Green's function has none (maximum principle), and the
  paper reports them for TV, but not for KL, at low resolution.
* The edge-following path (the paper's "simplest way"): from the source,
  repeatedly move to the neighbour with the smallest value among those below
  the current vertex (the largest decrease; ties to the lowest id); stop at
  the target (OK) or where no neighbour is lower (STUCK); STEP_LIMIT after
  n_v moves, TRUNCATED when the polyline would exceed max_pts points.
"""

import numpy as np

from .topology import vertex_neighbours

OK, STUCK, STEP_LIMIT, TRUNCATED = 0, 1, 2, 3


def local_minima(f, tri, interior_mask, target: int):
    """Sorted array of the spurious local minima of f (interior, != target)."""
    f = np.asarray(f, dtype=np.float64)
    n_v = len(f)
    nb = vertex_neighbours(n_v, tri)
    out = []
    for v in range(n_v):
        if not interior_mask[v] or v == target:
            continue
        if all(f[v] <= f[u] for u in nb[v]):
            out.append(v)
    return np.asarray(out, dtype=np.int64)


def edge_path(f, tri, xy, source: int, target: int, max_pts: int = 1 << 30):
    """Edge-following polyline (array of points) and status."""
    f = np.asarray(f, dtype=np.float64)
    n_v = len(f)
    nb = vertex_neighbours(n_v, tri)
    v = int(source)
    pts = [xy[v]]
    if v == target:
        return np.asarray(pts), OK
    for _ in range(n_v):
        best = -1
        for u in sorted(nb[v]):
            if f[u] < f[v] and (best < 0 or f[u] < f[best]):
                best = u
        if best < 0:
            return np.asarray(pts), STUCK
        if len(pts) >= max_pts:
            return np.asarray(pts), TRUNCATED
        v = best
        pts.append(xy[v])
        if v == target:
            return np.asarray(pts), OK
    return np.asarray(pts), STEP_LIMIT
