"""Triangle-based gradient-descent path tracing, Section IV (oracle, FP64 CPU).

The field f is piecewise linear over the triangles, so each triangle has one
constant gradient g = sum_i f_i grad(phi_i), grad(phi_i) = J e_i / (2A) with e_i
the edge opposite vertex i (counter-clockwise) and J the +90 degree rotation.
The path follows d = -g.  The paper describes the walk in prose (Section IV,
"Gradient-descent path generation"); this is the reading used everywhere:

* At a vertex v: if v is the target t, stop.  If v is a neighbour of t, the
  path lies on an edge incident on t: append t and stop.  Otherwise, among
  the triangles around v whose direction d points into the triangle from v
  (inside the corner wedge, inclusive), follow the steepest one (largest |g|,
  ties to the lowest triangle id) to the opposite edge.  If none qualifies,
  take the incident edge with the largest positive slope (f_v - f_u)/|v - u|
  (ties to the lowest u) to its other end; if no slope is positive the path is
  stuck in a local minimum.
* On an edge (a, b), coming from one triangle: if a or b is t, append t and
  stop (the path intersects an edge incident on the target).  Otherwise enter
  the triangle across the edge.  If its direction points into it, cross it to
  its exit edge.  If it does not (a valley edge, both sides pushing back) or
  there is no triangle across (a boundary edge), slide along the edge to its
  endpoint with the lower value (ties to the lower id).
* An exit whose barycentric coordinate is at most eps lands on the vertex.
* The walk stops with STEP_LIMIT after max_steps states (default 4 n_t) and
  with TRUNCATED when the polyline would exceed max_pts points.

The polyline starts at the source vertex and ends at the target vertex.
"""

import math

import numpy as np

from .topology import triangle_neighbours, vertex_neighbours, vertex_triangles

OK, STUCK_LOCAL_MIN, STEP_LIMIT, TRUNCATED = 0, 1, 2, 3


class Tracer:
    def __init__(self, xy: np.ndarray, tri: np.ndarray, eps: float = 1e-12):
        self.xy = np.asarray(xy, dtype=np.float64)
        self.tri = np.asarray(tri, dtype=np.int64)
        self.n_v = self.xy.shape[0]
        self.nbr = triangle_neighbours(self.tri)
        self.vtri = vertex_triangles(self.n_v, self.tri)
        self.vnb = vertex_neighbours(self.n_v, self.tri)
        self.eps = eps
        p0 = self.xy[self.tri[:, 0]]
        p1 = self.xy[self.tri[:, 1]]
        p2 = self.xy[self.tri[:, 2]]
        a2 = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p1[:, 1] - p0[:, 1]) * (p2[:, 0] - p0[:, 0])
        self.gphi = np.zeros((len(self.tri), 3, 2))
        for i, (pa, pb) in enumerate(((p1, p2), (p2, p0), (p0, p1))):
            e = pb - pa                                   # edge opposite vertex i
            self.gphi[:, i, 0] = -e[:, 1] / a2            # J e / (2A)
            self.gphi[:, i, 1] = e[:, 0] / a2

    def grad(self, t: int, f: np.ndarray) -> np.ndarray:
        v = self.tri[t]
        return f[v[0]] * self.gphi[t, 0] + f[v[1]] * self.gphi[t, 1] + f[v[2]] * self.gphi[t, 2]

    def _local(self, t: int, v: int) -> int:
        row = self.tri[t]
        return 0 if row[0] == v else (1 if row[1] == v else 2)

    def trace(self, f, q: int, target: int, max_pts: int = 1 << 30, max_steps: int = None):
        """Path from q to target on the field f: an array over all vertices, or
        an object indexed by vertex id (e.g. a PathOnlyField, which evaluates
        the divergence only at the vertices the walk reads)."""
        if not isinstance(f, PathOnlyField):
            f = np.asarray(f, dtype=np.float64)
        if max_steps is None:
            max_steps = 4 * len(self.tri)
        eps = self.eps
        xy = self.xy
        path = [tuple(xy[q])]

        def push(p):
            if len(path) >= max_pts:
                return False
            path.append((float(p[0]), float(p[1])))
            return True

        state = ("v", q)
        steps = 0
        while True:
            if steps >= max_steps:
                return np.asarray(path), STEP_LIMIT
            steps += 1
            if state[0] == "v":
                v = state[1]
                if v == target:
                    return np.asarray(path), OK
                if target in self.vnb[v]:
                    if not push(xy[target]):
                        return np.asarray(path), TRUNCATED
                    return np.asarray(path), OK
                best = None
                best_g = 0.0
                for t in self.vtri[v]:
                    g = self.grad(t, f)
                    gn = math.hypot(g[0], g[1])
                    if gn == 0.0:
                        continue
                    i = self._local(t, v)
                    j, k = (i + 1) % 3, (i + 2) % 3
                    aj = -(self.gphi[t, j] @ g)
                    ak = -(self.gphi[t, k] @ g)
                    tol = eps * gn * max(np.hypot(*self.gphi[t, j]), np.hypot(*self.gphi[t, k]))
                    if aj >= -tol and ak >= -tol and aj + ak > 0.0 and gn > best_g:
                        best, best_g = (t, i, max(aj, 0.0), max(ak, 0.0)), gn
                if best is not None:
                    t, i, aj, ak = best
                    j, k = (i + 1) % 3, (i + 2) % 3
                    s = 1.0 / (aj + ak)
                    lj, lk = s * aj, s * ak
                    vj, vk = int(self.tri[t, j]), int(self.tri[t, k])
                    if lj <= eps:
                        if not push(xy[vk]):
                            return np.asarray(path), TRUNCATED
                        state = ("v", vk)
                    elif lk <= eps:
                        if not push(xy[vj]):
                            return np.asarray(path), TRUNCATED
                        state = ("v", vj)
                    else:
                        if not push(lj * xy[vj] + lk * xy[vk]):
                            return np.asarray(path), TRUNCATED
                        state = ("e", t, i, lj, lk)
                    continue
                # edge fallback: steepest descending incident edge
                best_u, best_s = -1, 0.0
                for u in self.vnb[v]:
                    slope = (f[v] - f[u]) / math.hypot(xy[v, 0] - xy[u, 0], xy[v, 1] - xy[u, 1])
                    if slope > best_s:
                        best_u, best_s = u, slope
                if best_u < 0:
                    return np.asarray(path), STUCK_LOCAL_MIN
                if not push(xy[best_u]):
                    return np.asarray(path), TRUNCATED
                state = ("v", best_u)
                continue
            # edge state: left triangle t through the edge opposite local i,
            # at barycentric weights (la, lb) on endpoints a = tri[t, i+1], b = tri[t, i+2]
            _, t, i, la, lb = state
            a, b = int(self.tri[t, (i + 1) % 3]), int(self.tri[t, (i + 2) % 3])
            if a == target or b == target:
                if not push(xy[target]):
                    return np.asarray(path), TRUNCATED
                return np.asarray(path), OK
            t2 = int(self.nbr[t, i])
            slide = t2 < 0
            if not slide:
                g2 = self.grad(t2, f)
                gn2 = math.hypot(g2[0], g2[1])
                c2 = 3 - self._local(t2, a) - self._local(t2, b)
                rc = -(self.gphi[t2, c2] @ g2)
                tol = eps * gn2 * np.hypot(*self.gphi[t2, c2])
                slide = not (rc > tol)
            if slide:
                low = a if (f[a] < f[b] or (f[a] == f[b] and a < b)) else b
                if not push(xy[low]):
                    return np.asarray(path), TRUNCATED
                state = ("v", low)
                continue
            ia, ib = self._local(t2, a), self._local(t2, b)
            ra = -(self.gphi[t2, ia] @ g2)
            rb = -(self.gphi[t2, ib] @ g2)
            sa = la / -ra if ra < 0.0 else math.inf
            sb = lb / -rb if rb < 0.0 else math.inf
            if math.isinf(min(sa, sb)):          # no exit edge found: treat as a valley edge
                low = a if (f[a] < f[b] or (f[a] == f[b] and a < b)) else b
                if not push(xy[low]):
                    return np.asarray(path), TRUNCATED
                state = ("v", low)
                continue
            c = int(self.tri[t2, c2])
            if sa <= sb:
                s = sa
                lb2 = max(lb + s * rb, 0.0)
                lc2 = max(s * rc, 0.0)
                tot = lb2 + lc2
                lb2, lc2 = lb2 / tot, lc2 / tot
                if lb2 <= eps:
                    nxt = ("v", c)
                elif lc2 <= eps:
                    nxt = ("v", b)
                else:
                    nxt = None
                exit_local, w_other = ia, {b: lb2, c: lc2}
            else:
                s = sb
                la2 = max(la + s * ra, 0.0)
                lc2 = max(s * rc, 0.0)
                tot = la2 + lc2
                la2, lc2 = la2 / tot, lc2 / tot
                if la2 <= eps:
                    nxt = ("v", c)
                elif lc2 <= eps:
                    nxt = ("v", a)
                else:
                    nxt = None
                exit_local, w_other = ib, {a: la2, c: lc2}
            if nxt is not None:
                if not push(xy[nxt[1]]):
                    return np.asarray(path), TRUNCATED
                state = nxt
                continue
            e1 = int(self.tri[t2, (exit_local + 1) % 3])
            e2 = int(self.tri[t2, (exit_local + 2) % 3])
            l1, l2 = w_other[e1], w_other[e2]
            if not push(l1 * xy[e1] + l2 * xy[e2]):
                return np.asarray(path), TRUNCATED
            state = ("e", t2, exit_local, l1, l2)


class PathOnlyField:
    """The field of one target evaluated only where the walk reads it: the
    paper's CPU scheme (Section V, Table I), which computes KL or TV only at
    the vertices relevant to the path, from the precomputed Poisson kernel.
    f[x] is Eq. 35 (KL, weighted by row x, 0 log 0 = 0) or Eq. 34 (TV) for
    rows x and t of P, computed on first use and kept."""

    def __init__(self, P, t: int, kind: str = "kl"):
        self.P = P
        self.Pt = np.asarray(P[t], dtype=np.float64)
        self.kind = kind
        self.cache = {}

    def __getitem__(self, x):
        x = int(x)
        v = self.cache.get(x)
        if v is None:
            px = np.asarray(self.P[x], dtype=np.float64)
            if self.kind == "kl":
                nz = px > 0.0
                with np.errstate(divide="ignore"):
                    v = float(np.sum(px[nz] * np.log(px[nz] / self.Pt[nz])))
            else:
                v = float(np.sum(np.abs(px - self.Pt)))
            self.cache[x] = v
        return v

    @property
    def evaluated(self) -> int:
        return len(self.cache)
