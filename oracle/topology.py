"""Mesh topology for the discrete setting of Section IV (oracle, FP64 CPU).

Boundary vertices B are the endpoints of edges with exactly one incident
triangle; interior vertices I are the rest (Section IV, the n = k + m split
used by the block form Eq. 18).  The caller's boundary loops must cover
exactly B, each consecutive pair being a boundary edge; their concatenation
fixes the column order of the Poisson kernel.  Interior vertices keep
increasing vertex-id order.
"""

import numpy as np


class TopologyError(ValueError):
    pass


def edge_triangle_counts(tri: np.ndarray):
    """Map undirected edge (a, b), a < b -> number of incident triangles."""
    counts = {}
    for t in tri:
        for e in range(3):
            a, b = int(t[e]), int(t[(e + 1) % 3])
            key = (a, b) if a < b else (b, a)
            counts[key] = counts.get(key, 0) + 1
    return counts


def split_boundary(n_v: int, tri: np.ndarray, loops):
    """Return (B, I): boundary ids in loop order, interior ids ascending.

    Raises TopologyError if the loops disagree with the topological boundary.
    """
    counts = edge_triangle_counts(tri)
    if any(c > 2 for c in counts.values()):
        raise TopologyError("non-manifold edge")
    bedges = {e for e, c in counts.items() if c == 1}
    bverts = set()
    for a, b in bedges:
        bverts.add(a)
        bverts.add(b)
    order = [int(v) for l in loops for v in l]
    if len(order) != len(set(order)):
        raise TopologyError("a vertex appears twice in the loops")
    if set(order) != bverts:
        raise TopologyError("loops do not match the topological boundary")
    for l in loops:
        for i in range(len(l)):
            a, b = int(l[i]), int(l[(i + 1) % len(l)])
            key = (a, b) if a < b else (b, a)
            if key not in bedges:
                raise TopologyError(f"loop step {a}->{b} is not a boundary edge")
    B = np.asarray(order, dtype=np.int64)
    used = np.zeros(n_v, dtype=bool)
    used[tri.reshape(-1)] = True
    if not used.all():
        raise TopologyError("vertex not used by any triangle")
    isb = np.zeros(n_v, dtype=bool)
    isb[B] = True
    I = np.nonzero(~isb)[0].astype(np.int64)
    return B, I


def vertex_neighbours(n_v: int, tri: np.ndarray):
    nb = [set() for _ in range(n_v)]
    for t in tri:
        a, b, c = int(t[0]), int(t[1]), int(t[2])
        nb[a].update((b, c))
        nb[b].update((a, c))
        nb[c].update((a, b))
    return [sorted(s) for s in nb]


def vertex_triangles(n_v: int, tri: np.ndarray):
    vt = [[] for _ in range(n_v)]
    for ti, t in enumerate(tri):
        for v in t:
            vt[int(v)].append(ti)
    return vt


def triangle_neighbours(tri: np.ndarray) -> np.ndarray:
    """nbr[t, i] = triangle across the edge opposite local vertex i, or -1."""
    owner = {}
    for ti, t in enumerate(tri):
        for i in range(3):
            a, b = int(t[(i + 1) % 3]), int(t[(i + 2) % 3])
            key = (a, b) if a < b else (b, a)
            owner.setdefault(key, []).append((ti, i))
    nbr = -np.ones((len(tri), 3), dtype=np.int64)
    for lst in owner.values():
        if len(lst) == 2:
            (t0, i0), (t1, i1) = lst
            nbr[t0, i0] = t1
            nbr[t1, i1] = t0
    return nbr
