"""Synthetic planar triangle meshes standing in for the paper's domains.

The paper meshes its domains with the Triangle package (Section V); those
domains are not available, so two seeded families stand in for them:

* ``disk_rings``: the unit disk as a centre vertex plus ``n_rings`` concentric
  rings of ``n_seg`` vertices each (radii j/n_rings, angles 2*pi*i/n_seg,
  aligned across rings).  The innermost ring is a fan around the centre; every
  annular quad is split on the diagonal (ring j, i) -> (ring j+1, i+1).  The
  quads are isosceles trapezoids, so the mesh is Delaunay.
* ``grid_obstacles``: the unit square cut into N x N cells of side h = 1/N,
  each cell split on its (i, j) -> (i+1, j+1) diagonal, with axis-aligned
  rectangular blocks of whole cells removed as obstacles (holes).
* ``cell_domain``: any union of whole grid cells (a boolean cell mask), each
  cell split on the same diagonal, its boundary loops traced along the cell
  edges; ``serpentine`` builds a long winding corridor from it (a maze-like
  domain whose harmonic measures decay by hundreds of orders of magnitude
  along the corridor) and ``strip`` a single straight corridor.
* ``convex_holes``: the unit disk minus a few convex regular polygons, meshed
  as the Delaunay triangulation of a jittered hexagonal point set plus points
  spaced along every boundary loop (a stand-in for the paper's "Convex Holes"
  domain meshed at low resolution, n = 175, Section V).  Unlike the grid, no
  edge weight is exactly zero, and the Delaunay property keeps every interior
  edge weight non-negative.

Every mesh is returned with counter-clockwise triangles and its boundary loops:
the outer loop counter-clockwise, one clockwise loop per obstacle (the domain
lies to the left of every loop).  Concatenating the loops fixes the column
order of the Poisson kernel.  Nothing here computes any quantity of the
divergence-distance method.
"""

import math
from dataclasses import dataclass, field

import numpy as np

from .rng import SplitMix64


@dataclass
class Mesh:
    xy: np.ndarray          # float64 [n_v, 2]
    tri: np.ndarray         # int32 [n_t, 3], counter-clockwise
    loops: list             # list of int32 arrays (vertex ids), outer loop first
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_v(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_t(self) -> int:
        return int(self.tri.shape[0])

    def loop_arrays(self):
        """(loop_idx int32[k], loop_off int64[n_loops+1]) as passed to dd_load_mesh."""
        idx = np.concatenate([np.asarray(l, dtype=np.int32) for l in self.loops])
        off = np.zeros(len(self.loops) + 1, dtype=np.int64)
        off[1:] = np.cumsum([len(l) for l in self.loops])
        return idx, off

    def boundary_flags(self) -> np.ndarray:
        flags = np.zeros(self.n_v, dtype=bool)
        for l in self.loops:
            flags[np.asarray(l)] = True
        return flags


def disk_rings(n_rings: int = 16, n_seg: int = 128) -> Mesh:
    """Concentric-ring triangulation of the unit disk (n = 1 + n_rings*n_seg)."""
    n_v = 1 + n_rings * n_seg
    xy = np.zeros((n_v, 2), dtype=np.float64)

    def vid(j, i):  # ring j in 1..n_rings, segment i (mod n_seg)
        return 1 + (j - 1) * n_seg + (i % n_seg)

    for j in range(1, n_rings + 1):
        r = j / n_rings
        for i in range(n_seg):
            a = 2.0 * math.pi * i / n_seg
            xy[vid(j, i)] = (r * math.cos(a), r * math.sin(a))
    tris = []
    for i in range(n_seg):
        tris.append((0, vid(1, i), vid(1, i + 1)))
    for j in range(1, n_rings):
        for i in range(n_seg):
            a, b = vid(j, i), vid(j + 1, i)
            c, d = vid(j + 1, i + 1), vid(j, i + 1)
            tris.append((a, b, c))
            tris.append((a, c, d))
    tri = np.asarray(tris, dtype=np.int32)
    loop = np.asarray([vid(n_rings, i) for i in range(n_seg)], dtype=np.int32)
    return Mesh(xy=xy, tri=tri, loops=[loop], name=f"disk_r{n_rings}_s{n_seg}",
                meta={"n_rings": n_rings, "n_seg": n_seg})


def draw_obstacles(rng: SplitMix64, N: int, count: int, wmin: int, wmax: int,
                   square: bool, max_tries: int = 100000):
    """Seeded non-overlapping obstacle blocks (i0, j0, w, h) in whole cells.

    Each block keeps at least one free cell between itself and the outer
    boundary and between itself and every other block, so that all boundary
    loops stay vertex-disjoint.  Overlapping draws are rejected and redrawn.
    """
    blocks = []
    tries = 0
    while len(blocks) < count:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("could not place obstacles")
        w = rng.randint(wmin, wmax)
        h = w if square else rng.randint(wmin, wmax)
        if w + 2 > N or h + 2 > N:
            continue
        i0 = rng.randint(1, N - 1 - w)
        j0 = rng.randint(1, N - 1 - h)
        ok = True
        for (a0, b0, aw, ah) in blocks:
            # dilate the new block by one cell; it must not touch an existing block
            if i0 - 1 < a0 + aw and a0 < i0 + w + 1 and j0 - 1 < b0 + ah and b0 < j0 + h + 1:
                ok = False
                break
        if ok:
            blocks.append((i0, j0, w, h))
    return blocks


def grid_obstacles(N: int, blocks) -> Mesh:
    """Unit-square grid with N x N cells, diagonal split, minus obstacle blocks."""
    inside = np.zeros((N + 1, N + 1), dtype=bool)      # vertex strictly inside a block
    cell_free = np.ones((N, N), dtype=bool)            # [j, i]
    for (i0, j0, w, h) in blocks:
        inside[j0 + 1:j0 + h, i0 + 1:i0 + w] = True
        cell_free[j0:j0 + h, i0:i0 + w] = False
    ids = -np.ones((N + 1, N + 1), dtype=np.int64)
    keep = ~inside
    ids[keep] = np.arange(int(keep.sum()))
    jj, ii = np.nonzero(keep)
    hstep = 1.0 / N
    xy = np.stack([ii * hstep, jj * hstep], axis=1).astype(np.float64)
    cj, ci = np.nonzero(cell_free)
    v00 = ids[cj, ci]
    v10 = ids[cj, ci + 1]
    v11 = ids[cj + 1, ci + 1]
    v01 = ids[cj + 1, ci]
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tri = np.empty((2 * len(cj), 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    outer = []
    for i in range(0, N):
        outer.append(ids[0, i])
    for j in range(0, N):
        outer.append(ids[j, N])
    for i in range(N, 0, -1):
        outer.append(ids[N, i])
    for j in range(N, 0, -1):
        outer.append(ids[j, 0])
    loops = [np.asarray(outer, dtype=np.int32)]
    for (i0, j0, w, h) in blocks:
        l = []
        for j in range(j0, j0 + h):           # up the left side
            l.append(ids[j, i0])
        for i in range(i0, i0 + w):           # right along the top
            l.append(ids[j0 + h, i])
        for j in range(j0 + h, j0, -1):       # down the right side
            l.append(ids[j, i0 + w])
        for i in range(i0 + w, i0, -1):       # left along the bottom
            l.append(ids[j0, i])
        loops.append(np.asarray(l, dtype=np.int32))
    return Mesh(xy=xy, tri=tri, loops=loops, name=f"grid_N{N}_o{len(blocks)}",
                meta={"N": N, "blocks": list(blocks), "ids": ids})


def cell_domain(free: np.ndarray, h: float, name: str = "cells", meta=None) -> Mesh:
    """Mesh of the union of the free cells free[j, i] (cell (i, j) spans
    [i h, (i+1) h] x [j h, (j+1) h]), each split on its (i, j) -> (i+1, j+1)
    diagonal.  Boundary loops follow the cell edges with the domain on their
    left (outer loop counter-clockwise and first, holes clockwise).  Cells
    that touch only at a corner would pinch the boundary and are rejected."""
    free = np.asarray(free, dtype=bool)
    H, W = free.shape
    used = np.zeros((H + 1, W + 1), dtype=bool)
    cj, ci = np.nonzero(free)
    for dj in (0, 1):
        for di in (0, 1):
            used[cj + dj, ci + di] = True
    ids = -np.ones((H + 1, W + 1), dtype=np.int64)
    ids[used] = np.arange(int(used.sum()))
    jj, ii = np.nonzero(used)
    xy = np.stack([ii * h, jj * h], axis=1).astype(np.float64)
    v00, v10, v11, v01 = ids[cj, ci], ids[cj, ci + 1], ids[cj + 1, ci + 1], ids[cj + 1, ci]
    tri = np.empty((2 * len(cj), 3), dtype=np.int32)
    tri[0::2] = np.stack([v00, v10, v11], axis=1)
    tri[1::2] = np.stack([v00, v11, v01], axis=1)

    def is_free(j, i):
        return 0 <= j < H and 0 <= i < W and free[j, i]

    nxt = {}                                     # directed boundary edges, domain on the left
    for j, i in zip(cj.tolist(), ci.tolist()):
        sides = (((j - 1, i), (j, i), (j, i + 1)),            # bottom: (i, j) -> (i+1, j)
                 ((j, i + 1), (j, i + 1), (j + 1, i + 1)),    # right
                 ((j + 1, i), (j + 1, i + 1), (j + 1, i)),    # top
                 ((j, i - 1), (j + 1, i), (j, i)))            # left
        for (nj, ni), a, b in sides:
            if not is_free(nj, ni):
                u, v = int(ids[a]), int(ids[b])
                if u in nxt:
                    raise ValueError("cells touching at a corner pinch the boundary")
                nxt[u] = v
    loops, seen = [], set()
    for start in sorted(nxt):
        if start in seen:
            continue
        loop, u = [], start
        while u not in seen:
            seen.add(u)
            loop.append(u)
            u = nxt[u]
        loops.append(np.asarray(loop, dtype=np.int32))

    def area2(l):
        p = xy[l]
        return float(np.sum(p[:, 0] * np.roll(p[:, 1], -1) - np.roll(p[:, 0], -1) * p[:, 1]))

    loops.sort(key=lambda l: -area2(l))          # the one counter-clockwise loop first
    return Mesh(xy=xy, tri=tri, loops=loops, name=name, meta=dict(meta or {}, ids=ids))


def serpentine(n_corr: int, corr_w: int, corr_len: int) -> Mesh:
    """A winding corridor: n_corr vertical corridors of corr_w x corr_len cells,
    joined at alternate ends through corr_w-wide gaps in the one-cell walls
    between them (each wall hangs from the bottom or the top edge).  The
    path from one end to the other is about n_corr (corr_len + 1) cells long,
    so harmonic measures across it fall by about exp(-pi L / w) for a path of
    length L in corridors of width w."""
    W = n_corr * corr_w + (n_corr - 1)
    Hc = corr_len
    free = np.ones((Hc, W), dtype=bool)
    for c in range(n_corr - 1):
        x = c * (corr_w + 1) + corr_w
        if c % 2 == 0:
            free[:Hc - corr_w, x] = False        # wall from the bottom, gap at the top
        else:
            free[corr_w:, x] = False             # wall from the top, gap at the bottom
    return cell_domain(free, 1.0 / max(W, Hc), name=f"serpentine_{n_corr}x{corr_w}x{corr_len}",
                       meta={"n_corr": n_corr, "corr_w": corr_w, "corr_len": corr_len, "N": max(W, Hc)})


def strip(w: int, length: int) -> Mesh:
    """A straight corridor of w x length cells (cell side 1 / length)."""
    return cell_domain(np.ones((w, length), dtype=bool), 1.0 / length, name=f"strip_{w}x{length}",
                       meta={"w": w, "length": length, "N": length})


def snap_to_vertex(xy: np.ndarray, p) -> int:
    """Nearest vertex to point p; ties go to the lowest vertex id."""
    d2 = (xy[:, 0] - p[0]) ** 2 + (xy[:, 1] - p[1]) ** 2
    return int(np.argmin(d2))


def _polygon_contains(poly: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Points strictly inside a counter-clockwise convex polygon."""
    inside = np.ones(len(pts), dtype=bool)
    for a in range(len(poly)):
        p0, p1 = poly[a], poly[(a + 1) % len(poly)]
        e = p1 - p0
        inside &= e[0] * (pts[:, 1] - p0[1]) - e[1] * (pts[:, 0] - p0[0]) > 0.0
    return inside


def _polygon_distance(poly: np.ndarray, pts: np.ndarray) -> np.ndarray:
    """Distance from each point to the polygon's boundary."""
    d = np.full(len(pts), np.inf)
    for a in range(len(poly)):
        p0, p1 = poly[a], poly[(a + 1) % len(poly)]
        e = p1 - p0
        s = np.clip(((pts - p0) @ e) / (e @ e), 0.0, 1.0)
        d = np.minimum(d, np.linalg.norm(pts - p0 - s[:, None] * e, axis=1))
    return d


def convex_holes(n_goal: int = 175, n_holes: int = 4, seed: int = 1) -> Mesh:
    """Unit disk minus convex polygonal holes, Delaunay-meshed with about n_goal vertices.

    Spacing h is chosen so that the lattice points (free area over the
    hexagonal cell area sqrt(3)/2 h^2) plus the boundary points (perimeter
    over h) come to about n_goal vertices.  Holes are
    regular 3- to 5-gons of circumradius 0.08..0.18, kept 0.1 from the outer
    circle and 0.12 from each other; they are drawn before h is used, so one
    seed gives the same domain at every resolution.  Outer-circle points are spaced at most h apart (along the
    arc); every hole edge is cut into pieces of length <= h.  Lattice points are jittered by up to
    0.2 h and dropped within 0.6 h of any boundary, so that the diametral
    circle of every boundary segment is empty and each boundary segment is a
    Delaunay edge (checked).  Triangles whose centroid falls in a hole are
    removed.  Needs scipy (Qhull) for the triangulation.
    """
    from scipy.spatial import Delaunay

    rng = SplitMix64(seed)
    # n_goal ~ A / (sqrt(3)/2 h^2) + perimeter / h with A ~ 0.8 pi and a
    # perimeter ~ 2 pi + 2.5 (circle plus holes): solve the quadratic for h
    c2 = math.sqrt(3.0) / 2.0 * n_goal
    per, area = 2.0 * math.pi + 2.5, 0.8 * math.pi
    h = (per + math.sqrt(per * per + 4.0 * c2 * area)) / (2.0 * c2)
    holes = []
    tries = 0
    while len(holes) < n_holes:
        tries += 1
        if tries > 100000:
            raise RuntimeError("could not place holes")
        r = 0.6 * math.sqrt(rng.uniform())
        th = 2.0 * math.pi * rng.uniform()
        c = (r * math.cos(th), r * math.sin(th))
        rad = 0.08 + 0.10 * rng.uniform()
        sides = rng.randint(3, 5)
        rot = 2.0 * math.pi * rng.uniform()
        if math.hypot(*c) + rad > 0.9:
            continue
        if any(math.hypot(c[0] - d[0], c[1] - d[1]) < rad + e + 0.12 for d, e, _ in holes):
            continue
        poly = np.array([(c[0] + rad * math.cos(rot + 2.0 * math.pi * i / sides),
                          c[1] + rad * math.sin(rot + 2.0 * math.pi * i / sides)) for i in range(sides)])
        holes.append((c, rad, poly))

    pts = []
    loops = []

    def add_loop(loop_pts, reverse):
        ids = list(range(len(pts), len(pts) + len(loop_pts)))
        pts.extend(loop_pts)
        if reverse:          # a hole is walked clockwise: the domain on the left
            ids = ids[:1] + ids[1:][::-1]
        loops.append(np.asarray(ids, dtype=np.int32))

    # the outer circle: points on the circle itself (a point on a chord would
    # lie on the convex hull's edge and drop out of the triangulation)
    n_out = max(8, int(math.ceil(2.0 * math.pi / h)))
    add_loop([np.array((math.cos(2.0 * math.pi * i / n_out), math.sin(2.0 * math.pi * i / n_out)))
              for i in range(n_out)], False)
    for _, _, poly in holes:
        walk = []
        for a in range(len(poly)):
            p0, p1 = poly[a], poly[(a + 1) % len(poly)]
            pieces = max(1, int(math.ceil(np.linalg.norm(p1 - p0) / h)))
            walk.extend(p0 + (p1 - p0) * (s / pieces) for s in range(pieces))
        add_loop(walk, True)

    dy = h * math.sqrt(3.0) / 2.0
    rows = int(math.ceil(1.0 / dy)) + 1
    cols = int(math.ceil(1.0 / h)) + 1
    lattice = []
    for j in range(-rows, rows + 1):
        for i in range(-cols, cols + 1):
            jx = (2.0 * rng.uniform() - 1.0) * 0.2 * h
            jy = (2.0 * rng.uniform() - 1.0) * 0.2 * h
            lattice.append((i * h + (0.5 * h if j & 1 else 0.0) + jx, j * dy + jy))
    lattice = np.asarray(lattice)
    keep = np.hypot(lattice[:, 0], lattice[:, 1]) < 1.0 - 0.6 * h
    for _, _, poly in holes:
        keep &= ~_polygon_contains(poly, lattice) & (_polygon_distance(poly, lattice) >= 0.6 * h)
    xy = np.concatenate([np.asarray(pts), lattice[keep]])

    tri = Delaunay(xy).simplices.astype(np.int32)
    cen = xy[tri].mean(axis=1)
    drop = np.zeros(len(tri), dtype=bool)
    for _, _, poly in holes:
        drop |= _polygon_contains(poly, cen)
    tri = tri[~drop]
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    cw = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]) < 0.0
    tri[cw] = tri[cw][:, [0, 2, 1]]
    edges = {(min(u, v), max(u, v)) for t in tri.tolist() for u, v in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0]))}
    for l in loops:
        for u, v in zip(l.tolist(), np.roll(l, -1).tolist()):
            if (min(u, v), max(u, v)) not in edges:
                raise RuntimeError("a boundary segment is not a Delaunay edge")
    return Mesh(xy=xy, tri=tri, loops=loops, name=f"holes{n_goal}_s{seed}",
                meta={"n_goal": n_goal, "h": h, "holes": [(c, rad, len(p)) for c, rad, p in holes]})
