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


def snap_to_vertex(xy: np.ndarray, p) -> int:
    """Nearest vertex to point p; ties go to the lowest vertex id."""
    d2 = (xy[:, 0] - p[0]) ** 2 + (xy[:, 1] - p[1]) ** 2
    return int(np.argmin(d2))
