"""Small hand-built meshes for oracle pins (test helpers, no method arithmetic)."""
import math

import numpy as np

from synthetic.meshes import Mesh, grid_obstacles


def plain_grid(N: int) -> Mesh:
    return grid_obstacles(N, [])


def hexagon() -> Mesh:
    """Regular hexagon of six equilateral triangles around a centre vertex."""
    xy = [(0.0, 0.0)] + [(math.cos(math.pi / 3 * i), math.sin(math.pi / 3 * i)) for i in range(6)]
    tri = [(0, 1 + i, 1 + (i + 1) % 6) for i in range(6)]
    return Mesh(np.asarray(xy), np.asarray(tri, dtype=np.int32), [np.arange(1, 7, dtype=np.int32)], "hexagon")


def random_delaunay_disk(n_rings: int, n_seg: int) -> Mesh:
    from synthetic.meshes import disk_rings
    return disk_rings(n_rings, n_seg)
