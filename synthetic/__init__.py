"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

Holds random draws and mesh generators only; none of the divergence-distance
arithmetic lives here.
"""
from .rng import SplitMix64
from .meshes import Mesh, disk_rings, grid_obstacles, draw_obstacles, snap_to_vertex
from . import workloads
