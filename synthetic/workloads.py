"""Seeded synthetic workloads: meshes plus target and source vertex draws.

Base seed 170802845 (the paper's arXiv number); workload i uses base + i.
Point-valued targets and sources are snapped to their nearest vertex (ties to
the lowest id); a source that snaps onto the target or onto a boundary vertex
is redrawn.  Targets are always interior vertices (a boundary target has an
infinite KL row, Section IV, Eq. 33).

Workloads (sizes follow the paper's range of domains, Tables I-II, widened):
  disk        16 rings x 128 segments (n = 2,049, k = 128); target nearest
              (0.3, 0.2); 32 sources r = 0.95*sqrt(u), theta = 2*pi*v.
  grid140     h = 1/140, 8 square obstacles of side 7..21 cells;
              64 interior targets; 256 interior sources per target.
  grid450     h = 1/450, 24 rectangles with sides 9..36 cells; 1024 targets.
  batch64     64 grids, n log-uniform in [5k, 100k], 0..16 obstacles each,
              16..256 targets per domain, 64 sources per target.
  serving     8 grids, n log-uniform in [10k, 500k]; query draws.
"""

import math
from dataclasses import dataclass, field

import numpy as np

from .meshes import Mesh, disk_rings, draw_obstacles, grid_obstacles, snap_to_vertex
from .rng import SplitMix64

BASE_SEED = 170802845


@dataclass
class Workload:
    name: str
    mesh: Mesh
    targets: np.ndarray                  # int32 [T]
    sources: np.ndarray                  # int32 [T, S]
    meta: dict = field(default_factory=dict)


def _interior_ids(mesh: Mesh) -> np.ndarray:
    return np.nonzero(~mesh.boundary_flags())[0].astype(np.int32)


def draw_targets(rng: SplitMix64, mesh: Mesh, T: int) -> np.ndarray:
    interior = _interior_ids(mesh)
    return np.asarray([interior[rng.choice(len(interior))] for _ in range(T)], dtype=np.int32)


def draw_sources(rng: SplitMix64, mesh: Mesh, targets: np.ndarray, S: int) -> np.ndarray:
    interior = _interior_ids(mesh)
    out = np.empty((len(targets), S), dtype=np.int32)
    for a, t in enumerate(targets):
        for s in range(S):
            while True:
                v = interior[rng.choice(len(interior))]
                if v != t:
                    break
            out[a, s] = v
    return out


def disk(n_rings: int = 16, n_seg: int = 128, n_sources: int = 32, seed: int = BASE_SEED + 0) -> Workload:
    mesh = disk_rings(n_rings, n_seg)
    rng = SplitMix64(seed)
    bflag = mesh.boundary_flags()
    t = snap_to_vertex(mesh.xy, (0.3, 0.2))
    src = []
    while len(src) < n_sources:
        r = 0.95 * math.sqrt(rng.uniform())
        th = 2.0 * math.pi * rng.uniform()
        v = snap_to_vertex(mesh.xy, (r * math.cos(th), r * math.sin(th)))
        if v == t or bflag[v]:
            continue
        src.append(v)
    return Workload("disk", mesh, np.asarray([t], dtype=np.int32),
                    np.asarray([src], dtype=np.int32),
                    meta={"target_point": (0.3, 0.2)})


def grid(N: int, n_obst: int, wmin: int, wmax: int, square: bool, T: int, S: int,
         seed: int, name: str) -> Workload:
    rng = SplitMix64(seed)
    blocks = draw_obstacles(rng, N, n_obst, wmin, wmax, square)
    mesh = grid_obstacles(N, blocks)
    targets = draw_targets(rng, mesh, T)
    sources = draw_sources(rng, mesh, targets, S) if S > 0 else np.zeros((T, 0), np.int32)
    return Workload(name, mesh, targets, sources, meta={"N": N, "blocks": blocks})


def grid140(T: int = 64, S: int = 256) -> Workload:
    """h = 1/140 with 8 square obstacles (side 0.05..0.15 = 7..21 cells)."""
    return grid(140, 8, 7, 21, True, T, S, BASE_SEED + 1, "grid140")


def grid450(T: int = 1024, S: int = 0) -> Workload:
    """h = 1/450 with 24 rectangular obstacles (sides 9..36 cells)."""
    return grid(450, 24, 9, 36, False, T, S, BASE_SEED + 2, "grid450")


def small_grid(N: int = 24, n_obst: int = 2, T: int = 4, S: int = 8, seed: int = BASE_SEED + 100) -> Workload:
    """Small grid with obstacles for fast tests (several tiles, ragged k)."""
    wmax = max(2, N // 6)
    return grid(N, n_obst, 2, wmax, False, T, S, seed, f"grid{N}")


def batch64(n_domains: int = 64, seed: int = BASE_SEED + 3, S: int = 64):
    """Uneven domains: n log-uniform in [5k, 100k], 0..16 obstacles, 16..256 targets."""
    rng = SplitMix64(seed)
    out = []
    for d in range(n_domains):
        n_goal = math.exp(math.log(5e3) + rng.uniform() * (math.log(1e5) - math.log(5e3)))
        N = max(16, int(round(math.sqrt(n_goal))) - 1)
        n_obst = rng.randint(0, 16)
        wmax = max(3, N // 10)
        wmin = max(2, N // 40)
        T = rng.randint(16, 256)
        sub_seed = rng.next_u64()
        out.append(grid(N, n_obst, wmin, wmax, False, T, S, sub_seed, f"batch{d}"))
    return out


def serving_domains(n_domains: int = 8, seed: int = BASE_SEED + 4):
    """Resident domains for the serving loop: n log-uniform in [10k, 500k]."""
    rng = SplitMix64(seed)
    out = []
    for d in range(n_domains):
        n_goal = math.exp(math.log(1e4) + rng.uniform() * (math.log(5e5) - math.log(1e4)))
        N = max(32, int(round(math.sqrt(n_goal))) - 1)
        n_obst = rng.randint(0, 16)
        wmax = max(3, N // 12)
        wmin = max(2, N // 50)
        sub_seed = rng.next_u64()
        out.append(grid(N, n_obst, wmin, wmax, False, 0, 0, sub_seed, f"serve{d}"))
    return out


def serving_queries(domains, rate_qps: float = 2000.0, duration_s: float = 10.0,
                    seed: int = BASE_SEED + 5):
    """Poisson arrivals; each query = (time, domain, interior target, S log-uniform in [1, 1024])."""
    rng = SplitMix64(seed)
    q = []
    tnow = 0.0
    while True:
        tnow += -math.log(1.0 - rng.uniform()) / rate_qps
        if tnow >= duration_s:
            break
        d = rng.choice(len(domains))
        mesh = domains[d].mesh
        interior = _interior_ids(mesh)
        t = int(interior[rng.choice(len(interior))])
        S = max(1, min(1024, int(math.floor(math.exp(rng.uniform() * math.log(1024.0))))))
        srcs = []
        for _ in range(S):
            while True:
                v = int(interior[rng.choice(len(interior))])
                if v != t:
                    break
            srcs.append(v)
        q.append((tnow, d, t, np.asarray(srcs, dtype=np.int32)))
    return q
