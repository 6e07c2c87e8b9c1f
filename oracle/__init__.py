"""FP64 CPU oracle for the divergence-distance hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously correct restatements of what the paper computes, each
function citing its passage (Chen, Gotsman & Hormann, "Path Planning with
Divergence-Based Distance Functions"):

  topology.py    boundary/interior split of a triangle mesh (Section IV)
  laplacian.py   cotangent Laplacian L^c and its A- and Z-scaled variants (Section IV)
  poisson.py     discrete Poisson kernel P = [-L_II^-1 L_IB ; I] (Eq. 32-33)
  divergence.py  TV and KL fields (Eq. 34-35, with Eq. 16-17 for the direction)
  trace.py       triangle-based gradient-descent path tracing (Section IV)
  greens.py      Dirichlet Green's function column D_Ip (Eq. 21), for path agreement
  hausdorff.py   Hausdorff distance between polylines

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  It shares no code with the CUDA library and never calls
it; the product path does not fall back to it.
"""
