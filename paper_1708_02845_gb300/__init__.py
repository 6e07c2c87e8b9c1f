"""Divergence-distance path planning on GB300 (sm_103a).

Chen, Gotsman & Hormann, "Path Planning with Divergence-Based Distance
Functions": the Poisson kernel of a triangulated planar domain (Eq. 32-33),
the TV and KL divergence fields of a target (Eq. 34-35) and triangle-walking
gradient-descent paths (Section IV).  The work runs in libdd.so (CUDA C ABI,
include/dd.h); `paper_1708_02845_gb300.dd` is its ctypes binding and
`paper_1708_02845_gb300.build` compiles it.
"""

__version__ = "0.1.0"
