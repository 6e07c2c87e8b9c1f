"""Helpers for the GPU parity tests (call libdd through its C ABI)."""
import numpy as np

FLOOR_FP32 = 1e-2      # relative-error floor of the FP32 field path
TOL_FP32 = 1e-5        # relative tolerance of the FP32 field path


def ctx_and_lib():
    import torch
    from paper_1708_02845_gb300.build import build
    build()
    from paper_1708_02845_gb300 import dd
    ctx = dd.dd_create(0, torch.cuda.current_stream().cuda_stream)
    return dd, ctx


def load(dd, ctx, mesh):
    idx, off = mesh.loop_arrays()
    return dd.dd_load_mesh(ctx, mesh.xy, mesh.tri, idx, off)


def field_error(got, ref, floor=FLOOR_FP32):
    """max |g - r| / max(|r|, floor) over entries where the reference is finite."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    fin = np.isfinite(ref)
    return float(np.max(np.abs(got[fin] - ref[fin]) / np.maximum(np.abs(ref[fin]), floor)))


def mean_edge(mesh):
    e = np.concatenate([mesh.tri[:, [0, 1]], mesh.tri[:, [1, 2]], mesh.tri[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.mean(np.hypot(*(mesh.xy[e[:, 0]] - mesh.xy[e[:, 1]]).T)))
