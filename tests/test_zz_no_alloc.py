"""dd_distance_noalloc against dd_distance, through the C ABI (GPU).

The no-allocation entry point is for callers that may not call cudaMalloc,
such as a robot's real-time control loop that allocates only at start-up or
a plugin whose host framework owns all device memory.  It must give the same
fields as the regular entry point; two calls in a row check that the shared
fixed scratch array is reused correctly.  This file is collected last.
"""
import numpy as np
import pytest

from synthetic import workloads
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_dd_distance():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    try:
        wl = workloads.small_grid(37, 3, T=70, S=1, seed=777)
        mesh = wl.mesh
        mid = load(dd, ctx, mesh)
        dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
        info = dd.dd_mesh_info(ctx, mid)
        n_v, k, k_pad = info["n_v"], info["k"], info["k_pad"]
        P = torch.zeros((n_v, k), dtype=torch.float32, device="cuda")
        dd.dd_get_poisson_kernel(ctx, mid, P)
        dd.dd_sync(ctx)
        Pp = torch.zeros((n_v, k_pad), dtype=torch.float32, device="cuda")
        Pp[:, :k] = P
        stream = torch.cuda.current_stream().cuda_stream
        for targets in (wl.targets[:3], wl.targets[3:70]):      # stream kernel, then tile kernel
            T = len(targets)
            ref = torch.empty((2, T, n_v), dtype=torch.float32, device="cuda")
            dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, ref)
            dd.dd_sync(ctx)
            dt = torch.as_tensor(np.asarray(targets, dtype=np.int32), device="cuda")
            got = torch.full((2, T, n_v), float("nan"), dtype=torch.float32, device="cuda")
            dd.dd_distance_noalloc(Pp, n_v, k_pad, dt, T, dd.DD_F_KL | dd.DD_F_TV, got, stream)
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            for a in range(T):
                assert field_error(g[0, a], r[0, a]) <= TOL_FP32
                assert field_error(g[1, a], r[1, a]) <= TOL_FP32
        with pytest.raises(dd.DDError):
            big = torch.zeros(300, dtype=torch.int32, device="cuda")
            dd.dd_distance_noalloc(Pp, n_v, 4096, big, 300, 1, got, stream)
    finally:
        dd.dd_destroy(ctx)
