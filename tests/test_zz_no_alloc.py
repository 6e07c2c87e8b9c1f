"""dd_distance_noalloc against dd_distance and the oracle, through the C ABI (GPU).

The no-allocation entry point is for callers that may not call cudaMalloc,
such as a robot's real-time control loop that allocates only at start-up or
a plugin whose host framework owns all device memory.  It must give the same
fields as the regular entry point, bit for bit, and those fields must meet
the FP32 tolerance against the FP64 oracle.  Two calls in a row -- two
targets (the streaming kernel), then 67 (the tile kernel and the exact
recompute) -- check that the shared fixed scratch array is reused correctly.
A target id out of range and misaligned pointers are refused with DD_EINVAL,
and a call after a refused one is correct again.  This file is collected
last.
"""
import numpy as np
import pytest

from oracle.divergence import kl_field_fast, tv_field
from oracle.poisson import PoissonOracle
from synthetic import workloads
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_matches_dd_distance_and_oracle():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    try:
        wl = workloads.small_grid(37, 3, T=70, S=1, seed=777)
        mesh = wl.mesh
        po = PoissonOracle(mesh.xy, mesh.tri, mesh.loops)
        P64 = po.full()
        mid = load(dd, ctx, mesh)
        dd.dd_set_poisson_kernel(ctx, mid, P64)          # the device stores the oracle's kernel in FP32
        info = dd.dd_mesh_info(ctx, mid)
        n_v, k, k_pad = info["n_v"], info["k"], info["k_pad"]
        P = torch.zeros((n_v, k), dtype=torch.float32, device="cuda")
        dd.dd_get_poisson_kernel(ctx, mid, P)
        dd.dd_sync(ctx)
        Pp = torch.zeros((n_v, k_pad), dtype=torch.float32, device="cuda")
        Pp[:, :k] = P
        stream = torch.cuda.current_stream().cuda_stream
        mask = dd.DD_F_KL | dd.DD_F_TV

        def both(targets):
            T = len(targets)
            ref = torch.empty((2, T, n_v), dtype=torch.float32, device="cuda")
            dd.dd_distance(ctx, mid, targets, mask, dd.DD_PREC_FP32, ref)
            dd.dd_sync(ctx)
            dt = torch.as_tensor(np.asarray(targets, dtype=np.int32), device="cuda")
            got = torch.full((2, T, n_v), float("nan"), dtype=torch.float32, device="cuda")
            dd.dd_distance_noalloc(Pp, n_v, k_pad, dt, T, mask, got, stream)
            return got.cpu().numpy(), ref.cpu().numpy()

        for targets in (wl.targets[:2], wl.targets[3:70]):      # streaming kernel, then tile kernel
            g, r = both(targets)
            assert np.array_equal(g, r)                         # the same arithmetic, bit for bit
            for a, t in enumerate(targets):
                assert field_error(g[0, a], kl_field_fast(P64, P64[t])) <= TOL_FP32
                assert field_error(g[1, a], tv_field(P64, P64[t])) <= TOL_FP32
                assert g[0, a, t] == 0.0 and g[1, a, t] == 0.0

        out = torch.empty((2, 3, n_v), dtype=torch.float32, device="cuda")
        for bad in ([int(wl.targets[0]), n_v, int(wl.targets[1])], [-1, int(wl.targets[0]), int(wl.targets[1])]):
            dt = torch.as_tensor(np.asarray(bad, dtype=np.int32), device="cuda")
            with pytest.raises(dd.DDError):                     # detected on the device, never read
                dd.dd_distance_noalloc(Pp, n_v, k_pad, dt, 3, mask, out, stream)
        dt = torch.as_tensor(np.asarray(wl.targets[:3], dtype=np.int32), device="cuda")
        with pytest.raises(dd.DDError):                         # P not 16-byte aligned
            flat = Pp.reshape(-1)
            dd.dd_distance_noalloc(flat[1:], n_v, k_pad, dt, 3, mask, out, stream)
        with pytest.raises(dd.DDError):                         # beyond the fixed scratch
            big = torch.zeros(300, dtype=torch.int32, device="cuda")
            dd.dd_distance_noalloc(Pp, n_v, 4096, big, 300, 1, out, stream)
        g, r = both(wl.targets[:3])                             # a good call after the refused ones
        assert np.array_equal(g, r)
    finally:
        dd.dd_destroy(ctx)
