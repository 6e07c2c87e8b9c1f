"""GPU parity of libdd against the FP64 oracle, through the C ABI.

Tolerances: Poisson kernel entries within the FP32 rounding of the oracle's
value plus 1e-12 (solver); fields |g - r| / max(|r|, 1e-2) <= 1e-5 (FP32
path) with D(t, t) = 0 exactly; traced paths within half a mean edge length
(Hausdorff) of the oracle's paths with identical status codes.
"""
import math

import numpy as np
import pytest

from oracle.divergence import kl_field_fast, tv_field
from oracle.hausdorff import hausdorff
from oracle.poisson import PoissonOracle
from oracle.trace import Tracer
from synthetic import workloads
from synthetic.meshes import grid_obstacles
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load, mean_edge

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    yield dd, ctx
    dd.dd_destroy(ctx)


CASES = {
    "disk": lambda: workloads.disk(),
    "grid24": lambda: workloads.small_grid(24, 2, T=5, S=8),
    "grid37": lambda: workloads.small_grid(37, 3, T=70, S=4, seed=777),
    "grid140": lambda: workloads.grid140(T=8, S=32),
}

_cache = {}


def case(name):
    if name not in _cache:
        wl = CASES[name]()
        po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
        _cache[name] = (wl, po, po.full())
    return _cache[name]


@pytest.mark.parametrize("name", list(CASES))
def test_poisson_kernel_matches_oracle(env, name):
    dd, ctx = env
    wl, po, P = case(name)
    mid = load(dd, ctx, wl.mesh)
    iters, resid = dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    assert resid <= 1e-15
    got = np.empty((wl.mesh.n_v, po.k), dtype=np.float32)
    dd.dd_get_poisson_kernel(ctx, mid, got)
    ref32 = np.where(P < np.finfo(np.float32).tiny, 0.0, P)
    err = np.abs(got.astype(np.float64) - ref32)
    assert np.all(err <= 1.2e-7 * np.abs(ref32) + 1e-12), float((err - 1.2e-7 * np.abs(ref32)).max())
    assert np.abs(got.astype(np.float64).sum(axis=1) - 1.0).max() < 1e-5
    dd.dd_unload_mesh(ctx, mid)


def _fields(dd, ctx, mid, n_v, targets, host=False):
    T = len(targets)
    if host:
        out = np.empty((2, T, n_v), dtype=np.float32)
        dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, out)
        return out
    out = torch.empty((2, T, n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, out)
    dd.dd_sync(ctx)
    return out.cpu().numpy()


@pytest.mark.parametrize("name,T", [("disk", 1), ("grid24", 1), ("grid24", 2), ("grid24", 5),
                                    ("grid37", 3), ("grid37", 70), ("grid140", 1), ("grid140", 2),
                                    ("grid140", 8)])
def test_fields_on_oracle_kernel(env, name, T):
    """Field kernels alone: the oracle's P installed, fields vs the oracle's fields."""
    dd, ctx = env
    wl, po, P = case(name)
    targets = list(wl.targets[:T]) if len(wl.targets) >= T else [int(po.I[(i * 7919) % po.m]) for i in range(T)]
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    got = _fields(dd, ctx, mid, wl.mesh.n_v, targets)
    for a, t in enumerate(targets):
        ref_kl = kl_field_fast(P, P[t])
        ref_tv = tv_field(P, P[t])
        assert field_error(got[0, a], ref_kl) <= TOL_FP32
        assert field_error(got[1, a], ref_tv) <= TOL_FP32
        assert got[0, a, t] == 0.0 and got[1, a, t] == 0.0
        inf = ~np.isfinite(ref_kl)
        assert np.all(got[0, a][inf] >= 87.0)            # +inf rows: log argument clamped at FLT_MIN
        assert np.all(np.isfinite(got[:, a]))
    dd.dd_unload_mesh(ctx, mid)


def test_fast_log_spread(env):
    """The hardware mantissa log's error spread stays inside the bound the FP32
    streaming pass relies on (measured over all 2^23 mantissas)."""
    dd, _ = env
    spread = dd.dd_check_fast_log()
    assert 0.0 < spread <= dd.DD_FAST_LOG_SPREAD, spread


@pytest.mark.parametrize("name", ["disk", "grid140"])
def test_stream_pass_against_table_path(env, name):
    """One target (streaming kernel, hardware mantissa log with exact recompute
    of rows below DD_EXACT_BELOW) against the same target among three (tile
    kernel, one-number log2 first pass with exact recompute of pairs below
    DD_TILE_EXACT_BELOW): rows where both are exact agree to FP32 summation
    rounding, rows where one is exact within ln2 * DD_FAST_LOG_SPREAD plus
    rounding, the rest within the sum of both first passes' bounds."""
    dd, ctx = env
    wl, po, P = case(name)
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    n = wl.mesh.n_v
    for t in list(wl.targets[:4]):
        others = [int(po.I[(i * 7919) % po.m]) for i in (1, 2)]
        one = _fields(dd, ctx, mid, n, [t])
        three = _fields(dd, ctx, mid, n, [t] + others)
        kl1, kl3 = one[0, 0].astype(np.float64), three[0, 0].astype(np.float64)
        assert np.all(np.abs(one[1, 0] - three[1, 0]) <= 2e-6 * np.maximum(three[1, 0], 1.0))   # TV: summation order
        near = kl3 < dd.DD_EXACT_BELOW
        assert np.all(np.abs(kl1 - kl3)[near] <= 2e-6 * np.maximum(kl3[near], 1e-2))
        between = ~near & (kl3 < dd.DD_TILE_EXACT_BELOW)
        bound = math.log(2.0) * dd.DD_FAST_LOG_SPREAD + 1e-6 * kl3[between]
        assert np.all(np.abs(kl1 - kl3)[between] <= bound)
        far = (kl3 >= dd.DD_TILE_EXACT_BELOW) & np.isfinite(kl3)
        k = P.shape[1]
        bound = (2 * math.log(2.0) * dd.DD_FAST_LOG_SPREAD + 2.0 ** -24 * (2 * math.log(k) + 2 * kl3[far] + 2)
                 + 1e-6 * kl3[far])
        assert np.all(np.abs(kl1 - kl3)[far] <= bound)
        assert one[0, 0, t] == 0.0
    dd.dd_unload_mesh(ctx, mid)


@pytest.mark.parametrize("name", ["disk", "grid24", "grid140"])
def test_end_to_end_fields(env, name):
    """Poisson kernel by the device solver, then fields, vs the oracle."""
    dd, ctx = env
    wl, po, P = case(name)
    mid = load(dd, ctx, wl.mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    targets = list(wl.targets[:4])
    got = _fields(dd, ctx, mid, wl.mesh.n_v, targets, host=True)
    for a, t in enumerate(targets):
        assert field_error(got[0, a], kl_field_fast(P, P[t])) <= TOL_FP32
        assert field_error(got[1, a], tv_field(P, P[t])) <= TOL_FP32
    dd.dd_unload_mesh(ctx, mid)


@pytest.mark.parametrize("name,f", [("disk", "kl"), ("disk", "tv"), ("grid140", "kl"), ("grid24", "kl")])
def test_trace_parity(env, name, f):
    dd, ctx = env
    wl, po, P = case(name)
    mesh = wl.mesh
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    tr = Tracer(mesh.xy, mesh.tri)
    h = mean_edge(mesh)
    fbit = dd.DD_F_KL if f == "kl" else dd.DD_F_TV
    n_t = len(wl.targets)                     # every target of the case (grid140: 8 x 32 paths)
    for a in range(n_t):
        t = int(wl.targets[a])
        srcs = wl.sources[a]
        S, max_pts = len(srcs), 4096
        xy = np.zeros((S, max_pts, 2), dtype=np.float32)
        ln = np.zeros(S, dtype=np.int32)
        st = np.zeros(S, dtype=np.int32)
        dd.dd_trace(ctx, mid, t, fbit, srcs, max_pts, xy, ln, st)
        ref = kl_field_fast(P, P[t]) if f == "kl" else tv_field(P, P[t])
        for s, q in enumerate(srcs):
            path, status = tr.trace(ref, int(q), t, max_pts=max_pts)
            assert st[s] == status, (t, int(q), st[s], status)
            assert np.allclose(xy[s, 0], mesh.xy[q], atol=1e-6)
            if status == 0:
                assert np.allclose(xy[s, ln[s] - 1], mesh.xy[t], atol=1e-6)
            assert hausdorff(xy[s, :ln[s]], path, h / 10) <= 0.5 * h
    dd.dd_unload_mesh(ctx, mid)


def test_query_host_equals_device(env):
    dd, ctx = env
    wl, po, P = case("grid24")
    mesh = wl.mesh
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    T, S, mp = len(wl.targets), wl.sources.shape[1], 512
    hf = np.zeros((2, T, mesh.n_v), np.float32)
    hxy = np.zeros((T * S, mp, 2), np.float32)
    hl = np.zeros(T * S, np.int32)
    hs = np.zeros(T * S, np.int32)
    dd.dd_query(ctx, mid, wl.targets, wl.sources, 3, 0, dd.DD_F_KL, mp, hf, hxy, hl, hs)
    df = torch.zeros((2, T, mesh.n_v), dtype=torch.float32, device="cuda")
    dxy = torch.zeros((T * S, mp, 2), dtype=torch.float32, device="cuda")
    dl = torch.zeros(T * S, dtype=torch.int32, device="cuda")
    ds = torch.zeros(T * S, dtype=torch.int32, device="cuda")
    dd.dd_query(ctx, mid, wl.targets, wl.sources, 3, 0, dd.DD_F_KL, mp, df, dxy, dl, ds)
    dd.dd_sync(ctx)
    assert np.array_equal(hf, df.cpu().numpy())
    assert np.array_equal(hl, dl.cpu().numpy()) and np.array_equal(hs, ds.cpu().numpy())
    for i in range(T * S):
        assert np.array_equal(hxy[i, :hl[i]], dxy[i, :hl[i]].cpu().numpy())
    dd.dd_unload_mesh(ctx, mid)


def test_query_host_chunks_equal_device(env):
    """With host field buffers and many targets the fields are computed in
    chunks of targets, each chunk copied back while the next is computed:
    fields (pinned and pageable buffers), lengths, statuses and paths equal
    the device-buffer call's bit for bit."""
    dd, ctx = env
    wl = workloads.grid140(T=1, S=1)
    mesh = wl.mesh
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    interior = np.nonzero(~mesh.boundary_flags())[0]
    rng = np.random.default_rng(140300)
    T, S, mp = 300, 2, 1024
    targets = rng.choice(interior, T, replace=False).astype(np.int32)
    src = rng.choice(interior, (T, S)).astype(np.int32)
    df = torch.zeros((2, T, mesh.n_v), dtype=torch.float32, device="cuda")
    dxy = torch.zeros((T * S, mp, 2), dtype=torch.float32, device="cuda")
    dl = torch.zeros(T * S, dtype=torch.int32, device="cuda")
    ds = torch.zeros(T * S, dtype=torch.int32, device="cuda")
    dd.dd_query(ctx, mid, targets, src, 3, 0, dd.DD_F_KL, mp, df, dxy, dl, ds)
    dd.dd_sync(ctx)
    ref = df.cpu().numpy()
    for pinned in (True, False):
        hf = torch.zeros((2, T, mesh.n_v), dtype=torch.float32)
        if pinned:
            hf = hf.pin_memory()
        hxy = np.zeros((T * S, mp, 2), np.float32)
        hl = np.zeros(T * S, np.int32)
        hs = np.zeros(T * S, np.int32)
        dd.dd_query(ctx, mid, targets, src, 3, 0, dd.DD_F_KL, mp, hf.numpy(), hxy, hl, hs)
        assert np.array_equal(hf.numpy(), ref), pinned
        assert np.array_equal(hl, dl.cpu().numpy()) and np.array_equal(hs, ds.cpu().numpy())
        for i in range(0, T * S, 7):
            assert np.array_equal(hxy[i, :hl[i]], dxy[i, :hl[i]].cpu().numpy())
    dd.dd_unload_mesh(ctx, mid)


def test_errors(env):
    dd, ctx = env
    wl, po, P = case("grid24")
    mesh = wl.mesh
    mid = load(dd, ctx, mesh)
    out = torch.empty((1, 1, mesh.n_v), dtype=torch.float32, device="cuda")
    with pytest.raises(dd.DDError) as e:
        dd.dd_distance(ctx, mid, [int(wl.targets[0])], dd.DD_F_KL, 0, out)
    assert e.value.status == dd.DD_ESTATE
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    with pytest.raises(dd.DDError) as e:
        dd.dd_distance(ctx, mid, [int(po.B[0])], dd.DD_F_KL, 0, out)
    assert e.value.status == dd.DD_EINVAL
    with pytest.raises(dd.DDError) as e:
        dd.dd_distance(ctx, mid, [int(wl.targets[0])], 8, 0, out)      # no such field bit
    assert e.value.status == dd.DD_EINVAL
    with pytest.raises(dd.DDError) as e:
        dd.dd_distance(ctx, 99, [int(wl.targets[0])], 1, 0, out)
    assert e.value.status == dd.DD_EINVAL
    with pytest.raises(dd.DDError) as e:
        dd.dd_poisson_kernel(ctx, mid, 1e-30, 3)
    assert e.value.status == dd.DD_ENOTCONV
    dd.dd_unload_mesh(ctx, mid)


def test_every_tile_shape_bit_identical(env, monkeypatch):
    """The tile shapes sum every (row, target) in the same order (32-term
    chunks, compensated across 64-column partial sums), so their fields are
    bit-identical -- the three staged shapes and the pipelined shape on the
    tiled copy of P, for KL+TV, KL alone and TV alone, on 70 targets (a
    ragged second target tile) of a mesh whose row and column counts are not
    multiples of the tiles; they match the oracle.  Replacing P replaces the
    tiled copy: the pipelined shape then matches the oracle on the new P."""
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    targets = [int(t) for t in wl.targets]
    assert len(targets) > 64 and len(targets) % 64 and wl.mesh.n_v % 128

    def fields(shape, f_mask):
        monkeypatch.setenv("DD_TILE_SHAPE", str(shape))
        nf = 2 if f_mask == (dd.DD_F_KL | dd.DD_F_TV) else 1
        out = torch.empty((nf, len(targets), wl.mesh.n_v), dtype=torch.float32, device="cuda")
        dd.dd_distance(ctx, mid, targets, f_mask, dd.DD_PREC_FP32, out)
        dd.dd_sync(ctx)
        return out.cpu().numpy()

    for f_mask in (dd.DD_F_KL | dd.DD_F_TV, dd.DD_F_KL, dd.DD_F_TV):
        outs = [fields(shape, f_mask) for shape in range(4)]
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        if f_mask == (dd.DD_F_KL | dd.DD_F_TV):
            for a, t in enumerate(targets):
                assert field_error(outs[3][0, a], kl_field_fast(P, P[t])) <= TOL_FP32
                assert field_error(outs[3][1, a], tv_field(P, P[t])) <= TOL_FP32
                assert outs[3][0, a, t] == 0.0 and outs[3][1, a, t] == 0.0
    # a new P (rows still distributions): the tiled copy follows it
    P2 = 0.5 * (P + P[:, ::-1])
    dd.dd_set_poisson_kernel(ctx, mid, np.ascontiguousarray(P2))
    o = fields(3, dd.DD_F_KL | dd.DD_F_TV)
    monkeypatch.delenv("DD_TILE_SHAPE")
    for a, t in enumerate(targets[:8]):
        assert field_error(o[0, a], kl_field_fast(P2, P2[t])) <= TOL_FP32
        assert field_error(o[1, a], tv_field(P2, P2[t])) <= TOL_FP32
    dd.dd_unload_mesh(ctx, mid)


def test_more_targets_than_one_recompute_window(env):
    """1,100 targets (repeats included) on grid37: the exact recompute scans
    its row blocks' first-pass values in windows of 1,024 targets and stages
    the flagging targets in groups of 16, so this crosses a window and runs
    many groups; every field (KL and TV) matches the oracle's, and a repeated
    target gives identical rows."""
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    rng = np.random.default_rng(1100)
    pool = [int(t) for t in wl.targets]
    targets = [pool[i] for i in rng.integers(0, len(pool), 1100)]
    out = torch.empty((2, len(targets), wl.mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, out)
    dd.dd_sync(ctx)
    o = out.cpu().numpy()
    refs = {}
    for a, t in enumerate(targets):
        if t not in refs:
            refs[t] = (kl_field_fast(P, P[t]), tv_field(P, P[t]), a)
        kl, tv, first = refs[t]
        assert field_error(o[0, a], kl) <= TOL_FP32
        assert field_error(o[1, a], tv) <= TOL_FP32
        assert np.array_equal(o[:, a], o[:, first])
    dd.dd_unload_mesh(ctx, mid)


def test_load_latency_hook(env):
    """dd_load_latency: a dependent-load chase through a buffer that fits L2
    is faster than one through a buffer far larger than L2 (DRAM), both
    positive; sizes outside [4096, 2^32] or not a multiple of 128 are refused."""
    dd, ctx = env
    l2 = dd.dd_load_latency(ctx, 16 << 20, 20000)
    dram = dd.dd_load_latency(ctx, 1 << 30, 20000)
    assert 0.0 < l2 < dram
    for nbytes, steps in ((1000, 10), (4096 + 64, 10), ((1 << 32) + 128, 10), (4096, 0)):
        with pytest.raises(dd.DDError) as e:
            dd.dd_load_latency(ctx, nbytes, steps)
        assert e.value.status == dd.DD_EINVAL


def test_kernel_timing_hook(env):
    """dd_kernel_timing: per-kernel CUDA-event totals of the launches on the
    context's stream, one entry per kernel of a dd_query, none once disabled."""
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    targets = [int(t) for t in wl.targets[:8]]
    src = np.asarray(wl.sources)[:8]
    n = wl.mesh.n_v
    f = torch.empty((2, 8, n), dtype=torch.float32, device="cuda")
    xy = torch.empty((8 * src.shape[1], 512, 2), dtype=torch.float32, device="cuda")
    ln = torch.empty(8 * src.shape[1], dtype=torch.int32, device="cuda")
    st = torch.empty(8 * src.shape[1], dtype=torch.int32, device="cuda")
    dd.dd_query(ctx, mid, targets, src, 3, dd.DD_PREC_FP32, dd.DD_F_KL, 512, f, xy, ln, st)   # tunes once
    dd.dd_kernel_timing(ctx, 1)
    for _ in range(3):
        dd.dd_query(ctx, mid, targets, src, 3, dd.DD_PREC_FP32, dd.DD_F_KL, 512, f, xy, ln, st)
    got = dd.dd_kernel_timing(ctx, 0)
    for name in ("stage_targets_kernel", "field_tile_kernel", "fix_kl_kernel", "trace_kernel"):
        assert got[name][0] == 3 and got[name][1] > 0.0, (name, got)
    assert "rates_kernel" not in got        # few paths per field: the walk forms the rates it needs
    dd.dd_query(ctx, mid, targets, src, 3, dd.DD_PREC_FP32, dd.DD_F_KL, 512, f, xy, ln, st)
    assert dd.dd_kernel_timing(ctx, 2) == {}
    dd.dd_unload_mesh(ctx, mid)


def test_query_host_output_kinds(env):
    """dd_query into device memory, pinned host memory (paths moved by the copy
    kernel, also at a 4-byte-aligned offset) and pageable host memory: the
    same fields, lengths, statuses and path prefixes."""
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    targets = [int(t) for t in wl.targets[:6]]
    src = np.asarray(wl.sources)[:6]
    n, S, mp = wl.mesh.n_v, src.shape[1], 301            # odd max_pts: rows not 16-byte aligned

    def run(kind):
        if kind == "device":
            mk = lambda shape, dt: torch.empty(shape, dtype=dt, device="cuda")
        elif kind == "pageable":
            mk = lambda shape, dt: torch.empty(shape, dtype=dt)
        else:
            def mk(shape, dt, off=(kind == "pinned_offset")):
                flat = torch.empty(int(np.prod(shape)) + 1, dtype=dt).pin_memory()
                return flat[1:].view(shape) if off else flat[:-1].view(shape)
        f = mk((2, 6, n), torch.float32)
        xy = mk((6 * S, mp, 2), torch.float32)
        ln = mk((6 * S,), torch.int32)
        st = mk((6 * S,), torch.int32)
        dd.dd_query(ctx, mid, targets, src, 3, dd.DD_PREC_FP32, dd.DD_F_KL, mp, f, xy, ln, st)
        dd.dd_sync(ctx)
        return f.cpu().numpy(), xy.cpu().numpy(), ln.cpu().numpy(), st.cpu().numpy()

    ref = run("device")
    for kind in ("pinned", "pinned_offset", "pageable"):
        f, xy, ln, st = run(kind)
        assert np.array_equal(f, ref[0]) and np.array_equal(ln, ref[2]) and np.array_equal(st, ref[3]), kind
        for i in range(len(ln)):
            assert np.array_equal(xy[i, :ln[i]], ref[1][i, :ln[i]]), (kind, i)
    dd.dd_unload_mesh(ctx, mid)


def test_degenerate_inputs(env):
    """Empty and degenerate calls: no targets, no sources, ids out of range and
    max_pts < 2 are DD_EINVAL; a source equal to its target is a one-point OK
    path; max_pts = 2 truncates a long path to its first two points; a source
    on the boundary traces without error from the source's position."""
    dd, ctx = env
    wl, po, P = case("grid24")
    mesh = wl.mesh
    mid = load(dd, ctx, mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    t = int(wl.targets[0])
    out = torch.empty((2, 1, mesh.n_v), dtype=torch.float32, device="cuda")
    xy = torch.empty((4, 1024, 2), dtype=torch.float32, device="cuda")
    ln = torch.empty(4, dtype=torch.int32, device="cuda")
    st = torch.empty(4, dtype=torch.int32, device="cuda")
    for call in (lambda: dd.dd_distance(ctx, mid, [], 3, 0, out),
                 lambda: dd.dd_distance(ctx, mid, [mesh.n_v], 3, 0, out),
                 lambda: dd.dd_trace(ctx, mid, t, dd.DD_F_KL, [], 64, xy, ln, st),
                 lambda: dd.dd_trace(ctx, mid, t, dd.DD_F_KL, [mesh.n_v], 64, xy, ln, st),
                 lambda: dd.dd_trace(ctx, mid, t, dd.DD_F_KL, [t], 1, xy, ln, st),
                 lambda: dd.dd_query(ctx, mid, [t], np.zeros((1, 0), np.int32), 3, 0, 1, 64, out, xy, ln, st)):
        with pytest.raises(dd.DDError) as e:
            call()
        assert e.value.status == dd.DD_EINVAL
    far = int(po.I[np.argmax(np.hypot(*(mesh.xy[po.I] - mesh.xy[t]).T))])
    boundary = int(po.B[len(po.B) // 2])
    dd.dd_trace(ctx, mid, t, dd.DD_F_KL, [t, far, far, boundary], 1024, xy, ln, st)
    dd.dd_sync(ctx)
    L, S_ = ln.cpu().numpy(), st.cpu().numpy()
    X = xy.cpu().numpy()
    assert L[0] == 1 and S_[0] == dd.DD_TRACE_OK and np.allclose(X[0, 0], mesh.xy[t])
    assert S_[1] == dd.DD_TRACE_OK and L[1] > 2
    assert np.allclose(X[1, 0], mesh.xy[far]) and np.allclose(X[1, L[1] - 1], mesh.xy[t])
    assert np.allclose(X[3, 0], mesh.xy[boundary]) and S_[3] in (dd.DD_TRACE_OK, dd.DD_TRACE_STUCK)
    dd.dd_trace(ctx, mid, t, dd.DD_F_KL, [far], 2, xy, ln, st)
    dd.dd_sync(ctx)
    assert ln.cpu().numpy()[0] == 2 and st.cpu().numpy()[0] == dd.DD_TRACE_TRUNCATED
    dd.dd_unload_mesh(ctx, mid)
