"""GPU parity of the sparse fields (Section V: P sparsified by eliminating
the entries below a threshold relative to their row's maximum; DD_PREC_SPARSE
after dd_sparsify) and of the merged-bin extension (DD_PREC_SPARSE_MERGED)
against the FP64 oracle, through the C ABI.

The oracle decides which entries a row keeps in FP64 on the FP64 kernel, the
device in FP32 on its FP32 copy; the two can differ only on entries whose
FP64 value lies within FP32 rounding of theta x (row max): relative
BORDER = 8 x 2^-24 (the rounding of the stored entry, of theta, of the
row maximum and of their product, each at most 2^-24, with margin).  Rows
holding such an entry are left out of the comparison (a target holding one
is not used), and the kept counts agree up to the number of such entries.
Everything else: the fields to the FP32 tolerance |g - r| / max(|r|, 1e-2)
<= 1e-5, and exactly 0 at the target.
"""
import numpy as np
import pytest

from oracle import sparse
from oracle.poisson import PoissonOracle
from synthetic import workloads
from synthetic.meshes import convex_holes
from tests._gpu import TOL_FP32, ctx_and_lib, field_error, load

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BORDER = 8.0 * 2.0 ** -24

CASES = {
    "disk": lambda: workloads.disk(),
    "grid37": lambda: workloads.small_grid(37, 3, T=6, S=2, seed=777),
    "holes2000": lambda: workloads.Workload("holes2000", convex_holes(2000, seed=3), np.zeros(0, np.int32),
                                            np.zeros((0, 0), np.int32)),
}
_cache = {}


def case(name):
    if name not in _cache:
        wl = CASES[name]()
        po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
        _cache[name] = (wl, po, po.full())
    return _cache[name]


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    dd, ctx = ctx_and_lib()
    yield dd, ctx
    dd.dd_destroy(ctx)


def _targets(po, count):
    ids = po.I
    return [int(ids[i]) for i in np.linspace(0, len(ids) - 1, count + 2).astype(int)[1:-1]]


def _border(P, theta):
    """[rows][k]: entries within FP32 rounding of their row's threshold (the
    FP64 and FP32 decisions may differ there)."""
    P = np.asarray(P, dtype=np.float64)
    thr = theta * P.max(axis=1, keepdims=True)
    return np.abs(P - thr) <= BORDER * thr


def _check_sparse(dd, got, P, th, targets, merged=False):
    """Compare [3][T][n] fields (KL, TV, KLT) with the oracle on the rows no
    borderline entry can change; returns the share of rows left out."""
    bad_rows = _border(P, th).any(axis=1)
    used = 0
    for a, t in enumerate(targets):
        assert not bad_rows[t], "a target holds a borderline entry: choose another"
        if merged:
            refs = (sparse.merged_kl_field(P, t, th), sparse.merged_tv_field(P, t, th),
                    sparse.merged_klt_field(P, t, th))
            rows = np.ones(P.shape[0], bool)                  # only the target's decision matters
        else:
            refs = (sparse.sparse_kl_field(P, t, th), sparse.sparse_tv_field(P, t, th),
                    sparse.sparse_klt_field(P, t, th))
            rows = ~bad_rows
        used += 1
        for f, (r, lo) in enumerate(zip(refs, (80.0, None, 50.0))):
            g = got[f, a]
            assert field_error(g[rows], r[rows]) <= TOL_FP32, (f, field_error(g[rows], r[rows]))
            assert g[t] == 0.0
            inf = ~np.isfinite(r) & rows
            if inf.any():
                assert np.all(g[inf] >= lo)
    assert used == len(targets)
    return float(np.mean(bad_rows))


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("theta", [None, 0.05])
def test_sparse_fields_on_oracle_kernel(env, name, theta):
    dd, ctx = env
    wl, po, P = case(name)
    th = sparse.default_theta(wl.mesh.n_v) if theta is None else theta
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    kept, nbytes = dd.dd_sparsify(ctx, mid, -1.0 if theta is None else theta)
    mask = sparse.keep_mask(P, th)
    assert abs(kept - int(mask.sum())) <= int(_border(P, th).sum())
    assert nbytes == (wl.mesh.n_v + 1) * 8 + kept * 6
    targets = _targets(po, 5)
    T, n = len(targets), wl.mesh.n_v
    out = torch.empty((3, T, n), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_SPARSE, out)
    one = torch.empty((1, T, n), dtype=torch.float32, device="cuda")
    two = torch.empty((1, T, n), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KLT, dd.DD_PREC_SPARSE, one)
    dd.dd_distance(ctx, mid, targets, dd.DD_F_TV, dd.DD_PREC_SPARSE, two)
    mrg = torch.empty((3, T, n), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_SPARSE_MERGED, mrg)
    dd.dd_sync(ctx)
    got = out.cpu().numpy()
    # the same kernel arithmetic alone or together
    assert np.array_equal(one.cpu().numpy()[0], got[2]) and np.array_equal(two.cpu().numpy()[0], got[1])
    assert _check_sparse(dd, got, P, th, targets) < 0.01
    _check_sparse(dd, mrg.cpu().numpy(), P, th, targets, merged=True)
    dd.dd_unload_mesh(ctx, mid)


def test_klt_dense_and_traced(env):
    """DD_F_KLT on the dense FP32 path: the target-weighted KL of the oracle,
    laid out after KL and TV, and traceable by dd_query."""
    from oracle.fdiv import kl_reverse_field
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    targets = [int(t) for t in wl.targets[:3]]
    S = 2
    n = wl.mesh.n_v
    f3 = torch.empty((3, 3, n), dtype=torch.float32, device="cuda")
    f2 = torch.empty((2, 3, n), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_FP32, f3)
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, f2)
    xy = torch.empty((3 * S, 512, 2), dtype=torch.float32, device="cuda")
    ln = torch.empty(3 * S, dtype=torch.int32, device="cuda")
    st = torch.empty(3 * S, dtype=torch.int32, device="cuda")
    src = np.asarray(wl.sources)[:3, :S]
    fq = torch.empty((2, 3, n), dtype=torch.float32, device="cuda")
    dd.dd_query(ctx, mid, targets, src, dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_FP32, dd.DD_F_KLT, 512, fq, xy, ln, st)
    xy2, ln2, st2 = torch.empty_like(xy), torch.empty_like(ln), torch.empty_like(st)
    dd.dd_trace_fields(ctx, mid, f3[2].contiguous(), targets, src, 512, xy2, ln2, st2)
    dd.dd_sync(ctx)
    g3, g2 = f3.cpu().numpy(), f2.cpu().numpy()
    assert np.array_equal(g3[:2], g2)
    assert np.array_equal(fq.cpu().numpy()[1], g3[2]) and np.array_equal(fq.cpu().numpy()[0], g3[1])
    for a, t in enumerate(targets):
        r = kl_reverse_field(P, P[t])
        assert field_error(g3[2, a], r) <= TOL_FP32
        assert g3[2, a, t] == 0.0
        assert np.all(g3[2, a][~np.isfinite(r)] >= 50.0)
    assert torch.equal(st, st2) and torch.equal(ln, ln2)
    assert (st.cpu().numpy() == dd.DD_TRACE_OK).all()
    dd.dd_unload_mesh(ctx, mid)


def test_sparse_theta_zero_is_dense(env):
    """theta = 0 keeps every positive entry of the target row: the dense
    fields wherever they are finite."""
    from oracle.divergence import kl_field_fast, tv_field
    from oracle.fdiv import kl_reverse_field
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    kept, _ = dd.dd_sparsify(ctx, mid, 0.0)
    assert kept == int((P >= np.finfo(np.float32).tiny).sum())     # stored P flushes below FLT_MIN
    t = _targets(po, 2)
    a = torch.empty((3, 2, wl.mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, t, dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_SPARSE, a)
    dd.dd_sync(ctx)
    a = a.cpu().numpy()
    for i, ti in enumerate(t):
        assert field_error(a[0, i], kl_field_fast(P, P[ti])) <= TOL_FP32
        assert field_error(a[1, i], tv_field(P, P[ti])) <= TOL_FP32
        assert field_error(a[2, i], kl_reverse_field(P, P[ti])) <= TOL_FP32
    dd.dd_unload_mesh(ctx, mid)


def test_sparse_states_and_errors(env):
    dd, ctx = env
    wl, po, P = case("grid37")
    mid = load(dd, ctx, wl.mesh)
    t = _targets(po, 1)
    out = np.empty((1, wl.mesh.n_v), dtype=np.float32)
    with pytest.raises(dd.DDError):                     # no kernel yet
        dd.dd_sparsify(ctx, mid)
    dd.dd_set_poisson_kernel(ctx, mid, P)
    with pytest.raises(dd.DDError):                     # not sparsified yet
        dd.dd_distance(ctx, mid, t, dd.DD_F_KL, dd.DD_PREC_SPARSE, out)
    for bad in (1.0, 2.0, float("nan")):
        with pytest.raises(dd.DDError):
            dd.dd_sparsify(ctx, mid, bad)
    dd.dd_sparsify(ctx, mid)
    dd.dd_distance(ctx, mid, t, dd.DD_F_KL, dd.DD_PREC_SPARSE, out)   # host output
    dev = torch.empty((1, wl.mesh.n_v), dtype=torch.float32, device="cuda")
    dd.dd_distance(ctx, mid, t, dd.DD_F_KL, dd.DD_PREC_SPARSE, dev)
    dd.dd_sync(ctx)
    assert np.array_equal(out, dev.cpu().numpy())
    dd.dd_set_poisson_kernel(ctx, mid, P)               # replacing P discards the sparse rows
    with pytest.raises(dd.DDError):
        dd.dd_distance(ctx, mid, t, dd.DD_F_KL, dd.DD_PREC_SPARSE, out)
    dd.dd_unload_mesh(ctx, mid)


def test_sparse_end_to_end_grid140(env):
    """Device PCG, dd_sparsify, sparse fields and a traced query against the
    oracle's own FP64 kernel of the same mesh."""
    dd, ctx = env
    wl = workloads.grid140(T=3, S=8)
    mesh = wl.mesh
    P = PoissonOracle(mesh.xy, mesh.tri, mesh.loops).full()
    mid = load(dd, ctx, mesh)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    th = sparse.default_theta(mesh.n_v)
    kept, _ = dd.dd_sparsify(ctx, mid)
    mask = sparse.keep_mask(P, th)
    assert abs(kept - int(mask.sum())) <= int(_border(P, th).sum())
    assert 0.5 < 1.0 - kept / P.size < 0.99
    targets = [int(t) for t in wl.targets]
    S = wl.sources.shape[1]
    f = torch.empty((3, len(targets), mesh.n_v), dtype=torch.float32, device="cuda")
    xy = torch.empty((len(targets) * S, 1024, 2), dtype=torch.float32, device="cuda")
    ln = torch.empty(len(targets) * S, dtype=torch.int32, device="cuda")
    st = torch.empty(len(targets) * S, dtype=torch.int32, device="cuda")
    dd.dd_query(ctx, mid, targets, wl.sources, dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_SPARSE,
                dd.DD_F_KLT, 1024, f, xy, ln, st)
    dd.dd_sync(ctx)
    assert _check_sparse(dd, f.cpu().numpy(), P, th, targets) < 0.01
    # the query traced exactly what dd_trace_fields traces on the same sparse field
    xy2, ln2, st2 = torch.empty_like(xy), torch.empty_like(ln), torch.empty_like(st)
    dd.dd_trace_fields(ctx, mid, f[2].contiguous(), targets, wl.sources, 1024, xy2, ln2, st2)
    dd.dd_sync(ctx)
    assert torch.equal(st, st2) and torch.equal(ln, ln2)
    stn, lnn, xyn = st.cpu().numpy(), ln.cpu().numpy(), xy.cpu().numpy()
    for i in np.nonzero(stn == dd.DD_TRACE_OK)[0]:
        assert np.allclose(xyn[i, lnn[i] - 1], mesh.xy[targets[i // S]], atol=1e-6)
    dd.dd_unload_mesh(ctx, mid)
