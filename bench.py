"""Benchmark of the online divergence-distance path (fields + traced paths).

One step = one dd_query over a batch of the grid450 workload (the largest
configuration that fits one GPU): KL and TV fields of 1,024 interior targets
over all n = 192,360 vertices (k = 3,936 boundary columns, P = 3.0 GB FP32)
on the FP32 path, and 1,024 x 16 paths traced on the KL fields.  The Poisson
kernel is computed once per domain before timing (the paper's preprocessing)
and reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one process per GPU under torch.distributed.run; every rank
processes its own target batches (weak scaling, no data-path collective).
`--impl reference` times the FP64 CPU oracle on a bounded sample of the
same workload (rank 0 only).

The JSON line: `value` from CUDA events around each step (inputs resident,
P far larger than L2, L2 also flushed between steps outside the events),
`e2e` through the same call with pinned host buffers, `kernels` (live
per-kernel times from the library's own events), `roofline` for the
dominant kernel, `clocks` sampled during the timed region (measured once
more, with `remeasured`, if they show a slowdown or a clock lock),
`error_vs_oracle` (every result of the step against the FP64 oracle on
sampled rows), `step_bf16x3` (the same step with the KL fields from the
split-BF16 tensor-core GEMM), `cpu_baseline` (the oracle on every host core,
full fields and the paper's path-only scheme), and with no `--section` the
grid140 step, the grid450 single-target, sparse and other-divergence
passes, the batch, serving and census measurements.
"""

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "distance fields/s (KL+TV, one target over all vertices) with traced paths"
UNIT = "fields/s"
# the query-step workloads: targets per step, sources per target, polyline capacity
WORKLOADS = {
    "grid450": {"T": 1024, "S": 16, "max_pts": 4096,
                "desc": "grid450: unit square h=1/450, 24 rectangular obstacles, n=%d, k=%d; %d targets x (KL+TV) "
                        "+ %dx%d KL paths per step"},
    "grid140": {"T": 64, "S": 256, "max_pts": 1024,
                "desc": "grid140: unit square h=1/140, 8 square obstacles, n=%d, k=%d; %d targets x (KL+TV) "
                        "+ %dx%d KL paths per step"},
}
HEADLINE = "grid450"
# kernels one dd_query step launches at most: target staging, the targets in
# the tiled layout, field tile, exact KL recompute near the targets, triangle
# rates and vertex decisions (only when 128 or more paths share a field),
# path walk
STEP_LAUNCHES = 7
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from
# ncu captures of the step's kernels (means over the captured query steps);
# absent where no capture of the current kernel exists; used only when the
# step runs the captured (T, S).  grid450's tile launch (the pipelined tile
# on the tiled copy of P) reads each pair of row tiles from DRAM about once:
# the 16 CTAs of one pair run together and share it through L2.
TRAFFIC = {
    "grid140": {},
    "grid450": {"T": 1024, "S": 16, "field_tile_kernel": 9287471001, "trace_kernel": 307644416},
}
# the same for one field_stream_kernel launch of the grid450 single-target pass
STREAM_TRAFFIC_BYTES = 3035740160    # 3,032,217,088 read + 3,523,072 written (4 n k_pad = 3.03 GB of P)
N_BATCHES = 4
# sampled rows and targets for the error against the FP64 oracle (Green's rows)
ERR_ROWS, ERR_TARGETS = 256, 128


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the job's time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_workload(name: str, T: int, S: int):
    from synthetic import workloads
    return getattr(workloads, name)(T=T, S=S)


def workload_batches(rank: int, name: str = HEADLINE):
    from synthetic import workloads
    from synthetic.rng import SplitMix64
    w = WORKLOADS[name]
    wl = make_workload(name, w["T"], w["S"])
    # rank 0 starts with the workload's own batch; every other batch (and all of
    # another rank's) is drawn from a rank-seeded stream, so ranks share no work
    batches = [(wl.targets, wl.sources)] if rank == 0 else []
    rng = SplitMix64(workloads.BASE_SEED + 1000 + rank)
    while len(batches) < N_BATCHES:
        t = workloads.draw_targets(rng, wl.mesh, w["T"])
        s = workloads.draw_sources(rng, wl.mesh, t, w["S"])
        batches.append((t, s))
    return wl, batches


def sm_count(device_index: int) -> int:
    import torch
    try:
        return int(torch.cuda.get_device_properties(device_index).multi_processor_count)
    except Exception:
        return 0


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def clocks_rejected(clocks) -> bool:
    """True for a clock record that invalidates a timing: hw_slowdown,
    hw_thermal_slowdown or sw_thermal_slowdown active, or the median SM clock
    under 80 % of its maximum with no reason active (a leftover clock lock).
    sw_power_cap is kept (normal under load on this part)."""
    bad = {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}
    reasons = set(clocks.get("reasons") or [])
    if reasons & bad:
        return True
    sm, mx = clocks.get("sm_mhz"), clocks.get("sm_max_mhz")
    return bool(sm and mx and sm < 0.8 * mx and not reasons)


def roof_tile(n_v, k, T, tile_ms, sms, sm_mhz, traffic):
    """The field tile kernel against the FP32 pipe's rate: per (row, column,
    target) 4 FP32 operations -- KL one addition (the log2 ratio) and one
    multiply-add, TV two additions -- against 128 FP32 lanes x clock per SM
    (one operation per lane per clock; a packed FP32x2 instruction does two
    and holds the pipe twice as long)."""
    ops = 4.0 * n_v * k * T
    peak_alu = sms * 128 * sm_mhz * 1e6 / 1e12
    achieved = ops / (tile_ms / 1e3) / 1e12
    return {"kernel": "field_tile_kernel", "bound": "alu", "achieved": round(achieved, 3), "peak": round(peak_alu, 3),
            "unit": "T FP32 operations/s", "frac": round(achieved / peak_alu, 4), "traffic": traffic,
            "algorithmic_fp32_ops": ops, "ms_per_launch": round(tile_ms, 4),
            "peak_source": f"{sms} SMs (read from the device) x 128 FP32 lanes x {sm_mhz:.0f} MHz (median SM clock "
                           "sampled in the timed region), one FP32 operation per lane per clock",
            "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch" if traffic else
                              "no ncu capture of this kernel on this workload"}


_LOAD_NS = {}


def load_latency(dd, ctx):
    """ns per dependent global load (L1 bypassed), measured once per run by
    dd_load_latency: a 32 MB cycle (L2 hits after a warm-up pass) and a 1 GB
    one (DRAM)."""
    if not _LOAD_NS:
        try:
            _LOAD_NS["l2"] = round(dd.dd_load_latency(ctx, 32 << 20, 200000), 1)
            _LOAD_NS["dram"] = round(dd.dd_load_latency(ctx, 1 << 30, 100000), 1)
        except Exception as e:     # a measurement, not a result: report why it is missing
            _LOAD_NS["error"] = str(e)
    return _LOAD_NS


def roof_walk(walk_ms, walk_points, max_points, traffic, lat=None):
    """The walk: a chain of dependent gathers per path (one triangle record and
    one rate vector per crossing), bounded by the longest path's chain of
    dependent L2 round trips, not by a bandwidth.  With the measured latency
    of one dependent L2 load: the floor of one such load per point of the
    longest path, and the step's time in those loads."""
    us_pt = walk_ms * 1e3 / max(max_points, 1)
    out = {"kernel": "trace_kernel", "bound": "latency", "ms_per_launch": round(walk_ms, 4),
           "points_per_s": round(walk_points / (walk_ms / 1e3), 1), "longest_path_points": int(max_points),
           "us_per_point_of_longest_path": round(us_pt, 4), "traffic": traffic,
           "note": "one dependent record + rate gather per crossing; the launch lasts as long as its longest path"}
    if lat and "l2" in lat:
        out["dependent_load_ns"] = {"l2": lat["l2"], "dram": lat["dram"], "source": "dd_load_latency, CUDA events"}
        out["floor_ms_one_l2_load_per_point"] = round(max_points * lat["l2"] / 1e6, 4)
        out["l2_loads_per_point"] = round(us_pt * 1e3 / lat["l2"], 2)
    return out


def query_step(dd, ctx, dev, stream, flush, args, rank, world, local_rank, name, pk, pk_kind):
    """Load the workload, compute its Poisson kernel, then time K dd_query steps
    (T targets x KL+TV fields + T x S KL paths) with CUDA events on the
    context stream, per-kernel times from the library's events, clocks
    sampled meanwhile; then the same call end to end with pinned host buffers."""
    import torch
    w = WORKLOADS[name]
    T, S, max_pts = w["T"], w["S"], w["max_pts"]
    wl, batches = workload_batches(rank, name)
    mesh = wl.mesh
    idx, off = mesh.loop_arrays()
    mid = dd.dd_load_mesh(ctx, mesh.xy, mesh.tri, idx, off)
    info = dd.dd_mesh_info(ctx, mid)
    t0 = time.perf_counter()
    iters, resid = dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
    preproc_s = time.perf_counter() - t0
    n_v, k = info["n_v"], info["k"]

    fields = torch.empty((2, T, n_v), dtype=torch.float32, device=dev)
    pxy = torch.empty((T * S, max_pts, 2), dtype=torch.float32, device=dev)
    plen = torch.empty(T * S, dtype=torch.int32, device=dev)
    pst = torch.empty(T * S, dtype=torch.int32, device=dev)

    def step(i):
        tg, sr = batches[i % len(batches)]
        dd.dd_query(ctx, mid, tg, sr, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, dd.DD_F_KL, max_pts,
                    fields, pxy, plen, pst)

    for i in range(args.warmup):
        flush.fill_(float(i))
        step(i)
    dd.dd_sync(ctx)
    torch.cuda.synchronize()

    # fields vs tracing on the same stream (untimed for the metric)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tg, sr = batches[0]
    split_f, split_t = [], []
    for r in range(2):
        flush.fill_(1.0)
        ev[0].record(stream)
        dd.dd_distance(ctx, mid, tg, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, fields)
        ev[1].record(stream)
        dd.dd_trace_fields(ctx, mid, fields[0], tg, sr, max_pts, pxy, plen, pst)
        ev[2].record(stream)
        torch.cuda.synchronize()
        split_f.append(ev[0].elapsed_time(ev[1]))
        split_t.append(ev[1].elapsed_time(ev[2]))
    field_ms, trace_ms = statistics.median(split_f), statistics.median(split_t)

    # timed region: K steps, L2 flushed between steps (outside the step events)
    def timed_region():
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        sampler = ClockSampler(local_rank if "CUDA_VISIBLE_DEVICES" not in os.environ else 0)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        sampler.start()
        time.sleep(0.3)
        dd.dd_kernel_timing(ctx, 1)      # per-kernel CUDA events on this stream, live over the timed steps
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            step(args.warmup + i)
            ends[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        kernel_ms = dd.dd_kernel_timing(ctx, 0)
        clocks = sampler.stop()
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        return kernel_ms, clocks, float(sum(step_ms)), wall

    kernel_ms, clocks, dev_ms, wall = timed_region()
    # a region that saw a thermal or hardware slowdown, or SM clocks far below
    # their maximum with no reason given, is measured once more (every rank
    # takes the same decision)
    remeasured = None
    if max_over_ranks(1.0 if clocks_rejected(clocks) else 0.0, dev if world > 1 else None) > 0.0:
        first = {"reasons": clocks.get("reasons"), "sm_mhz": clocks.get("sm_mhz"),
                 "ms_per_step": round(dev_ms / args.steps, 4)}
        kernel_ms, clocks, dev_ms, wall = timed_region()
        remeasured = {"first": first}
    if world > 1:
        import torch.distributed as dist
        dev_ms = max_over_ranks(dev_ms, dev)
        dist.barrier()
    status = pst.cpu().numpy()
    lens = plen.cpu().numpy()

    # end to end through the same C-ABI call with host buffers
    hf = torch.empty((2, T, n_v), dtype=torch.float32).pin_memory()
    hxy = torch.empty((T * S, max_pts, 2), dtype=torch.float32).pin_memory()
    hl = torch.empty(T * S, dtype=torch.int32).pin_memory()
    hs = torch.empty(T * S, dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 10))
    for i in range(2):
        tg, sr = batches[i % len(batches)]
        dd.dd_query(ctx, mid, tg, sr, 3, 0, 1, max_pts, hf, hxy, hl, hs)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(e2e_steps):
        tg, sr = batches[i % len(batches)]
        dd.dd_query(ctx, mid, tg, sr, 3, 0, 1, max_pts, hf, hxy, hl, hs)
    e2e_s = time.perf_counter() - e0
    # into pinned host buffers the library moves exactly each path's defined
    # prefix (len points), plus the lengths and statuses (counted on the last
    # step's lengths)
    ln = hl.numpy()
    path_bytes = int(ln.astype(np.int64).sum()) * 8
    h2d = T * 4 + T * S * 4
    d2h = 2 * T * n_v * 4 + T * S * 8 + path_bytes
    del hf, hxy, hl, hs

    fields_per_step = 2 * T
    value = world * fields_per_step * args.steps / (dev_ms / 1e3)
    sm_mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    sms = sm_count(local_rank) or 152
    tot = sum(ms for _, ms in kernel_ms.values()) or 1.0
    kernels = {kn: {"launches": c, "ms_per_launch": round(ms / max(c, 1), 4), "share": round(ms / tot, 4)}
               for kn, (c, ms) in sorted(kernel_ms.items(), key=lambda kv: -kv[1][1])}
    per_launch = {kn: ms / max(c, 1) for kn, (c, ms) in kernel_ms.items()}
    traffic = TRAFFIC.get(name, {})
    if (traffic.get("T"), traffic.get("S")) != (T, S):
        traffic = {}
    tile_ms = per_launch.get("field_tile_kernel", field_ms)
    roof_t = roof_tile(n_v, k, T, tile_ms, sms, sm_mhz, traffic.get("field_tile_kernel"))
    walk_ms = per_launch.get("trace_kernel")
    walk_points = int(np.clip(lens, 0, None).sum())
    roof_w = (roof_walk(walk_ms, walk_points, int(lens.max()), traffic.get("trace_kernel"), load_latency(dd, ctx))
              if walk_ms else None)
    dom = max(kernel_ms, key=lambda kn: kernel_ms[kn][1]) if kernel_ms else "field_tile_kernel"
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["desc"] % (n_v, k, T, T, S), "n_v": n_v, "k": k, "targets_per_step": T,
                   "sources_per_target": S, "max_pts": max_pts, "precision": "FP32 fields (DD_PREC_FP32)",
                   "l2": "inputs larger than L2 (P = %.2f GB); L2 also flushed between steps (256 MB write outside "
                         "the step events)" % (4.0 * n_v * info["k_pad"] / 1e9),
                   "parallelism": f"replicas x{world}"},
        "paths_per_s": round(world * T * S * args.steps / (dev_ms / 1e3), 1),
        "kernel_split_ms": {"fields": round(field_ms, 4), "trace": round(trace_ms, 4)},
        "paths_ok_frac": float(np.mean(status == 0)), "max_path_pts": int(lens.max()),
        "preproc": {"pcg_iters": iters, "resid": resid, "seconds": round(preproc_s, 3)},
        "wall_s_timed_region": round(wall, 4),
        "roofline": roof_t if dom != "trace_kernel" or roof_w is None else roof_w,
        "roofline_walk": roof_w if dom != "trace_kernel" else None,
        "roofline_fields": roof_t if dom == "trace_kernel" else None, "peaks": pk_kind,
        "e2e": {"value": round(world * fields_per_step * e2e_steps / e2e_s, 1), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(sum(c for c, _ in kernel_ms.values())) or STEP_LAUNCHES * args.steps,
        "kernels": kernels,
        "clocks": clocks,
    }
    if "fix_kl_kernel" in per_launch:
        line["recompute_over_tile"] = round(per_launch["fix_kl_kernel"] / tile_ms, 4)
    line["tile_shapes"] = dd.dd_tuning_table().strip().splitlines()
    if remeasured is not None:
        line["remeasured"] = remeasured
    return {"line": line, "mid": mid, "wl": wl, "batches": batches, "fields": fields, "pxy": pxy, "plen": plen,
            "pst": pst, "T": T, "S": S, "max_pts": max_pts, "n_v": n_v, "k": k, "k_pad": info["k_pad"]}


def bf16x3_step(dd, ctx, q, flush, stream, args):
    """The same query step with DD_PREC_BF16X3: the KL fields from the split-BF16
    tensor-core GEMM (error bound 1e-4 of S_x, not the FP32 path's 1e-5: not
    the headline), TV from a TV-only FP32 tile pass, the paths traced on the
    GEMM's KL fields.  Reports its time, its kernels and the KL fields'
    largest deviation from the FP32 path's relative to max(|KL|, 1)."""
    import torch
    mid, batches, fields, T = q["mid"], q["batches"], q["fields"], q["T"]

    def step(i):
        tg, sr = batches[i % len(batches)]
        dd.dd_query(ctx, mid, tg, sr, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_BF16X3, dd.DD_F_KL, q["max_pts"],
                    fields, q["pxy"], q["plen"], q["pst"])

    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    dd.dd_kernel_timing(ctx, 1)
    ms = []
    for i in range(args.steps):
        flush.fill_(float(i))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(args.warmup + i)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    kt = dd.dd_kernel_timing(ctx, 0)
    tg, sr = batches[0]
    ref = torch.empty_like(fields)
    dd.dd_distance(ctx, mid, tg, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, ref)
    got = torch.empty_like(fields)
    dd.dd_distance(ctx, mid, tg, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_BF16X3, got)
    torch.cuda.synchronize()
    fin = ref[0] < 80.0
    dev = (got[0] - ref[0]).abs() / ref[0].abs().clamp(min=1.0)
    kl_dev = float(dev[fin].max().item())
    tv_same = bool(torch.equal(got[1], ref[1]))
    del ref, got
    dev_ms = float(sum(ms))
    return {"ms_per_step": round(dev_ms / args.steps, 4), "fields_per_s": round(2 * T * args.steps / (dev_ms / 1e3), 1),
            "kl_max_dev_vs_fp32": kl_dev, "tv_identical": tv_same,
            "kernels": {n: {"launches": c, "ms_per_launch": round(v / max(c, 1), 4)} for n, (c, v) in kt.items()},
            "note": "KL through the tensor-core GEMM (split BF16, 1e-4 bound), TV through a TV-only FP32 pass"}


class OracleRows:
    """FP64 oracle rows of P for sampled vertices and targets of one workload
    (Green's-row solves), and the dense fields between them."""

    def __init__(self, wl, targets, n_rows: int, seed: int):
        from oracle.poisson import PoissonOracle
        from synthetic.rng import SplitMix64
        t0 = time.perf_counter()
        po = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
        rng = SplitMix64(seed)
        interior = np.asarray(po.I)
        self.rows = np.array(sorted({int(interior[rng.choice(len(interior))]) for _ in range(n_rows)}), np.int64)
        self.targets = np.asarray(targets, np.int64)
        both = np.concatenate([self.rows, self.targets])
        R = po.rows(both)
        self.Px, self.Pt = R[:len(self.rows)], R[len(self.rows):]
        self.seconds = time.perf_counter() - t0
        self.n_v = wl.mesh.n_v

    def dense(self):
        """KL [T][R], TV [T][R], KLT [T][R] and S_x [T][R] = sum_b P[x,b] |log P[t,b]|."""
        from oracle.divergence import kl_field_fast, tv_field
        from oracle.fdiv import kl_reverse_field
        kl = np.stack([kl_field_fast(self.Px, pt) for pt in self.Pt])
        tv = np.stack([tv_field(self.Px, pt) for pt in self.Pt])
        klt = np.stack([kl_reverse_field(self.Px, pt) for pt in self.Pt])
        # a zero column (P[t,b] = 0) has P[x,b] = 0 on every interior row: its term is 0
        lg = np.abs(np.log(np.maximum(self.Pt, 1e-300)))
        sx = np.stack([(self.Px * lg[a][None, :]).sum(axis=1) for a in range(len(self.Pt))])
        return kl, tv, klt, sx


def rel_err(g, r, floor):
    """max and median of |g - r| / max(|r|, floor) over the finite reference entries."""
    g = np.asarray(g, np.float64)
    r = np.asarray(r, np.float64)
    fl = np.broadcast_to(np.asarray(floor, np.float64), r.shape)
    fin = np.isfinite(r) & np.isfinite(fl)
    e = np.abs(g[fin] - r[fin]) / np.maximum(np.abs(r[fin]), fl[fin])
    return {"max": float(e.max()), "median": float(np.median(e)), "n": int(e.size)}


def error_vs_oracle(dd, ctx, dev, q, orows):
    """Every field result of the step against the FP64 oracle on sampled rows:
    FP32 KL and TV (tolerance 1e-5 relative, floor 1e-2), split-BF16 KL
    (1e-4 relative, floor S_x = sum_b P[x,b] |log P[t,b]|)."""
    import torch
    mid, n_v = q["mid"], q["n_v"]
    tg = [int(t) for t in orows.targets]
    T = len(tg)
    out = torch.empty((2, T, n_v), dtype=torch.float32, device=dev)
    dd.dd_distance(ctx, mid, tg, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, out)
    g32 = out[:, :, torch.as_tensor(orows.rows, device=dev)].cpu().numpy()
    dd.dd_distance(ctx, mid, tg, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_BF16X3, out)
    gbf = out[:, :, torch.as_tensor(orows.rows, device=dev)].cpu().numpy()
    del out
    kl, tv, _, sx = orows.dense()
    res = {"sample": "%d sampled interior rows x %d targets of the step's first batch; oracle rows by Green's-row "
                     "solves (%.1f s)" % (len(orows.rows), T, orows.seconds),
           "fp32_kl": dict(rel_err(g32[0], kl, 1e-2), tol=1e-5, floor="1e-2"),
           "fp32_tv": dict(rel_err(g32[1], tv, 1e-2), tol=1e-5, floor="1e-2"),
           "bf16x3_kl": dict(rel_err(gbf[0], kl, sx), tol=1e-4, floor="S_x"),
           "bf16x3_tv": dict(rel_err(gbf[1], tv, 1e-2), tol=1e-5, floor="1e-2")}
    for key in ("fp32_kl", "fp32_tv", "bf16x3_kl", "bf16x3_tv"):
        res[key]["ok"] = bool(res[key]["max"] <= res[key]["tol"])
    return res


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1708_02845_gb300.build import build
    if rank == 0 or not os.path.exists(os.path.join(ROOT, "paper_1708_02845_gb300", "_lib", "libdd.so")):
        build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    from paper_1708_02845_gb300 import dd

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    ctx = dd.dd_create(local_rank, stream.cuda_stream)
    pk, pk_kind = peaks()
    flush = torch.empty((256 << 20) // 4, dtype=torch.float32, device=dev)
    if args.section in ("grid450", "batch", "serve", "census", "mid", "grid140", "maze"):
        if args.section == "grid450":
            st_sec, gm_sec = grid450_sections(dd, ctx, dev, stream, flush, pk, pk_kind)
            out = {"metric": "grid450 sections only", "stream": st_sec, "gemm": gm_sec}
        elif args.section == "grid140":
            out = query_step(dd, ctx, dev, stream, flush, args, rank, world, local_rank, "grid140", pk, pk_kind)["line"]
            out["metric"] = "grid140 step only"
        elif args.section == "batch":
            out = {"metric": "batch64 section only", "batch": batch_section(dd, ctx, dev, stream, flush, args)}
        elif args.section == "maze":
            out = {"metric": "maze section only", "maze": maze_section(dd, ctx, dev)}
        elif args.section == "census":
            out = {"metric": "census section only", "census": census_section(dd, ctx, dev)}
        elif args.section == "mid":
            out = {"metric": "grid300 section only", "mid": mid_section(dd, ctx, dev, stream, flush, pk, pk_kind)}
        else:
            out = {"metric": "serving section only", "serve": serve_section(dd, ctx, args, n_domains=8, seconds=10.0)}
        dd.dd_destroy(ctx)
        return out
    q = query_step(dd, ctx, dev, stream, flush, args, rank, world, local_rank, HEADLINE, pk, pk_kind)
    line = q["line"]
    line["step_bf16x3"] = bf16x3_step(dd, ctx, q, flush, stream, args)
    orows = None
    if args.oracle_errors and world == 1:
        orows = OracleRows(q["wl"], q["batches"][0][0][:ERR_TARGETS], ERR_ROWS, seed=170802845 + 77)
        line["error_vs_oracle"] = error_vs_oracle(dd, ctx, dev, q, orows)
    if args.section == "all" and world == 1:
        mid = q["mid"]
        for key in ("fields", "pxy"):
            q[key] = None
        torch.cuda.empty_cache()
        line["stream"], line["gemm"] = grid450_sections(dd, ctx, dev, stream, flush, pk, pk_kind, mid=mid,
                                                        wl=q["wl"], orows=orows)
        dd.dd_unload_mesh(ctx, mid)
        g140 = query_step(dd, ctx, dev, stream, flush, args, rank, world, local_rank, "grid140", pk, pk_kind)
        dd.dd_unload_mesh(ctx, g140["mid"])
        line["grid140"] = {kk: g140["line"][kk] for kk in ("value", "ms_per_step", "config", "paths_per_s",
                                                           "paths_ok_frac", "max_path_pts", "roofline",
                                                           "roofline_fields", "roofline_walk", "kernels", "e2e",
                                                           "clocks", "recompute_over_tile") if kk in g140["line"]}
        del g140
        torch.cuda.empty_cache()
        line["maze"] = maze_section(dd, ctx, dev)
        line["batch"] = batch_section(dd, ctx, dev, stream, flush, args)
        line["serve"] = serve_section(dd, ctx, args, n_domains=8, seconds=10.0)
        line["census"] = census_section(dd, ctx, dev)
    dd.dd_destroy(ctx)
    return line


def grid450_sections(dd, ctx, dev, stream, flush, pk, pk_kind, reps: int = 10, mid=None, wl=None, orows=None):
    """grid450 (n = 192,360, k = 3,936; P = 3.0 GB FP32, far above L2); the
    mesh of the headline step when given (mid, wl), else loaded and solved here.

    stream: single-target KL+TV sweeps; the streaming kernel reads P once per
      target, achieved GB/s = (4 n k_pad + 8 n) bytes / event-timed dd_distance.
    gemm: 1,024 targets, KL through the split-BF16 tcgen05 GEMM; algorithmic
      2 n k T flop (three BF16 products issued), against the FP32 CUDA-core
      path for the same KL fields.
    other_f_divergences, sparse: one target per call, one pass each."""
    import torch
    from synthetic import workloads
    T_big = 1024
    own = mid is None
    iters = resid = pre = None
    if own:
        wl = workloads.grid450(T=T_big)
        idx, off = wl.mesh.loop_arrays()
        mid = dd.dd_load_mesh(ctx, wl.mesh.xy, wl.mesh.tri, idx, off)
        t0 = time.perf_counter()
        iters, resid = dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
        pre = time.perf_counter() - t0
    info = dd.dd_mesh_info(ctx, mid)
    n_v, k, k_pad = info["n_v"], info["k"], info["k_pad"]

    def timed(fn, n_rep):
        ms = []
        for _ in range(n_rep):
            flush.fill_(0.5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    out1 = torch.empty((2, 1, n_v), dtype=torch.float32, device=dev)
    tl = [int(t) for t in wl.targets]
    for t in tl[:3]:
        dd.dd_distance(ctx, mid, [t], 3, 0, out1)
    it = iter(tl * 4)
    med = timed(lambda: dd.dd_distance(ctx, mid, [next(it)], 3, 0, out1), reps)
    nbytes = 4.0 * n_v * k_pad + 2 * 4.0 * n_v
    achieved = nbytes / (med / 1e3) / 1e9
    stream_sec = {"workload": "grid450 single target: n=%d, k_pad=%d, P=%.2f GB FP32" % (n_v, k_pad, 4.0 * n_v * k_pad / 1e9),
                  "kernel": "field_stream_kernel (+ stage_targets_kernel)", "bound": "hbm",
                  "achieved": round(achieved, 1), "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                  "frac": round(achieved / pk.get("hbm_gbs", 6672.5), 4), "peak_source": pk_kind,
                  "ms_per_field_pair": round(med, 4), "fields_per_s": round(2 / (med / 1e3), 1),
                  "traffic": STREAM_TRAFFIC_BYTES, "algorithmic_bytes": int(nbytes),
                  "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch, this workload",
                  "preproc": {"pcg_iters": iters, "resid": resid, "seconds": round(pre, 2)} if own else
                  "the headline step's kernel"}

    outk = torch.empty((1, T_big, n_v), dtype=torch.float32, device=dev)
    dd.dd_distance(ctx, mid, tl, dd.DD_F_KL, dd.DD_PREC_BF16X3, outk)   # builds the BF16 split of P once
    torch.cuda.synchronize()
    g_ms = timed(lambda: dd.dd_distance(ctx, mid, tl, dd.DD_F_KL, dd.DD_PREC_BF16X3, outk), 5)
    dd.dd_distance(ctx, mid, tl, dd.DD_F_KL, dd.DD_PREC_FP32, outk)     # first call runs the tile autotuner
    torch.cuda.synchronize()
    f_ms = timed(lambda: dd.dd_distance(ctx, mid, tl, dd.DD_F_KL, dd.DD_PREC_FP32, outk), 2)
    flop_alg = 2.0 * n_v * k * T_big
    tf_alg = flop_alg / (g_ms / 1e3) / 1e12
    tf_iss = 3 * tf_alg
    peak_bf16 = pk.get("bf16_tflops", 1916.1)
    gemm_sec = {"workload": "grid450, %d targets, KL only" % T_big, "kernel": "kl_gemm_kernel (+ split_targets_kernel)",
                "bound": "tensor", "achieved": round(tf_iss, 1), "achieved_algorithmic": round(tf_alg, 1),
                "peak": peak_bf16, "unit": "TFLOP/s", "frac": round(tf_iss / peak_bf16, 4), "peak_source": pk_kind,
                "ms": round(g_ms, 3), "kl_fields_per_s": round(T_big / (g_ms / 1e3), 1),
                "fp32_path_ms": round(f_ms, 3), "speedup_vs_fp32_path": round(f_ms / g_ms, 2), "traffic": None}
    # other f-divergences (Section VI): one target per call, one pass over P each
    out_f = torch.empty((1, n_v), dtype=torch.float32, device=dev)
    fams = [("chi2", dd.DD_DIV_CHI2, 0.0), ("hellinger", dd.DD_DIV_HELLINGER, 0.0), ("power2.5", dd.DD_DIV_POWER, 2.5),
            ("alpha0.5", dd.DD_DIV_ALPHA, 0.5), ("kl_reverse", dd.DD_DIV_KL_REVERSE, 0.0)]
    fdiv_sec = {"workload": stream_sec["workload"], "kernel": "fdiv_kernel (+ stage_targets_kernel)", "bound": "hbm",
                "unit": "GB/s", "peak": pk.get("hbm_gbs"), "peak_source": pk_kind, "families": {}}
    for name, fam, prm in fams:
        dd.dd_divergence(ctx, mid, [tl[0]], fam, prm, out_f)
        it2 = iter(tl * 4)
        ms_f = timed(lambda: dd.dd_divergence(ctx, mid, [next(it2)], fam, prm, out_f), reps)
        gbs = (4.0 * n_v * k_pad + 4.0 * n_v) / (ms_f / 1e3) / 1e9
        fdiv_sec["families"][name] = {"ms": round(ms_f, 4), "achieved": round(gbs, 1),
                                      "frac": round(gbs / pk.get("hbm_gbs", 6672.5), 4)}
    stream_sec["other_f_divergences"] = fdiv_sec
    klt_ms = fdiv_sec["families"]["kl_reverse"]["ms"]
    stream_sec["sparse"] = sparse_subsection(dd, ctx, dev, stream, flush, mid, n_v, k, k_pad, tl, pk, pk_kind, reps,
                                             dense_ms=med, dense_klt_ms=klt_ms, orows=orows)
    if own:
        dd.dd_unload_mesh(ctx, mid)
    return stream_sec, gemm_sec


def sparse_subsection(dd, ctx, dev, stream, flush, mid, n_v, k, k_pad, tl, pk, pk_kind, reps, dense_ms=None,
                      dense_klt_ms=None, orows=None):
    """Sparse fields of Section V (each row's entries below 1/sqrt(n) of its
    maximum eliminated), one target per call.  KL~ and TV~ read only the CSR
    copy of the sparsified P (csr_stream_kernel): algorithmic bytes of a call =
    6 B per kept entry (value + 16-bit column) + 8 B per row offset + the two
    output fields.  KLT~ reads the dense rows at the target's kept 4-column
    blocks (sparse_field_kernel): 16 B x n x listed blocks + the output.  With
    oracle rows: the device's sparse fields against the oracle's sparse fields
    (parity; rows with an entry within FP32 rounding of its threshold counted
    apart) and against the oracle's dense fields (the approximation), FP64,
    on the sampled rows."""
    import torch
    from oracle import sparse as osp
    t0 = time.perf_counter()
    kept, csr_bytes = dd.dd_sparsify(ctx, mid)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    P = torch.empty((n_v, k), dtype=torch.float32, device=dev)
    dd.dd_get_poisson_kernel(ctx, mid, P)
    theta32 = torch.tensor(1.0 / math.sqrt(n_v), dtype=torch.float32, device=dev)
    use = tl[:reps]

    def listed_blocks(t):
        row = torch.zeros(k_pad, dtype=torch.float32, device=dev)
        row[:k] = P[t]
        keep = (row >= theta32 * row.max()) & (row > 0)
        return int(keep.reshape(-1, 4).any(dim=1).sum().item())

    blocks = [listed_blocks(t) for t in use]
    del P
    out2 = torch.empty((2, 1, n_v), dtype=torch.float32, device=dev)
    out1 = torch.empty((1, 1, n_v), dtype=torch.float32, device=dev)
    for t in use[:3]:
        dd.dd_distance(ctx, mid, [t], 3, dd.DD_PREC_SPARSE, out2)
        dd.dd_distance(ctx, mid, [t], dd.DD_F_KLT, dd.DD_PREC_SPARSE, out1)
    torch.cuda.synchronize()

    def timed(fn):
        ms = []
        for t in use:
            flush.fill_(0.5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(t)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms

    ms_csr = timed(lambda t: dd.dd_distance(ctx, mid, [t], 3, dd.DD_PREC_SPARSE, out2))
    ms_klt = timed(lambda t: dd.dd_distance(ctx, mid, [t], dd.DD_F_KLT, dd.DD_PREC_SPARSE, out1))
    csr_alg = 6.0 * kept + 8.0 * (n_v + 1) + 8.0 * n_v
    g_csr = statistics.median([csr_alg / (m / 1e3) / 1e9 for m in ms_csr])
    g_klt = statistics.median([(16.0 * n_v * b + 4.0 * n_v) / (m / 1e3) / 1e9 for m, b in zip(ms_klt, blocks)])
    hbm = pk.get("hbm_gbs", 6672.5)
    res = {"reading": "Section V: each row's entries below max/sqrt(n) eliminated; KL~ over the field row's kept "
                      "entries, KLT~ over the target row's kept columns, TV~ between the sparsified rows",
           "sparsity": round(1.0 - kept / float(n_v * k), 4), "csr_bytes": int(csr_bytes),
           "dense_bytes": int(4 * n_v * k_pad), "build_seconds": round(build_s, 3),
           "kl_tv": {"kernel": "csr_stream_kernel (+ stage_targets_kernel, sparse_stage_kernel)", "bound": "hbm",
                     "ms_per_field_pair": round(statistics.median(ms_csr), 4), "achieved": round(g_csr, 1),
                     "peak": hbm, "unit": "GB/s", "frac": round(g_csr / hbm, 4), "peak_source": pk_kind,
                     "algorithmic_bytes": int(csr_alg),
                     "speedup_vs_dense": round(dense_ms / statistics.median(ms_csr), 2) if dense_ms else None},
           "klt": {"kernel": "sparse_field_kernel (+ stage_targets_kernel, sparse_stage_kernel)", "bound": "hbm",
                   "ms_per_field": round(statistics.median(ms_klt), 4), "achieved": round(g_klt, 1), "peak": hbm,
                   "unit": "GB/s", "frac": round(g_klt / hbm, 4), "listed_blocks_mean": round(float(np.mean(blocks)), 1),
                   "dense_blocks": int(k_pad // 4),
                   "speedup_vs_dense_klt": round(dense_klt_ms / statistics.median(ms_klt), 2) if dense_klt_ms else None},
           "traffic": None}
    if orows is not None:
        nt = 16
        tg = [int(t) for t in orows.targets[:nt]]
        out3 = torch.empty((3, nt, n_v), dtype=torch.float32, device=dev)
        dd.dd_distance(ctx, mid, tg, dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_SPARSE, out3)
        g = out3[:, :, torch.as_tensor(orows.rows, device=dev)].cpu().numpy()
        del out3
        theta = osp.default_theta(n_v)
        thr = theta * orows.Px.max(axis=1, keepdims=True)
        border_rows = (np.abs(orows.Px - thr) <= 8.0 * 2.0 ** -24 * thr).any(axis=1)
        par = {"kl": [], "tv": [], "klt": []}
        apx = {"kl": [], "tv": [], "klt": []}
        from oracle.divergence import kl_field_fast, tv_field
        from oracle.fdiv import kl_reverse_field
        R = len(orows.rows)
        for a in range(nt):
            Ps = np.vstack([orows.Px, orows.Pt[a][None, :]])
            refs = {"kl": osp.sparse_kl_field(Ps, R, theta)[:R], "tv": osp.sparse_tv_field(Ps, R, theta)[:R],
                    "klt": osp.sparse_klt_field(Ps, R, theta)[:R]}
            dense = {"kl": kl_field_fast(orows.Px, orows.Pt[a]), "tv": tv_field(orows.Px, orows.Pt[a]),
                     "klt": kl_reverse_field(orows.Px, orows.Pt[a])}
            for f, i in (("kl", 0), ("tv", 1), ("klt", 2)):
                ok = ~border_rows & np.isfinite(refs[f])
                par[f].append(np.abs(g[i, a][ok] - refs[f][ok]) / np.maximum(np.abs(refs[f][ok]), 1e-2))
                fin = np.isfinite(dense[f])
                apx[f].append(np.abs(g[i, a][fin] - dense[f][fin]) / np.maximum(np.abs(dense[f][fin]), 1e-2))
        res["parity_vs_oracle_sparse"] = {f: {"max": float(np.max(np.concatenate(v))),
                                              "median": float(np.median(np.concatenate(v))), "tol": 1e-5}
                                          for f, v in par.items()}
        res["parity_vs_oracle_sparse"]["rows_left_out"] = int(border_rows.sum())
        res["approximation_vs_oracle_dense"] = {f: {"max": float(np.max(np.concatenate(v))),
                                                    "median": float(np.median(np.concatenate(v)))}
                                                for f, v in apx.items()}
        res["error_sample"] = "%d sampled rows x %d targets, FP64 oracle rows, relative with floor 1e-2" % (R, nt)
    return res


def maze_section(dd, ctx, dev, n_targets: int = 64):
    """log P on a maze-like domain (Section V, Precision): a serpentine
    corridor of 6 x 4 x 40 cells whose kernel reaches 1e-76.  The device
    solve, the full-precision refinement (sweeps, seconds), and the FP32 KL
    and TV fields of targets spread over the maze against the oracle's
    subtraction-free kernel, before the refinement (log P[t,b] evaluated at
    FLT_MIN where FP32 P is 0) and after it."""
    import torch
    from oracle.divergence import kl_field_fast, tv_field
    from oracle.logpoisson import poisson_subtraction_free
    from synthetic.meshes import serpentine
    mesh = serpentine(6, 4, 40)
    t0 = time.perf_counter()
    P = poisson_subtraction_free(mesh.xy, mesh.tri, mesh.loops)
    oracle_s = time.perf_counter() - t0
    interior = np.nonzero(~mesh.boundary_flags())[0]
    targets = [int(interior[i]) for i in np.linspace(0, len(interior) - 1, n_targets).astype(int)]
    idx, off = mesh.loop_arrays()
    mid = dd.dd_load_mesh(ctx, mesh.xy, mesh.tri, idx, off)
    t0 = time.perf_counter()
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
    pcg_s = time.perf_counter() - t0
    out = torch.empty((2, len(targets), mesh.n_v), dtype=torch.float32, device=dev)

    def errors():
        dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, out)
        g = out.cpu().numpy().astype(np.float64)
        ek, et = [], []
        for a, t in enumerate(targets):
            rk, rt = kl_field_fast(P, P[t]), tv_field(P, P[t])
            fin = np.isfinite(rk)
            ek.append(np.max(np.abs(g[0, a][fin] - rk[fin]) / np.maximum(np.abs(rk[fin]), 1e-2)))
            et.append(np.max(np.abs(g[1, a] - rt) / np.maximum(np.abs(rt), 1e-2)))
        return {"kl_max": float(np.max(ek)), "kl_median": float(np.median(ek)), "tv_max": float(np.max(et))}

    before = errors()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sweeps, change = dd.dd_log_poisson_kernel(ctx, mid, 1e-14, 200000)
    refine_s = time.perf_counter() - t0
    after = errors()
    dd.dd_unload_mesh(ctx, mid)
    pos = P[P > 0]
    return {"workload": "serpentine maze 6 x 4 x 40 cells: n=%d, k=%d; %d targets spread over the interior"
                        % (mesh.n_v, sum(len(l) for l in mesh.loops), len(targets)),
            "kernel_min": float(pos.min()), "share_below_flt_min": round(float(np.mean(pos < 1.1754944e-38)), 4),
            "pcg_seconds": round(pcg_s, 3), "refine": {"sweeps": sweeps, "last_change": change,
                                                       "seconds": round(refine_s, 3)},
            "fields_vs_oracle_before_refinement": before, "fields_vs_oracle_after_refinement": after,
            "tolerance": "1e-5 relative, floor 1e-2", "oracle_seconds": round(oracle_s, 2)}


def mid_section(dd, ctx, dev, stream, flush, pk, pk_kind, reps: int = 8):
    """A mid-size grid for full ncu captures (a few GB on the device): N = 300
    with 12 obstacles (n = 86,449, k = 2,122, P = 0.73 GB, larger than L2).
    The single-target dense stream (KL+TV), the sparse pass (KL+TV, Section V),
    the split-BF16 KL GEMM, the FP32 KL+TV pass for 512 targets and the
    alpha (0.5) and reverse-KL fields of one target, each timed with CUDA
    events (L2 flushed before every launch)."""
    import torch
    from synthetic import workloads
    T = 512
    wl = workloads.grid(300, 12, 8, 30, False, T, 0, 170802845 + 400, "grid300")
    idx, off = wl.mesh.loop_arrays()
    mid = dd.dd_load_mesh(ctx, wl.mesh.xy, wl.mesh.tri, idx, off)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
    info = dd.dd_mesh_info(ctx, mid)
    n_v, k, k_pad = info["n_v"], info["k"], info["k_pad"]
    tl = [int(t) for t in wl.targets]

    def timed(fn, n_rep):
        ms = []
        for i in range(n_rep):
            flush.fill_(0.5)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(i)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    out1 = torch.empty((2, 1, n_v), dtype=torch.float32, device=dev)
    dd.dd_sparsify(ctx, mid)
    for prec in (dd.DD_PREC_FP32, dd.DD_PREC_SPARSE):
        dd.dd_distance(ctx, mid, [tl[0]], 3, prec, out1)
    dense_ms = timed(lambda i: dd.dd_distance(ctx, mid, [tl[i]], 3, dd.DD_PREC_FP32, out1), reps)
    sparse_ms = timed(lambda i: dd.dd_distance(ctx, mid, [tl[i]], 3, dd.DD_PREC_SPARSE, out1), reps)
    outk = torch.empty((1, T, n_v), dtype=torch.float32, device=dev)
    dd.dd_distance(ctx, mid, tl, 1, dd.DD_PREC_BF16X3, outk)
    gemm_ms = timed(lambda i: dd.dd_distance(ctx, mid, tl, 1, dd.DD_PREC_BF16X3, outk), 4)
    # the FP32 many-target pass (field tile kernel + exact recompute), KL+TV
    out2 = torch.empty((2, T, n_v), dtype=torch.float32, device=dev)
    dd.dd_distance(ctx, mid, tl, 3, dd.DD_PREC_FP32, out2)      # the first call runs the tile autotuner
    tile_ms = timed(lambda i: dd.dd_distance(ctx, mid, tl, 3, dd.DD_PREC_FP32, out2), 4)
    # two f-divergence families of the two-pass kernel, one target per call
    outd = torch.empty((1, n_v), dtype=torch.float32, device=dev)
    fdiv = {}
    for name, fam, prm in (("alpha0.5", dd.DD_DIV_ALPHA, 0.5), ("kl_reverse", dd.DD_DIV_KL_REVERSE, 0.0)):
        dd.dd_divergence(ctx, mid, [tl[0]], fam, prm, outd)
        f_ms = timed(lambda i: dd.dd_divergence(ctx, mid, [tl[i]], fam, prm, outd), reps)
        fdiv[name] = {"ms": round(f_ms, 4), "gbs": round(4.0 * n_v * k_pad / (f_ms / 1e3) / 1e9, 1)}
    dd.dd_unload_mesh(ctx, mid)
    issued = 3 * 2.0 * n_v * k * T / (gemm_ms / 1e3) / 1e12
    return {"workload": "grid300: n=%d, k=%d, P=%.2f GB FP32" % (n_v, k, 4.0 * n_v * k_pad / 1e9),
            "dense_stream_ms": round(dense_ms, 4),
            "dense_stream_gbs": round(4.0 * n_v * k_pad / (dense_ms / 1e3) / 1e9, 1),
            "sparse_ms": round(sparse_ms, 4), "gemm_T": T, "gemm_ms": round(gemm_ms, 4),
            "fp32_fields_ms": round(tile_ms, 4), "tile_shapes": dd.dd_tuning_table().strip().splitlines(),
            "f_divergences": fdiv,
            "gemm_tflops_issued": round(issued, 1), "peak_bf16": pk.get("bf16_tflops"), "peak_source": pk_kind}


def batch_section(dd, ctx, dev, stream, flush, args, S: int = 64, max_pts: int = 1536):
    """64 uneven grid domains (n log-uniform in [5k, 100k], 0..16 obstacles,
    16..256 targets each, 64 traced paths per target): one dd_query_batch per
    step -- all KL+TV fields in one persistent launch with autotuned tiles,
    all paths in one tracer launch."""
    import torch
    from synthetic import workloads
    wls = workloads.batch64(S=S)
    mids, Ts, tg, sr = [], [], [], []
    t0 = time.perf_counter()
    pcg_iters = 0
    for wl in wls:
        idx, off = wl.mesh.loop_arrays()
        mid = dd.dd_load_mesh(ctx, wl.mesh.xy, wl.mesh.tri, idx, off)
        it, _ = dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
        pcg_iters += it
        mids.append(mid)
        Ts.append(len(wl.targets))
        tg.append(np.asarray(wl.targets, np.int32))
        sr.append(np.asarray(wl.sources, np.int32).reshape(-1))
    pre = time.perf_counter() - t0
    tg = np.concatenate(tg)
    sr = np.concatenate(sr)
    n_vs = [wl.mesh.n_v for wl in wls]
    ks = [dd.dd_mesh_info(ctx, m)["k"] for m in mids]
    nT = int(sum(Ts))
    n_f = int(sum(2 * T * n for T, n in zip(Ts, n_vs)))
    out = torch.empty(n_f, dtype=torch.float32, device=dev)
    xy = torch.empty((nT * S, max_pts, 2), dtype=torch.float32, device=dev)
    ln = torch.empty(nT * S, dtype=torch.int32, device=dev)
    st = torch.empty(nT * S, dtype=torch.int32, device=dev)

    def q():
        dd.dd_query_batch(ctx, mids, Ts, tg, sr, S, 3, 1, max_pts, out, xy, ln, st)

    q()                       # first call runs the autotuner for new size classes
    for _ in range(2):
        q()
    torch.cuda.synchronize()
    ms = []
    dd.dd_kernel_timing(ctx, 1)
    for _ in range(max(3, min(args.steps, 10))):
        flush.fill_(0.25)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    kt = dd.dd_kernel_timing(ctx, 0)
    ktot = sum(v for _, v in kt.values()) or 1.0
    kernels = {n: {"launches": c, "ms_per_launch": round(v / max(c, 1), 4), "share": round(v / ktot, 4)}
               for n, (c, v) in sorted(kt.items(), key=lambda kv: -kv[1][1])}
    med = statistics.median(ms)
    stn = st.cpu().numpy()
    elem_targets = float(sum(T * n * k for T, n, k in zip(Ts, n_vs, ks)))
    for mid in mids:
        dd.dd_unload_mesh(ctx, mid)
    return {"workload": "batch64: %d grid domains, n %d..%d, k %d..%d, %d targets (16..256 per domain), %d paths"
                        % (len(wls), min(n_vs), max(n_vs), min(ks), max(ks), nT, nT * S),
            "ms_per_batch": round(med, 3), "fields_per_s": round(2 * nT / (med / 1e3), 1),
            "paths_per_s": round(nT * S / (med / 1e3), 1),
            "field_fp32_instructions_per_batch": 4.0 * elem_targets, "paths_ok_frac": float(np.mean(stn == 0)),
            "tile_shapes": dd.dd_tuning_table().strip().splitlines(), "kernels": kernels,
            "preproc": {"pcg_iters_total": pcg_iters, "seconds": round(pre, 2)},
            "launches_per_batch": round(sum(c for c, _ in kt.values()) / max(len(ms), 1), 2)}


def census_section(dd, ctx, dev, sizes=(175, 500, 2000, 10000, 40000), seeds=(1, 2, 3, 4),
                   max_targets: int = 1024):
    """Spurious-local-minimum census (Section V): on convex-holes Delaunay
    meshes of growing resolution (the same four domains at every size), the
    share of targets whose TV field, KL field and target-weighted KL field
    (the reverse direction, Sum_b P[t,b] log(P[t,b]/P[x,b])), the sparse KL,
    TV and target-weighted KL fields of Section V (each row's entries below
    1/sqrt(n) of its maximum eliminated, the weight row deciding the terms),
    and the merged-bin target-weighted KL (an extension: the target row's
    small entries merged into one bin), have an interior vertex other than
    the target with no lower neighbour.  All interior
    targets up to max_targets, else max_targets spread evenly over them.
    Everything runs through the library: the FP64 kernel solve, the FP32
    fields, the minimum test."""
    import torch
    from synthetic.meshes import convex_holes
    rows = []
    t0 = time.perf_counter()
    for n_goal in sizes:
        agg = {"n_goal": n_goal, "meshes": 0, "n_v": [], "k": [], "targets": 0,
               "tv": [0, 0], "kl": [0, 0], "kl_target_weighted": [0, 0], "kl_sparse": [0, 0], "tv_sparse": [0, 0],
               "kl_target_weighted_sparse": [0, 0], "kl_target_weighted_merged": [0, 0]}
        for seed in seeds:
            mesh = convex_holes(n_goal, seed=seed)
            idx, off = mesh.loop_arrays()
            mid = dd.dd_load_mesh(ctx, mesh.xy, mesh.tri, idx, off)
            dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
            interior = np.nonzero(~mesh.boundary_flags())[0]
            if len(interior) > max_targets:
                interior = interior[np.linspace(0, len(interior) - 1, max_targets).astype(np.int64)]
            targets = interior.astype(np.int32)
            T = len(targets)
            fields = torch.empty((2, T, mesh.n_v), dtype=torch.float32, device=dev)
            dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, fields)
            rev = torch.empty((T, mesh.n_v), dtype=torch.float32, device=dev)
            dd.dd_divergence(ctx, mid, targets, dd.DD_DIV_KL_REVERSE, 0.0, rev)
            dd.dd_sparsify(ctx, mid)
            sparse_f = torch.empty((3, T, mesh.n_v), dtype=torch.float32, device=dev)
            dd.dd_distance(ctx, mid, targets, dd.DD_F_KL | dd.DD_F_TV | dd.DD_F_KLT, dd.DD_PREC_SPARSE, sparse_f)
            merged_f = torch.empty((1, T, mesh.n_v), dtype=torch.float32, device=dev)
            dd.dd_distance(ctx, mid, targets, dd.DD_F_KLT, dd.DD_PREC_SPARSE_MERGED, merged_f)
            for name, f in (("kl", fields[0]), ("tv", fields[1]), ("kl_target_weighted", rev),
                            ("kl_sparse", sparse_f[0]), ("tv_sparse", sparse_f[1]),
                            ("kl_target_weighted_sparse", sparse_f[2]), ("kl_target_weighted_merged", merged_f[0])):
                c = dd.dd_local_minima(ctx, mid, f.contiguous(), targets, None)
                agg[name][0] += int(np.count_nonzero(c))
                agg[name][1] += int(c.sum())
            agg["meshes"] += 1
            agg["n_v"].append(mesh.n_v)
            agg["k"].append(dd.dd_mesh_info(ctx, mid)["k"])
            agg["targets"] += T
            dd.dd_unload_mesh(ctx, mid)
        for name in ("tv", "kl", "kl_target_weighted", "kl_sparse", "tv_sparse", "kl_target_weighted_sparse",
                     "kl_target_weighted_merged"):
            agg[name] = {"targets_with_minima": agg[name][0], "minima": agg[name][1],
                         "share": round(agg[name][0] / agg["targets"], 4)}
        rows.append(agg)
    return {"workload": "convex_holes(n, seed 1..4): unit disk minus 4 convex polygons, Delaunay; "
                        "all interior targets up to %d per mesh" % max_targets,
            "rows": rows, "paths": path_shapes(dd, ctx, dev), "seconds": round(time.perf_counter() - t0, 2)}


def path_shapes(dd, ctx, dev, n_goal: int = 10000, T: int = 32, S: int = 32, max_pts: int = 4096):
    """Fig. 2: paths that cut through triangles against paths along edges, on
    the same target-weighted KL fields of one convex-holes mesh: the share of
    paths that reach the target and the mean length of those that do."""
    import torch
    from synthetic.meshes import convex_holes
    from synthetic.rng import SplitMix64
    mesh = convex_holes(n_goal, seed=1)
    idx, off = mesh.loop_arrays()
    mid = dd.dd_load_mesh(ctx, mesh.xy, mesh.tri, idx, off)
    dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
    interior = np.nonzero(~mesh.boundary_flags())[0]
    rng = SplitMix64(170802845 + 7)
    targets = [int(interior[rng.choice(len(interior))]) for _ in range(T)]
    sources = np.array([[int(interior[rng.choice(len(interior))]) for _ in range(S)] for _ in range(T)], np.int32)
    f = torch.empty((1, T, mesh.n_v), dtype=torch.float32, device=dev)
    dd.dd_distance(ctx, mid, targets, dd.DD_F_KLT, dd.DD_PREC_FP32, f)
    out = {}
    for name, fn in (("triangles", dd.dd_trace_fields), ("edges", dd.dd_trace_edges)):
        xy = torch.empty((T * S, max_pts, 2), dtype=torch.float32, device=dev)
        ln = torch.empty(T * S, dtype=torch.int32, device=dev)
        st = torch.empty(T * S, dtype=torch.int32, device=dev)
        fn(ctx, mid, f[0].contiguous(), targets, sources, max_pts, xy, ln, st)
        torch.cuda.synchronize()
        xy, ln, st = xy.cpu().numpy(), ln.cpu().numpy(), st.cpu().numpy()
        lens = [float(np.sum(np.hypot(*np.diff(xy[i, :ln[i]], axis=0).T))) for i in range(T * S) if st[i] == 0]
        out[name] = {"ok_share": round(float(np.mean(st == 0)), 4), "mean_length": round(float(np.mean(lens)), 4),
                     "mean_points": round(float(np.mean(ln[st == 0])), 1)}
    out["edge_over_triangle_length"] = round(out["edges"]["mean_length"] / out["triangles"]["mean_length"], 4)
    out["workload"] = "convex_holes(%d, seed 1): n=%d; %d targets x %d sources on the target-weighted KL field" % (
        n_goal, mesh.n_v, T, S)
    dd.dd_unload_mesh(ctx, mid)
    return out


def serve_section(dd, ctx, args, n_domains: int, seconds: float, rate: float = 2000.0, max_pts: int = 2048):
    """Served (continuous batching) vs plain per-query form on the serving workload.

    Resident grid domains (n log-uniform in [10k, 500k]; n_domains smallest of
    the 8-domain recipe when fewer are asked), Poisson arrivals at `rate` q/s
    for `seconds`; each query = a random interior target plus S sources,
    S log-uniform in [1, 1024].  Both forms replay the arrivals in real time;
    latency = arrival -> paths in host memory."""
    from synthetic import workloads
    doms = workloads.serving_domains()
    order = sorted(range(len(doms)), key=lambda i: doms[i].mesh.n_v)[:n_domains]
    doms = [doms[i] for i in sorted(order)]
    t0 = time.perf_counter()
    mids, pre_dom = [], []
    for wl in doms:
        t1 = time.perf_counter()
        idx, off = wl.mesh.loop_arrays()
        mid = dd.dd_load_mesh(ctx, wl.mesh.xy, wl.mesh.tri, idx, off)
        t2 = time.perf_counter()
        it, _ = dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
        info = dd.dd_mesh_info(ctx, mid)
        pre_dom.append({"n_v": info["n_v"], "k": info["k"], "load_s": round(t2 - t1, 2), "pcg_iters": it,
                        "pcg_s": round(time.perf_counter() - t2, 2)})
        mids.append(mid)
    pre = time.perf_counter() - t0
    qs = workloads.serving_queries(doms, rate_qps=rate, duration_s=seconds)
    # ---- served
    sv = dd.dd_server_create(ctx, 32 << 30, n_slots=4, max_batch=256, max_pts=max_pts)
    lat = {}
    refused = 0
    start = time.perf_counter()
    pos = 0
    while pos < len(qs):
        now = time.perf_counter() - start
        while pos < len(qs) and qs[pos][0] <= now:
            t, d, tgt, src = qs[pos]
            if dd.dd_server_submit(sv, pos, mids[d], tgt, src) != dd.DD_OK:
                refused += 1
            pos += 1
        ids, sts, ls = dd.dd_server_poll(sv)
        for i, l in zip(ids, ls):
            lat[int(i)] = float(l)
        time.sleep(0.0002)
    dd.dd_server_wait_idle(sv, 600.0)
    served_wall = time.perf_counter() - start
    ids, sts, ls = dd.dd_server_poll(sv, 1 << 20)
    for i, l in zip(ids, ls):
        lat[int(i)] = float(l)
    paths_ok = []
    for i in list(lat.keys())[:200]:
        S = len(qs[i][3])
        _, _, st = dd.dd_server_take(sv, i, S, max_pts)
        paths_ok.append(float(np.mean(st == 0)))
    dd.dd_server_destroy(sv)
    L = np.asarray(list(lat.values()))
    # ---- plain per-query form (the same arrivals, one query at a time, host buffers)
    n_plain = len(qs)
    plat = []
    start = time.perf_counter()
    for i in range(n_plain):
        t, d, tgt, src = qs[i]
        while time.perf_counter() - start < t:
            pass
        S = len(src)
        hf = np.empty((1, 1, doms[d].mesh.n_v), np.float32)
        hxy = np.empty((S, max_pts, 2), np.float32)
        hl = np.empty(S, np.int32)
        hs = np.empty(S, np.int32)
        dd.dd_query(ctx, mids[d], [tgt], src.reshape(1, -1), dd.DD_F_KL, dd.DD_PREC_FP32, dd.DD_F_KL, max_pts,
                    hf, hxy, hl, hs)
        plat.append((time.perf_counter() - start - t) * 1e3)
    for mid in mids:
        dd.dd_unload_mesh(ctx, mid)
    PL = np.asarray(plat)
    return {"workload": "serving: %d resident grid domains (n %d..%d, k %d..%d), Poisson arrivals %.0f q/s for %.1f s, "
                        "S log-uniform in [1, 1024]" % (len(doms), min(w.mesh.n_v for w in doms),
                                                         max(w.mesh.n_v for w in doms),
                                                         min(sum(len(l) for l in w.mesh.loops) for w in doms),
                                                         max(sum(len(l) for l in w.mesh.loops) for w in doms),
                                                         rate, seconds),
            "served": {"queries": len(qs), "completed": int(L.size), "refused": refused,
                       "qps": round(L.size / served_wall, 1),
                       "p50_ms": round(float(np.percentile(L, 50)), 3), "p99_ms": round(float(np.percentile(L, 99)), 3),
                       "paths_ok_frac_sample": round(float(np.mean(paths_ok)), 4) if paths_ok else None,
                       "slots": 4, "max_batch": 256},
            "plain": {"queries": n_plain, "p50_ms": round(float(np.percentile(PL, 50)), 3),
                      "p99_ms": round(float(np.percentile(PL, 99)), 3),
                      "qps": round(n_plain / (time.perf_counter() - start), 1),
                      "form": "one dd_query per query (T=1, host buffers), in arrival order, all %d queries"
                              % n_plain},
            "preproc_s": round(pre, 2), "preproc_domains": pre_dom}


# ---------------------------------------------------------------- the oracle on the host cores
# The oracle's FP64 Poisson kernel of the workload lives in shared memory,
# filled by spawned workers (each factorises -L_II itself and solves a block of
# columns, Eq. 33); the same workers then time the oracle's fields (Eq. 34-35
# over every vertex) and paths, one task per core at a time.  Spawned, not
# forked: the parent has used CUDA by then.
_HOST = {}


def _host_init(name, shm_name, n, k):
    from multiprocessing import shared_memory
    w = WORKLOADS[name]
    wl = make_workload(name, w["T"], w["S"])
    shm = shared_memory.SharedMemory(name=shm_name)
    _HOST.update(wl=wl, shm=shm, P=np.ndarray((n, k), dtype=np.float64, buffer=shm.buf), po=None, tracer=None)


def _host_columns(cols):
    from oracle.poisson import PoissonOracle
    if _HOST["po"] is None:
        wl = _HOST["wl"]
        _HOST["po"] = PoissonOracle(wl.mesh.xy, wl.mesh.tri, wl.mesh.loops)
    po = _HOST["po"]
    c0, c1 = int(cols[0]), int(cols[-1]) + 1
    X = po.lu.solve(po.L_IB[:, c0:c1].toarray())       # -L_II X = L_IB
    P = _HOST["P"]
    P[po.I, c0:c1] = X
    P[np.asarray(po.B)[c0:c1], np.arange(c0, c1)] = 1.0
    return c1 - c0


def _host_tracer():
    from oracle.trace import Tracer
    if _HOST["tracer"] is None:
        wl = _HOST["wl"]
        _HOST["tracer"] = Tracer(wl.mesh.xy, wl.mesh.tri)
    return _HOST["tracer"]


def _host_fields(t, r0, r1, keep=False, chunk=4096):
    """KL and TV of target t over rows [r0, r1), in row chunks (oracle.divergence)."""
    from oracle.divergence import kl_field_fast, tv_field
    P = _HOST["P"]
    pt = np.array(P[t])
    kl = np.empty(r1 - r0) if keep else None
    for a in range(r0, r1, chunk):
        b = min(r1, a + chunk)
        f = kl_field_fast(P[a:b], pt)
        tv_field(P[a:b], pt)
        if keep:
            kl[a - r0:b - r0] = f
    return kl


def _host_full(args):
    """One target's KL+TV over every vertex and one path traced on the KL field."""
    t, q = args
    tr = _host_tracer()
    n = _HOST["P"].shape[0]
    c0 = time.perf_counter()
    kl = _host_fields(int(t), 0, n, keep=True)
    c1 = time.perf_counter()
    path, st = tr.trace(kl, int(q), int(t), max_pts=WORKLOADS[_HOST["wl"].name]["max_pts"])
    c2 = time.perf_counter()
    return c1 - c0, c2 - c1, int(st), len(path)


def _host_path_only(args):
    """The paper's CPU scheme (Section V, Table I): one path, KL evaluated only
    at the vertices the walk reads."""
    from oracle.trace import PathOnlyField
    t, q = args
    tr = _host_tracer()
    c0 = time.perf_counter()
    f = PathOnlyField(_HOST["P"], int(t), "kl")
    path, st = tr.trace(f, int(q), int(t), max_pts=WORKLOADS[_HOST["wl"].name]["max_pts"])
    return time.perf_counter() - c0, f.evaluated, int(st), len(path)


def _host_ref_task(args):
    """One core's share of a reference-arm step: strip j of n_strips of one
    target's KL+TV field, and one path by the path-only scheme."""
    t, j, n_strips, q = args
    n = _HOST["P"].shape[0]
    c0 = time.perf_counter()
    _host_fields(int(t), j * n // n_strips, (j + 1) * n // n_strips)
    c1 = time.perf_counter()
    s, ev, st, npts = _host_path_only((t, q))
    return c1 - c0, s, ev, st


class HostOracle:
    """The oracle's FP64 P of a workload in shared memory plus a spawned pool
    of one single-threaded worker per host core."""

    def __init__(self, name: str, cores: int):
        import multiprocessing
        from concurrent.futures import ProcessPoolExecutor
        from multiprocessing import shared_memory
        from oracle.topology import split_boundary
        w = WORKLOADS[name]
        wl = make_workload(name, w["T"], w["S"])
        n = wl.mesh.n_v
        k = len(split_boundary(n, wl.mesh.tri, wl.mesh.loops)[0])
        self.name, self.n, self.k, self.cores = name, n, k, cores
        self.shm = shared_memory.SharedMemory(create=True, size=n * k * 8)
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        try:
            self.pool = ProcessPoolExecutor(max_workers=cores, mp_context=multiprocessing.get_context("spawn"),
                                            initializer=_host_init, initargs=(name, self.shm.name, n, k))
            t0 = time.perf_counter()
            blocks = [b for b in np.array_split(np.arange(k), 2 * cores) if len(b)]
            list(self.pool.map(_host_columns, blocks))
            self.kernel_s = time.perf_counter() - t0
        finally:
            for v, val in saved.items():
                if val is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = val

    def map(self, fn, tasks):
        return list(self.pool.map(fn, tasks))

    def close(self):
        self.pool.shutdown()
        self.shm.close()
        self.shm.unlink()


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(name: str = HEADLINE):
    """fields/s of the oracle with every host core busy: each core takes one
    target of the step's first batch and computes its KL+TV over every vertex
    (then traces one path on the KL field); beside it the paper's CPU scheme,
    one path per core with KL evaluated only at the vertices the walk reads."""
    t0 = time.perf_counter()
    cores = host_cores()
    ho = HostOracle(name, cores)
    try:
        wl, batches = workload_batches(0, name)
        tg, sr = batches[0]
        full = ho.map(_host_full, [(int(tg[w]), int(sr[w][0])) for w in range(cores)])
        po = ho.map(_host_path_only, [(int(tg[w]), int(sr[w][1])) for w in range(cores)])
    finally:
        ho.close()
    field_s = statistics.mean(r[0] for r in full)
    return {"value": round(cores * 2.0 / field_s, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} targets of {name}'s first batch, one per core at once: KL+TV over all n = {ho.n} "
                      f"vertices each (FP64, from the oracle's P in shared memory, computed in "
                      f"{ho.kernel_s:.1f} s and not timed), then one path traced on the KL field",
            "full_field_trace_ms_per_path": round(1e3 * statistics.mean(r[1] for r in full), 2),
            "path_only": {"scheme": "Section V, Table I: KL only at the vertices the walk reads",
                          "ms_per_path": round(1e3 * statistics.mean(r[0] for r in po), 2),
                          "vertices_evaluated_per_path": round(float(np.mean([r[1] for r in po])), 1),
                          "points_per_path": round(float(np.mean([r[3] for r in po])), 1),
                          "ok_share": round(float(np.mean([r[2] == 0 for r in po])), 4)},
            "seconds": round(time.perf_counter() - t0, 2)}


def reference_arm(args):
    """The FP64 oracle as the reference arm, on every host core: per step each
    core takes one target of the step's batch (the GPU arm's targets, in
    order) and computes one eighth of its KL+TV field (rows j n/8 .. (j+1) n/8,
    j = step mod 8) and one path by the paper's path-only scheme.  The step's
    time is its wall time; fields/s counts each eighth as 1/8 field."""
    t0 = time.perf_counter()
    cores = host_cores()
    name = args.workload
    n_strips = 8
    ho = HostOracle(name, cores)
    try:
        wl, batches = workload_batches(0, name)

        def tasks(i):
            tg, sr = batches[i % len(batches)]
            base = (i // len(batches)) * cores
            return [(int(tg[(base + w) % len(tg)]), i % n_strips, n_strips, int(sr[(base + w) % len(tg)][0]))
                    for w in range(cores)]

        for i in range(args.warmup):
            ho.map(_host_ref_task, tasks(i))
        walls, evals = [], []
        for i in range(args.steps):
            c0 = time.perf_counter()
            res = ho.map(_host_ref_task, tasks(args.warmup + i))
            walls.append(time.perf_counter() - c0)
            evals.extend(r[2] for r in res)
    finally:
        ho.close()
    fields_per_step = cores * 2.0 / n_strips
    v = fields_per_step * args.steps / sum(walls)
    w = WORKLOADS[name]
    return {"metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * sum(walls) / args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w["desc"] % (ho.n, ho.k, w["T"], w["T"], w["S"]),
                       "sample": f"per step {cores} of the step's targets (one per core): 1/{n_strips} of the rows "
                                 "of each KL+TV field and one path by the path-only scheme"},
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(v, 4),
                             "sample": f"per step {cores} targets at once (one per core): KL+TV over 1/{n_strips} "
                                       "of the vertices + one path-only trace each; ms_per_step is the step's wall "
                                       "time",
                             "vertices_evaluated_per_path": round(float(np.mean(evals)), 1)},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "preproc_s": round(ho.kernel_s, 1), "seconds": round(time.perf_counter() - t0, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=HEADLINE,
                    help="query-step workload of the reference arm and the CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-errors", dest="oracle_errors", action="store_false",
                    help="skip the error of the step's results against the FP64 oracle")
    ap.add_argument("--section", choices=["all", "step", "grid140", "grid450", "batch", "serve", "census", "mid",
                                          "maze"],
                    default="all",
                    help="step: only the grid450 query step (with its split-BF16 form and oracle errors); grid140, "
                         "grid450 (single-target, sparse, other-divergence and GEMM passes), batch, serve, census, "
                         "mid (a grid300 case small enough for full ncu captures), maze (log P): only that part")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(reference_arm(args)))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1 and args.section in ("all", "step"):
            line["cpu_baseline"] = cpu_baseline(args.workload)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
