"""Benchmark of the online divergence-distance path (fields + traced paths).

One step = one dd_query over a batch of the grid140 workload: KL and TV
fields of 64 interior targets over all n = 18,174 vertices (k = 1,028
boundary columns) and 64 x 256 paths traced on the KL fields.  The Poisson
kernel is computed once per domain before timing (the paper's
preprocessing) and reported separately.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one process per GPU under torch.distributed.run; every rank
processes its own target batches (weak scaling, no data-path collective).
`--impl reference` times the FP64 CPU oracle on a bounded sample of the
same workload (rank 0 only).

The JSON line: `value` from CUDA events around each step (inputs resident,
L2 flushed between steps outside the events), `e2e` through the same call
with pinned host buffers, `kernels` (live per-kernel times from the
library's own events), `roofline` for the dominant kernel with
`roofline_fields` / `roofline_walk` for the other of the two, `clocks`
sampled during the timed region (measured once more, with `remeasured`, if
they show a slowdown or a clock lock), `cpu_baseline` (the oracle on every
host core), `step_bf16x3` (the same step on the split-BF16 path), and with
no `--section` the grid450, batch, serving and census measurements.
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
T_BATCH, S_PER_TARGET, MAX_PTS = 64, 256, 1024
# kernels one dd_query step launches: target staging, field tile, exact KL
# recompute near the targets, triangle rates, vertex decisions, path walk
STEP_LAUNCHES = 6
# bytes the walk gathers and stores per point it appends: one 64-B triangle
# record, one 16-B rate vector, one 8-B point
WALK_BYTES_PER_POINT = 88
# DRAM bytes (read + write) of one field_tile_kernel launch of this step, from an
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum); P is read once
TILE_TRAFFIC_BYTES = 77092352        # 75,064,576 read + 2,027,776 written (P is 4 n k_pad = 74.7 MB; 64x64 shape)
# the same for one trace_kernel launch (records and rates mostly served by L2)
WALK_TRAFFIC_BYTES = 31522560        # 31,330,816 read + 191,744 written
# the same for one field_stream_kernel launch of the grid450 single-target pass
STREAM_TRAFFIC_BYTES = 3035740160    # 3,032,217,088 read + 3,523,072 written (4 n k_pad = 3.03 GB of P)
N_BATCHES = 8


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


def workload_batches(rank: int):
    from synthetic import workloads
    from synthetic.rng import SplitMix64
    wl = workloads.grid140(T=T_BATCH, S=S_PER_TARGET)
    # rank 0 starts with the workload's own batch; every other batch (and all of
    # another rank's) is drawn from a rank-seeded stream, so ranks share no work
    batches = [(wl.targets, wl.sources)] if rank == 0 else []
    rng = SplitMix64(workloads.BASE_SEED + 1000 + rank)
    while len(batches) < N_BATCHES:
        t = workloads.draw_targets(rng, wl.mesh, T_BATCH)
        s = workloads.draw_sources(rng, wl.mesh, t, S_PER_TARGET)
        batches.append((t, s))
    return wl, batches


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
    if args.section in ("grid450", "batch", "serve", "census", "mid"):
        pk, pk_kind = peaks()
        flush = torch.empty((256 << 20) // 4, dtype=torch.float32, device=dev)
        if args.section == "grid450":
            st_sec, gm_sec = grid450_sections(dd, ctx, dev, stream, flush, pk, pk_kind)
            out = {"metric": "grid450 sections only", "stream": st_sec, "gemm": gm_sec}
        elif args.section == "batch":
            out = {"metric": "batch64 section only", "batch": batch_section(dd, ctx, dev, stream, flush, args)}
        elif args.section == "census":
            out = {"metric": "census section only", "census": census_section(dd, ctx, dev)}
        elif args.section == "mid":
            out = {"metric": "grid300 section only", "mid": mid_section(dd, ctx, dev, stream, flush, pk, pk_kind)}
        else:
            out = {"metric": "serving section only", "serve": serve_section(dd, ctx, args, n_domains=8, seconds=10.0)}
        dd.dd_destroy(ctx)
        return out
    wl, batches = workload_batches(rank)
    mesh = wl.mesh
    idx, off = mesh.loop_arrays()
    mid = dd.dd_load_mesh(ctx, mesh.xy, mesh.tri, idx, off)
    info = dd.dd_mesh_info(ctx, mid)
    t0 = time.perf_counter()
    iters, resid = dd.dd_poisson_kernel(ctx, mid, 1e-15, 20000)
    preproc_s = time.perf_counter() - t0
    n_v, k, k_pad = info["n_v"], info["k"], info["k_pad"]

    T, S = T_BATCH, S_PER_TARGET
    fields = torch.empty((2, T, n_v), dtype=torch.float32, device=dev)
    pxy = torch.empty((T * S, MAX_PTS, 2), dtype=torch.float32, device=dev)
    plen = torch.empty(T * S, dtype=torch.int32, device=dev)
    pst = torch.empty(T * S, dtype=torch.int32, device=dev)
    l2_bytes = 256 << 20
    flush = torch.empty(l2_bytes // 4, dtype=torch.float32, device=dev)

    def step(i):
        tg, sr = batches[i % len(batches)]
        dd.dd_query(ctx, mid, tg, sr, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, dd.DD_F_KL, MAX_PTS,
                    fields, pxy, plen, pst)

    for i in range(args.warmup):
        flush.fill_(float(i))
        step(i)
    dd.dd_sync(ctx)
    torch.cuda.synchronize()

    # per-kernel split on the same stream (untimed for the metric): fields vs tracing
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tg, sr = batches[0]
    split_f, split_t = [], []
    for r in range(3):
        flush.fill_(1.0)
        ev[0].record(stream)
        dd.dd_distance(ctx, mid, tg, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_FP32, fields)
        ev[1].record(stream)
        dd.dd_trace_fields(ctx, mid, fields[0], tg, sr, MAX_PTS, pxy, plen, pst)
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
    hxy = torch.empty((T * S, MAX_PTS, 2), dtype=torch.float32).pin_memory()
    hl = torch.empty(T * S, dtype=torch.int32).pin_memory()
    hs = torch.empty(T * S, dtype=torch.int32).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    for i in range(2):
        tg, sr = batches[i]
        dd.dd_query(ctx, mid, tg, sr, 3, 0, 1, MAX_PTS, hf, hxy, hl, hs)
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for i in range(e2e_steps):
        tg, sr = batches[i % len(batches)]
        dd.dd_query(ctx, mid, tg, sr, 3, 0, 1, MAX_PTS, hf, hxy, hl, hs)
    e2e_s = time.perf_counter() - e0
    # into pinned host buffers the library moves exactly each path's defined
    # prefix (len points), plus the lengths and statuses (counted on the last
    # step's lengths)
    ln = hl.numpy()
    path_bytes = int(ln.astype(np.int64).sum()) * 8
    h2d = T * 4 + T * S * 4
    d2h = 2 * T * n_v * 4 + T * S * 8 + path_bytes

    fields_per_step = 2 * T
    value = world * fields_per_step * args.steps / (dev_ms / 1e3)
    pk, pk_kind = peaks()
    # dominant kernel (largest device time over the timed steps) and its roofline
    sm_mhz = clocks.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    tot = sum(ms for _, ms in kernel_ms.values()) or 1.0
    kernels = {name: {"launches": n, "ms_per_launch": round(ms / max(n, 1), 4), "share": round(ms / tot, 4)}
               for name, (n, ms) in sorted(kernel_ms.items(), key=lambda kv: -kv[1][1])}
    dom = max(kernel_ms, key=lambda k: kernel_ms[k][1]) if kernel_ms else "field_tile_kernel"
    dom_ms = kernel_ms[dom][1] / max(kernel_ms[dom][0], 1) if kernel_ms else field_ms
    walk_ms = kernel_ms["trace_kernel"][1] / max(kernel_ms["trace_kernel"][0], 1) if "trace_kernel" in kernel_ms else None
    walk_steps = int(np.clip(lens, 0, None).sum())
    tile_ms = kernel_ms["field_tile_kernel"][1] / max(kernel_ms["field_tile_kernel"][0], 1) \
        if "field_tile_kernel" in kernel_ms else field_ms
    # field tile: per (x, b, t) KL one FADD (log2 ratio) + one FFMA, TV two FADD = 4 FP32 instructions
    ops = 4.0 * n_v * k * T
    hbm_peak = float(pk["hbm_gbs"])
    peak_alu = 152 * 128 * sm_mhz * 1e6 / 1e12
    roof_tile = {"kernel": "field_tile_kernel", "bound": "alu", "achieved": round(ops / (tile_ms / 1e3) / 1e12, 3),
                 "peak": round(peak_alu, 3), "unit": "T FP32 instructions/s",
                 "frac": round(ops / (tile_ms / 1e3) / 1e12 / peak_alu, 4), "traffic": TILE_TRAFFIC_BYTES,
                 "algorithmic_fp32_ops": ops, "ms_per_launch": round(tile_ms, 4),
                 "peak_source": f"152 SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz (median SM clock sampled), one "
                                "FP32 instruction per lane per clock",
                 "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch, this workload"}
    if walk_ms is not None:
        # walk: per point appended, one 64-B triangle record and one 16-B rate gathered, one 8-B point stored
        wbytes = WALK_BYTES_PER_POINT * walk_steps
        roof_walk = {"kernel": "trace_kernel", "bound": "hbm", "achieved": round(wbytes / (walk_ms / 1e3) / 1e9, 1),
                     "peak": hbm_peak, "unit": "GB/s", "frac": round(wbytes / (walk_ms / 1e3) / 1e9 / hbm_peak, 4),
                     "traffic": WALK_TRAFFIC_BYTES, "algorithmic_bytes": wbytes, "ms_per_launch": round(walk_ms, 4),
                     "peak_source": "measured HBM copy bandwidth, burst",
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch, this workload",
                     "note": "a chain of dependent gathers (latency-bound): the records and rates (39 MB) are "
                             "L2-resident, so the DRAM traffic is far below the gathered bytes and the frac "
                             "against HBM shows the distance from any bandwidth roofline"}
    else:
        roof_walk = None
    dom = max(kernel_ms, key=lambda k: kernel_ms[k][1]) if kernel_ms else "field_tile_kernel"
    roof = roof_walk if (dom == "trace_kernel" and roof_walk is not None) else roof_tile
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(dev_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "grid140: unit square h=1/140, 8 square obstacles, n=%d, k=%d; 64 targets x "
                               "(KL+TV) + 64x256 KL paths per step" % (n_v, k),
                   "n_v": n_v, "k": k, "targets_per_step": T, "sources_per_target": S, "max_pts": MAX_PTS,
                   "l2": "flushed between steps (256 MB write outside the step events)",
                   "parallelism": f"replicas x{world}"},
        "paths_per_s": round(world * T * S * args.steps / (dev_ms / 1e3), 1),
        "walk_steps_per_s": round(walk_steps / (walk_ms / 1e3), 1) if walk_ms else None,
        "kernel_split_ms": {"fields": round(field_ms, 4), "trace": round(trace_ms, 4)},
        "paths_ok_frac": float(np.mean(status == 0)), "max_path_pts": int(lens.max()),
        "preproc": {"pcg_iters": iters, "resid": resid, "seconds": round(preproc_s, 3)},
        "wall_s_timed_region": round(wall, 4),
        "roofline": roof, "roofline_fields": roof_tile if roof is not roof_tile else None,
        "roofline_walk": roof_walk if roof is not roof_walk else None, "peaks": pk_kind,
        "e2e": {"value": round(world * fields_per_step * e2e_steps / e2e_s, 1), "unit": UNIT,
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(sum(n for n, _ in kernel_ms.values())) or STEP_LAUNCHES * args.steps,
        "kernels": kernels,
        "clocks": clocks,
    }
    if remeasured is not None:
        line["remeasured"] = remeasured
    line["step_bf16x3"] = bf16x3_step(dd, ctx, mid, batches, fields, pxy, plen, pst, flush, stream, args, T, S, n_v)
    if args.stream and args.section == "all":
        line["stream"], line["gemm"] = grid450_sections(dd, ctx, dev, stream, flush, pk, pk_kind)
        line["batch"] = batch_section(dd, ctx, dev, stream, flush, args)
        line["serve"] = serve_section(dd, ctx, args, n_domains=5, seconds=3.0)
        line["census"] = census_section(dd, ctx, dev)
    dd.dd_destroy(ctx)
    return line


def bf16x3_step(dd, ctx, mid, batches, fields, pxy, plen, pst, flush, stream, args, T, S, n_v):
    """The same query step with DD_PREC_BF16X3: the KL fields from the split-BF16
    tensor-core GEMM (error bound 1e-4 of S_x, not the FP32 path's 1e-5: not
    the headline), TV from a TV-only FP32 tile pass, the paths traced on the
    GEMM's KL fields.  Reports its time and the KL fields' largest deviation
    from the FP32 path's relative to max(|KL|, 1)."""
    import torch

    def step(i):
        tg, sr = batches[i % len(batches)]
        dd.dd_query(ctx, mid, tg, sr, dd.DD_F_KL | dd.DD_F_TV, dd.DD_PREC_BF16X3, dd.DD_F_KL, MAX_PTS,
                    fields, pxy, plen, pst)

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
    r, g = ref.cpu().numpy().astype(np.float64), got.cpu().numpy().astype(np.float64)
    fin = r[0] < 80.0
    dev_ms = float(sum(ms))
    return {"ms_per_step": round(dev_ms / args.steps, 4), "fields_per_s": round(2 * T * args.steps / (dev_ms / 1e3), 1),
            "kl_max_dev_vs_fp32": float(np.max(np.abs(g[0][fin] - r[0][fin]) / np.maximum(np.abs(r[0][fin]), 1.0))),
            "tv_identical": bool(np.array_equal(g[1], r[1])),
            "kernels": {n: {"launches": c, "ms_per_launch": round(v / max(c, 1), 4)} for n, (c, v) in kt.items()},
            "note": "KL through the tensor-core GEMM (split BF16, 1e-4 bound), TV through a TV-only FP32 pass"}


def grid450_sections(dd, ctx, dev, stream, flush, pk, pk_kind, reps: int = 10):
    """grid450 (n = 192,360, k = 3,936; P = 3.0 GB FP32, far above L2).

    stream: single-target KL+TV sweeps; the streaming kernel reads P once per
      target, achieved GB/s = (4 n k_pad + 8 n) bytes / event-timed dd_distance.
    gemm: 1,024 targets, KL through the split-BF16 tcgen05 GEMM; algorithmic
      2 n k T flop (three BF16 products issued), against the FP32 CUDA-core
      path for the same KL fields."""
    import torch
    from synthetic import workloads
    T_big = 1024
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
                  "preproc": {"pcg_iters": iters, "resid": resid, "seconds": round(pre, 2)}}

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
    stream_sec["sparse"] = sparse_subsection(dd, ctx, dev, stream, flush, mid, n_v, k, k_pad, tl, pk, pk_kind, reps)
    stream_sec["sparse"]["speedup_vs_dense"] = round(med / stream_sec["sparse"]["ms_per_field_pair"], 2)
    dd.dd_unload_mesh(ctx, mid)
    return stream_sec, gemm_sec


def sparse_subsection(dd, ctx, dev, stream, flush, mid, n_v, k, k_pad, tl, pk, pk_kind, reps):
    """Sparse KL+TV of one target (Section V): the target row's entries below
    max/sqrt(n) merged into one bin; every row of P is read only at the
    4-column blocks holding the target's kept columns.  Algorithmic bytes of a
    launch = 16 B x n x (the target's listed blocks) + 8 B x n (row totals) +
    the two output fields; the listed blocks are counted on the host from the
    exported kernel.  Accuracy against the dense FP32 fields of the same
    targets."""
    import torch
    t0 = time.perf_counter()
    kept, blocks = dd.dd_sparsify(ctx, mid)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    P32 = np.empty((n_v, k), dtype=np.float32)
    dd.dd_get_poisson_kernel(ctx, mid, P32)
    theta = np.float32(1.0 / math.sqrt(n_v))
    use = tl[:reps]

    def listed_blocks(t):
        row = np.zeros(k_pad, np.float32)
        row[:k] = P32[t]
        keep = (row >= theta * row.max()) & (row > 0)
        return int(keep.reshape(-1, 4).any(axis=1).sum())

    out1 = torch.empty((2, 1, n_v), dtype=torch.float32, device=dev)
    for t in use[:3]:
        dd.dd_distance(ctx, mid, [t], 3, dd.DD_PREC_SPARSE, out1)
    torch.cuda.synchronize()
    ms, gbs = [], []
    for t in use:
        flush.fill_(0.5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        dd.dd_distance(ctx, mid, [t], 3, dd.DD_PREC_SPARSE, out1)
        e1.record(stream)
        torch.cuda.synchronize()
        m = e0.elapsed_time(e1)
        ms.append(m)
        gbs.append((16.0 * n_v * listed_blocks(t) + 8.0 * n_v + 8.0 * n_v) / (m / 1e3) / 1e9)
    med, g = statistics.median(ms), statistics.median(gbs)
    dense = torch.empty((3, 4, n_v), dtype=torch.float32, device=dev)
    sp = torch.empty_like(dense)
    dd.dd_distance(ctx, mid, tl[:4], 7, dd.DD_PREC_FP32, dense)
    dd.dd_distance(ctx, mid, tl[:4], 7, dd.DD_PREC_SPARSE, sp)
    torch.cuda.synchronize()
    d, s_ = dense.cpu().numpy().astype(np.float64), sp.cpu().numpy().astype(np.float64)
    rel = np.abs(s_ - d) / np.maximum(np.abs(d), 1e-2)
    interior = d[2] < 40.0          # KLT is +inf (returned large) on boundary rows
    return {"kernel": "sparse_field_kernel (+ stage_targets_kernel, sparse_stage_kernel)", "bound": "hbm",
            "achieved": round(g, 1), "peak": pk.get("hbm_gbs"), "unit": "GB/s",
            "frac": round(g / pk.get("hbm_gbs", 6672.5), 4), "peak_source": pk_kind,
            "ms_per_field_pair": round(med, 4), "fields_per_s": round(2 / (med / 1e3), 1),
            "speedup_vs_dense": None, "sparsity": round(1.0 - kept / float(n_v * k), 4),
            "listed_blocks_mean": round(float(np.mean([listed_blocks(t) for t in use])), 1),
            "dense_blocks": int(k_pad // 4), "build_seconds": round(build_s, 3),
            "vs_dense_fp32": {"kl_max_rel": float(np.max(rel[0])), "kl_median_rel": float(np.median(rel[0])),
                              "tv_max_rel": float(np.max(rel[1])), "tv_median_rel": float(np.median(rel[1])),
                              "klt_max_rel": float(np.max(rel[2][interior])),
                              "klt_median_rel": float(np.median(rel[2][interior]))},
            "traffic": None}


def mid_section(dd, ctx, dev, stream, flush, pk, pk_kind, reps: int = 8):
    """A mid-size grid for full ncu captures (a few GB on the device): N = 300
    with 12 obstacles (n = 86,449, k = 2,122, P = 0.73 GB, larger than L2).
    The single-target dense stream (KL+TV), the sparse pass (KL+TV, Section V)
    and the split-BF16 KL GEMM for 512 targets, each timed with CUDA events
    (L2 flushed before every launch)."""
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
    dd.dd_unload_mesh(ctx, mid)
    issued = 3 * 2.0 * n_v * k * T / (gemm_ms / 1e3) / 1e12
    return {"workload": "grid300: n=%d, k=%d, P=%.2f GB FP32" % (n_v, k, 4.0 * n_v * k_pad / 1e9),
            "dense_stream_ms": round(dense_ms, 4),
            "dense_stream_gbs": round(4.0 * n_v * k_pad / (dense_ms / 1e3) / 1e9, 1),
            "sparse_ms": round(sparse_ms, 4), "gemm_T": T, "gemm_ms": round(gemm_ms, 4),
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
    mids = []
    for wl in doms:
        idx, off = wl.mesh.loop_arrays()
        mid = dd.dd_load_mesh(ctx, wl.mesh.xy, wl.mesh.tri, idx, off)
        dd.dd_poisson_kernel(ctx, mid, 1e-15, 40000)
        mids.append(mid)
    pre = time.perf_counter() - t0
    qs = workloads.serving_queries(doms, rate_qps=rate, duration_s=seconds)
    # ---- served
    sv = dd.dd_server_create(ctx, 24 << 30, n_slots=3, max_batch=64, max_pts=max_pts)
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
    # ---- plain per-query form (same arrivals, one query at a time, host buffers)
    n_plain = min(len(qs), int(rate * min(seconds, 2.0)))
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
                       "slots": 3, "max_batch": 64},
            "plain": {"queries": n_plain, "p50_ms": round(float(np.percentile(PL, 50)), 3),
                      "p99_ms": round(float(np.percentile(PL, 99)), 3),
                      "qps": round(n_plain / (time.perf_counter() - start), 1),
                      "form": "one dd_query per query (T=1, host buffers), in arrival order, first %d queries"
                              % n_plain},
            "preproc_s": round(pre, 2)}


class OracleStep:
    """The FP64 oracle on a bounded sample of the grid140 step (fields/s)."""

    def __init__(self):
        from oracle.poisson import PoissonOracle
        from oracle.trace import Tracer
        from synthetic import workloads
        self.wl = workloads.grid140(T=T_BATCH, S=S_PER_TARGET)
        po = PoissonOracle(self.wl.mesh.xy, self.wl.mesh.tri, self.wl.mesh.loops)
        self.P = po.full()
        self.tracer = Tracer(self.wl.mesh.xy, self.wl.mesh.tri)

    def run(self, a: int, sample_paths: int):
        """KL+TV of target a over all vertices plus `sample_paths` of its 256 paths.

        Returns the seconds one real step-target (2 fields + 256 paths) would take."""
        from oracle.divergence import kl_field_fast, tv_field
        P = self.P
        a = a % len(self.wl.targets)
        t = int(self.wl.targets[a])
        c0 = time.perf_counter()
        kl = kl_field_fast(P, P[t])
        tv_field(P, P[t])
        c1 = time.perf_counter()
        for q in self.wl.sources[a][:sample_paths]:
            self.tracer.trace(kl, int(q), t, max_pts=MAX_PTS)
        c2 = time.perf_counter()
        return (c1 - c0) + (c2 - c1) / sample_paths * S_PER_TARGET


# The oracle on every host core: one process per core (spawned, so that a pool
# started after CUDA work does not inherit the parent's GPU context), each with
# its own OracleStep; a task is one target of the sample, timed in its worker.
_ORACLE = None


def _oracle_init():
    global _ORACLE
    _ORACLE = OracleStep()


def _oracle_task(args):
    a, sample_paths = args
    return _ORACLE.run(a, sample_paths)


def oracle_pool(cores: int):
    import multiprocessing
    from concurrent.futures import ProcessPoolExecutor
    # one thread per worker: the workers inherit this environment when spawned
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        pool = ProcessPoolExecutor(max_workers=cores, mp_context=multiprocessing.get_context("spawn"),
                                   initializer=_oracle_init)
        list(pool.map(_oracle_task, [(w, 1) for w in range(cores)]))      # every worker built its kernel
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(sample_paths: int = 16):
    """fields/s of the oracle with every host core busy: each core takes one
    grid140 target (KL+TV over all n plus sample_paths of its 256 paths,
    scaled to the full per-target work)."""
    t0 = time.perf_counter()
    cores = host_cores()
    pool = oracle_pool(cores)
    per_target = list(pool.map(_oracle_task, [(cores + w, sample_paths) for w in range(cores)]))
    pool.shutdown()
    return {"value": round(cores * 2.0 / statistics.mean(per_target), 4), "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{cores} targets of grid140, one per core at once: KL+TV over all n plus {sample_paths} "
                      f"of {S_PER_TARGET} paths each, scaled to 2 fields + {S_PER_TARGET} paths per target",
            "seconds": round(time.perf_counter() - t0, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-stream", dest="stream", action="store_false",
                    help="skip the grid450 measurements (single-target HBM stream, BF16 tensor-core KL)")
    ap.add_argument("--section", choices=["all", "step", "grid450", "batch", "serve", "census", "mid"], default="all",
                    help="step: only the grid140 query step; grid450 / batch / serve / census / mid: only that part "
                         "(mid: a grid300 case small enough for full ncu captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return
        t0 = time.perf_counter()
        cores = host_cores()
        pool = oracle_pool(cores)
        for i in range(args.warmup):
            list(pool.map(_oracle_task, [(i * cores + w, 2) for w in range(cores)]))
        # per step every core takes one target; a step's time = the mean scaled per-target time
        step_s = []
        for i in range(args.steps):
            res = list(pool.map(_oracle_task, [((args.warmup + i) * cores + w, 4) for w in range(cores)]))
            step_s.append(statistics.mean(res))
        pool.shutdown()
        v = cores * 2.0 * args.steps / sum(step_s)
        line = {"metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(1e3 * sum(step_s) / args.steps, 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "impl": "reference",
                "config": {"workload": "grid140 (as --impl ours); per step one target per host core: KL+TV over "
                                       "all n and 4 of its 256 paths, scaled to the full per-target work"},
                "cpu_baseline": {"kind": "oracle", "cores": cores, "value": round(v, 4),
                                 "sample": f"per step {cores} targets at once (one per core): KL+TV over all n + "
                                           "4 of 256 paths each, scaled"},
                "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                "seconds": round(time.perf_counter() - t0, 1)}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    line = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1 and args.section in ("all", "step"):
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
