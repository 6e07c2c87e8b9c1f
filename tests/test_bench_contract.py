"""bench.py's step measurement on the CPU with a stand-in library and
stand-in CUDA events: the JSON line carries the contract's keys with
consistent values, the dominant kernel's roofline is chosen from the live
per-kernel times (the tile kernel against the FP32 issue rate of the
device's SM count, the walk against its latency chain), and a timed region
whose clocks show a slowdown is measured once more.  (The numbers are the stand-ins'; the GPU run gives the
real ones.)"""
import json
import os
import sys
import time
import types

import numpy as np
import pytest

torch = pytest.importorskip("torch")
sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


class _Event:
    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = time.perf_counter()

    def elapsed_time(self, other):
        return max((other.t - self.t) * 1e3, 1e-3)


def _fake_dd(n_v, k, kernel_ms):
    m = types.ModuleType("paper_1708_02845_gb300.dd")
    m.DD_F_KL, m.DD_F_TV, m.DD_F_KLT = 1, 2, 4
    m.DD_PREC_FP32, m.DD_PREC_BF16X3, m.DD_PREC_SPARSE = 0, 1, 2
    m.dd_create = lambda dev, stream=0: object()
    m.dd_destroy = lambda ctx: None
    m.dd_sync = lambda ctx: None
    m.dd_load_mesh = lambda ctx, xy, tri, idx, off: 0
    m.dd_mesh_info = lambda ctx, mid: {"n_v": n_v, "k": k, "k_pad": (k + 3) // 4 * 4}
    m.dd_poisson_kernel = lambda ctx, mid, rtol, it: (24, 2e-16)
    m.timing = {"on": False}

    def query(ctx, mid, tg, sr, f, prec, tf, max_pts, fields, xy, ln, st):
        fields.fill_(0.5)
        ln.fill_(12)
        st.zero_()

    def distance(ctx, mid, tg, f, prec, out):
        out.fill_(0.5)

    def kernel_timing(ctx, mode):
        if mode == 1:
            m.timing["on"] = True
            return {}
        on, m.timing["on"] = m.timing["on"], False
        return dict(kernel_ms) if on else {}

    m.dd_query = query
    m.dd_distance = distance
    m.dd_unload_mesh = lambda ctx, mid: None
    m.dd_trace_fields = lambda ctx, mid, f, tg, sr, max_pts, xy, ln, st: None
    m.dd_kernel_timing = kernel_timing
    m.dd_tuning_table = lambda: "rows<=2^18 k_pad<=2^12 T<=2^8: 64x64\n"
    m.dd_load_latency = lambda ctx, nbytes, steps: 150.0 if nbytes < (64 << 20) else 410.0
    return m


@pytest.fixture
def stand_ins(monkeypatch):
    def install(n_v, k, kernel_ms, clock_records):
        import paper_1708_02845_gb300 as pkg
        import paper_1708_02845_gb300.build as b
        fake = _fake_dd(n_v, k, kernel_ms)
        monkeypatch.setitem(sys.modules, "paper_1708_02845_gb300.dd", fake)
        monkeypatch.setattr(pkg, "dd", fake, raising=False)
        monkeypatch.setattr(b, "build", lambda *a, **kw: "")
        real_empty = torch.empty

        def empty(*a, device=None, **kw):
            return real_empty(*a, **kw)

        monkeypatch.setattr(torch, "empty", empty)
        monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
        monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
        monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
        monkeypatch.setattr(torch.cuda, "Event", _Event)
        monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: types.SimpleNamespace(cuda_stream=0))
        records = list(clock_records)
        monkeypatch.setattr(bench.ClockSampler, "start", lambda self: None)
        monkeypatch.setattr(bench.ClockSampler, "stop", lambda self: records.pop(0) if records else
                            {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3})
        monkeypatch.setitem(bench.WORKLOADS, bench.HEADLINE, dict(bench.WORKLOADS[bench.HEADLINE], **SMALL))
        monkeypatch.setattr(bench, "sm_count", lambda dev: 148)
        monkeypatch.setattr(bench, "_LOAD_NS", {})
        return fake
    return install


# the headline workload's mesh with fewer targets and sources per step (host memory)
SMALL = {"T": 64, "S": 4, "max_pts": 256}


def _args(steps=3):
    return types.SimpleNamespace(steps=steps, warmup=3, section="step", oracle_errors=False, no_cpu_baseline=True,
                                 gpus=1, impl="ours", workload=bench.HEADLINE)


KERNELS = {"stage_targets_kernel": (3, 0.04), "field_tile_kernel": (3, 6.7), "fix_kl_kernel": (3, 0.6),
           "rates_kernel": (3, 0.075), "vertex_decision_kernel": (3, 0.17), "trace_kernel": (3, 1.0)}
GOOD = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}
N_V, K = 192360, 3936


def test_step_line_keeps_the_contract(stand_ins):
    stand_ins(N_V, K, KERNELS, [GOOD])
    line = bench.run_ours(_args(), 0, 1, 0)
    json.dumps(line)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks",
                "kernels"):
        assert key in line, key
    T, S = SMALL["T"], SMALL["S"]
    assert line["metric"] == bench.METRIC and line["unit"] == "fields/s" and line["n_gpus"] == 1
    assert line["steps"] == 3 and line["warmup"] == 3 and line["higher_is_better"] is True
    assert line["config"]["workload"].startswith("grid450") and line["vs_baseline"] is None
    assert abs(line["value"] - 2 * T / (line["ms_per_step"] / 1e3)) <= 1e-3 * line["value"] + 1.0
    r = line["roofline"]
    assert r["kernel"] == "field_tile_kernel" and r["bound"] == "alu" and r["traffic"] is None
    assert r["algorithmic_fp32_ops"] == 4.0 * N_V * K * T
    assert abs(r["ms_per_launch"] - 6.7 / 3) < 1e-4
    assert abs(r["peak"] - 148 * 128 * 2070e6 / 1e12) < 1e-3            # the device's SM count
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-3
    w = line["roofline_walk"]
    assert w["kernel"] == "trace_kernel" and w["bound"] == "latency" and w["longest_path_points"] == 12
    # against one dependent L2 load per point of the longest path (150 ns from the latency hook)
    assert w["dependent_load_ns"]["l2"] == 150.0 and w["dependent_load_ns"]["dram"] == 410.0
    assert abs(w["floor_ms_one_l2_load_per_point"] - 12 * 150.0 / 1e6) < 1e-6
    assert abs(w["l2_loads_per_point"] - w["us_per_point_of_longest_path"] * 1e3 / 150.0) < 0.01
    assert line["roofline_fields"] is None and line["gpu_launches"] == 18
    assert abs(line["recompute_over_tile"] - 0.6 / 6.7) < 1e-3
    e = line["e2e"]
    assert e["unit"] == "fields/s" and e["h2d_bytes_per_step"] == T * 4 + T * S * 4
    assert e["d2h_bytes_per_step"] == 2 * T * N_V * 4 + T * S * 8 + T * S * 12 * 8
    assert "remeasured" not in line and line["clocks"] == GOOD
    assert line["step_bf16x3"]["tv_identical"] is True


def test_walk_named_when_it_dominates(stand_ins):
    k = dict(KERNELS, trace_kernel=(3, 9.0))
    stand_ins(N_V, K, k, [GOOD])
    line = bench.run_ours(_args(), 0, 1, 0)
    assert line["roofline"]["kernel"] == "trace_kernel" and line["roofline"]["bound"] == "latency"
    assert line["roofline_fields"]["kernel"] == "field_tile_kernel" and line["roofline_walk"] is None


def test_throttled_region_is_measured_again(stand_ins):
    hot = {"sm_mhz": 1500.0, "sm_max_mhz": 2070.0, "reasons": ["hw_thermal_slowdown"], "samples": 3}
    stand_ins(N_V, K, KERNELS, [hot, GOOD])
    line = bench.run_ours(_args(), 0, 1, 0)
    assert line["remeasured"]["first"]["reasons"] == ["hw_thermal_slowdown"]
    assert line["clocks"] == GOOD
    assert np.isfinite(line["value"])


def test_reference_arm_line():
    """`--impl reference` times the oracle on the host cores and prints the
    same metric, unit and direction as the library's line, with its own
    cpu_baseline and an e2e that moves no bytes."""
    import subprocess
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--workload", "grid140"], capture_output=True, text=True, timeout=600,
                       cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["value"] > 0 and line["steps"] == 2
    assert line["config"]["workload"].startswith("grid140") and line["ms_per_step"] > 0
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
