"""Benchmark: spin configurations per second into the exact table g(E, M) on one GB300.

Workload (one step): the 6x6 square torus with J = +1 on all 72 bonds (N = 36, 2^36
configurations) enumerated into its int64 table g(E, M) by isg_enumerate, followed by isg_thermo
on 256 temperatures in [0.5, 5] at h = 0 in FP64 (Eq. 2). Inputs are synthetic and seeded.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on the launching
stream, an L2 flush (a 256 MiB write) between steps outside the events, a barrier and
synchronisation around the timed region, max over ranks. Under torchrun every rank runs the
same workload on its own GPU (replicas, weak scaling), so `value` is the configurations of all
ranks per second of the slowest rank. With --shard the ranks share the one torus instead
(strong scaling): each step, every rank enumerates its share of the 2^36 configurations
(isg_enumerate_rank), one NCCL all-reduce sums the int64 tables, and every rank runs the
thermodynamics on the summed table; `value` is 2^36 per second of the slowest rank.

`--impl reference` runs the CPU oracle (oracle/, plain C, all host cores) on a bounded sample of
the same workload and reports the same metric, extrapolated from the sample to a full step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "spin configs/sec into exact g(E,M) on 1 GB300, % INT roofline; batched vs plain"
UNIT = "configs/s"
WORKLOAD = ("6x6 square torus (periodic), J=+1 on 72 bonds, N=36, 2^36 configurations -> int64 g(E,M); "
            "then FP64 thermodynamics on 256 T in [0.5,5] at h=0")
T_GRID = np.linspace(0.5, 5.0, 256)
H_GRID = np.array([0.0])
SM_MAX_MHZ_FALLBACK = 2070.0
# Algorithmic integer operations per configuration of the Gray-step method: one update of the
# bin address and one counter increment.
OPS_PER_CONFIG = 2
# DRAM traffic of one enumeration launch on this workload from the committed ncu capture
# (profiles/enumerate_kernel_torus6x6.md), valid only for the kernel's device code it was taken on
# (enum_core.cuh and enum_kernels.cuh; a changed kernel reports no traffic until re-captured).
TRAFFIC_BYTES = 34816          # dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu: 34.82 KB read, 0 written)
TRAFFIC_SOURCES_SHA = "0d5e8403033bc6bd"


def kernel_sources_sha() -> str:
    h = hashlib.sha256()
    for f in ("enum_core.cuh", "enum_kernels.cuh"):
        with open(os.path.join(ROOT, "paper_1110_2561_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples every 25 ms while running (the sampler is
    started, and its first sample awaited, before the timed region begins)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu = gpu_id
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "25"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
            self.lines.clear()                 # keep only samples taken during the timed region
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ------------------------------------------------------------------------------ GPU (isg) arm
def run_isg(args):
    import torch
    import torch.distributed as dist
    from paper_1110_2561_gb300 import isg, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    lat = workloads.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    shape = isg.table_shape(gh)
    tuned = isg.isg_autotune(gh, torch.cuda.current_stream())
    tuned_fields = {k: tuned[k] for k in ("stride_residue", "block_threads", "ctas_per_sm", "lane_model")} if tuned else {}
    plan = isg.isg_debug_plan(gh, **tuned_fields)
    # --shard-bits k (profiling case): each step enumerates shard 0 of 2^k with q - k inner bits,
    # so the launch has the same number of warp tasks as the full one
    shard = dict(shard_bits=args.shard_bits, shard_lo=0, shard_hi=1,
                 inner_bits=max(plan["b"], plan["q"] - args.shard_bits)) if args.shard_bits else {}
    n_configs = 1 << (lat.n - args.shard_bits)
    stream = torch.cuda.current_stream()
    g = torch.zeros(shape, dtype=torch.int64, device=dev)
    outs = tuple(torch.empty((len(T_GRID), 1), dtype=torch.float64, device=dev) for _ in range(5))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    peaks = isg.isg_probe_peaks(stream)
    sharded = args.shard and world > 1
    if args.shard and shard:
        raise SystemExit("--shard and --shard-bits exclude each other")

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        if sharded:
            isg.isg_enumerate_rank(gh, rank, world, g, stream, autotune=1)
            dist.all_reduce(g, op=dist.ReduceOp.SUM)
        else:
            isg.isg_enumerate(gh, g, stream, autotune=1, **shard)
        if ev:
            ev[1].record(stream)
        isg.isg_thermo(g, gh, T_GRID, H_GRID, isg.ISG_FP64, stream, out=outs)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # correctness of the last warm-up result (cheap invariants; parity lives in the tests)
    gc = g.cpu().numpy()
    assert int(gc.sum()) == n_configs
    if not shard:
        assert all(int(gc[:, m].sum()) == math.comb(lat.n, m) for m in range(lat.n + 1))

    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    uuid = str(getattr(torch.cuda.get_device_properties(dev), "uuid", local))
    gpu_id = uuid if uuid.startswith("GPU-") or uuid.isdigit() else "GPU-" + uuid
    with ClockSampler(gpu_id) as clk:
        torch.cuda.nvtx.range_push("isg_timed")       # lets ncu select exactly the timed launches
        for k in range(args.steps):
            flush.fill_(k & 0xFF)                      # L2 flush between timed steps, outside the events
            step(evs[k])
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(c) for a, b, c in evs]
    enum_ms = [a.elapsed_time(b) for a, b, c in evs]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())

    # end to end through the public API with host buffers (copies inside the timed region)
    e2e_steps = max(1, min(args.steps, 5))
    h2d = plan["blob_bytes"] + T_GRID.nbytes + H_GRID.nbytes
    d2h = int(np.prod(shape)) * 8 + 5 * len(T_GRID) * len(H_GRID) * 8
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        if sharded:                                   # host share, summed over the ranks through the GPUs
            part = isg.isg_enumerate_rank(gh, rank, world, None, stream, autotune=1)
            t = torch.from_numpy(part).to(dev)
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            gh_host = t.cpu().numpy()
        else:
            gh_host = isg.isg_enumerate(gh, None, stream, autotune=1, **shard)  # host table: D2H inside
        isg.isg_thermo(gh_host, gh, T_GRID, H_GRID, isg.ISG_FP64, stream)  # host g: H2D inside, host outputs
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    assert np.array_equal(gh_host, gc)

    isg.isg_device_status(stream)                     # the kernels' self-check of every device-output step
    clocks = clk.summary()
    if rank == 0:
        ms_per_step = total_ms / args.steps
        ranks_counted = 1 if sharded else world      # replicas: every rank its own torus
        value = ranks_counted * n_configs / (ms_per_step * 1e-3)
        enum_s = statistics.mean(enum_ms) * 1e-3     # with --shard: this rank's share plus the all-reduce
        rank_configs = n_configs // world if sharded else n_configs   # enumerated by one rank per step
        sm_max = clocks.get("sm_max_mhz") or measured_peaks().get("sm_max_mhz") or SM_MAX_MHZ_FALLBACK
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        alu_peak = sms * 4 * 32 * sm_max * 1e6                     # 4 schedulers x 32 lanes per SM per clock
        red_peak = sms * 32 * sm_max * 1e6                         # one 32-lane shared reduction per SM per clock
        achieved_ops = OPS_PER_CONFIG * rank_configs / enum_s
        traffic = TRAFFIC_BYTES if TRAFFIC_SOURCES_SHA == kernel_sources_sha() and not sharded else None
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong" if sharded else "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD if not shard else f"shard 0 of 2^{args.shard_bits} of: " + WORKLOAD,
                       "parallelism": f"shard{world}" if sharded else f"replicas{world}",
                       "l2": "flushed between steps (256 MiB write)",
                       "plan": {k: plan[k] for k in ("q", "b", "tasks", "threads", "copies", "ctas_per_sm", "G",
                                                     "n_e_compact", "stride", "lane_model", "lane_cost",
                                                     "lane_cost_index_order")},
                       "autotuned": tuned_fields},
            # the binding unit: one shared-memory reduction per configuration; the shared-memory
            # pipe executes one warp-wide (32-lane) reduction per clock per SM
            "roofline": {"bound": "smem_atomic", "achieved": rank_configs / enum_s / 1e9,
                         "peak": red_peak / 1e9, "unit": "Gred/s", "frac": rank_configs / enum_s / red_peak,
                         "traffic": traffic, "kernel": f"enumerate_kernel<{plan['b']}>",
                         "work_per_config": "1 red.shared.add.u32 (plus 1 integer add)",
                         "peak_source": f"{sms} SMs x 32 lanes/clk x {sm_max:.0f} MHz (unit counts and clock)",
                         "peak_measured": peaks["red_conflict_free"] / 1e9,
                         "frac_of_measured": rank_configs / enum_s / peaks["red_conflict_free"],
                         "peak_measured_scattered": peaks["red_scattered"] / 1e9,
                         "match_any_aggregated": peaks["match_aggregated"] / 1e9,
                         "peak_measured_source": "isg_probe_peaks (red.shared.add.u32, measured in this run)"},
            "roofline_alu": {"bound": "alu", "achieved": achieved_ops / 1e9, "peak": alu_peak / 1e9, "unit": "Gop/s",
                             "frac": achieved_ops / alu_peak, "ops_per_config": OPS_PER_CONFIG,
                             "peak_source": f"{sms} SMs x 128 lanes/clk x {sm_max:.0f} MHz (unit counts and clock)"},
            "enumerate_ms": statistics.mean(enum_ms), "thermo_ms": statistics.mean(
                [b.elapsed_time(c) for a, b, c in evs]),
            "e2e": {"value": ranks_counted * n_configs / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            # this library's kernels, all ranks: the enumeration, then the thermodynamics: one
            # kernel when every field is zero and the table has at most 1024 energy bins (the
            # per-energy path), else the ln g conversion and the grid kernel
            "gpu_launches": (1 + (1 if np.all(H_GRID == 0) and shape[0] <= 1024 else 2)) * args.steps * world,
            "clocks": clocks,
        }
        # the other workloads and the oracle baseline at N = 1 only (the scaling runs time the
        # headline step alone)
        if not args.no_extras and world == 1:
            line["workloads"] = extra_measurements(stream, dev)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------------------ other workloads
def _event_ms(fn, stream, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def extra_measurements(stream, dev):
    """The other workloads of the method, measured once each (not part of the timed step):
    4x4 free lattice latency, 4096 EA instances batched vs per-instance, and the 3x3x4 cubic
    torus thermodynamics on a 512 x 256 (T, h) grid in FP32 vs FP64."""
    import torch
    from paper_1110_2561_gb300 import isg, workloads

    out = {}
    # 4x4 free ferromagnet: enumerate + FP64 thermodynamics on 64 temperatures, one call each
    lat = workloads.square(4, 4, False)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
    T = np.linspace(0.5, 5, 64)
    o64 = tuple(torch.empty((64, 1), dtype=torch.float64, device=dev) for _ in range(5))

    def small_step():
        isg.isg_enumerate(gh, g, stream)
        isg.isg_thermo(g, gh, T, [0.0], isg.ISG_FP64, stream, out=o64)
    pe = isg.prepare_enumerate(gh, g, stream)
    pt = isg.prepare_thermo(g, gh, T, [0.0], o64, isg.ISG_FP64, stream)

    def prepared_step():
        pe()
        pt()

    def host_us(fn, n=200):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / n * 1e6
    def latency_us(fn, n=200):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(n):
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts) * 1e6
    out["square4x4_free"] = {
        "what": "isg_enumerate (65,536 configurations) + isg_thermo (64 T, FP64), device buffers",
        "latency_us": latency_us(prepared_step),
        "back_to_back_us_per_call": host_us(prepared_step),
        "back_to_back_us_per_call_python_binding": host_us(small_step)}
    # EA +-J batch: one prepared batch (graph replay) vs a loop of per-instance launches
    lats = workloads.ea_instances()
    hs = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    configs = sum(1 << l.n for l in lats)
    b = isg.Batch(hs, autotune=1)
    bat_ms = _event_ms(lambda: b.run(stream), stream, 3)
    b.status(stream)
    b.close()
    outs = [torch.zeros(isg.table_shape(h), dtype=torch.int64, device=dev) for h in hs]

    def plain():
        for h, t in zip(hs, outs):
            isg.isg_enumerate(h, t, stream)
    pl_ms = _event_ms(plain, stream, 2)
    out["ea_4096_batched_vs_plain"] = {
        "instances": len(lats), "configs": configs,
        "batched_ms": bat_ms, "batched_instances_per_s": len(lats) / (bat_ms * 1e-3),
        "batched_configs_per_s": configs / (bat_ms * 1e-3),
        "plain_ms": pl_ms, "plain_instances_per_s": len(lats) / (pl_ms * 1e-3),
        "plain_configs_per_s": configs / (pl_ms * 1e-3), "speedup": pl_ms / bat_ms}
    # spin-flip symmetry halving (a NEXT row, reported apart from the headline): half the visits
    lat = workloads.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
    sym_ms = _event_ms(lambda: isg.isg_enumerate(gh, g, stream, autotune=1, symmetry=1), stream, 5)
    b = isg.Batch(hs, autotune=1, symmetry=1)
    bsym_ms = _event_ms(lambda: b.run(stream), stream, 3)
    b.status(stream)
    b.close()
    out["symmetry_halving"] = {
        "what": "enumerate only spin N-1 up, add the M -> -M mirror (exact for any couplings)",
        "torus6x6_ms": sym_ms, "torus6x6_effective_configs_per_s": (1 << 36) / (sym_ms * 1e-3),
        "torus6x6_enumerated_configs_per_s": (1 << 35) / (sym_ms * 1e-3),
        "ea_4096_batched_ms": bsym_ms, "ea_4096_batched_instances_per_s": len(lats) / (bsym_ms * 1e-3),
        "ea_4096_effective_configs_per_s": configs / (bsym_ms * 1e-3)}
    # derived physics: the temperature of the specific-heat maximum of the 6x6 torus (h = 0)
    lat = workloads.square(6, 6, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
    isg.isg_enumerate(gh, g, stream, autotune=1)
    stream.synchronize()                              # the table is ready before the clock starts
    t0 = time.perf_counter()
    tc, cmax = isg.isg_specific_heat_peak(g, gh, 0.0, 1.0, 4.0, isg.ISG_FP64, stream)
    out["torus6x6_specific_heat_peak"] = {"T_peak": tc, "C_peak": cmax, "ms": (time.perf_counter() - t0) * 1e3}
    # derived physics: Binder-cumulant crossing of the 4x4 and 6x6 tori (h = 0, 2001 T in [1.5, 3.5])
    Tb = np.linspace(1.5, 3.5, 2001)
    ub = []
    for L in (4, 6):
        lb = workloads.square(L, L, True)
        hb = isg.isg_graph_create(lb.n, lb.edges)
        gb = torch.zeros(isg.table_shape(hb), dtype=torch.int64, device=dev)
        isg.isg_enumerate(hb, gb, stream, autotune=1)
        ob = tuple(torch.empty((len(Tb), 1), dtype=torch.float64, device=dev) for _ in range(4))
        mag_ms = _event_ms(lambda: isg.isg_magnetisation(gb, hb, Tb, [0.0], isg.ISG_FP64, stream, out=ob), stream, 5)
        ub.append(ob[3][:, 0].cpu().numpy())
    dub = ub[1] - ub[0]
    k = int(np.nonzero(np.diff(np.sign(dub)))[0][0])
    t_cross = Tb[k] + (Tb[k + 1] - Tb[k]) * dub[k] / (dub[k] - dub[k + 1])
    out["torus_binder_crossing_4x4_6x6"] = {"T_cross": float(t_cross), "U4_at_cross": float(ub[0][k]),
                                            "isg_magnetisation_ms_2001T": mag_ms}
    # split-and-convolve (a variant of the full enumeration, reported apart from the headline):
    # the same exact tables from 2^|S| * sum 2^|C| visits
    split = {}
    for name, lat in (("torus6x6", workloads.square(6, 6, True)), ("cubic3x3x4", workloads.cubic(3, 3, 4, True)),
                      ("torus7x7", workloads.square(7, 7, True)), ("torus8x8", workloads.square(8, 8, True))):
        hs = isg.isg_graph_create(lat.n, lat.edges)
        gs = torch.zeros(isg.table_shape(hs), dtype=torch.int64, device=dev)
        plan_s = isg.isg_split_plan(hs)
        ms = _event_ms(lambda: isg.isg_enumerate_split(hs, gs, stream), stream, 3)
        tot = sum(int(v) for v in gs.cpu().numpy().ravel())       # 2^64 for N = 64: Python integers
        split[name] = {"N": lat.n, "ms": ms, "boundary_spins": plan_s["boundary_spins"],
                       "components": plan_s["components"], "largest_component": plan_s["largest_component"],
                       "visits": plan_s["visits"], "effective_configs_per_s": 2.0 ** lat.n / (ms * 1e-3),
                       "visits_per_s": plan_s["visits"] / (ms * 1e-3), "sum_g_equals_2^N": tot == 2 ** lat.n}
    # the EA ensemble as a prepared batch with options.split (instances whose split models less
    # work go through split launches inside the captured graph), beside the plain prepared batch
    hs_e = [isg.isg_graph_create(l.n, l.edges) for l in lats]
    t0 = time.perf_counter()
    bsp = isg.Batch(hs_e, split=1)
    create_s = time.perf_counter() - t0
    sb_ms = _event_ms(lambda: bsp.run(stream), stream, 3)
    bsp.status(stream)
    bsp.close()
    split["ea_4096_prepared_batch"] = {"instances": len(lats), "ms": sb_ms, "create_s": create_s,
                                       "instances_per_s": len(lats) / (sb_ms * 1e-3),
                                       "effective_configs_per_s": configs / (sb_ms * 1e-3),
                                       "plain_prepared_batch_ms": bat_ms, "speedup": bat_ms / sb_ms}
    out["split_and_convolve"] = split
    # derived physics at sizes only the split reaches: exact tables of the L x L tori (L >= 6 by
    # split-and-convolve), their specific-heat maxima, and the Binder-cumulant crossings of
    # neighbouring sizes (both approach the infinite-lattice 2 / ln(1 + sqrt 2) = 2.269)
    Tb = np.linspace(1.8, 3.0, 2401)
    series, u4 = {}, {}
    t0 = time.perf_counter()
    for L in range(4, 9):
        lf = workloads.square(L, L, True)
        hf = isg.isg_graph_create(lf.n, lf.edges)
        tab = isg.isg_enumerate_split(hf) if L >= 6 else isg.isg_enumerate(hf)
        tp, cpk = isg.isg_specific_heat_peak(tab, hf, 0.0, 1.5, 3.5, isg.ISG_FP64)
        u4[L] = isg.isg_magnetisation(tab, hf, Tb, [0.0], isg.ISG_FP64)[3][:, 0]
        series[f"{L}x{L}"] = {"N": lf.n, "T_peak": tp, "C_peak_per_spin": cpk / lf.n}
    for L in range(4, 8):
        d = u4[L + 1] - u4[L]
        k = np.nonzero(np.diff(np.sign(d)))[0]
        if len(k):
            k = int(k[0])
            series[f"binder_crossing_{L}x{L}_{L + 1}x{L + 1}"] = float(Tb[k] + (Tb[k + 1] - Tb[k]) * d[k] / (d[k] - d[k + 1]))
    series["seconds"] = time.perf_counter() - t0
    out["finite_size_series_tori"] = series
    # cubic 3x3x4 torus: thermodynamics on 512 T x 256 h, FP32 vs FP64
    lat = workloads.cubic(3, 3, 4, True)
    gh = isg.isg_graph_create(lat.n, lat.edges)
    g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
    enum_ms = _event_ms(lambda: isg.isg_enumerate(gh, g, stream, autotune=1), stream, 3)
    T = np.linspace(0.5, 8, 512)
    h = np.linspace(-2, 2, 256)
    r64 = tuple(torch.empty((512, 256), dtype=torch.float64, device=dev) for _ in range(5))
    r32 = tuple(torch.empty((512, 256), dtype=torch.float64, device=dev) for _ in range(5))
    t64 = _event_ms(lambda: isg.isg_thermo(g, gh, T, h, isg.ISG_FP64, stream, out=r64), stream, 5)
    t32 = _event_ms(lambda: isg.isg_thermo(g, gh, T, h, isg.ISG_FP32, stream, out=r32), stream, 5)
    names = ("logZ", "E", "M", "C", "chi")
    err = {}
    for k, nm in enumerate(names):
        d = (r32[k] - r64[k]).abs()
        err[nm] = {"max_abs": float(d.max()), "max_rel": float((d / r64[k].abs().clamp_min(1e-300)).max()),
                   "max_rel_of_grid_max": float(d.max() / r64[k].abs().max())}
    m64 = tuple(torch.empty((512, 256), dtype=torch.float64, device=dev) for _ in range(4))
    m32 = tuple(torch.empty((512, 256), dtype=torch.float64, device=dev) for _ in range(4))
    tm64 = _event_ms(lambda: isg.isg_magnetisation(g, gh, T, h, isg.ISG_FP64, stream, out=m64), stream, 5)
    tm32 = _event_ms(lambda: isg.isg_magnetisation(g, gh, T, h, isg.ISG_FP32, stream, out=m32), stream, 5)
    for k, nm in enumerate(("absM", "M2", "M4", "binder")):
        d = (m32[k] - m64[k]).abs()
        err[nm] = {"max_abs": float(d.max()), "max_rel": float((d / m64[k].abs().clamp_min(1e-300)).max()),
                   "max_rel_of_grid_max": float(d.max() / m64[k].abs().max())}
    out["cubic3x3x4_thermo"] = {"enumerate_ms": enum_ms, "enumerate_configs_per_s": (1 << 36) / (enum_ms * 1e-3),
                                "grid": "512 T in [0.5,8] x 256 h in [-2,2]", "fp64_ms": t64, "fp32_ms": t32,
                                "fp32_speedup": t64 / t32, "magnetisation_fp64_ms": tm64,
                                "magnetisation_fp32_ms": tm32, "fp32_vs_fp64": err}
    # the request stream: 2000 requests enumerating every configuration (the serving workload's
    # count), and shorter streams of the same seed with symmetry halving and split service
    out["serving"] = {"every_configuration_2000": serve_stream(2000, 50.0, 20.0, 0.0),
                      "symmetry_halving_200": serve_stream(200, 50.0, 20.0, 0.0, 1),
                      "split_work_ratio_0.25_200": serve_stream(200, 50.0, 20.0, 0.25)}
    return out


# ------------------------------------------------------------------------------ CPU oracle
def oracle_step(lat, sample_configs: int, threads: int):
    """One bounded step of the oracle: the first `sample_configs` configurations of the workload,
    then the FP64 thermodynamics on the full grid from the (exact) table. Returns the seconds of
    each part."""
    import oracle
    t0 = time.perf_counter()
    g = oracle.g_masks(lat.n, lat.edges, 0, sample_configs, threads=threads)
    t1 = time.perf_counter()
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    oracle.thermo(lat.n, e_min, g, T_GRID, H_GRID)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1


def calibrate_sample(lat, threads: int, seconds: float) -> int:
    import oracle
    n = 1 << 20
    while True:
        t0 = time.perf_counter()
        oracle.g_masks(lat.n, lat.edges, 0, n, threads=threads)
        dt = time.perf_counter() - t0
        if dt > 0.5 or n >= 1 << 34:
            break
        n <<= 1
    target = int(n * seconds / max(dt, 1e-6))
    return max(1 << 20, min(1 << lat.n, 1 << max(20, target.bit_length() - 1)))


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def cpu_workloads(threads: int, rate: float) -> dict:
    """The oracle on the other workloads, each a bounded sample extrapolated to the whole: the 4x4
    free lattice whole on one thread (enumeration and the 64-T thermodynamics); the 4096 EA
    instances by OpenMP O1 over two instances of each shape; the 3x3x4 cubic torus's enumeration
    (OpenMP O1) and its FP64 thermodynamics on one core (4 of the 512 temperatures, all 256
    fields). `rate`: the OpenMP O1 rate measured just before (configurations/s), which sizes each
    enumeration sample to about a second."""
    import oracle
    from paper_1110_2561_gb300 import workloads
    out = {}
    lat = workloads.square(4, 4, False)
    t0 = time.perf_counter()
    g = oracle.g_masks(lat.n, lat.edges, threads=1)
    t1 = time.perf_counter()
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    oracle.thermo(lat.n, e_min, g, np.linspace(0.5, 5, 64), [0.0])
    t2 = time.perf_counter()
    out["square4x4_free"] = {"what": "O1 on one thread (65,536 configurations) + FP64 thermodynamics on 64 T, one core",
                             "enumerate_us": (t1 - t0) * 1e6, "thermo_us": (t2 - t1) * 1e6}
    lats = workloads.ea_instances()
    per_shape = {}
    for l in lats:
        per_shape.setdefault(l.n, []).append(l)
    total_s, sampled = 0.0, []
    budget = 1 << max(20, int(rate * 0.5).bit_length() - 1)      # about half a second per instance
    for n, group in sorted(per_shape.items()):
        k = min(len(group), 2)
        cut = min(1 << n, budget)
        t0 = time.perf_counter()
        for l in group[:k]:
            oracle.g_masks(l.n, l.edges, 0, cut, threads=threads)
        dt = (time.perf_counter() - t0) / k * ((1 << n) / cut)
        total_s += dt * len(group)
        sampled.append(f"{k} of the {len(group)} N={n} instances ({cut} configurations each)")
    out["ea_4096"] = {"what": f"OpenMP O1 ({threads} threads), instance by instance",
                      "sample": "; ".join(sampled) + "; extrapolated to all 4096", "seconds": total_s,
                      "instances_per_s": len(lats) / total_s}
    lat = workloads.cubic(3, 3, 4, True)
    cut = 1 << max(20, int(rate).bit_length() - 1)               # about a second
    t0 = time.perf_counter()
    g = oracle.g_masks(lat.n, lat.edges, 0, cut, threads=threads)
    t_enum = time.perf_counter() - t0
    e_min, _, _ = oracle.bins(lat.n, lat.edges)
    T, h = np.linspace(0.5, 8, 512), np.linspace(-2, 2, 256)
    t0 = time.perf_counter()
    oracle.thermo(lat.n, e_min, g, T[::128], h)          # the sample's table: the same shape and sparsity
    t_thermo = (time.perf_counter() - t0) * (len(T) / len(T[::128]))
    out["cubic3x3x4"] = {"what": f"OpenMP O1 ({threads} threads) on the first {cut} configurations; FP64 thermodynamics "
                                 f"on one core over that sample's table, 4 of 512 T x 256 h, extrapolated",
                         "enumerate_configs_per_s": cut / t_enum, "thermo_s_512x256": t_thermo}
    return out


def cpu_baseline(seconds: float):
    import oracle
    from paper_1110_2561_gb300 import workloads
    lat = workloads.square(6, 6, True)
    threads = os.cpu_count() or 1
    sample = calibrate_sample(lat, threads, seconds)
    t_enum, t_thermo = oracle_step(lat, sample, threads)
    full_step = t_enum * ((1 << lat.n) / sample) + t_thermo
    # one thread: one to two seconds of O1 on the same torus
    cut = 1 << 22
    while True:
        t0 = time.perf_counter()
        oracle.g_masks(lat.n, lat.edges, 0, cut, threads=1)
        dt1 = time.perf_counter() - t0
        if dt1 > 1.0 or cut >= 1 << 30:
            break
        cut <<= 1
    return {"value": (1 << lat.n) / full_step, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {sample} of 2^36 configurations ({t_enum:.2f} s, O1 popcount oracle, {threads} OpenMP "
                      f"threads) plus the full FP64 thermodynamics ({t_thermo:.3f} s); rate extrapolated to a full step",
            "cpu": cpu_model(),
            "single_thread_configs_per_s": cut / dt1,
            "single_thread_sample": f"first {cut} configurations of the 6x6 torus, O1 on one thread ({dt1:.2f} s)",
            "workloads": cpu_workloads(threads, sample / t_enum)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_1110_2561_gb300 import workloads
    import oracle
    oracle.build()
    lat = workloads.square(6, 6, True)
    threads = os.cpu_count() or 1
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup)))
    sample = calibrate_sample(lat, threads, per_step)
    for _ in range(args.warmup):
        oracle_step(lat, sample, threads)
    ext = []
    for _ in range(args.steps):
        t_enum, t_thermo = oracle_step(lat, sample, threads)
        ext.append(t_enum * ((1 << lat.n) / sample) + t_thermo)
    ms_per_step = 1e3 * statistics.mean(ext)
    value = (1 << lat.n) / (ms_per_step * 1e-3)
    desc = (f"each step: first {sample} of 2^36 configurations (O1 popcount oracle, {threads} OpenMP threads) plus "
            f"the full FP64 thermodynamics, extrapolated to a full step")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ serving mode
def serve_stream(n_requests: int, rate: float, step_ms: float, split_ratio: float, symmetry: int = 0,
                 lane_model: int = 1) -> dict:
    """Poisson stream of lattice requests (seeded; N uniform in 16..38, square / triangular / cubic,
    periodic or free, J uniform in {-2,-1,1,2}) submitted at their arrival times to isg_server;
    latency percentiles, throughput and offered vs achieved load (configurations counted into the
    tables; with symmetry the server enumerates about half of them, reported apart)."""
    from paper_1110_2561_gb300 import isg, workloads

    reqs = workloads.serving_stream(n_requests, rate_per_s=rate)
    graphs = [isg.isg_graph_create(r.lattice.n, r.lattice.edges) for r in reqs]
    srv = isg.Server(step_ms=step_ms, split_work_ratio=split_ratio, symmetry=symmetry, lane_model=lane_model)
    warm = srv.submit(isg.isg_graph_create(20, workloads.square(4, 5, True).edges))
    srv.wait(warm)
    srv.result(warm)
    tickets = []
    t0 = time.perf_counter()
    for r, g in zip(reqs, graphs):
        delay = r.arrival_s - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(srv.submit(g))
    lat, queued, configs = [], [], 0
    bad = 0
    for t, r in zip(tickets, reqs):
        srv.wait(t)
        g, times = srv.result(t)
        lat.append(times[2])
        queued.append(times[0])
        configs += 1 << r.lattice.n
        if sum(int(v) for v in g.ravel()) != 1 << r.lattice.n:
            bad += 1
    st = srv.stats()
    elapsed = time.perf_counter() - t0
    srv.close()
    span_arrivals = reqs[-1].arrival_s - reqs[0].arrival_s
    lat_ms = np.array(lat) * 1e3
    return {
        "workload": f"{n_requests} requests, Poisson {rate}/s, N uniform 16..38, square/triangular/cubic, "
                    "periodic or free, J uniform in {-2,-1,1,2} (seeded)",
        "p50_ms": float(np.percentile(lat_ms, 50)), "p90_ms": float(np.percentile(lat_ms, 90)),
        "p99_ms": float(np.percentile(lat_ms, 99)), "max_ms": float(lat_ms.max()),
        "mean_queue_ms": float(np.mean(queued) * 1e3),
        "offered_configs_per_s": configs / max(1e-9, span_arrivals),
        "achieved_configs_per_s": configs / max(1e-9, elapsed),
        "device_busy_frac": st["device_ms"] * 1e-3 / max(1e-9, elapsed),
        "steps": int(st["steps"]), "step_ms": step_ms, "invariant_failures": bad,
        "split_work_ratio": split_ratio, "symmetry": symmetry, "lane_model": lane_model,
    }


def run_serving(args):
    """The request-stream benchmark (one JSON line)."""
    import torch

    torch.cuda.set_device(0)
    line = {"metric": "serving latency and throughput (continuous batching)", "unit": "ms"}
    line.update(serve_stream(args.requests, args.rate, args.step_ms, args.split_ratio, args.symmetry, args.lane_model))
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------ profiling cases
def run_profile_case(args):
    """Small cases of the other kernels for ncu captures: W untimed + K timed launches each."""
    import torch
    from paper_1110_2561_gb300 import isg, workloads

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    res = {"case": args.profile_case}
    if args.profile_case in ("ea-batch", "ea-batch-tuned", "ea-split-batch"):
        lats = workloads.ea_instances()
        if args.profile_case != "ea-split-batch":
            lats = lats[:256]                                     # shuffled order: all four shapes
        tuned = {"autotune": 1} if args.profile_case == "ea-batch-tuned" else {}
        if args.profile_case == "ea-split-batch":
            tuned = {"split": 1}                                  # all 4096, the 5x6 ones by split launches
        b = isg.Batch([isg.isg_graph_create(l.n, l.edges) for l in lats], **tuned)
        for _ in range(args.warmup):
            b.run(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("isg_timed")        # lets ncu skip the autotuner's trial launches
        res["ms"] = _event_ms(lambda: b.run(stream), stream, args.steps)
        torch.cuda.nvtx.range_pop()
        res["configs_per_s"] = sum(1 << l.n for l in lats) / (res["ms"] * 1e-3)
        b.status(stream)
        b.close()
    elif args.profile_case == "cubic-thermo":
        lat = workloads.cubic(3, 3, 4, True)
        gh = isg.isg_graph_create(lat.n, lat.edges)
        g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
        isg.isg_enumerate(gh, g, stream)
        T, h = np.linspace(0.5, 8, 512), np.linspace(-2, 2, 256)
        outs = tuple(torch.empty((512, 256), dtype=torch.float64, device=dev) for _ in range(5))
        for prec, name in ((isg.ISG_FP64, "fp64_ms"), (isg.ISG_FP32, "fp32_ms")):
            for _ in range(args.warmup):
                isg.isg_thermo(g, gh, T, h, prec, stream, out=outs)
            res[name] = _event_ms(lambda: isg.isg_thermo(g, gh, T, h, prec, stream, out=outs), stream, args.steps)
    elif args.profile_case == "small-thermo":
        # the 4x4 free lattice's FP64 thermodynamics on 64 temperatures at h = 0 (a clustered grid)
        lat = workloads.square(4, 4, False)
        gh = isg.isg_graph_create(lat.n, lat.edges)
        g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
        isg.isg_enumerate(gh, g, stream)
        outs = tuple(torch.empty((64, 1), dtype=torch.float64, device=dev) for _ in range(5))
        call = isg.prepare_thermo(g, gh, np.linspace(0.5, 5, 64), [0.0], outs, isg.ISG_FP64, stream)
        for _ in range(args.warmup):
            call()
        res["fp64_ms"] = _event_ms(call, stream, args.steps)
    elif args.profile_case == "small-pair":
        # the 4x4 free lattice's prepared call pair (enumerate + FP64 thermodynamics on 64 T at
        # h = 0) as the default benchmark times it; the timed pairs inside the NVTX range isg_timed
        lat = workloads.square(4, 4, False)
        gh = isg.isg_graph_create(lat.n, lat.edges)
        g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
        outs = tuple(torch.empty((64, 1), dtype=torch.float64, device=dev) for _ in range(5))
        pe = isg.prepare_enumerate(gh, g, stream)
        pt = isg.prepare_thermo(g, gh, np.linspace(0.5, 5, 64), [0.0], outs, isg.ISG_FP64, stream)
        for _ in range(args.warmup):
            pe()
            pt()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("isg_timed")
        res["pair_ms"] = _event_ms(lambda: (pe(), pt()), stream, args.steps)
        torch.cuda.nvtx.range_pop()
    elif args.profile_case in ("cubic-enumerate", "torus-enumerate"):
        # the full enumeration of the 3x3x4 (or 6x6) torus, autotuned as in the benchmark; with
        # --shard-bits k, shard 0 of 2^k with q - k inner bits (the full launch's task count)
        lat = workloads.cubic(3, 3, 4, True) if args.profile_case == "cubic-enumerate" else workloads.square(6, 6, True)
        gh = isg.isg_graph_create(lat.n, lat.edges)
        g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
        res["tuned"] = isg.isg_autotune(gh, stream)
        tf = {k: res["tuned"][k] for k in ("stride_residue", "block_threads", "ctas_per_sm", "lane_model")}
        res["plan"] = isg.isg_debug_plan(gh, **tf)
        shard = {}
        if args.shard_bits:
            shard = dict(shard_bits=args.shard_bits, shard_lo=0, shard_hi=1,
                         inner_bits=max(res["plan"]["b"], res["plan"]["q"] - args.shard_bits))
            res["shard_plan"] = isg.isg_debug_plan(gh, **tf, **shard)
        for _ in range(args.warmup):
            isg.isg_enumerate(gh, g, stream, autotune=1, **shard)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("isg_timed")
        res["ms"] = _event_ms(lambda: isg.isg_enumerate(gh, g, stream, autotune=1, **shard), stream, args.steps)
        torch.cuda.nvtx.range_pop()
        res["configs_per_s"] = 2.0 ** (36 - args.shard_bits) / (res["ms"] * 1e-3)
        isg.isg_device_status(stream)
    elif args.profile_case in ("split-torus6x6", "split-torus7x7", "split-torus8x8", "split-cubic3x3x4"):
        lat = {"split-torus6x6": workloads.square(6, 6, True), "split-torus7x7": workloads.square(7, 7, True),
               "split-torus8x8": workloads.square(8, 8, True), "split-cubic3x3x4": workloads.cubic(3, 3, 4, True)}[
                   args.profile_case]
        gh = isg.isg_graph_create(lat.n, lat.edges)
        g = torch.zeros(isg.table_shape(gh), dtype=torch.int64, device=dev)
        for _ in range(args.warmup):
            isg.isg_enumerate_split(gh, g, stream)
        res["ms"] = _event_ms(lambda: isg.isg_enumerate_split(gh, g, stream), stream, args.steps)
        res["sum_ok"] = sum(int(v) for v in g.cpu().numpy().ravel()) == 2 ** lat.n    # 2^64: Python integers
    else:
        raise SystemExit(f"unknown profile case {args.profile_case}")
    torch.cuda.synchronize()
    print(json.dumps(res), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("isg", "reference"), default="isg")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the oracle timing leg")
    ap.add_argument("--no-extras", action="store_true", help="skip the other workloads' measurements")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target seconds of the oracle sample")
    ap.add_argument("--serving", action="store_true", help="run the request-stream (serving) benchmark instead")
    ap.add_argument("--profile-case", choices=("ea-batch", "ea-batch-tuned", "ea-split-batch", "cubic-thermo", "small-thermo", "small-pair", "cubic-enumerate", "torus-enumerate",
                                               "split-torus6x6",
                                               "split-torus7x7", "split-torus8x8", "split-cubic3x3x4"),
                    default=None,
                    help="run only a small case of another kernel (for ncu captures)")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--step-ms", type=float, default=20.0)
    ap.add_argument("--split-ratio", type=float, default=0.0,
                    help="serving: serve requests whose split-and-convolve work is below this fraction by split launches")
    ap.add_argument("--symmetry", type=int, choices=(0, 1), default=0,
                    help="serving: enumerate each tile-served request's half with spin N-1 up and mirror it")
    ap.add_argument("--lane-model", type=int, choices=(0, 1), default=1,
                    help="serving: the quick lane search for requests of at least 36 spins (1, the server's "
                         "default) or the index order (0)")
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: the ranks share the one torus (strong scaling, NCCL all-reduce per step)")
    ap.add_argument("--shard-bits", type=int, default=0,
                    help="profiling case: enumerate only shard 0 of 2^k per step (not a benchmark line); also for "
                         "the cubic-enumerate and torus-enumerate profile cases")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "isg":
        ap.error("at least 3 warm-up steps")
    if args.profile_case:
        run_profile_case(args)
    elif args.serving:
        run_serving(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_isg(args)


if __name__ == "__main__":
    main()
