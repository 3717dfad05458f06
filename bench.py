"""Benchmark of the cost-table search on the scene-scale workload.

Workload (the paper's scene scale, Sec. I: 5.27 M Gaussians, 59 FP32 channels):
N = 5,270,000 synthetic Gaussians, reserve ratios 0.1..1.0 (10 kept sets),
bit-widths {2,3,4,5,6,8,10,12,14,16}, groups of 4,096, 0-1 ILP at 40 MB.

One step = the whole hot path over one scene whose attributes are resident in
HBM: validation, importance rank, Morton order, slab relayout
(mgs_scene_create), kept lists and the fused cost kernel (mgs_plan_create +
mgs_plan_launch), the table's copy to pinned host memory, and the budget solve
(mgs_solve_budget).  `value` = cost-table evaluations (element x ratio x
bit-width) per second over the timed steps; `e2e` = the same metric through
the one-call API from pinned host buffers (attribute upload and table
download inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own scene (seed + rank): scenes are
independent, so the work is sharded with no collective on the data path
(weak scaling); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2604_26799_gb300 import synth  # noqa: E402

WORKLOAD = synth.SCENE
METRIC = "cost-table evals/s"
UNIT = "evals/s"
N_CH = synth.N_CHANNELS
ALU_OPS_PER_EVAL = 12        # fma, 2 clamps, round, int->float, sub, mul, sub, e^2, |e|, max|e|, histogram
LANES_PER_SM_CLK = 128       # 4 SM sub-partitions x 32 lanes, one warp-instruction each per clock


def evals_of(w: synth.Workload, n: int | None = None) -> int:
    n = w.n if n is None else n
    keep = synth.keep_counts(n, list(w.ratios))
    return int(keep.sum()) * N_CH * len(w.bits)


def algorithmic_bytes(w: synth.Workload) -> int:
    """Bytes the cost kernel must read per launch: every kept element's 59 channels (4 B)
    once per ratio, plus its 4-byte kept index once per channel chunk read; and write
    the table."""
    keep = synth.keep_counts(w.n, list(w.ratios))
    groups = sum((int(k) + w.group_size - 1) // w.group_size for k in keep)
    items = groups * N_CH
    table = items * len(w.bits) * (8 * 3 + 4) + items * 12
    return int(keep.sum()) * N_CH * 4 + table


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return ws, rank, local


def reduce_max(value: float, world: int) -> float:
    """Max over ranks (identity on one process)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self) -> dict:
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        mx = max(r[1] for r in rows)
        load = [r for r in rows if r[0] >= 0.5 * mx] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in load for i, v in enumerate(r[2]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in load), "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)) | {"source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# ---------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(n_sample: int, seed: int):
    """The oracle as it stands, on the first-ratio grid of a smaller scene of the
    same distributions (the full scene would take hours of one CPU core)."""
    import oracle
    w = WORKLOAD
    attrs, imp = synth.make_scene(n_sample, seed)
    keep = synth.keep_counts(n_sample, list(w.ratios))
    t0 = time.perf_counter()
    oracle.cost_table(attrs, imp, keep, list(w.bits), w.group_size)
    dt = time.perf_counter() - t0
    ev = int(keep.sum()) * N_CH * len(w.bits)
    return ev, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_sample = int(os.environ.get("MGS_ORACLE_SAMPLE", "120000"))
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample(20_000, seed=1)
    total_ev, total_t = 0, 0.0
    for s in range(args.steps):
        ev, dt = oracle_sample(n_sample, seed=s)
        total_ev += ev
        total_t += dt
    value = total_ev / total_t
    sample = (f"{n_sample} Gaussians per step (of {WORKLOAD.n}), same distributions and grid "
              f"(10 ratios x 10 bit-widths, G={WORKLOAD.group_size}); oracle.cost_table, 1 thread")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_block(args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def config_block(n_gpus: int) -> dict:
    w = WORKLOAD
    return {"workload": w.name, "n_gaussians": w.n, "channels": N_CH,
            "reserve_ratios": [f"{p}/{q}" for p, q in w.ratios], "bits": list(w.bits),
            "group_size": w.group_size, "budget_bytes": w.budget_bytes,
            "parallelism": f"replicas x{n_gpus}" if n_gpus > 1 else "1 GPU",
            "l2": "inputs larger than L2 (1.24 GB attributes, 1.5 GB slabs per scene)"}


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args):
    import torch
    from paper_2604_26799_gb300 import mgs

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    w = WORKLOAD
    attrs_np, imp_np = synth.make_scene(w.n, seed=w.seed + rank)
    keep = w.keep()
    grid = mgs.Grid(keep, list(w.bits), w.group_size)
    attrs_d = torch.from_numpy(attrs_np).to(dev)
    imp_d = torch.from_numpy(imp_np).to(dev)
    attrs_h = torch.from_numpy(attrs_np).pin_memory()
    imp_h = torch.from_numpy(imp_np).pin_memory()
    del attrs_np
    ctx = mgs.mgs_create(dev.index)
    L = mgs.mgs_table_layout_for(w.n, N_CH, grid)
    table_d = torch.empty(L.total_bytes, dtype=torch.uint8, device=dev)
    table_h = torch.empty(L.total_bytes, dtype=torch.uint8).pin_memory()
    table_np = table_h.numpy()
    opts = mgs.solve_opts()
    st = torch.cuda.Stream(device=dev)
    evals = evals_of(w)
    kernel_ms: list[float] = []
    phase = {"scene": [], "plan": [], "kernel": [], "d2h": [], "solve": []}

    def step(record: bool):
        with torch.cuda.stream(st):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            e[0].record(st)
            scene = mgs.mgs_scene_create(ctx, attrs_d, imp_d, stream=st)
            e[1].record(st)
            plan = mgs.mgs_plan_create(ctx, [scene], grid, [table_d], use_graph=False, stream=st)
            e[2].record(st)
            mgs.mgs_plan_launch(plan, st)
            e[3].record(st)
            table_h.copy_(table_d, non_blocking=True)
            e[4].record(st)
            e[4].synchronize()
            t0 = time.perf_counter()
            sol = mgs.mgs_solve_budget(table_np, L, grid, w.budget_bytes, opts)
            t_solve = time.perf_counter() - t0
            mgs.mgs_plan_destroy(plan)
            mgs.mgs_scene_destroy(scene)
        if record:
            phase["scene"].append(e[0].elapsed_time(e[1]))
            phase["plan"].append(e[1].elapsed_time(e[2]))
            phase["kernel"].append(e[2].elapsed_time(e[3]))
            phase["d2h"].append(e[3].elapsed_time(e[4]))
            phase["solve"].append(1000 * t_solve)
            kernel_ms.append(e[2].elapsed_time(e[3]))
        return sol

    # pick the tile shape for this grid on this GPU (one-time, before the timed region)
    tune = None
    if not args.no_autotune:
        sc = mgs.mgs_scene_create(ctx, attrs_d, imp_d, stream=st)
        chosen, ms_cfg = mgs.mgs_autotune(ctx, sc, grid, stream=st)
        mgs.mgs_scene_destroy(sc)
        tune = {"chosen": mgs.mgs_tile_config_name(chosen),
                "ms": {mgs.mgs_tile_config_name(i): round(float(t), 3)
                       for i, t in enumerate(ms_cfg) if t > 0}}
    for _ in range(args.warmup):
        sol = step(False)
    torch.cuda.synchronize()
    barrier(ws)
    launches0 = mgs.mgs_kernel_launches()
    with ClockSampler(dev.index) as clk:
        torch.cuda.synchronize()
        barrier(ws)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(st)
        for _ in range(args.steps):
            sol = step(True)
        ev1.record(st)
        torch.cuda.synchronize()
        barrier(ws)
    launches = (mgs.mgs_kernel_launches() - launches0) // args.steps
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = reduce_max(ms, ws)
    clocks = clk.summary()

    # e2e: the one-call public API from pinned host buffers
    e2e_ms = None
    if rank == 0 or True:
        def e2e_step():
            scene = mgs.mgs_scene_create(ctx, attrs_h, imp_h, stream=st)
            mgs.mgs_build_cost_table(ctx, scene, grid, table_h, stream=st)
            s = mgs.mgs_solve_budget(table_np, L, grid, w.budget_bytes, opts)
            mgs.mgs_scene_destroy(scene)
            return s
        e2e_step()
        torch.cuda.synchronize()
        barrier(ws)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        e2e_ms = reduce_max(1000 * (time.perf_counter() - t0) / args.steps, ws)

    # plain per-configuration loop on the same scene (comparator), table only
    plain_ms = fused_ms = None
    if not args.no_plain:
        scene = mgs.mgs_scene_create(ctx, attrs_d, imp_d, stream=st)
        with torch.cuda.stream(st):
            mgs.mgs_build_cost_table(ctx, scene, grid, table_d, stream=st)   # kept lists cached
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            mgs.mgs_build_cost_table_plain(ctx, scene, grid, table_d, stream=st)
            b.record(st)
            b.synchronize()
            plain_ms = a.elapsed_time(b)
            a.record(st)
            mgs.mgs_build_cost_table(ctx, scene, grid, table_d, stream=st)
            b.record(st)
            b.synchronize()
            fused_ms = a.elapsed_time(b)
        mgs.mgs_scene_destroy(scene)

    peaks = measured_peaks()
    k_ms = statistics.mean(kernel_ms)
    k_bytes = algorithmic_bytes(w)
    hbm_gbs = k_bytes / (k_ms * 1e-3) / 1e9
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12   # T ops/s
    alu_achieved = evals * ALU_OPS_PER_EVAL / (k_ms * 1e-3) / 1e12
    traffic = None
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(prof):
        try:
            traffic = json.load(open(prof)).get("k_cost_bytes_per_launch")
        except (OSError, ValueError):
            traffic = None

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        n_sample = int(os.environ.get("MGS_ORACLE_SAMPLE", "120000"))
        ev, dt = oracle_sample(n_sample, seed=99)
        cpu = {"value": ev / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle.cost_table on {n_sample} Gaussians of the same distributions and grid, "
                         f"{dt:.1f} s of one core"}

    if rank == 0:
        value = evals * ws / (ms_max * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_block(ws),
            "roofline": {"bound": "alu", "achieved": alu_achieved, "peak": alu_peak, "unit": "Tops/s",
                         "frac": alu_achieved / alu_peak, "traffic": traffic,
                         "kernel": "k_cost", "ops_per_eval": ALU_OPS_PER_EVAL,
                         "peak_source": f"{n_sm} SMs x {LANES_PER_SM_CLK} lanes x {sm_mhz:.0f} MHz"},
            "hbm": {"achieved": hbm_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": hbm_gbs / peaks["hbm_gbs"], "bytes_per_launch": k_bytes,
                    "peak_source": peaks["source"]},
            "kernel_ms": k_ms,
            "phase_ms": {k: statistics.mean(v) for k, v in phase.items()},
            "table_evals_per_s": evals / (k_ms * 1e-3),
            "entries_per_s": int(L.n_items) * len(w.bits) / (ms_max * 1e-3),
            "plain_loop_table_ms": plain_ms, "fused_table_ms": fused_ms,
            "solution": {"r_index": sol["r_index"], "est_bytes": sol["est_bytes"],
                         "objective": sol["objective"], "lp_bound": sol["lp_bound"]},
            "e2e": {"value": evals * ws / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(attrs_h.numel() * 4 + imp_h.numel() * 4),
                    "d2h_bytes_per_step": int(L.total_bytes), "ms_per_step": e2e_ms},
            "gpu_launches": int(launches),
            "autotune": tune,
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    mgs.mgs_destroy(ctx)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mgs", choices=["mgs", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-loop comparator")
    ap.add_argument("--no-autotune", action="store_true", help="use the default tile shape")
    ap.add_argument("--n", type=int, default=None,
                    help="scene size override (smaller cases for profiling; default 5,270,000)")
    args = ap.parse_args()
    if args.n is not None:
        global WORKLOAD
        import dataclasses
        WORKLOAD = dataclasses.replace(synth.SCENE, n=args.n,
                                       name=synth.SCENE.name.replace("N=5.27M", f"N={args.n}"))
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
