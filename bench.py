"""Benchmark of the cost-table search on the scene-scale workload.

Workload (the paper's scene scale, Sec. I: 5.27 M Gaussians, 59 FP32 channels):
N = 5,270,000 synthetic Gaussians, reserve ratios 0.1..1.0 (10 kept sets),
bit-widths {2,3,4,5,6,8,10,12,14,16}, groups of 4,096, 0-1 ILP at 40 MB.

One step = the whole hot path over one scene whose attributes are resident in
HBM: validation, importance rank, Morton order, slab relayout
(mgs_scene_create), kept lists and the fused cost kernel (mgs_plan_create +
mgs_plan_launch), and the budget solve on the device
(mgs_solve_budgets_device, whose chosen options come back to the host).
`value` = cost-table evaluations (element x ratio x bit-width) per second over
the timed steps; `e2e` = the same metric through the same calls from pinned
host buffers (each step uploads its attributes and importance and reads its
solution back), with step i+1's scene created on a second stream while step i
runs; the serial figure is reported beside it.

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
import tempfile
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
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms while running.
    Started before the warm-up (nvidia-smi takes a while to start); mark() and
    unmark() bracket the timed region, whose samples the summary reports."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")
    t0 = t1 = None

    def mark(self):
        self.t0 = time.time()

    def unmark(self):
        self.t1 = time.time()

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples: a temporary file, or where MGS_CLOCKS_CSV says (kept)
        self.keep = os.environ.get("MGS_CLOCKS_CSV")
        if self.keep:
            self.path = self.keep
        else:
            fd, self.path = tempfile.mkstemp(prefix=f"mgs_clocks_gpu{gpu_index}_", suffix=".csv")
            os.close(fd)

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
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
        import datetime
        rows = []
        with open(self.path) as fh:
            lines = fh.read().splitlines()
        if not self.keep:
            try:
                os.remove(self.path)
            except OSError:
                pass
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((float(parts[1]), float(parts[2]), parts[5:9], ts))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        if self.t0 is not None and self.t1 is not None:
            inside = [r for r in rows if self.t0 - 0.05 <= r[3] <= self.t1 + 0.05]
            if not inside:   # the nearest sample to the timed region
                inside = [min(rows, key=lambda r: abs(r[3] - 0.5 * (self.t0 + self.t1)))]
            rows = inside
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
def cpu_info() -> dict:
    """Host CPU model and core count (the GPU machine is an Arm Grace host)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and ":" in line:
                model = (model + " / " if model else "") + line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return {"cpu_model": model or platform.processor() or platform.machine(), "host_cores": os.cpu_count()}


def cpu_baseline(attrs: np.ndarray, imp: np.ndarray) -> dict:
    """The oracle as it stands: the full scene-scale table on every host core
    (threaded over its independent items), and a bounded sample on one core."""
    import oracle
    w = WORKLOAD
    cores = os.cpu_count() or 1
    keep = w.keep()
    full = os.environ.get("MGS_ORACLE_FULL", "1") != "0"
    if full:
        t0 = time.perf_counter()
        oracle.cost_table(attrs, imp, keep, list(w.bits), w.group_size, threads=cores)
        dt_all = time.perf_counter() - t0
        ev_all = evals_of(w)
        sample_all = (f"the full table of the timed workload ({w.n} Gaussians, 10 ratios x 10 bit-widths), "
                      f"oracle.cost_table on {cores} threads, {dt_all:.1f} s including its rank and Morton sorts")
    else:
        n_s = int(os.environ.get("MGS_ORACLE_SAMPLE_ALL", "1000000"))
        ev_all, dt_all = oracle_sample(n_s, seed=98, threads=cores)
        sample_all = f"{n_s} Gaussians of the same distributions and grid on {cores} threads, {dt_all:.1f} s"
    n_sample = int(os.environ.get("MGS_ORACLE_SAMPLE", "120000"))
    ev1, dt1 = oracle_sample(n_sample, seed=99)
    sample_1 = (f"oracle.cost_table on {n_sample} Gaussians of the same distributions and "
                f"grid, {dt1:.1f} s of one core")
    return {"value": ev_all / dt_all, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample_all,
            "cores_all": {"cores": cores, "value": ev_all / dt_all, "sample": sample_all},
            "cores_1": {"cores": 1, "value": ev1 / dt1, "sample": sample_1}, **cpu_info()}


def kernel_counters() -> dict:
    """ncu figures of the current cost kernel (profiles/k_cost_counters.json): they
    apply only while the kernel source is the one they were taken from."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_cost_counters.json")
    src = os.path.join(ROOT, "paper_2604_26799_gb300", "csrc", "cost.cu")
    try:
        c = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return {}
    if c.get("cost_cu_sha256") != sha:
        return {"note": "kernel changed since the counters were taken"}
    return c


def oracle_sample(n_sample: int, seed: int, threads: int = 1):
    """The oracle as it stands, on the first-ratio grid of a smaller scene of the
    same distributions (the full scene would take hours of one CPU core)."""
    import oracle
    w = WORKLOAD
    attrs, imp = synth.make_scene(n_sample, seed)
    keep = synth.keep_counts(n_sample, list(w.ratios))
    t0 = time.perf_counter()
    oracle.cost_table(attrs, imp, keep, list(w.bits), w.group_size, threads=threads)
    dt = time.perf_counter() - t0
    ev = int(keep.sum()) * N_CH * len(w.bits)
    return ev, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n_sample = int(os.environ.get("MGS_ORACLE_SAMPLE", "600000"))
    cores = os.cpu_count() or 1
    for _ in range(args.warmup if args.warmup < 1 else 1):
        oracle_sample(20_000, seed=1, threads=cores)
    total_ev, total_t = 0, 0.0
    for s in range(args.steps):
        ev, dt = oracle_sample(n_sample, seed=s, threads=cores)
        total_ev += ev
        total_t += dt
    value = total_ev / total_t
    sample = (f"{n_sample} Gaussians per step (of {WORKLOAD.n}), same distributions and grid "
              f"(10 ratios x 10 bit-widths, G={WORKLOAD.group_size}); oracle.cost_table on {cores} threads")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": config_block(args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             **cpu_info()},
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
    opts = mgs.solve_opts()
    st = torch.cuda.Stream(device=dev)
    evals = evals_of(w)
    kernel_ms: list[float] = []
    phase = {"scene": [], "plan": [], "kernel": [], "solve": []}

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
            # the budget solve on the device; only the chosen options come back
            sol = mgs.mgs_solve_budgets_device(ctx, table_d, L, grid, [w.budget_bytes], opts, stream=st)[0]
            e[4].record(st)
            mgs.mgs_plan_destroy(plan)
            mgs.mgs_scene_destroy(scene)
        if record:
            e[4].synchronize()
            phase["scene"].append(e[0].elapsed_time(e[1]))
            phase["plan"].append(e[1].elapsed_time(e[2]))
            phase["kernel"].append(e[2].elapsed_time(e[3]))
            phase["solve"].append(e[3].elapsed_time(e[4]))
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
    with ClockSampler(dev.index) as clk:
        for _ in range(args.warmup):   # nvidia-smi starts meanwhile
            sol = step(False)
        torch.cuda.synchronize()
        barrier(ws)
        launches0 = mgs.mgs_kernel_launches()
        clk.mark()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(st)
        for _ in range(args.steps):
            sol = step(True)
        ev1.record(st)
        torch.cuda.synchronize()
        clk.unmark()
        barrier(ws)
    launches = (mgs.mgs_kernel_launches() - launches0) // args.steps
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_max = reduce_max(ms, ws)
    clocks = clk.summary()

    # e2e: the public API from pinned host buffers.  Serial: one step after the
    # other.  Pipelined (the figure reported): step i+1's scene is created (its
    # upload, validation, Morton sort and relayout) on a second stream while
    # step i's cost table and solve run; every step still uploads its own
    # inputs and reads its own solution back to the host.
    st2 = torch.cuda.Stream(device=dev)

    def e2e_step():
        scene = mgs.mgs_scene_create(ctx, attrs_h, imp_h, stream=st)
        mgs.mgs_build_cost_table(ctx, scene, grid, table_d, stream=st)
        s = mgs.mgs_solve_budgets_device(ctx, table_d, L, grid, [w.budget_bytes], opts, stream=st)[0]
        mgs.mgs_scene_destroy(scene)
        return s

    from concurrent.futures import ThreadPoolExecutor

    def e2e_create():
        # scene creation (upload, validation, sort, relayout) on the second stream,
        # from an ingest thread: the call waits for its validation result on the
        # host, which must not hold up the thread that launches the cost table
        scene = mgs.mgs_scene_create(ctx, attrs_h, imp_h, stream=st2)
        ready = torch.cuda.Event()
        ready.record(st2)
        return scene, ready

    def e2e_pipelined(k):
        sols = []
        with ThreadPoolExecutor(max_workers=1) as ingest:
            nxt = ingest.submit(e2e_create)
            for i in range(k):
                scene, ready = nxt.result()
                st.wait_event(ready)
                mgs.mgs_build_cost_table(ctx, scene, grid, table_d, stream=st)
                if i + 1 < k:
                    nxt = ingest.submit(e2e_create)
                sols.append(mgs.mgs_solve_budgets_device(ctx, table_d, L, grid, [w.budget_bytes], opts,
                                                         stream=st)[0])
                mgs.mgs_scene_destroy(scene)
        return sols

    e2e_step()
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_serial_ms = reduce_max(1000 * (time.perf_counter() - t0) / args.steps, ws)
    e2e_pipelined(2)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    e2e_sols = e2e_pipelined(args.steps)
    torch.cuda.synchronize()
    e2e_ms = reduce_max(1000 * (time.perf_counter() - t0) / args.steps, ws)
    e2e_same = all(x["r_index"] == sol["r_index"] and x["objective"] == sol["objective"] for x in e2e_sols)

    # the host-to-device copy alone (pinned attributes and importance), for the e2e budget
    h2d_ms = []
    with torch.cuda.stream(st):
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            attrs_d.copy_(attrs_h, non_blocking=True)
            imp_d.copy_(imp_h, non_blocking=True)
            b.record(st)
            b.synchronize()
            h2d_ms.append(a.elapsed_time(b))
    h2d_ms = statistics.median(h2d_ms)

    # the host solver on the same table (comparator for the device solve)
    table_np = table_d.cpu().numpy()
    t0 = time.perf_counter()
    host_sol = mgs.mgs_solve_budget(table_np, L, grid, w.budget_bytes, opts)
    host_solve_ms = 1000 * (time.perf_counter() - t0)
    same_as_host = (host_sol["r_index"] == sol["r_index"] and host_sol["objective"] == sol["objective"]
                    and bool((host_sol["choice"] == sol["choice"]).all()))
    del table_np

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
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline, hbm = kernel_rooflines(evals, k_ms, k_bytes, n_sm, peaks)
    counters = kernel_counters()
    roofline["traffic"] = counters.get("traffic_bytes_per_launch")
    roofline["executed_instr_per_eval"] = counters.get("executed_instr_per_eval")
    roofline["counters_source"] = counters.get("note")

    # the other workloads of the metric, one GPU: the large single scene, the batched
    # persistent launch and the served job stream
    workloads = None
    if rank == 0 and ws == 1 and not args.no_workloads:
        del table_d
        torch.cuda.empty_cache()
        src = SourceScene(torch, dev)
        workloads = {"large": large_record(torch, mgs, ctx, src, 3, 1),
                     "batch": batch_record(torch, mgs, ctx, src, 3, 1),
                     "serve": serve_record(torch, mgs, ctx, src, int(os.environ.get("MGS_SERVE_JOBS", "120")),
                                           args.slice_items)}
        del src
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        cpu = cpu_baseline(attrs_h.numpy(), imp_h.numpy())

    if rank == 0:
        value = evals * ws / (ms_max * 1e-3)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config_block(ws),
            "roofline": roofline,
            "hbm": hbm,
            "kernel_ms": k_ms,
            "phase_ms": {k: statistics.mean(v) for k, v in phase.items()},
            "table_evals_per_s": evals / (k_ms * 1e-3),
            "entries_per_s": int(L.n_items) * len(w.bits) / (ms_max * 1e-3),
            "plain_loop_table_ms": plain_ms, "fused_table_ms": fused_ms,
            "host_solve_ms": host_solve_ms, "device_solve_equals_host": same_as_host,
            "solution": {"r_index": sol["r_index"], "est_bytes": sol["est_bytes"],
                         "objective": sol["objective"], "lp_bound": sol["lp_bound"]},
            "e2e": {"value": evals * ws / (e2e_ms * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": int(attrs_h.numel() * 4 + imp_h.numel() * 4),
                    "h2d_copy_ms": h2d_ms,
                    "h2d_gbs": (attrs_h.numel() * 4 + imp_h.numel() * 4) / (h2d_ms * 1e-3) / 1e9,
                    "d2h_bytes_per_step": int(sol["choice"].nbytes) + 48 * len(w.ratios), "ms_per_step": e2e_ms,
                    "pipelined": "step i+1's scene creation (upload included) on a second stream, from an ingest thread, during step i",
                    "serial_ms_per_step": e2e_serial_ms, "solutions_equal_device_step": e2e_same},
            "gpu_launches": int(launches),
            "autotune": tune,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "workloads": workloads,
        }
        print(json.dumps(line))
    mgs.mgs_destroy(ctx)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# Other workloads (one JSON line each; the default is the scene-scale search)
# ---------------------------------------------------------------------------
def _events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def kernel_rooflines(evals: int, k_ms: float, k_bytes: int, n_sm: int, peaks: dict) -> tuple[dict, dict]:
    """ALU-issue roofline (the bound of the cost kernel) and the HBM fraction with
    algorithmic bytes, for a cost-kernel time of k_ms."""
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    alu_peak = n_sm * LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12   # T ops/s
    alu = evals * ALU_OPS_PER_EVAL / (k_ms * 1e-3) / 1e12
    gbs = k_bytes / (k_ms * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": alu, "peak": alu_peak, "unit": "Tops/s", "frac": alu / alu_peak,
            "kernel": "k_cost", "ops_per_eval": ALU_OPS_PER_EVAL,
            "peak_source": f"{n_sm} SMs x {LANES_PER_SM_CLK} lanes x {sm_mhz:.0f} MHz"}
    hbm = {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
           "bytes_per_launch": k_bytes, "peak_source": peaks["source"]}
    return roof, hbm


def grid_bytes(keeps, G: int, n_bits: int) -> int:
    """Algorithmic bytes of a cost launch over kept sets `keeps`: every kept element's
    59 channels once per ratio (4 B each), plus the table written."""
    total = 0
    for keep in keeps:
        groups = sum((int(k) + G - 1) // G for k in keep)
        items = groups * N_CH
        total += int(np.sum(keep)) * N_CH * 4 + items * n_bits * (8 * 3 + 4) + items * 12
    return total


class SourceScene:
    """One generated 6 M-Gaussian scene (the large workload's) feeding the batched and
    served workloads too: their scenes are row ranges of it (same distributions), so
    the default run generates it once."""

    def __init__(self, torch, dev):
        w = synth.LARGE
        a, imp = synth.make_scene(w.n, seed=w.seed)
        self.n = w.n
        self.h_attrs = torch.from_numpy(a).pin_memory()
        self.h_imp = torch.from_numpy(imp).pin_memory()
        self.d_attrs = self.h_attrs.to(dev)
        self.d_imp = self.h_imp.to(dev)
        del a, imp

    def rows(self, n: int, i: int, device: bool):
        """Scene i of size n: a contiguous row range."""
        off = (i * 1_000_003) % (self.n - n + 1)
        a, imp = (self.d_attrs, self.d_imp) if device else (self.h_attrs, self.h_imp)
        return a[off:off + n], imp[off:off + n]


def batch_record(torch, mgs, ctx, src: SourceScene, steps: int, warmup: int) -> dict:
    """16 scenes of uneven size (log-uniform 3e5..6e6), 10 ratios x 10 bit-widths, in one
    persistent launch replayed from a CUDA graph; group sizes 1024 / 4096 / 16384, tile
    shape autotuned per group size.  Compared with one launch per scene."""
    dev = src.d_attrs.device
    sizes = [int(x) for x in synth.batch_sizes(16, 300_000, 6_000_000, seed=3)]
    bits = list(synth.SCENE.bits)
    st = torch.cuda.Stream(device=dev)
    scenes = []
    for i, n in enumerate(sizes):
        a, imp = src.rows(n, i, device=True)
        scenes.append(mgs.mgs_scene_create(ctx, a, imp, stream=st))
    keeps = [synth.keep_counts(n, list(synth.tenths())) for n in sizes]
    evals = sum(int(k.sum()) for k in keeps) * N_CH * len(bits)
    peaks = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    per_g = {}
    with ClockSampler(dev.index) as clk:
        for G in (1024, 4096, 16384):
            grids = [mgs.Grid(k, bits, G) for k in keeps]
            lays = [mgs.mgs_table_layout_for(n, N_CH, g) for n, g in zip(sizes, grids)]
            tables = [torch.empty(L.total_bytes, dtype=torch.uint8, device=dev) for L in lays]
            big = int(np.argmax(sizes))
            chosen, _ = mgs.mgs_autotune(ctx, scenes[big], grids[big], stream=st)
            with torch.cuda.stream(st):
                plan = mgs.mgs_plan_create(ctx, scenes, grids, tables, use_graph=True, stream=st)
                singles = [mgs.mgs_plan_create(ctx, [sc], [g], [t], use_graph=False, stream=st)
                           for sc, g, t in zip(scenes, grids, tables)]
                for _ in range(max(1, warmup)):
                    mgs.mgs_plan_launch(plan, st)
                    for p in singles:
                        mgs.mgs_plan_launch(p, st)
                a, b = _events(torch)
                if G == 4096:
                    clk.mark()
                a.record(st)
                for _ in range(steps):
                    mgs.mgs_plan_launch(plan, st)
                b.record(st)
                b.synchronize()
                if G == 4096:
                    clk.unmark()
                batched_ms = a.elapsed_time(b) / steps
                a.record(st)
                for _ in range(steps):
                    for p in singles:
                        mgs.mgs_plan_launch(p, st)
                b.record(st)
                b.synchronize()
                seq_ms = a.elapsed_time(b) / steps
                mgs.mgs_plan_destroy(plan)
                for p in singles:
                    mgs.mgs_plan_destroy(p)
            roof, hbm = kernel_rooflines(evals, batched_ms, grid_bytes(keeps, G, len(bits)), n_sm, peaks)
            per_g[str(G)] = {"tile": mgs.mgs_tile_config_name(chosen), "batched_graph_ms": batched_ms,
                             "batched_evals_per_s": evals / (batched_ms * 1e-3),
                             "one_launch_per_scene_ms": seq_ms, "roofline": roof, "hbm": hbm}
            del tables
            torch.cuda.synchronize()
    for sc in scenes:
        mgs.mgs_scene_destroy(sc)
    best_g = max(per_g, key=lambda g: per_g[g]["batched_evals_per_s"])
    best = per_g[best_g]
    return {"metric": METRIC, "value": best["batched_evals_per_s"], "unit": UNIT, "steps": steps,
            "warmup": warmup, "ms_per_step": best["batched_graph_ms"], "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched: 16 scenes, N log-uniform 3e5..6e6 (total %d), 10 ratios x "
                                   "10 bit-widths, one persistent launch in a CUDA graph, G swept "
                                   "1024/4096/16384 (best reported)" % sum(sizes), "sizes": sizes,
                       "best_group_size": int(best_g)},
            "evals_per_pass": evals, "roofline": best["roofline"], "hbm": best["hbm"],
            "per_group_size": per_g, "clocks": clk.summary()}


def serve_record(torch, mgs, ctx, src: SourceScene, n_jobs: int, slice_items: int) -> dict:
    """Poisson job stream (20 jobs/s; N log-uniform 1e5..6e6; budget U[5, 60] MB; each a
    10 x 10 search) through the continuous-batching server; p50/p99 time from submission to
    the ILP answer.  Compared with a one-job-at-a-time plain per-(ratio, bit-width) loop fed
    the same arrivals (its service times measured per scene)."""
    dev = src.d_attrs.device
    t_arr, job_sizes, budgets = synth.poisson_arrivals(n_jobs, 20.0, seed=7)
    # a pool of resident host scenes; job j uses the pool scene closest to its drawn size
    pool_n = sorted({int(x) for x in np.quantile(job_sizes, np.linspace(0, 1, 12))})
    pool = [(*src.rows(n, i, device=False), n) for i, n in enumerate(pool_n)]
    pick = [int(np.argmin([abs(np.log(p[2]) - np.log(n)) for p in pool])) for n in job_sizes]
    bits = list(synth.SCENE.bits)
    grids = [mgs.Grid(synth.keep_counts(p[2], list(synth.tenths())), bits, 4096) for p in pool]
    opts = mgs.solve_opts()
    # warm-up: one job per pool scene (also the plain loop's service time per scene)
    plain_service = []
    st = torch.cuda.Stream(device=dev)
    for (a, imp, n), g in zip(pool, grids):
        L = mgs.mgs_table_layout_for(n, N_CH, g)
        tab = torch.empty(L.total_bytes, dtype=torch.uint8).pin_memory()
        t0 = time.perf_counter()
        sc = mgs.mgs_scene_create(ctx, a, imp, stream=st)
        mgs.mgs_build_cost_table_plain(ctx, sc, g, tab, stream=st)
        mgs.mgs_solve_budget(tab.numpy(), L, g, 30e6, opts)
        mgs.mgs_scene_destroy(sc)
        plain_service.append(time.perf_counter() - t0)
    srv = mgs.mgs_server_create(ctx, max_jobs=8, solver_threads=8, hbm_budget_bytes=120 << 30,
                                slice_items=slice_items)
    ids = []
    with ClockSampler(dev.index) as clk:
        time.sleep(0.3)   # nvidia-smi starts
        clk.mark()
        t_start = time.perf_counter()
        for j in range(n_jobs):
            now = time.perf_counter() - t_start
            if t_arr[j] > now:
                time.sleep(t_arr[j] - now)
            a, imp, n = pool[pick[j]]
            ids.append(mgs.mgs_server_submit(srv, a, imp, grids[pick[j]], float(budgets[j]), opts))
        res = [mgs.mgs_server_wait(srv, i, timeout_ms=600_000) for i in ids]
        clk.unmark()
    stats = mgs.mgs_server_stats(srv)
    mgs.mgs_server_destroy(srv)
    lat = np.array([r["t_done"] - r["t_submit"] for r in res])
    # where the latency goes: waiting for admission, ingest, compute, solve
    stages = {}
    for name, a_, b_ in (("admit_wait", "t_submit", "t_admit"), ("ingest", "t_admit", "t_ready"),
                         ("compute", "t_ready", "t_table"), ("solve", "t_table", "t_done")):
        d_ = np.array([r[b_] - r[a_] for r in res])
        stages[name] = {"p50_s": float(np.percentile(d_, 50)), "p99_s": float(np.percentile(d_, 99))}
    slow = int(np.argmax(lat))
    stages["slowest_job"] = {"n": int(pool[pick[slow]][2]),
                             **{k: float(res[slow][v] - res[slow]["t_submit"])
                                for k, v in (("admit", "t_admit"), ("ready", "t_ready"), ("table", "t_table"),
                                             ("done", "t_done"))}}
    ok = sum(1 for r in res if r["status"] == 0)
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    # the plain loop, one job at a time, same arrivals
    finish, plain_lat = 0.0, []
    for j in range(n_jobs):
        start = max(t_arr[j], finish)
        finish = start + plain_service[pick[j]]
        plain_lat.append(finish - t_arr[j])
    plain_lat = np.array(plain_lat)
    keeps = [synth.keep_counts(pool[pick[j]][2], list(synth.tenths())) for j in range(n_jobs)]
    evals = sum(int(k.sum()) for k in keeps) * N_CH * len(bits)
    peaks = measured_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    # whole-job figures over the served span: the arrival rate, not the GPU, sets it
    roof, hbm = kernel_rooflines(evals, span * 1e3, grid_bytes(keeps, 4096, len(bits)), n_sm, peaks)
    roof["bound"] = "arrival rate (20 jobs/s): whole-job evals over the served span"
    return {
        "metric": "served search latency (submission to ILP answer)", "unit": "s",
        "value": float(np.percentile(lat, 50)), "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)), "jobs_per_s": n_jobs / span, "jobs_ok": ok,
        "jobs": n_jobs, "evals_per_s": evals / span, "higher_is_better": False,
        "plain_loop_p50_s": float(np.percentile(plain_lat, 50)),
        "plain_loop_p99_s": float(np.percentile(plain_lat, 99)),
        "server": stats, "stages": stages, "data": "synthetic", "roofline": roof, "hbm": hbm,
        "clocks": clk.summary(),
        "config": {"workload": "serving: Poisson 20 jobs/s, N log-uniform 1e5..6e6 (12-scene pool), "
                               "budget U[5,60] MB, 10 ratios x 10 bit-widths, G 4096",
                   "pool_sizes": pool_n, "slice_items": slice_items}}


def large_record(torch, mgs, ctx, src: SourceScene, steps: int, warmup: int) -> dict:
    """6 M Gaussians, 20 ratios (0.05..1.00), bit-widths 1..16, groups of 2048; ILP at 8 budgets."""
    dev = src.d_attrs.device
    w = synth.LARGE
    a_d, i_d = src.d_attrs, src.d_imp
    grid = mgs.Grid(w.keep(), list(w.bits), w.group_size)
    st = torch.cuda.Stream(device=dev)
    L = mgs.mgs_table_layout_for(w.n, N_CH, grid)
    tab = torch.empty(L.total_bytes, dtype=torch.uint8, device=dev)
    sc = mgs.mgs_scene_create(ctx, a_d, i_d, stream=st)
    chosen, _ = mgs.mgs_autotune(ctx, sc, grid, stream=st)
    mgs.mgs_scene_destroy(sc)
    budgets = [10e6, 20e6, 40e6, 60e6, 80e6, 120e6, 160e6, 240e6]
    phase = {"scene": [], "kernel": [], "solve_8_budgets": []}
    evals = int(w.keep().sum()) * N_CH * len(w.bits)
    total = 0.0
    with ClockSampler(dev.index) as clk:
        for step in range(warmup + steps):
            if step == warmup:
                clk.mark()
            with torch.cuda.stream(st):
                e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                e[0].record(st)
                sc = mgs.mgs_scene_create(ctx, a_d, i_d, stream=st)
                plan = mgs.mgs_plan_create(ctx, [sc], grid, [tab], stream=st)
                e[1].record(st)
                mgs.mgs_plan_launch(plan, st)
                e[2].record(st)
                sols = mgs.mgs_solve_budgets_device(ctx, tab, L, grid, budgets, mgs.solve_opts(), stream=st)
                e[3].record(st)
                mgs.mgs_plan_destroy(plan)
                mgs.mgs_scene_destroy(sc)
            e[3].synchronize()
            if step >= warmup:
                phase["scene"].append(e[0].elapsed_time(e[1]))
                phase["kernel"].append(e[1].elapsed_time(e[2]))
                phase["solve_8_budgets"].append(e[2].elapsed_time(e[3]))
                total += e[0].elapsed_time(e[3])
        clk.unmark()
    # the host solver on the same table, for comparison
    tab_np = tab.cpu().numpy()
    t0 = time.perf_counter()
    host = mgs.mgs_solve_budgets(tab_np, L, grid, budgets, mgs.solve_opts())
    host_ms = 1000 * (time.perf_counter() - t0)
    same = all(a["r_index"] == b["r_index"] and a["objective"] == b["objective"] for a, b in zip(sols, host))
    ms = total / steps
    k_ms = statistics.mean(phase["kernel"])
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    roof, hbm = kernel_rooflines(evals, k_ms, grid_bytes([w.keep()], w.group_size, len(w.bits)), n_sm,
                                 measured_peaks())
    return {"metric": METRIC, "value": evals / (ms * 1e-3), "unit": UNIT, "steps": steps, "warmup": warmup,
            "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name}, "tile": mgs.mgs_tile_config_name(chosen),
            "kernel_evals_per_s": evals / (k_ms * 1e-3), "roofline": roof, "hbm": hbm,
            "phase_ms": {k: statistics.mean(v) for k, v in phase.items()},
            "host_solve_8_budgets_ms": host_ms, "device_solve_equals_host": same, "clocks": clk.summary(),
            "solutions": [{"budget": b, "r_index": s["r_index"], "est_bytes": s["est_bytes"]}
                          for b, s in zip(budgets, sols)]}


def _one_record(args, which: str):
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    ctx = mgs.mgs_create(0)
    src = SourceScene(torch, dev)
    if which == "batch":
        rec = batch_record(torch, mgs, ctx, src, args.steps, args.warmup)
    elif which == "serve":
        rec = serve_record(torch, mgs, ctx, src, int(os.environ.get("MGS_SERVE_JOBS", "120")), args.slice_items)
    else:
        rec = large_record(torch, mgs, ctx, src, args.steps, args.warmup)
    mgs.mgs_destroy(ctx)
    rec["n_gpus"] = 1
    print(json.dumps(rec))
    return 0


def run_batch(args):
    return _one_record(args, "batch")


def run_serve(args):
    return _one_record(args, "serve")


def run_large(args):
    return _one_record(args, "large")


def run_preprocess(args):
    """Preprocessing of the scene-scale scene (5.27 M Gaussians x 59 channels): Euler
    replacement and I_g = I_d * V_norm^beta.  HBM-bound: reported against the measured
    copy bandwidth with the algorithmic bytes (read 59 channels + I_d, write 58 + I_g)."""
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    w = WORKLOAD
    a, imp = synth.make_scene(w.n, seed=w.seed)
    a_d, i_d = torch.from_numpy(a).to(dev), torch.from_numpy(imp).to(dev)
    out = torch.empty((w.n, N_CH - 1), dtype=torch.float32, device=dev)
    ig = torch.empty(w.n, dtype=torch.float32, device=dev)
    ctx = mgs.mgs_create(0)
    st = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2 between steps
    times = []
    for step in range(args.warmup + args.steps):
        with torch.cuda.stream(st):
            flush.fill_(step & 255)
            e0, e1 = _events(torch)
            e0.record(st)
            mgs.mgs_preprocess(ctx, a_d, i_d, 1.0, out, ig, stream=st)
            e1.record(st)
        e1.synchronize()
        if step >= args.warmup:
            times.append(e0.elapsed_time(e1))
    mgs.mgs_destroy(ctx)
    ms = statistics.mean(times)
    bytes_alg = w.n * 4 * (N_CH + 1 + (N_CH - 1) + 1)
    peaks = measured_peaks()
    gbs = bytes_alg / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu:
        import oracle
        n_s = 1_000_000
        t0 = time.perf_counter()
        oracle.preprocess(a[:n_s], imp[:n_s], 1.0)
        dt = time.perf_counter() - t0
        cpu = {"value": n_s / dt, "unit": "Gaussians/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle.preprocess on the first {n_s} Gaussians, {dt:.2f} s of one core"}
    print(json.dumps({"metric": "preprocessed Gaussians/s", "value": w.n / (ms * 1e-3), "unit": "Gaussians/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"preprocess N={w.n}, 59 -> 58 channels, beta 1",
                                 "l2": "flushed (256 MB write) before every step"},
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                                   "bytes_per_launch": bytes_alg, "peak_source": peaks["source"]},
                      "gpu_launches": 6, "cpu_baseline": cpu}))


def run_raht(args):
    """RAHT of 10 channels (SH DC, opacity, log-scales, rotation) of the scene-scale
    scene at octree depth 16: voxel means and 48 merge steps.  Measured per call with
    the scene resident; HBM roofline with the algorithmic bytes (read the channels of
    every Gaussian, write V - 1 AC vectors)."""
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    w = WORKLOAD
    a, imp = synth.make_scene(w.n, seed=w.seed)
    channels = [3, 4, 5, 51, 52, 53, 54, 55, 56, 57]
    depth = 16
    ctx = mgs.mgs_create(0)
    st = torch.cuda.Stream(device=dev)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(imp).to(dev), stream=st)
    ac = torch.empty((w.n, len(channels)), dtype=torch.float32, device=dev)
    times, V = [], 0
    for step in range(args.warmup + args.steps):
        with torch.cuda.stream(st):
            e0, e1 = _events(torch)
            e0.record(st)
            _, _, V = mgs.mgs_raht(ctx, scene, channels, depth, ac_out=ac, stream=st)
            e1.record(st)
        e1.synchronize()
        if step >= args.warmup:
            times.append(e0.elapsed_time(e1))
    mgs.mgs_scene_destroy(scene)
    mgs.mgs_destroy(ctx)
    ms = statistics.mean(times)
    bytes_alg = w.n * len(channels) * 4 + (V - 1) * len(channels) * 4
    peaks = measured_peaks()
    gbs = bytes_alg / (ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu:
        import oracle
        n_s = 1_000_000
        t0 = time.perf_counter()
        oracle.raht(a[:n_s], channels, depth)
        dt = time.perf_counter() - t0
        cpu = {"value": n_s / dt, "unit": "Gaussians/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle.raht on the first {n_s} Gaussians (depth {depth}), {dt:.2f} s of one core"}
    print(json.dumps({"metric": "RAHT Gaussians/s", "value": w.n / (ms * 1e-3), "unit": "Gaussians/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"RAHT N={w.n}, depth {depth}, {len(channels)} channels",
                                 "voxels": V},
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": gbs / peaks["hbm_gbs"], "traffic": None,
                                   "bytes_per_launch": bytes_alg, "peak_source": peaks["source"]},
                      "cpu_baseline": cpu}))


def run_raht_search(args):
    """The search in the RAHT domain (Sec. III-D/F): for every reserve ratio of the
    scene-scale grid, the RAHT of the kept set's 7 important channels (SH DC, opacity,
    log-scales) at depth 16, the cost table of its AC coefficients (10 bit-widths,
    G = 4096) and the device budget solve; tau by the rule of mgs_solve_budget."""
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    w = WORKLOAD
    a, imp = synth.make_scene(w.n, seed=w.seed)
    channels = [3, 4, 5, 51, 52, 53, 54]
    depth, budget = 16, 7e6
    bits = list(w.bits)
    keep = w.keep()
    ctx = mgs.mgs_create(0)
    st = torch.cuda.Stream(device=dev)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(imp).to(dev), stream=st)
    ac = torch.empty((w.n, len(channels)), dtype=torch.float32, device=dev)
    opts = mgs.solve_opts(const_bytes=4.0 * len(channels))       # the DC coefficients in FP32
    times, phases, evals, pick = [], {"raht": 0.0, "table": 0.0, "solve": 0.0}, 0, None
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        per_r, ev = [], 0
        ph = {"raht": 0.0, "table": 0.0, "solve": 0.0}
        with torch.cuda.stream(st):
            for K in keep:
                e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
                e[0].record(st)
                _, acv, V = mgs.mgs_raht(ctx, scene, channels, depth, ac_out=ac, stream=st, keep=int(K))
                e[1].record(st)
                grid = mgs.Grid([V - 1], bits, w.group_size)
                L = mgs.mgs_table_layout_for(V - 1, len(channels), grid)
                tab = torch.empty(L.total_bytes, dtype=torch.uint8, device=dev)
                mgs.mgs_build_cost_table_coeffs(ctx, acv, grid, tab, stream=st)
                e[2].record(st)
                sol = mgs.mgs_solve_budgets_device(ctx, tab, L, grid, [budget], opts, stream=st)[0]
                e[3].record(st)
                e[3].synchronize()
                ph["raht"] += e[0].elapsed_time(e[1])
                ph["table"] += e[1].elapsed_time(e[2])
                ph["solve"] += e[2].elapsed_time(e[3])
                ev += (V - 1) * len(channels) * len(bits)
                per_r.append((int(sol["ratio_status"][0]), float(sol["objective"]), float(sol["est_bytes"])))
        dt = (time.perf_counter() - t0) * 1e3
        if step >= args.warmup:
            times.append(dt)
            for k in ph:
                phases[k] += ph[k] / args.steps
            evals = ev
        best, largest = -1, -1
        for r, (status, obj, _) in enumerate(per_r):
            if status < 0:
                continue
            largest = r
            if status == 1:
                continue
            if best < 0 or obj <= per_r[best][1]:
                best = r
        pick = best if best >= 0 else largest
    mgs.mgs_scene_destroy(scene)
    mgs.mgs_destroy(ctx)
    ms = statistics.mean(times)
    print(json.dumps({"metric": "RAHT-domain search: AC cost-table evals/s", "value": evals / (ms * 1e-3),
                      "unit": "evals/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"RAHT search N={w.n}, 10 ratios, depth {depth}, {len(channels)} "
                                             f"channels, b={bits}, G={w.group_size}, budget {budget:.0f} B"},
                      "phase_ms": phases, "tau_index": pick}))


def run_encode(args):
    """The block coder (Alg. 1's actual size S_a): quantise the kept half of the
    scene-scale scene (59 channels, G = 4096) with widths drawn around 8 bits and
    write the whole stream (mgs_encode_config)."""
    import numpy as np
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    w = WORKLOAD
    a, imp = synth.make_scene(w.n, seed=w.seed)
    C = a.shape[1]
    keep, G = w.n // 2, w.group_size
    ng = (keep + G - 1) // G
    q = np.clip(np.rint(np.random.default_rng(9).normal(8, 3, size=(C, ng))), 1, 16).astype(np.uint8)
    ctx = mgs.mgs_create(0)
    st = torch.cuda.Stream(device=dev)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(imp).to(dev), stream=st)
    out = torch.empty(mgs.mgs_encode_bound(keep, G, C), dtype=torch.uint8, device=dev)
    d_bits = torch.from_numpy(q).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    times, total = [], 0
    launches0 = None
    for step in range(args.warmup + args.steps):
        with torch.cuda.stream(st):
            flush.fill_(step & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if step == args.warmup:
                launches0 = mgs.mgs_kernel_launches()
            e0.record(st)
            total = mgs.mgs_encode_config(ctx, scene, keep, G, d_bits, out, stream=st)
            e1.record(st)
            e1.synchronize()
        if step >= args.warmup:
            times.append(e0.elapsed_time(e1))
    launches = (mgs.mgs_kernel_launches() - launches0) // args.steps
    mgs.mgs_scene_destroy(scene)
    mgs.mgs_destroy(ctx)
    ms = statistics.mean(times)
    codes = keep * C
    peaks = measured_peaks()
    alg = codes * 4 + keep * 4 + total           # attribute reads, kept positions, stream written once
    gbs = alg / (ms * 1e-3) / 1e9
    print(json.dumps({"metric": "block coder: codes encoded/s", "value": codes / (ms * 1e-3),
                      "unit": "codes/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "higher_is_better": True, "dtype": "u16", "data": "synthetic",
                      "config": {"workload": f"encode N={w.n}, keep {keep}, {C} channels, G={G}, "
                                             "widths ~ N(8, 3) clipped to 1..16", "l2": "flushed"},
                      "stream_bytes": int(total), "bits_per_code": 8.0 * total / codes,
                      "gpu_launches": int(launches),
                      "roofline": {"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                   "frac": gbs / peaks["hbm_gbs"], "traffic": None, "bytes_per_launch": int(alg),
                                   "peak_source": peaks["source"]}}))


def run_calibrated(args):
    """Alg. 1 end to end with real compression at scene scale: the cost table of
    the 10 x 10 grid, then the S_Delta calibration loop (mgs_search_calibrated)
    at a 40 MB budget, with the paper's linear estimator (sum P Q) and, for
    comparison, the entropy-bound estimator."""
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    w = WORKLOAD
    a, imp = synth.make_scene(w.n, seed=w.seed)
    ctx = mgs.mgs_create(0)
    st = torch.cuda.Stream(device=dev)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(imp).to(dev), stream=st)
    grid = mgs.Grid(w.keep(), list(w.bits), w.group_size)
    L = mgs.mgs_table_layout_for(w.n, a.shape[1], grid)
    tab = torch.empty(L.total_bytes, dtype=torch.uint8, device=dev)
    budget = w.budget_bytes
    res = {}
    for name, model in (("fixed", mgs.MGS_RATE_FIXED), ("entropy", mgs.MGS_RATE_ENTROPY)):
        times, tab_ms, out = [], [], None
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            with torch.cuda.stream(st):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                mgs.mgs_build_cost_table(ctx, scene, grid, tab, stream=st)
                e1.record(st)
                out = mgs.mgs_search_calibrated(ctx, scene, grid, tab, L, budget, tolerance=0.05,
                                                max_rounds=8, init_bits=8,
                                                opts=mgs.solve_opts(rate_model=model), stream=st)
            dt = (time.perf_counter() - t0) * 1e3
            if step >= args.warmup:
                times.append(dt)
                tab_ms.append(e0.elapsed_time(e1))
        res[name] = dict(ms=statistics.mean(times), table_ms=statistics.mean(tab_ms), r_index=out["r_index"],
                         rounds=int(out["rounds"]), actual_bytes=out["actual_bytes"],
                         size_error=(out["actual_bytes"] - budget) / budget,
                         ratio_rounds=[int(x) for x in out["ratio_rounds"]],
                         ratio_status=[int(x) for x in out["ratio_status"]])
    mgs.mgs_scene_destroy(scene)
    mgs.mgs_destroy(ctx)
    f = res["fixed"]
    print(json.dumps({"metric": "Alg. 1 with real compression: time to a calibrated configuration",
                      "value": f["ms"], "unit": "ms", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": f["ms"], "higher_is_better": False, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"calibrated search N={w.n}, 10 ratios x {len(w.bits)} widths, "
                                             f"G={w.group_size}, budget {budget:.0f} B, tolerance 5 %"},
                      "fixed_rate": f, "entropy_rate": res["entropy"]}))


def run_vq(args):
    """SH vector quantisation (Sec. III-D) at scene scale: 50 mini-batches of
    65536 of the 45 SH-rest coefficients of 5.27 M Gaussians against a
    4096-entry codebook, then the assignment of every vector."""
    import numpy as np
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    w = WORKLOAD
    attrs, _ = synth.make_scene(w.n, seed=w.seed)
    x = np.ascontiguousarray(attrs[:, 6:51])
    del attrs
    n, D = x.shape
    K, iters, batch = synth.VQ_K, synth.VQ_ITERS, synth.VQ_BATCH
    cb0 = x[synth.vq_init_rows(n, K, seed=1)]
    bt = synth.vq_batches(n, iters, batch, seed=2)
    ctx = mgs.mgs_create(0)
    st = torch.cuda.Stream(device=dev)
    xd = torch.from_numpy(x).to(dev)
    btd = torch.from_numpy(bt).to(dev)
    cb0d = torch.from_numpy(cb0).to(dev)
    cbd = torch.empty_like(cb0d)
    cnt = torch.empty(K, dtype=torch.int64, device=dev)
    idx = torch.empty(n, dtype=torch.int32, device=dev)
    times, train_ms, assign_ms = [], [], []
    launches0 = None
    for step in range(args.warmup + args.steps):
        with torch.cuda.stream(st):
            cbd.copy_(cb0d)
            cnt.zero_()
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            if step == args.warmup:
                launches0 = mgs.mgs_kernel_launches()
            e[0].record(st)
            mgs.mgs_vq_train(ctx, xd, cbd, cnt, btd, stream=st)
            e[1].record(st)
            mgs.mgs_vq_assign(ctx, xd, cbd, index_out=idx, stream=st)
            e[2].record(st)
            e[2].synchronize()
        if step >= args.warmup:
            times.append(e[0].elapsed_time(e[2]))
            train_ms.append(e[0].elapsed_time(e[1]))
            assign_ms.append(e[1].elapsed_time(e[2]))
    launches = (mgs.mgs_kernel_launches() - launches0) // args.steps
    ms = statistics.mean(times)
    evals = (iters * batch + n) * K                       # (vector, centre) scores
    ops = evals * (D + 1)                                 # D fmaf for the dot, one for the score
    peaks = measured_peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    alu_peak = n_sm * LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    a_ms = statistics.mean(assign_ms)
    vq_scores, vq_rescored = mgs.mgs_vq_stats(ctx)
    # the assignment is a contraction on the tensor cores (TF32): 2 D flops per
    # score, against the measured bf16 peak scaled by the nominal TF32/BF16
    # ratio (1.1 / 2.25 PFLOP/s dense)
    tf32_peak = peaks["bf16_tflops"] * 1.1 / 2.25
    tc_achieved = 2.0 * D * n * K / (a_ms * 1e-3) / 1e12
    cpu = None
    if not args.no_cpu:
        import oracle
        rows = np.random.default_rng(5).choice(n, 2000, replace=False)
        t0 = time.perf_counter()
        oracle.vq_assign(x[rows], cb0)
        dt = time.perf_counter() - t0
        cpu = {"value": 2000 * K / dt, "unit": "scores/s", "cores": 1, "kind": "oracle",
               "sample": f"oracle.vq_assign of 2000 of the vectors against the 4096 entries, {dt:.1f} s of one core"}
    mgs.mgs_destroy(ctx)
    print(json.dumps({"metric": "SH vector quantisation: vector-entry scores/s", "value": evals / (ms * 1e-3),
                      "unit": "scores/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"SH VQ N={n}, D={D}, K={K}, {iters} mini-batches of {batch}, "
                                             "then every vector assigned"},
                      "train_ms": statistics.mean(train_ms), "assign_ms": a_ms, "gpu_launches": int(launches),
                      "rescored_per_vector": vq_rescored / max(1, vq_scores // K),
                      "roofline": {"bound": "tensor", "achieved": tc_achieved, "peak": tf32_peak,
                                   "unit": "TFLOP/s", "frac": tc_achieved / tf32_peak, "traffic": None,
                                   "kernel": "k_vq_assign_tc", "flops_per_score": 2 * D,
                                   "peak_source": f"{peaks['source']} bf16 {peaks['bf16_tflops']} TFLOP/s x 1.1/2.25"},
                      "alu_issue_peak_tops": alu_peak,
                      "cpu_baseline": cpu}))


def run_solvers(args):
    """The 0-1 ILP of the scene-scale cost table at 40 MB three ways: the flat
    multiple-choice knapsack on the device and on the host (the same answer),
    and the paper's hierarchical solve (channel widths, then each channel's
    groups within its share of the budget).  Time, Omega and estimated size."""
    import torch
    from paper_2604_26799_gb300 import mgs
    dev = torch.device("cuda", 0)
    w = WORKLOAD
    a, imp = synth.make_scene(w.n, seed=w.seed)
    ctx = mgs.mgs_create(0)
    st = torch.cuda.Stream(device=dev)
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(a).to(dev), torch.from_numpy(imp).to(dev), stream=st)
    grid = mgs.Grid(w.keep(), list(w.bits), w.group_size)
    L = mgs.mgs_table_layout_for(w.n, a.shape[1], grid)
    tab = torch.empty(L.total_bytes, dtype=torch.uint8, device=dev)
    mgs.mgs_build_cost_table(ctx, scene, grid, tab, stream=st)
    st.synchronize()
    host = tab.cpu().numpy()
    opts = mgs.solve_opts()
    res = {}
    for name, fn in (("flat_device", lambda: mgs.mgs_solve_budgets_device(ctx, tab, L, grid, [w.budget_bytes], opts,
                                                                         stream=st)[0]),
                     ("flat_host", lambda: mgs.mgs_solve_budget(host, L, grid, w.budget_bytes, opts)),
                     ("hierarchical_host", lambda: mgs.mgs_solve_hierarchical(host, L, grid, w.budget_bytes, opts))):
        times, sol = [], None
        for step in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            sol = fn()
            if step >= args.warmup:
                times.append((time.perf_counter() - t0) * 1e3)
        res[name] = {"ms": statistics.median(times), "r_index": int(sol["r_index"]),
                     "objective": float(sol["objective"]), "est_bytes": float(sol["est_bytes"]),
                     "lp_bound": float(sol["lp_bound"])}
    mgs.mgs_scene_destroy(scene)
    mgs.mgs_destroy(ctx)
    f = res["flat_device"]
    print(json.dumps({"metric": "0-1 ILP at the budget: time to a configuration", "value": f["ms"], "unit": "ms",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": f["ms"],
                      "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": f"solvers on the scene-scale table (N={w.n}, 10 ratios x "
                                             f"{len(w.bits)} widths, G={w.group_size}), budget {w.budget_bytes:.0f} B"},
                      "solvers": res,
                      "hierarchical_objective_over_flat": res["hierarchical_host"]["objective"] / f["objective"]}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mgs", choices=["mgs", "reference"])
    ap.add_argument("--workload", default="scene", choices=["scene", "batch", "serve", "large", "preprocess", "raht", "raht_search",
                             "encode", "calibrated", "vq", "solvers"],
                    help="scene: the scene-scale search (default); batch: 16 uneven scenes in one "
                         "graph-replayed launch; serve: Poisson job stream through the server; "
                         "large: 6 M Gaussians x 20 ratios x 16 bit-widths; preprocess: Euler "
                         "replacement and view-independent importance of the scene-scale scene; "
                         "raht: RAHT of 10 channels of the scene-scale scene at depth 16; "
                         "raht_search: the search over RAHT AC tables for every ratio; "
                         "encode: the block coder on half the scene; calibrated: Alg. 1 with "
                         "real compression (the S_Delta loop) at 40 MB; vq: mini-batch k-means "
                         "of the SH coefficients and the assignment of every vector; solvers: the flat "
                         "0-1 ILP (device, host) against the hierarchical solve")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--slice-items", type=int, default=40_000,
                    help="serve: cost-table work items per batched launch")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-loop comparator")
    ap.add_argument("--no-autotune", action="store_true", help="use the default tile shape")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the large, batched and served sub-records of the default run")
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
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "preprocess":
        return run_preprocess(args)
    if args.workload == "raht":
        return run_raht(args)
    if args.workload == "raht_search":
        return run_raht_search(args)
    if args.workload == "encode":
        return run_encode(args)
    if args.workload == "calibrated":
        return run_calibrated(args)
    if args.workload == "vq":
        return run_vq(args)
    if args.workload == "solvers":
        return run_solvers(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
