"""Thin ctypes binding of include/mgs.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device
buffers are torch tensors (their data_ptr is passed); host buffers are numpy
arrays or torch CPU tensors.  Nothing here computes any step of the method:
it all runs in libmgs.so, and importing this module fails loudly when the
library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libmgs.so")

MGS_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NONFINITE", -3: "RANGE", -4: "OUT_OF_MEMORY", -5: "CUDA",
          -6: "INFEASIBLE", -7: "TIMEOUT", -8: "BUSY"}
MGS_MAX_RATIOS = 64
MGS_MAX_OPTIONS = 16
MGS_RATE_ENTROPY, MGS_RATE_FIXED = 0, 1
MGS_NORM_SSE, MGS_NORM_L2, MGS_NORM_L1, MGS_NORM_LINF = 0, 1, 2, 3


class MgsError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{ERRORS.get(status, status)}: {message}")
        self.status = status


class mgs_grid(ctypes.Structure):
    _fields_ = [("n_ratios", ctypes.c_int32), ("keep", ctypes.POINTER(ctypes.c_int64)),
                ("n_bits", ctypes.c_int32), ("bits", ctypes.POINTER(ctypes.c_int32)),
                ("group_size", ctypes.c_int32)]


class mgs_table_layout(ctypes.Structure):
    _fields_ = [("n_items", ctypes.c_int64), ("n_bits", ctypes.c_int32),
                ("n_ratios", ctypes.c_int32), ("n_channels", ctypes.c_int32),
                ("group_size", ctypes.c_int32),
                ("item_begin", ctypes.c_int64 * (MGS_MAX_RATIOS + 1)),
                ("n_groups", ctypes.c_int64 * MGS_MAX_RATIOS),
                ("off_sse", ctypes.c_int64), ("off_l1", ctypes.c_int64),
                ("off_hbits", ctypes.c_int64), ("off_linf", ctypes.c_int64),
                ("off_count", ctypes.c_int64), ("off_vmin", ctypes.c_int64),
                ("off_vmax", ctypes.c_int64), ("total_bytes", ctypes.c_int64)]


class mgs_solve_opts(ctypes.Structure):
    _fields_ = [("rate_model", ctypes.c_int32), ("norm", ctypes.c_int32),
                ("const_bytes", ctypes.c_double), ("meta_bytes_per_group", ctypes.c_double),
                ("delta_bytes", ctypes.c_double)]


class mgs_solution(ctypes.Structure):
    _fields_ = [("r_index", ctypes.c_int32), ("est_bytes", ctypes.c_double),
                ("objective", ctypes.c_double), ("lp_bound", ctypes.c_double),
                ("choice", ctypes.c_void_p), ("ratio_status", ctypes.c_void_p),
                ("ratio_objective", ctypes.c_void_p), ("ratio_bytes", ctypes.c_void_p),
                ("ratio_lp_bound", ctypes.c_void_p)]


class mgs_calib_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_double), ("tolerance", ctypes.c_double),
                ("max_rounds", ctypes.c_int32), ("init_bits", ctypes.c_int32),
                ("solve", mgs_solve_opts)]


class mgs_calib_result(ctypes.Structure):
    _fields_ = [("r_index", ctypes.c_int32), ("rounds", ctypes.c_int32),
                ("actual_bytes", ctypes.c_double), ("est_bytes", ctypes.c_double),
                ("objective", ctypes.c_double), ("bits", ctypes.c_void_p),
                ("ratio_status", ctypes.c_void_p), ("ratio_rounds", ctypes.c_void_p),
                ("ratio_actual", ctypes.c_void_p), ("ratio_delta", ctypes.c_void_p),
                ("ratio_objective", ctypes.c_void_p)]


class mgs_server_opts(ctypes.Structure):
    _fields_ = [("max_jobs", ctypes.c_int32), ("solver_threads", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("slice_items", ctypes.c_int64)]


class mgs_job(ctypes.Structure):
    _fields_ = [("attrs", ctypes.c_void_p), ("importance", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("n_channels", ctypes.c_int32), ("grid", mgs_grid), ("budget_bytes", ctypes.c_double),
                ("opts", mgs_solve_opts), ("table_out", ctypes.c_void_p)]


class mgs_job_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("r_index", ctypes.c_int32), ("est_bytes", ctypes.c_double),
                ("objective", ctypes.c_double), ("lp_bound", ctypes.c_double), ("n_choice", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_ready", ctypes.c_double),
                ("t_table", ctypes.c_double), ("t_done", ctypes.c_double)]


_lib = None

# name -> argtypes (all return mgs_status unless listed in _RESTYPE)
_P = ctypes.c_void_p
_SIGS = {
    "mgs_create": [ctypes.c_int32, ctypes.POINTER(_P)],
    "mgs_destroy": [_P],
    "mgs_last_error": [],
    "mgs_version": [],
    "mgs_kernel_launches": [],
    "mgs_scene_create": [_P, _P, _P, ctypes.c_int64, ctypes.c_int32, _P, ctypes.POINTER(_P)],
    "mgs_scene_destroy": [_P],
    "mgs_scene_info": [_P, _P, _P, _P],
    "mgs_scene_morton": [_P, _P, _P, _P],
    "mgs_table_layout_for": [ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(mgs_grid),
                             ctypes.POINTER(mgs_table_layout)],
    "mgs_build_cost_table": [_P, _P, ctypes.POINTER(mgs_grid), _P, _P],
    "mgs_build_cost_table_plain": [_P, _P, ctypes.POINTER(mgs_grid), _P, _P],
    "mgs_debug_fail_allocation": [ctypes.c_int64],
    "mgs_debug_allocations": [],
    "mgs_debug_cost_plan": [ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_int32],
    "mgs_vq_set_wait_limit": [_P, ctypes.c_int64],
    "mgs_build_cost_table_probe": [_P, _P, ctypes.POINTER(mgs_grid), _P, _P, ctypes.c_int64, _P,
                                   ctypes.c_int64, _P],
    "mgs_build_cost_tables_batched": [_P, ctypes.c_int32, _P, _P, _P, _P],
    "mgs_quantize_groups": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P],
    "mgs_quantize_groups_noalloc": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P],
    "mgs_plan_create": [_P, ctypes.c_int32, _P, _P, _P, ctypes.c_int32, _P, ctypes.POINTER(_P)],
    "mgs_plan_launch": [_P, _P],
    "mgs_plan_destroy": [_P],
    "mgs_plan_info": [_P, _P, _P, _P],
    "mgs_tile_config_count": [],
    "mgs_server_create": [_P, ctypes.POINTER(mgs_server_opts), ctypes.POINTER(_P)],
    "mgs_server_submit": [_P, ctypes.POINTER(mgs_job), ctypes.POINTER(ctypes.c_int64)],
    "mgs_server_wait": [_P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(mgs_job_result), _P,
                        ctypes.c_int64],
    "mgs_server_stats": [_P, _P, _P, _P, _P],
    "mgs_server_destroy": [_P],
    "mgs_tile_config_name": [ctypes.c_int32],
    "mgs_set_tile_config": [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32],
    "mgs_autotune": [_P, _P, ctypes.POINTER(mgs_grid), _P, _P, _P],
    "mgs_estimate_size": [_P, ctypes.POINTER(mgs_table_layout), ctypes.POINTER(mgs_grid),
                          ctypes.c_int32, _P, ctypes.POINTER(mgs_solve_opts),
                          ctypes.POINTER(ctypes.c_double)],
    "mgs_solve_budget": [_P, ctypes.POINTER(mgs_table_layout), ctypes.POINTER(mgs_grid),
                         ctypes.c_double, ctypes.POINTER(mgs_solve_opts),
                         ctypes.POINTER(mgs_solution)],
    "mgs_solve_budgets": [_P, ctypes.POINTER(mgs_table_layout), ctypes.POINTER(mgs_grid),
                          ctypes.c_int32, _P, ctypes.POINTER(mgs_solve_opts), _P],
    "mgs_solve_hierarchical": [_P, ctypes.POINTER(mgs_table_layout), ctypes.POINTER(mgs_grid),
                               ctypes.c_double, ctypes.POINTER(mgs_solve_opts), _P],
    "mgs_build_cost_table_coeffs": [_P, _P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(mgs_grid), _P, _P],
    "mgs_raht": [_P, _P, _P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _P, _P, _P, _P],
    "mgs_preprocess": [_P, _P, _P, ctypes.c_int64, ctypes.c_double, _P, _P, _P, _P],
    "mgs_encode_config": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P, ctypes.c_int64, _P, _P, _P],
    "mgs_encode_bound": [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32],
    "mgs_vq_assign": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P],
    "mgs_vq_train": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, ctypes.c_int32,
                     ctypes.c_int32, _P, _P],
    "mgs_vq_retain": [_P, _P, ctypes.c_int64, ctypes.c_int32, _P, _P],
    "mgs_vq_set_tensor_cores": [_P, ctypes.c_int32],
    "mgs_vq_stats": [_P, _P, _P],
    "mgs_search_calibrated": [_P, _P, ctypes.POINTER(mgs_grid), _P, ctypes.POINTER(mgs_table_layout),
                              ctypes.POINTER(mgs_calib_opts), ctypes.POINTER(mgs_calib_result), _P],
    "mgs_solve_budgets_device": [_P, _P, ctypes.POINTER(mgs_table_layout), ctypes.POINTER(mgs_grid),
                                 ctypes.c_int32, _P, ctypes.POINTER(mgs_solve_opts), _P, _P],
}
_RESTYPE = {"mgs_last_error": ctypes.c_char_p, "mgs_version": ctypes.c_char_p,
            "mgs_tile_config_name": ctypes.c_char_p, "mgs_tile_config_count": ctypes.c_int32,
            "mgs_kernel_launches": ctypes.c_int64, "mgs_debug_allocations": ctypes.c_int64, "mgs_encode_bound": ctypes.c_int64}


def lib():
    """Load libmgs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, ctypes.c_int32)
        _lib = L
    return _lib


def _check(status: int):
    if status != MGS_OK:
        raise MgsError(status, lib().mgs_last_error().decode(errors="replace"))


def _ptr(x) -> int | None:
    """Address of a torch tensor or numpy array (None for None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Grid:
    """Keeps the ctypes arrays of an mgs_grid alive."""

    def __init__(self, keep, bits, group_size: int):
        self.keep = np.ascontiguousarray(keep, dtype=np.int64)
        self.bits = np.ascontiguousarray(bits, dtype=np.int32)
        self.group_size = int(group_size)
        self.c = mgs_grid(len(self.keep), self.keep.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          len(self.bits), self.bits.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          self.group_size)


def mgs_version() -> str:
    return lib().mgs_version().decode()


def mgs_debug_fail_allocation(nth: int):
    """Make the nth device allocation from now on fail (0 disarms); tests only."""
    _check(lib().mgs_debug_fail_allocation(int(nth)))


def mgs_debug_allocations() -> int:
    return int(lib().mgs_debug_allocations())


def mgs_debug_cost_plan(config: int, bits) -> dict:
    """The cost kernel's histogram plan for a tile configuration and bit-widths
    (host only; tests of the planner)."""
    b = np.ascontiguousarray(bits, dtype=np.int32)
    n = lib().mgs_debug_cost_plan(int(config), b.shape[0], b.ctypes.data, None, 0)
    if n < 0:
        raise MgsError(-1, lib().mgs_last_error().decode(errors="replace"))
    out = np.zeros(n, dtype=np.int32)
    lib().mgs_debug_cost_plan(int(config), b.shape[0], b.ctypes.data, out.ctypes.data, n)
    k = b.shape[0]
    per = out[9:9 + 5 * k].reshape(k, 5)
    units = out[9 + 5 * k:].reshape(-1, 3)
    return dict(smem=int(out[0]), budget=int(out[1]), concurrent=bool(out[2]), a_words=int(out[3]),
                b_words=int(out[4]), n_small=int(out[5]), n_lane=int(out[6]), n_direct=int(out[7]),
                mode=per[:, 0], off=per[:, 1], words=per[:, 2], windows=per[:, 3], rwindows=per[:, 4],
                units=units)


def mgs_vq_set_wait_limit(ctx: int, cycles: int):
    _check(lib().mgs_vq_set_wait_limit(ctx, int(cycles)))


def mgs_kernel_launches() -> int:
    return lib().mgs_kernel_launches()


def mgs_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().mgs_create(device, ctypes.byref(h)))
    return h.value


def mgs_destroy(ctx: int):
    _check(lib().mgs_destroy(ctx))


def mgs_scene_create(ctx: int, attrs, importance, stream=None) -> int:
    n, C = attrs.shape
    h = ctypes.c_void_p()
    _check(lib().mgs_scene_create(ctx, _ptr(attrs), _ptr(importance), n, C, _stream(stream),
                                  ctypes.byref(h)))
    return h.value


def mgs_scene_destroy(scene: int):
    _check(lib().mgs_scene_destroy(scene))


def mgs_scene_info(scene: int) -> tuple[int, int, int]:
    n, c, b = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().mgs_scene_info(scene, ctypes.addressof(n), ctypes.addressof(c), ctypes.addressof(b)))
    return n.value, c.value, b.value


def mgs_scene_morton(scene: int, codes=None, order=None, stream=None):
    _check(lib().mgs_scene_morton(scene, _ptr(codes), _ptr(order), _stream(stream)))


def mgs_table_layout_for(n: int, n_channels: int, grid: Grid) -> mgs_table_layout:
    L = mgs_table_layout()
    _check(lib().mgs_table_layout_for(n, n_channels, ctypes.byref(grid.c), ctypes.byref(L)))
    return L


def mgs_build_cost_table(ctx: int, scene: int, grid: Grid, table, stream=None):
    _check(lib().mgs_build_cost_table(ctx, scene, ctypes.byref(grid.c), _ptr(table), _stream(stream)))


def mgs_build_cost_table_plain(ctx: int, scene: int, grid: Grid, table, stream=None):
    _check(lib().mgs_build_cost_table_plain(ctx, scene, ctypes.byref(grid.c), _ptr(table),
                                            _stream(stream)))


def mgs_build_cost_table_probe(ctx: int, scene: int, grid: Grid, table, hist=None, codes=None,
                               stream=None):
    """The fused table plus what its kernel counted: hist (device uint32 /
    int32 tensor, [n_items][sum 2^b]) and codes (device int16 tensor), either may
    be None.  Layouts as in include/mgs.h."""
    def entries(x):
        return 0 if x is None else int(x.numel() if hasattr(x, "numel") else x.size)

    hc, cc = entries(hist), entries(codes)
    _check(lib().mgs_build_cost_table_probe(ctx, scene, ctypes.byref(grid.c), _ptr(table), _ptr(hist), hc,
                                            _ptr(codes), cc, _stream(stream)))


def _grids(grids, n):
    """One Grid, or a list of Grids (one per scene), as a C array of mgs_grid."""
    if isinstance(grids, Grid):
        grids = [grids] * n
    arr = (mgs_grid * n)(*[g.c for g in grids])
    return arr, grids   # keep the Grid objects (and their arrays) alive


def mgs_build_cost_tables_batched(ctx: int, scenes: list[int], grids, tables: list, stream=None):
    sc = (ctypes.c_void_p * len(scenes))(*scenes)
    tb = (ctypes.c_void_p * len(tables))(*[_ptr(t) for t in tables])
    ga, _keep = _grids(grids, len(scenes))
    _check(lib().mgs_build_cost_tables_batched(ctx, len(scenes), sc, ctypes.addressof(ga), tb,
                                               _stream(stream)))


def mgs_quantize_groups(ctx: int, scene: int, keep: int, group_size: int, bits, codes, minmax,
                        stream=None):
    _check(lib().mgs_quantize_groups(ctx, scene, keep, group_size, _ptr(bits), _ptr(codes),
                                     _ptr(minmax), _stream(stream)))


def mgs_encode_bound(keep: int, group_size: int, n_channels: int) -> int:
    return int(lib().mgs_encode_bound(int(keep), int(group_size), int(n_channels)))


def mgs_encode_config(ctx: int, scene: int, keep: int, group_size: int, bits, stream_out=None,
                      block_bytes=None, stream=None) -> int:
    """Encode one configuration (bits [C, n_groups] uint8, host or device) into
    stream_out (a device uint8 tensor, or None to measure only); block_bytes
    (int32 [C, n_groups], host or device) receives each block's size.
    Returns the stream's length in bytes."""
    total = ctypes.c_int64()
    cap = 0 if stream_out is None else int(stream_out.numel())
    _check(lib().mgs_encode_config(ctx, scene, int(keep), int(group_size), _ptr(bits),
                                   _ptr(stream_out), cap, _ptr(block_bytes),
                                   ctypes.addressof(total), _stream(stream)))
    return total.value


def mgs_vq_assign(ctx: int, x, codebook, index_out=None, score_out=None, stream=None):
    """Nearest codebook entry of each row of x [n, D] (device tensors).
    Returns (index int32 [n], score or None)."""
    import torch
    n, D = x.shape
    if index_out is None:
        index_out = torch.empty(n, dtype=torch.int32, device=x.device)
    _check(lib().mgs_vq_assign(ctx, _ptr(x), n, D, _ptr(codebook), codebook.shape[0], _ptr(index_out),
                               _ptr(score_out), _stream(stream)))
    return index_out, score_out


def mgs_vq_train(ctx: int, x, codebook, counts, batches, assign_out=None, stream=None):
    """Mini-batch k-means over the rows of x: one update per row of `batches`
    [iters, batch] (device int32).  codebook [K, D] and counts [K] (int64) are
    updated in place."""
    n, D = x.shape
    iters, b = batches.shape
    _check(lib().mgs_vq_train(ctx, _ptr(x), n, D, _ptr(codebook), codebook.shape[0], _ptr(counts),
                              _ptr(batches), iters, b, _ptr(assign_out), _stream(stream)))


def mgs_vq_set_tensor_cores(ctx: int, enable: bool):
    """Score on the tensor cores with exact re-scoring (default) or on the CUDA cores."""
    _check(lib().mgs_vq_set_tensor_cores(ctx, int(bool(enable))))


def mgs_vq_stats(ctx: int) -> tuple[int, int]:
    """(scores, exactly re-scored entries) of the tensor path since the last call."""
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().mgs_vq_stats(ctx, ctypes.addressof(a), ctypes.addressof(b)))
    return a.value, b.value


def mgs_vq_retain(ctx: int, rows, K: int, index, stream=None):
    _check(lib().mgs_vq_retain(ctx, _ptr(rows), int(rows.shape[0]), int(K), _ptr(index), _stream(stream)))


def mgs_plan_create(ctx: int, scenes: list[int], grids, tables: list, use_graph: bool = False,
                    stream=None) -> int:
    sc = (ctypes.c_void_p * len(scenes))(*scenes)
    tb = (ctypes.c_void_p * len(tables))(*[_ptr(t) for t in tables])
    ga, _keep = _grids(grids, len(scenes))
    h = ctypes.c_void_p()
    _check(lib().mgs_plan_create(ctx, len(scenes), sc, ctypes.addressof(ga), tb, int(use_graph),
                                 _stream(stream), ctypes.byref(h)))
    return h.value


def mgs_plan_launch(plan: int, stream=None):
    _check(lib().mgs_plan_launch(plan, _stream(stream)))


def mgs_plan_destroy(plan: int):
    _check(lib().mgs_plan_destroy(plan))


def mgs_plan_info(plan: int) -> tuple[int, int, int]:
    w, l, c = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(lib().mgs_plan_info(plan, ctypes.addressof(w), ctypes.addressof(l), ctypes.addressof(c)))
    return w.value, l.value, c.value


def mgs_tile_config_count() -> int:
    return lib().mgs_tile_config_count()


def mgs_tile_config_name(i: int) -> str:
    return lib().mgs_tile_config_name(i).decode()


def mgs_set_tile_config(ctx: int, group_size: int, n_bits: int, config: int):
    _check(lib().mgs_set_tile_config(ctx, group_size, n_bits, config))


def mgs_autotune(ctx: int, scene: int, grid: Grid, stream=None) -> tuple[int, np.ndarray]:
    chosen = ctypes.c_int32(-1)
    ms = np.full(mgs_tile_config_count(), -1.0, dtype=np.float32)
    _check(lib().mgs_autotune(ctx, scene, ctypes.byref(grid.c), _stream(stream),
                              ctypes.addressof(chosen), ms.ctypes.data))
    return chosen.value, ms


def mgs_quantize_groups_noalloc(ctx: int, scene: int, keep: int, group_size: int, bits, codes,
                                minmax, stream=None):
    """mgs_quantize_groups for callers that cannot allocate device memory (static scratch)."""
    _check(lib().mgs_quantize_groups_noalloc(ctx, scene, keep, group_size, _ptr(bits), _ptr(codes),
                                             _ptr(minmax), _stream(stream)))


def mgs_server_create(ctx: int, max_jobs: int = 8, solver_threads: int = 4,
                      hbm_budget_bytes: int = 64 << 30, slice_items: int = 20000) -> int:
    h = ctypes.c_void_p()
    o = mgs_server_opts(max_jobs, solver_threads, hbm_budget_bytes, slice_items)
    _check(lib().mgs_server_create(ctx, ctypes.byref(o), ctypes.byref(h)))
    return h.value


def mgs_server_submit(server: int, attrs, importance, grid: Grid, budget_bytes: float, opts,
                      table_out=None) -> int:
    """attrs / importance (and table_out, a host buffer of the table layout's
    total_bytes, if given): host buffers that stay alive until the job is done."""
    n, C = attrs.shape
    j = mgs_job(_ptr(attrs), _ptr(importance), n, C, grid.c, float(budget_bytes), opts, _ptr(table_out))
    jid = ctypes.c_int64()
    _check(lib().mgs_server_submit(server, ctypes.byref(j), ctypes.byref(jid)))
    return jid.value


def mgs_server_wait(server: int, job_id: int, timeout_ms: int = 60000, max_choice: int = 0) -> dict:
    r = mgs_job_result()
    ch = np.zeros(max(max_choice, 1), dtype=np.uint8)
    _check(lib().mgs_server_wait(server, job_id, timeout_ms, ctypes.byref(r), ch.ctypes.data,
                                 max_choice))
    out = {k: getattr(r, k) for k, _ in mgs_job_result._fields_}
    out["choice"] = ch[:min(max_choice, r.n_choice)].copy()
    if r.status != MGS_OK:
        out["error"] = lib().mgs_last_error().decode(errors="replace")
    return out


def mgs_server_stats(server: int) -> dict:
    a, b, c, d = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().mgs_server_stats(server, ctypes.addressof(a), ctypes.addressof(b),
                                  ctypes.addressof(c), ctypes.addressof(d)))
    return dict(launches=a.value, work_items=b.value, in_flight=c.value, used_bytes=d.value)


def mgs_server_destroy(server: int):
    _check(lib().mgs_server_destroy(server))


def solve_opts(rate_model: int = MGS_RATE_ENTROPY, norm: int = MGS_NORM_SSE,
               const_bytes: float = 0.0, meta_bytes_per_group: float = 9.0,
               delta_bytes: float = 0.0) -> mgs_solve_opts:
    return mgs_solve_opts(rate_model, norm, const_bytes, meta_bytes_per_group, delta_bytes)


def mgs_estimate_size(table_host, layout: mgs_table_layout, grid: Grid, r_index: int, choice,
                      opts: mgs_solve_opts) -> float:
    out = ctypes.c_double()
    ch = np.ascontiguousarray(choice, dtype=np.uint8)
    _check(lib().mgs_estimate_size(_ptr(table_host), ctypes.byref(layout), ctypes.byref(grid.c),
                                   r_index, ch.ctypes.data, ctypes.byref(opts), ctypes.byref(out)))
    return out.value


def mgs_solve_budget(table_host, layout: mgs_table_layout, grid: Grid, budget_bytes: float,
                     opts: mgs_solve_opts) -> dict:
    nr = layout.n_ratios
    max_items = max(int(layout.item_begin[r + 1] - layout.item_begin[r]) for r in range(nr))
    choice = np.zeros(max(max_items, 1), dtype=np.uint8)
    st = np.zeros(nr, dtype=np.int32)
    obj = np.zeros(nr)
    byt = np.zeros(nr)
    lp = np.zeros(nr)
    sol = mgs_solution(-1, 0.0, 0.0, 0.0, choice.ctypes.data, st.ctypes.data, obj.ctypes.data,
                       byt.ctypes.data, lp.ctypes.data)
    rc = lib().mgs_solve_budget(_ptr(table_host), ctypes.byref(layout), ctypes.byref(grid.c),
                                float(budget_bytes), ctypes.byref(opts), ctypes.byref(sol))
    if rc not in (MGS_OK, -6):
        _check(rc)
    r = sol.r_index
    n_items = int(layout.item_begin[r + 1] - layout.item_begin[r]) if r >= 0 else 0
    return dict(status=rc, r_index=r, est_bytes=sol.est_bytes, objective=sol.objective,
                lp_bound=sol.lp_bound, choice=choice[:n_items].copy(), ratio_status=st,
                ratio_objective=obj, ratio_bytes=byt, ratio_lp_bound=lp)


def mgs_solve_budgets(table_host, layout: mgs_table_layout, grid: Grid, budgets, opts) -> list[dict]:
    """One solution per budget; the item hulls are shared."""
    return _solve_many(lambda *a: lib().mgs_solve_budgets(_ptr(table_host), *a), layout, grid, budgets, opts)


def mgs_solve_hierarchical(table_host, layout: mgs_table_layout, grid: "Grid", budget_bytes: float,
                           opts: mgs_solve_opts) -> dict:
    """The hierarchical (channel, then group) solve of Sec. III-F on a host table."""
    return _solve_many(lambda lay, g, nb, bud, o, sols: lib().mgs_solve_hierarchical(
        _ptr(table_host), lay, g, ctypes.c_double.from_address(bud).value, o, sols),
        layout, grid, [budget_bytes], opts)[0]


def mgs_solve_budgets_device(ctx: int, table, layout: mgs_table_layout, grid: Grid, budgets, opts,
                             stream=None) -> list[dict]:
    """mgs_solve_budgets computed on the device; `table` may be a device tensor or host array."""
    return _solve_many(lambda *a: lib().mgs_solve_budgets_device(ctx, _ptr(table), *a, _stream(stream)),
                       layout, grid, budgets, opts)


def mgs_search_calibrated(ctx: int, scene: int, grid: "Grid", table, layout: mgs_table_layout,
                          budget_bytes: float, tolerance: float = 0.05, max_rounds: int = 8,
                          init_bits: int = 8, opts: mgs_solve_opts | None = None,
                          stream=None) -> dict:
    """Alg. 1 with real compression (see mgs.h).  `table` is the scene's device
    cost table for `grid`.  The default estimator is Eq. (eq:size_estim)'s
    linear sum P Q (MGS_RATE_FIXED).  Returns the chosen ratio, its widths
    [C, n_groups] and the per-ratio record; r_index is -1 when no ratio
    converged."""
    if opts is None:
        opts = solve_opts(rate_model=MGS_RATE_FIXED)
    nr = layout.n_ratios
    C = layout.n_channels
    max_items = max(int(layout.item_begin[r + 1] - layout.item_begin[r]) for r in range(nr))
    bits = np.zeros(max(max_items, 1), dtype=np.uint8)
    st = np.zeros(nr, dtype=np.int32)
    rounds = np.zeros(nr, dtype=np.int32)
    act, dl, ob = np.zeros(nr), np.zeros(nr), np.zeros(nr)
    res = mgs_calib_result(-1, 0, 0.0, 0.0, 0.0, bits.ctypes.data, st.ctypes.data, rounds.ctypes.data,
                           act.ctypes.data, dl.ctypes.data, ob.ctypes.data)
    co = mgs_calib_opts(float(budget_bytes), float(tolerance), int(max_rounds), int(init_bits), opts)
    rc = lib().mgs_search_calibrated(ctx, scene, ctypes.byref(grid.c), _ptr(table), ctypes.byref(layout),
                                     ctypes.byref(co), ctypes.byref(res), _stream(stream))
    if rc not in (MGS_OK, -6):
        _check(rc)
    r = res.r_index
    ng = int(layout.n_groups[r]) if r >= 0 else 0
    return dict(r_index=r, rounds=res.rounds, actual_bytes=res.actual_bytes, est_bytes=res.est_bytes,
                objective=res.objective, bits=bits[:C * ng].reshape(C, ng).copy() if r >= 0 else None,
                ratio_status=st, ratio_rounds=rounds, ratio_actual=act, ratio_delta=dl,
                ratio_objective=ob)


def _solve_many(call, layout: mgs_table_layout, grid: Grid, budgets, opts) -> list[dict]:
    nb = len(budgets)
    nr = layout.n_ratios
    max_items = max(int(layout.item_begin[r + 1] - layout.item_begin[r]) for r in range(nr))
    bud = np.ascontiguousarray(budgets, dtype=np.float64)
    keep = []
    sols = (mgs_solution * nb)()
    for i in range(nb):
        arrs = (np.zeros(max(max_items, 1), dtype=np.uint8), np.zeros(nr, dtype=np.int32),
                np.zeros(nr), np.zeros(nr), np.zeros(nr))
        keep.append(arrs)
        sols[i] = mgs_solution(-1, 0.0, 0.0, 0.0, *[a.ctypes.data for a in arrs])
    rc = call(ctypes.byref(layout), ctypes.byref(grid.c), nb, bud.ctypes.data, ctypes.byref(opts),
              ctypes.addressof(sols))
    if rc not in (MGS_OK, -6):
        _check(rc)
    out = []
    for i in range(nb):
        r = sols[i].r_index
        n_items = int(layout.item_begin[r + 1] - layout.item_begin[r]) if r >= 0 else 0
        ch, st, ob, by, lp = keep[i]
        out.append(dict(r_index=r, est_bytes=sols[i].est_bytes, objective=sols[i].objective,
                        lp_bound=sols[i].lp_bound, choice=ch[:n_items].copy(), ratio_status=st,
                        ratio_objective=ob, ratio_bytes=by, ratio_lp_bound=lp))
    return out


def table_views(buf, layout: mgs_table_layout) -> dict:
    """Typed views of a table buffer (torch uint8 tensor or numpy uint8 array)."""
    ni, nb = int(layout.n_items), int(layout.n_bits)

    def view(off, count, dtype, shape):
        if isinstance(buf, np.ndarray):
            return buf[off:off + count * np.dtype(dtype).itemsize].view(dtype).reshape(shape)
        import torch
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32}[dtype]
        return buf[off:off + count * np.dtype(dtype).itemsize].view(tdt).reshape(shape)

    return dict(sse=view(layout.off_sse, ni * nb, np.float64, (ni, nb)),
                l1=view(layout.off_l1, ni * nb, np.float64, (ni, nb)),
                hbits=view(layout.off_hbits, ni * nb, np.float64, (ni, nb)),
                linf=view(layout.off_linf, ni * nb, np.float32, (ni, nb)),
                cnt=view(layout.off_count, ni, np.int32, (ni,)),
                vmin=view(layout.off_vmin, ni, np.float32, (ni,)),
                vmax=view(layout.off_vmax, ni, np.float32, (ni,)))


def mgs_preprocess(ctx: int, attrs, view_importance, beta: float, attrs_out=None, importance_out=None,
                   stream=None):
    """Euler replacement and importance I_g = I_d * V_norm^beta on the device.

    attrs: [n, 59] float32 device tensor; returns (attrs_out [n, 58], importance_out [n], V_q)."""
    import torch
    n = int(attrs.shape[0])
    if attrs_out is None:
        attrs_out = torch.empty((n, 58), dtype=torch.float32, device=attrs.device)
    if importance_out is None:
        importance_out = torch.empty(n, dtype=torch.float32, device=attrs.device)
    vq = ctypes.c_float()
    _check(lib().mgs_preprocess(ctx, _ptr(attrs), _ptr(view_importance), n, float(beta), _ptr(attrs_out),
                                _ptr(importance_out), ctypes.byref(vq), _stream(stream)))
    return attrs_out, importance_out, vq.value


def mgs_raht(ctx: int, scene: int, channels, depth: int, ac_out=None, stream=None, keep: int = 0):
    """RAHT of a resident scene's channels (keep > 0: of the `keep` most important Gaussians):
    (DC [n_c] numpy, AC [V - 1, n_c] device tensor, V)."""
    import torch
    n, _, _ = mgs_scene_info(scene)
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    nc = int(ch.shape[0])
    if ac_out is None:
        ac_out = torch.empty((max(n - 1, 1), nc), dtype=torch.float32, device="cuda")
    dc = np.empty(nc, dtype=np.float32)
    nv = ctypes.c_int64()
    _check(lib().mgs_raht(ctx, scene, ch.ctypes.data, nc, int(depth), int(keep), dc.ctypes.data, _ptr(ac_out),
                          ctypes.byref(nv), _stream(stream)))
    return dc, ac_out[:nv.value - 1], nv.value


def mgs_build_cost_table_coeffs(ctx: int, coeffs, grid: "Grid", table, stream=None):
    """Cost table of a [m, n_channels] float32 device array, groups in array order."""
    m, nc = int(coeffs.shape[0]), int(coeffs.shape[1])
    _check(lib().mgs_build_cost_table_coeffs(ctx, _ptr(coeffs), m, nc, ctypes.byref(grid.c), _ptr(table),
                                             _stream(stream)))
