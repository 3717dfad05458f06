"""CPU oracle for the MesonGS++ cost table and budget solve.

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg.  The product path (the package and its CUDA
library) never imports it, and it imports nothing from the product.

  oracle.c   C reference of the quantiser, entropy bound, Morton order, ranks,
             of the preprocessing (importance I_g, Euler angles), RAHT, the
             block coder that gives a configuration's actual size, and the
             vector quantisation of the SH coefficients (assignment, mini-batch
             k-means)
             (compiled with gcc -O2 -ffp-contract=off, no fast-math)
  mckp.py    exact references of the 0-1 ILP (brute force, DP) and the tau rule
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NONFINITE, ERR_RANGE, ERR_NOMEM = 0, -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (plain gcc, strict FP)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-ffp-contract=off", "-fno-fast-math",
           "-fexcess-precision=standard", "-Wall", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def load(path: str):
    """Load an oracle shared library from `path` and declare its signatures."""
    L = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32 = ctypes.c_int64, ctypes.c_int32
    L.oracle_rank.argtypes = [P, i64, P]
    L.oracle_morton.argtypes = [P, i64, i32, P, P]
    L.oracle_kept.argtypes = [P, P, i64, i64, P]
    L.oracle_kept.restype = i64
    L.oracle_group_cost.argtypes = [P, i64, P, i32, P, P, P, P, P, P, P]
    L.oracle_cost_table.argtypes = [P, P, i64, i32, P, i32, P, i32, i32, P, P, P, P, P, P, P]
    L.oracle_cost_table_mt.argtypes = [P, P, i64, i32, P, i32, P, i32, i32, P, P, P, P, P, P, P, i32]
    L.oracle_quantize.argtypes = [P, P, i64, i32, i64, i32, P, P, P]
    L.oracle_euler.argtypes = [P, P]
    L.oracle_euler.restype = None
    L.oracle_preprocess.argtypes = [P, i64, i32, P, ctypes.c_double, P, P, P]
    L.oracle_raht.argtypes = [P, i64, i32, P, i32, i32, P, i64, P, P, P, P, P]
    L.oracle_rans_lanes.argtypes = [i64]
    L.oracle_rans_lanes.restype = i32
    L.oracle_block_bound.argtypes = [i64, i32]
    L.oracle_block_bound.restype = i64
    L.oracle_encode_block.argtypes = [P, i64, i32, ctypes.c_float, ctypes.c_float, P, i64]
    L.oracle_encode_block.restype = i64
    L.oracle_decode_block.argtypes = [P, i64, i64, P, P, P, P]
    L.oracle_decode_block.restype = i64
    L.oracle_encode_config.argtypes = [P, P, i64, i32, i64, i32, P, P, i64, P]
    L.oracle_encode_config.restype = i64
    L.oracle_vq_assign.argtypes = [P, i64, i32, P, i32, P, P]
    L.oracle_vq_update.argtypes = [P, i64, i32, P, i32, P, P, i32, P]
    for f in (L.oracle_vq_assign, L.oracle_vq_update):
        f.restype = ctypes.c_int
    for f in (L.oracle_rank, L.oracle_morton, L.oracle_group_cost, L.oracle_cost_table, L.oracle_cost_table_mt,
              L.oracle_quantize, L.oracle_preprocess, L.oracle_raht):
        f.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load(build())
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class OracleError(RuntimeError):
    def __init__(self, code: int):
        super().__init__(f"oracle status {code}")
        self.code = code


def _check(rc: int):
    if rc != OK:
        raise OracleError(rc)


def rank(importance: np.ndarray, L=None) -> np.ndarray:
    imp = np.ascontiguousarray(importance, dtype=np.float32)
    out = np.empty(imp.shape[0], dtype=np.int32)
    _check((L or lib()).oracle_rank(_p(imp), imp.shape[0], _p(out)))
    return out


def morton(attrs: np.ndarray, L=None) -> tuple[np.ndarray, np.ndarray]:
    """Return (codes[i] uint64, order[p] int64) for attrs [n, C] (channels 0..2 = position)."""
    a = np.ascontiguousarray(attrs, dtype=np.float32)
    n, C = a.shape
    codes = np.empty(n, dtype=np.uint64)
    order = np.empty(n, dtype=np.int64)
    _check((L or lib()).oracle_morton(_p(a), n, C, _p(codes), _p(order)))
    return codes, order


def kept(rank_: np.ndarray, order: np.ndarray, keep: int) -> np.ndarray:
    r = np.ascontiguousarray(rank_, dtype=np.int32)
    o = np.ascontiguousarray(order, dtype=np.int64)
    out = np.empty(max(int(keep), 1), dtype=np.int64)
    k = lib().oracle_kept(_p(r), _p(o), o.shape[0], int(keep), _p(out))
    return out[:k]


def group_cost(vals: np.ndarray, bits, want_codes: bool = False, L=None) -> dict:
    v = np.ascontiguousarray(vals, dtype=np.float32)
    b = np.ascontiguousarray(bits, dtype=np.int32)
    nb = b.shape[0]
    out = dict(sse=np.empty(nb), l1=np.empty(nb), linf=np.empty(nb, dtype=np.float32),
               hbits=np.empty(nb), vmin=np.empty(1, dtype=np.float32),
               vmax=np.empty(1, dtype=np.float32))
    codes = np.empty((nb, v.shape[0]), dtype=np.uint16) if want_codes else None
    _check((L or lib()).oracle_group_cost(_p(v), v.shape[0], _p(b), nb, _p(out["sse"]), _p(out["l1"]),
                                   _p(out["linf"]), _p(out["hbits"]), _p(out["vmin"]),
                                   _p(out["vmax"]), _p(codes) if codes is not None else None))
    out["vmin"] = float(out["vmin"][0])
    out["vmax"] = float(out["vmax"][0])
    if codes is not None:
        out["codes"] = codes
    return out


def n_groups(keep: int, G: int) -> int:
    return (int(keep) + G - 1) // G


def cost_table(attrs, importance, keep, bits, G, threads: int = 1) -> dict:
    """Whole table, items ordered [r][c][g]; per-option arrays shaped [n_items, n_b].
    threads > 1 spreads the independent items over that many threads (same entries)."""
    a = np.ascontiguousarray(attrs, dtype=np.float32)
    imp = np.ascontiguousarray(importance, dtype=np.float32)
    k = np.ascontiguousarray(keep, dtype=np.int64)
    b = np.ascontiguousarray(bits, dtype=np.int32)
    n, C = a.shape
    n_items = sum(C * n_groups(x, G) for x in k)
    nb = b.shape[0]
    out = dict(sse=np.empty((n_items, nb)), l1=np.empty((n_items, nb)),
               linf=np.empty((n_items, nb), dtype=np.float32), hbits=np.empty((n_items, nb)),
               cnt=np.empty(n_items, dtype=np.int32), vmin=np.empty(n_items, dtype=np.float32),
               vmax=np.empty(n_items, dtype=np.float32))
    args = (_p(a), _p(imp), n, C, _p(k), k.shape[0], _p(b), nb, int(G), _p(out["sse"]), _p(out["l1"]),
            _p(out["linf"]), _p(out["hbits"]), _p(out["cnt"]), _p(out["vmin"]), _p(out["vmax"]))
    if threads > 1:
        _check(lib().oracle_cost_table_mt(*args, int(threads)))
    else:
        _check(lib().oracle_cost_table(*args))
    return out


def quantize(attrs, importance, keep: int, G: int, q_bits: np.ndarray):
    """Codes [C, keep] uint16 and min/max [C, n_groups, 2] for one chosen configuration."""
    a = np.ascontiguousarray(attrs, dtype=np.float32)
    imp = np.ascontiguousarray(importance, dtype=np.float32)
    n, C = a.shape
    ng = n_groups(keep, G)
    qb = np.ascontiguousarray(q_bits, dtype=np.uint8).reshape(C, ng)
    codes = np.empty((C, max(int(keep), 1)), dtype=np.uint16)
    mm = np.empty((C, max(ng, 1), 2), dtype=np.float32)
    _check(lib().oracle_quantize(_p(a), _p(imp), n, C, int(keep), int(G), _p(qb), _p(codes),
                                 _p(mm)))
    return codes[:, :keep], mm[:, :ng]


def euler(q, L=None) -> np.ndarray:
    """Euler angles [phi, theta, psi] (FP64) of the quaternion q = [w, x, y, z]."""
    qq = np.ascontiguousarray(q, dtype=np.float64).reshape(4)
    e = np.empty(3)
    (L or lib()).oracle_euler(_p(qq), _p(e))
    return e


def preprocess(attrs, view_importance, beta: float, L=None):
    """(attrs [n, 58] FP32 with Euler angles, I_g [n] FP32, V_q) for attrs [n, 59]."""
    a = np.ascontiguousarray(attrs, dtype=np.float32)
    imp = np.ascontiguousarray(view_importance, dtype=np.float32)
    n, C = a.shape
    out = np.empty((n, C - 1), dtype=np.float32)
    ig = np.empty(n, dtype=np.float32)
    vq = np.empty(1)
    _check((L or lib()).oracle_preprocess(_p(a), n, C, _p(imp), float(beta), _p(out), _p(ig), _p(vq)))
    return out, ig, float(vq[0])


def raht(attrs, channels, depth: int, L=None, weights: bool = False, importance=None, keep: int = 0,
         ranges: bool = False):
    """(DC [n_c], AC [V - 1, n_c], V) of the RAHT of `channels` at octree depth `depth`
    (FP64); with weights=True also the merge weight w1 + w2 of every AC, and with
    ranges=True (after the weights) the largest |value| of a Gaussian under each AC's
    merged node [V - 1, n_c].  keep > 0 transforms the kept set of the `keep` most
    important Gaussians only."""
    a = np.ascontiguousarray(attrs, dtype=np.float32)
    imp = None if importance is None else np.ascontiguousarray(importance, dtype=np.float32)
    ch = np.ascontiguousarray(channels, dtype=np.int32)
    n, C = a.shape
    dc = np.empty(ch.shape[0])
    ac = np.empty((max(n - 1, 1), ch.shape[0]))
    aw = np.empty(max(n - 1, 1), dtype=np.int64)
    ar = np.empty((max(n - 1, 1), ch.shape[0])) if ranges else None
    nv = np.empty(1, dtype=np.int64)
    _check((L or lib()).oracle_raht(_p(a), n, C, _p(ch), ch.shape[0], int(depth),
                                    _p(imp) if imp is not None else None, int(keep), _p(dc), _p(ac), _p(aw),
                                    _p(ar) if ranges else None, _p(nv)))
    V = int(nv[0])
    out = (dc, ac[:V - 1], V)
    if weights:
        out += (aw[:V - 1],)
    if ranges:
        out += (ar[:V - 1],)
    return out


def rans_lanes(n: int, L=None) -> int:
    return int((L or lib()).oracle_rans_lanes(int(n)))


def encode_block(codes, b: int, mn: float, mx: float, L=None) -> bytes:
    """One (channel, group) block of codes in the block format (oracle.c)."""
    L = L or lib()
    c = np.ascontiguousarray(codes, dtype=np.uint16)
    cap = int(L.oracle_block_bound(c.shape[0], int(b)))
    out = np.zeros(cap, dtype=np.uint8)
    sz = L.oracle_encode_block(_p(c), c.shape[0], int(b), float(mn), float(mx), _p(out), cap)
    if sz < 0:
        raise OracleError(int(sz))
    return out[:sz].tobytes()


def decode_block(buf: bytes, n: int, L=None):
    """Inverse of encode_block: (codes, b, min, max, bytes consumed)."""
    L = L or lib()
    a = np.frombuffer(bytes(buf) + b"\0", dtype=np.uint8)
    codes = np.zeros(max(int(n), 1), dtype=np.uint16)
    b = ctypes.c_int32()
    mn, mx = ctypes.c_float(), ctypes.c_float()
    used = L.oracle_decode_block(_p(a), len(buf), int(n), _p(codes), ctypes.byref(b),
                                 ctypes.byref(mn), ctypes.byref(mx))
    if used < 0:
        raise OracleError(int(used))
    return codes[:n], b.value, mn.value, mx.value, int(used)


def encode_config(attrs, importance, keep: int, G: int, q_bits: np.ndarray, L=None):
    """Quantise one configuration and encode every (channel, group) block in
    (c, g) order: (stream bytes, block sizes [C][n_groups])."""
    L = L or lib()
    a = np.ascontiguousarray(attrs, dtype=np.float32)
    imp = np.ascontiguousarray(importance, dtype=np.float32)
    n, C = a.shape
    ng = n_groups(keep, G)
    qb = np.ascontiguousarray(q_bits, dtype=np.uint8).reshape(C, ng)
    cap = 0
    for g in range(ng):
        ln = min(G, keep - g * G)
        cap += int(sum(L.oracle_block_bound(ln, int(qb[c, g])) for c in range(C)))
    out = np.zeros(max(cap, 1), dtype=np.uint8)
    sizes = np.zeros((C, ng), dtype=np.int64)
    tot = L.oracle_encode_config(_p(a), _p(imp), n, C, int(keep), int(G), _p(qb), _p(out), cap,
                                 _p(sizes))
    if tot < 0:
        raise OracleError(int(tot))
    return out[:tot].tobytes(), sizes


def vq_assign(x, codebook, L=None):
    """Nearest codebook entry per row of x [n, D]: (index int32 [n], score f32 [n])."""
    L = L or lib()
    xa = np.ascontiguousarray(x, dtype=np.float32)
    cb = np.ascontiguousarray(codebook, dtype=np.float32)
    n, D = xa.shape
    idx = np.empty(max(n, 1), dtype=np.int32)
    sc = np.empty(max(n, 1), dtype=np.float32)
    _check(L.oracle_vq_assign(_p(xa), n, D, _p(cb), cb.shape[0], _p(idx), _p(sc)))
    return idx[:n], sc[:n]


def vq_train(x, codebook, batches, counts=None, L=None):
    """Mini-batch k-means: one update per row of `batches` [iters, b] (row indices
    into x).  Returns (codebook, counts, assignments [iters, b])."""
    L = L or lib()
    xa = np.ascontiguousarray(x, dtype=np.float32)
    cb = np.array(codebook, dtype=np.float32, copy=True, order="C")
    K, D = cb.shape
    cnt = np.zeros(K, dtype=np.int64) if counts is None else np.array(counts, dtype=np.int64, copy=True)
    bt = np.ascontiguousarray(batches, dtype=np.int32).reshape(-1, np.shape(batches)[-1])
    asg = np.empty(bt.shape, dtype=np.int32)
    for t in range(bt.shape[0]):
        row = np.ascontiguousarray(bt[t])
        out = np.empty(max(row.shape[0], 1), dtype=np.int32)
        _check(L.oracle_vq_update(_p(xa), xa.shape[0], D, _p(cb), K, _p(cnt), _p(row), row.shape[0],
                                  _p(out)))
        asg[t] = out[:row.shape[0]]
    return cb, cnt, asg
