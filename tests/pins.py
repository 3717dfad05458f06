"""Pins of the CPU oracle: closed forms, library-routine reductions and
invariants of the group-wise quantiser (Sec. III-D), the entropy bound
(Sec. III-F "Size Estimator") and the Morton order (Sec. III-G).

Each check takes an oracle library handle so the same checks can be run
against deliberately broken copies of the oracle (tests/test_oracle_mutants.py)
to show that a plausible mistake fails at least one of them.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.stats import entropy as scipy_entropy

import oracle


def check_grid(L, b_data: int, b_q: int):
    """Data c_k = k / 2^b_data, k = 0..2^b_data (so min 0, max 1, range 1).

    With R = 1: S = 2^-b_q exactly, max/S = 2^b_q, Z = 0, and c/S = k * 2^(b_q - b_data)
    exactly, so the code is round-half-even(k * 2^(b_q - b_data)) clamped to 2^b_q - 1,
    the reconstruction is q * 2^-b_q and the error is exact in double.
    """
    n = (1 << b_data) + 1
    k = np.arange(n, dtype=np.float64)
    vals = (k / float(1 << b_data)).astype(np.float32)
    out = oracle.group_cost(vals, [b_q], want_codes=True, L=L)
    expect_q = np.minimum(np.rint(k * 2.0 ** (b_q - b_data)), (1 << b_q) - 1)
    assert np.array_equal(out["codes"][0].astype(np.int64), expect_q.astype(np.int64)), (b_data, b_q)
    err = expect_q / float(1 << b_q) - k / float(1 << b_data)
    assert math.isclose(out["sse"][0], float(np.sum(err * err)), rel_tol=1e-12, abs_tol=0.0)
    assert math.isclose(out["l1"][0], float(np.sum(np.abs(err))), rel_tol=1e-12)
    assert out["linf"][0] == np.float32(np.max(np.abs(err)))
    counts = np.bincount(expect_q.astype(np.int64))
    counts = counts[counts > 0]
    expect_h = n * scipy_entropy(counts, base=2)
    assert math.isclose(out["hbits"][0], expect_h, rel_tol=1e-10, abs_tol=1e-9)
    if b_q == b_data:
        # closed form: 2^b - 1 singletons and one pair -> n log2 n - 2 bits; SSE = 4^-b.
        assert math.isclose(out["hbits"][0], n * math.log2(n) - 2.0, rel_tol=1e-10)
        assert math.isclose(out["sse"][0], 4.0 ** (-b_q), rel_tol=1e-12)
    assert out["vmin"] == 0.0 and out["vmax"] == 1.0


def check_dyadic(L, j: int, off: int, b: int):
    """Data c_k = (k - off) / 2^j, k = 0..2^j: range 1, min -off/2^j, max (2^j - off)/2^j.

    Every FP32 operation of the quantiser is exact on these inputs (dyadic values with
    few bits), so the result must equal the paper's formula evaluated in exact rational
    arithmetic: S = R / 2^b, Z = round(2^b - max / S), q = round(clamp(c / S + Z)),
    c_hat = (q - Z) * S, with round = nearest, ties to even.
    """
    from fractions import Fraction as F
    n = (1 << j) + 1
    vals_q = [F(k - off, 1 << j) for k in range(n)]
    vals = np.array([float(v) for v in vals_q], dtype=np.float32)
    out = oracle.group_cost(vals, [b], want_codes=True, L=L)
    m, M = min(vals_q), max(vals_q)
    S = (M - m) / (1 << b)
    Z = round((1 << b) - M / S)
    top = (1 << b) - 1
    q = [round(min(max(v / S + Z, F(0)), F(top))) for v in vals_q]
    err = [(F(qk) - Z) * S - v for qk, v in zip(q, vals_q)]
    assert out["codes"][0].astype(np.int64).tolist() == q, (j, off, b)
    assert math.isclose(out["sse"][0], float(sum(e * e for e in err)), rel_tol=1e-12)
    assert math.isclose(out["l1"][0], float(sum(abs(e) for e in err)), rel_tol=1e-12)
    assert out["linf"][0] == np.float32(float(max(abs(e) for e in err)))
    counts = np.bincount(np.array(q))
    counts = counts[counts > 0]
    expect_h = n * scipy_entropy(counts, base=2) if counts.size > 1 else 0.0
    assert math.isclose(out["hbits"][0], expect_h, rel_tol=1e-10, abs_tol=1e-9)


def check_constant(L, value: float, n: int, bits):
    vals = np.full(n, value, dtype=np.float32)
    out = oracle.group_cost(vals, bits, want_codes=True, L=L)
    assert np.all(out["codes"] == 0)
    assert np.all(out["sse"] == 0.0) and np.all(out["l1"] == 0.0) and np.all(out["linf"] == 0.0)
    assert np.all(out["hbits"] == 0.0)
    assert out["vmin"] == np.float32(value) and out["vmax"] == np.float32(value)


def check_invariants(L, vals: np.ndarray, bits):
    """Properties that hold for any finite group."""
    vals = np.asarray(vals, dtype=np.float32)
    n = vals.shape[0]
    out = oracle.group_cost(vals, bits, want_codes=True, L=L)
    assert out["vmin"] == vals.min() and out["vmax"] == vals.max()
    order = np.argsort(vals, kind="stable")
    R = np.float32(vals.max()) - np.float32(vals.min())
    for k, b in enumerate(bits):
        q = out["codes"][k].astype(np.int64)
        assert q.min() >= 0 and q.max() <= (1 << b) - 1
        # monotone: a larger value never gets a smaller code
        assert np.all(np.diff(q[order]) >= 0)
        # entropy bound equals n * H(histogram of the codes) (library routine)
        counts = np.bincount(q)
        counts = counts[counts > 0]
        assert counts.sum() == n
        expect_h = n * scipy_entropy(counts, base=2) if counts.size > 1 else 0.0
        assert math.isclose(out["hbits"][k], expect_h, rel_tol=1e-10, abs_tol=1e-9)
        assert out["hbits"][k] <= n * min(b, math.log2(n)) + 1e-9
        S = float(R) / float(1 << b)
        if R > 0 and S > 1e-30:
            # the max lands at 2^b - 1, the min at 0: Z places the range on the code grid
            assert q[np.argmax(vals)] == (1 << b) - 1
            assert q[np.argmin(vals)] <= 1
            # every reconstruction lies within 1.5 steps (the top code within 1.5 S,
            # the rest within S/2, plus FP32 rounding of the arithmetic)
            slack = 1.5 * S + 4e-7 * float(max(abs(vals.min()), abs(vals.max())))
            assert float(out["linf"][k]) <= slack * (1 + 1e-6), (b, out["linf"][k], S)
        lin = float(out["linf"][k])
        assert out["sse"][k] <= n * lin * lin * (1 + 1e-12) + 1e-300
        assert out["l1"][k] <= n * lin * (1 + 1e-12) + 1e-300
        assert lin * lin <= out["sse"][k] * (1 + 1e-12) + 1e-300
        assert out["l1"][k] >= lin * (1 - 1e-12)


def check_uniform_noise(L, seed: int = 1):
    """Textbook: uniform data, step S -> mean squared error ~ S^2 / 12, mean |e| ~ S / 4.

    The top half-step above 2^b - 1 is clamped (S divides by 2^b); at b >= 8 that
    tail moves the means by under 5%.
    """
    rng = np.random.default_rng(seed)
    vals = rng.uniform(-3.0, 5.0, size=65536).astype(np.float32)
    for b in (8, 10, 12):
        out = oracle.group_cost(vals, [b], L=L)
        S = (float(vals.max()) - float(vals.min())) / (1 << b)
        mse = out["sse"][0] / vals.shape[0]
        assert 0.9 < mse / (S * S / 12.0) < 1.1, (b, mse, S)
        mae = out["l1"][0] / vals.shape[0]
        assert 0.9 < mae / (S / 4.0) < 1.1


def check_two_point(L, m: float, M: float, bits):
    vals = np.array([m, M, M, m, M], dtype=np.float32)
    out = oracle.group_cost(vals, bits, want_codes=True, L=L)
    for k, b in enumerate(bits):
        q = out["codes"][k]
        assert np.all(q[[1, 2, 4]] == (1 << b) - 1)
        assert np.all(q[[0, 3]] <= 1)


def spread_bits(v: np.ndarray) -> np.ndarray:
    """Spread the 21 low bits of v to every third bit (mask-and-shift method)."""
    x = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    x = (x | (x << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    x = (x | (x << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    x = (x | (x << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    x = (x | (x << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    x = (x | (x << np.uint64(2))) & np.uint64(0x1249249249249249)
    return x


def check_morton_lattice(L, seed: int = 3, n: int = 2000):
    """Positions on the 2^-21 lattice of [0, 1]: the axis code is the lattice index."""
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, 1 << 21, size=(n, 3)).astype(np.int64)
    idx[0] = 0
    idx[1] = (1 << 21) - 1
    pos = idx.astype(np.float64) / float(1 << 21)
    pos[1] = 1.0  # the max maps to t = 1 and is clamped to 2^21 - 1
    attrs = np.zeros((n, 5), dtype=np.float32)
    attrs[:, :3] = pos.astype(np.float32)
    attrs[:, 3:] = rng.standard_normal((n, 2)).astype(np.float32)
    # duplicates exercise the index tiebreak
    attrs[10] = attrs[20]
    idx[10] = idx[20]
    codes, order = oracle.morton(attrs, L=L)
    expect = (spread_bits(idx[:, 0]) | (spread_bits(idx[:, 1]) << np.uint64(1))
              | (spread_bits(idx[:, 2]) << np.uint64(2)))
    assert np.array_equal(codes, expect)
    expect_order = np.lexsort((np.arange(n), expect))
    assert np.array_equal(order, expect_order)


def check_rank(L, seed: int = 4, n: int = 5000):
    rng = np.random.default_rng(seed)
    imp = np.exp(rng.standard_normal(n)).astype(np.float32)
    imp[100:200] = imp[50]  # ties
    imp[300] = 0.0
    imp[301] = -0.0
    r = oracle.rank(imp, L=L)
    order = np.lexsort((np.arange(n), -imp.astype(np.float64)))
    expect = np.empty(n, dtype=np.int64)
    expect[order] = np.arange(n)
    assert np.array_equal(r.astype(np.int64), expect)


# ---- preprocessing (Sec. III-A view-independent importance, Sec. III-D Euler) ----

def quat_matrix(q) -> np.ndarray:
    """Textbook rotation matrix of a unit quaternion [w, x, y, z] (Hamilton convention)."""
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def euler_matrix(e) -> np.ndarray:
    """The decoder's rotation matrix from [phi, theta, psi] printed in Sec. III-D:
    R = Rz(psi) Ry(theta) Rx(phi), written entry by entry."""
    (sf, cf), (st, ct), (sp, cp) = [(math.sin(a), math.cos(a)) for a in e]
    return np.array([[ct * cp, -cf * sp + sf * st * cp, sf * sp + cf * st * cp],
                     [ct * sp, cf * cp + sf * st * sp, -sf * cp + cf * st * sp],
                     [-st, sf * ct, cf * ct]])


def check_euler_axes(L):
    """A rotation by a about one axis gives that angle alone."""
    for a in (-2.5, -0.7, 0.0, 0.3, 1.2, 3.0):
        h = a / 2
        assert np.allclose(oracle.euler([math.cos(h), math.sin(h), 0, 0], L=L), [a, 0, 0], atol=1e-12)
        assert np.allclose(oracle.euler([math.cos(h), 0, 0, math.sin(h)], L=L), [0, 0, a], atol=1e-12)
        if abs(a) < math.pi / 2:
            assert np.allclose(oracle.euler([math.cos(h), 0, math.sin(h), 0], L=L), [0, a, 0], atol=1e-12)


def check_euler_roundtrip(L, seed: int = 5, n: int = 400):
    """The decoder's matrix of the encoded angles is the quaternion's own rotation
    (away from gimbal lock), and q, -q and 3q give the same angles."""
    rng = np.random.default_rng(seed)
    done = 0
    while done < n:
        q = rng.standard_normal(4)
        e = oracle.euler(q, L=L)
        if abs(abs(e[1]) - math.pi / 2) < 1e-3:
            continue
        assert np.allclose(euler_matrix(e), quat_matrix(q), atol=1e-12), q
        assert np.allclose(oracle.euler(-q, L=L), e, atol=1e-12)
        assert np.allclose(oracle.euler(3.0 * q, L=L), e, atol=1e-12)
        assert -math.pi <= e[0] <= math.pi and -math.pi / 2 <= e[1] <= math.pi / 2
        done += 1


def pre_scene(n: int, seed: int):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, 59)).astype(np.float32)
    a[:, 52:55] = rng.normal(-4.0, 1.0, (n, 3)).astype(np.float32)
    imp = rng.lognormal(0.0, 1.0, n).astype(np.float32)
    return a, imp


def check_preprocess(L, seed: int = 6, n: int = 1000):
    """Channels pass through; V_q is numpy's lower 0.9-quantile of the volumes;
    beta = 0 leaves the importance unchanged; beta = 1 scales it by min(V / V_q, 1)."""
    a, imp = pre_scene(n, seed)
    out, ig0, vq = oracle.preprocess(a, imp, 0.0, L=L)
    assert np.array_equal(out[:, :55], a[:, :55])
    assert np.array_equal(ig0, imp)
    vol = np.exp(a[:, 52:55].astype(np.float64).sum(axis=1))
    assert vq == np.quantile(vol, 0.9, method="lower")
    _, ig1, _ = oracle.preprocess(a, imp, 1.0, L=L)
    expect = (imp.astype(np.float64) * np.minimum(vol / vq, 1.0)).astype(np.float32)
    assert np.allclose(ig1, expect, rtol=2e-7, atol=0)
    # the Gaussians at or above V_q keep their view-dependent score
    top = vol >= vq
    assert np.array_equal(ig1[top], imp[top]) and top.sum() == n - (9 * (n - 1)) // 10
    _, ig2, _ = oracle.preprocess(a, imp, 2.0, L=L)
    assert np.allclose(ig2, (imp * np.minimum(vol / vq, 1.0) ** 2).astype(np.float32), rtol=2e-7)
    for i in range(0, n, 97):
        assert np.allclose(out[i, 55:58], oracle.euler(a[i, 55:59], L=L).astype(np.float32), atol=0)


# ---- RAHT (Sec. III-D) ----

def check_raht_example(L):
    """Three voxels at depth 1, (0,0,0) = 1, (1,0,0) = 2, (0,1,0) = 4: the x-merge of
    the first two, then the y-merge of that node (weight 2) with the third."""
    a = np.zeros((3, 4), np.float32)
    a[:, :3] = [[0, 0, 0], [1, 0, 0], [0, 1, 0]]
    a[:, 3] = [1.0, 2.0, 4.0]
    dc, ac, V = oracle.raht(a, [3], 1, L=L)
    d1 = 3.0 / math.sqrt(2.0)
    assert V == 3
    assert math.isclose(ac[0, 0], 1.0 / math.sqrt(2.0), rel_tol=1e-14)
    assert math.isclose(ac[1, 0], (math.sqrt(2.0) * 4.0 - d1) / math.sqrt(3.0), rel_tol=1e-14)
    assert math.isclose(dc[0], 7.0 / math.sqrt(3.0), rel_tol=1e-14)


def check_raht_ranges(L, seed: int = 11, n: int = 2500):
    """The largest |value| under each AC's node: the hand example gives 2 for the
    first merge and 4 for the root; in general it is the largest |x| of the
    Gaussians in the voxels the node covers (a Morton-contiguous run of voxels,
    found here by brute force from the voxel codes), and every AC lies within
    sqrt(w) of it (DC^2 + AC^2 of a node is at most w times its largest |mean|^2)."""
    a = np.zeros((3, 4), np.float32)
    a[:, :3] = [[0, 0, 0], [1, 0, 0], [0, 1, 0]]
    a[:, 3] = [1.0, -2.0, 4.0]
    dc, ac, V, w, r = oracle.raht(a, [3], 1, L=L, weights=True, ranges=True)
    assert V == 3 and list(w) == [2, 3] and list(r[:, 0]) == [2.0, 4.0]
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, (n, 5)).astype(np.float32)
    a[:, 3:] = (rng.standard_normal((n, 2)) * rng.uniform(0.1, 10, (n, 1))).astype(np.float32)
    depth = 5
    dc, ac, V, w, r = oracle.raht(a, [3, 4], depth, L=L, weights=True, ranges=True)
    assert np.all(np.abs(ac) <= np.sqrt(w)[:, None] * r * (1 + 1e-12))
    codes, order = oracle.morton(a, L=L)
    vc = (codes[order] >> np.uint64(3 * (21 - depth))).astype(np.uint64)
    uniq = np.unique(vc)
    big = np.zeros((len(uniq), 2))
    np.maximum.at(big, np.searchsorted(uniq, vc), np.abs(a[order][:, 3:5].astype(np.float64)))
    # node of a merge at step s: voxels whose codes agree above bit s; its range is
    # the largest |x| over them.  The oracle lists ACs step by step in ascending code.
    expect = []
    for s_ in range(3 * depth):
        prefix = uniq >> np.uint64(s_ + 1)
        cur = uniq >> np.uint64(s_)
        for p in np.unique(prefix):
            sel = prefix == p
            if len(np.unique(cur[sel])) == 2:
                expect.append(big[sel].max(axis=0))
    assert np.array_equal(np.array(expect), r)


def voxel_means(attrs, channels, depth, L):
    """Voxel codes and FP64 means, from the Morton codes and numpy grouping."""
    codes, order = oracle.morton(attrs, L=L)
    vc = codes[order] >> np.uint64(3 * (21 - depth))
    uniq, start = np.unique(vc, return_index=True)
    vals = attrs[order][:, channels].astype(np.float64)
    counts = np.diff(np.append(start, len(vc)))
    means = np.add.reduceat(vals, start, axis=0) / counts[:, None]
    return uniq, means


def check_raht_orthonormal(L, seed: int = 8, n: int = 3000):
    """Leaf weights 1 make the transform orthonormal: the energy of the voxel
    means equals DC^2 + sum AC^2, and DC = sum / sqrt(V)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, (n, 6)).astype(np.float32)
    a[:, 3:] = rng.standard_normal((n, 3)).astype(np.float32)
    for depth in (3, 6, 10):
        dc, ac, V = oracle.raht(a, [3, 4, 5], depth, L=L)
        uniq, means = voxel_means(a, [3, 4, 5], depth, L)
        assert V == len(uniq) and ac.shape == (V - 1, 3)
        energy = (means ** 2).sum(axis=0)
        assert np.allclose(dc ** 2 + (ac ** 2).sum(axis=0), energy, rtol=1e-11, atol=0)
        assert np.allclose(dc, means.sum(axis=0) / math.sqrt(V), rtol=1e-12, atol=1e-12)


def check_raht_constant_and_dedup(L, seed: int = 9, n: int = 2000):
    """A constant channel has no AC energy; Gaussians sharing a voxel enter as their mean."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, (n, 5)).astype(np.float32)
    a[:, 3] = 2.5
    dc, ac, V = oracle.raht(a, [3], 7, L=L)
    assert np.all(np.abs(ac) < 1e-12) and math.isclose(dc[0], 2.5 * math.sqrt(V), rel_tol=1e-13)
    a[:, 4] = (rng.integers(-1000, 1000, n) / 64.0).astype(np.float32)   # dyadic: +1 is exact
    b = np.concatenate([a, a], axis=0)              # every Gaussian twice: same voxels
    b[n:, 4] += 1.0                                  # the copies differ by 1 in channel 4
    dc1, ac1, V1 = oracle.raht(a, [4], 7, L=L)
    dc2, ac2, V2 = oracle.raht(b, [4], 7, L=L)
    assert V1 == V2
    assert np.allclose(dc2, dc1 + 0.5 * math.sqrt(V1), rtol=1e-12)   # every mean moved by 0.5
    assert np.allclose(ac2, ac1, atol=1e-10)


def check_raht_keep(L, seed: int = 10, n: int = 3000, keep: int = 1200):
    """The RAHT of a kept set equals the RAHT of those Gaussians alone when they
    span the whole scene's bounding box (the bbox extremes are made the most
    important, so both use the same voxel grid)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(0, 1, (n, 5)).astype(np.float32)
    imp = rng.uniform(0, 1, n).astype(np.float32)
    ext = np.unique(np.concatenate([np.argmin(a[:, :3], axis=0), np.argmax(a[:, :3], axis=0)]))
    imp[ext] = 2.0 + np.arange(len(ext))
    dc, ac, V = oracle.raht(a, [3, 4], 9, L=L, importance=imp, keep=keep)
    top = np.sort(np.lexsort((np.arange(n), -imp))[:keep])     # the `keep` most important, index order
    dc2, ac2, V2 = oracle.raht(a[top], [3, 4], 9, L=L)
    assert V == V2 and np.array_equal(dc, dc2) and np.array_equal(ac, ac2)


# ---- block coder (actual size S_a of Alg. 1) ---------------------------------

RANS_L = 1 << 23


def read_block_py(buf: bytes, n: int):
    """Independent pure-Python reader of the block format (slow: small n).

    Returns (codes, b, min, max, bytes used, table) with table = {code: f}
    (None for raw or R = 0 blocks).  Every field is parsed from the format's
    definition: metadata, mode byte, gamma-coded table in LSB-first bit
    order, lane states, then the rANS bytes in decoding order.
    """
    import struct
    b = buf[0]
    mn, mx = struct.unpack("<ff", bytes(buf[1:9]))
    if np.float32(mx) - np.float32(mn) == np.float32(0.0):
        return [0] * n, b, mn, mx, 9, None
    mode = buf[9]
    bits = [(byte >> t) & 1 for byte in buf[10:] for t in range(8)]
    if mode == 0:
        codes = [sum(bits[i * b + j] << j for j in range(b)) for i in range(n)]
        return codes, b, mn, mx, 10 + (n * b + 7) // 8, None
    assert mode == 1, mode
    pos = 0

    def gamma():
        nonlocal pos
        zeros = 0
        while bits[pos] == 0:
            zeros += 1
            pos += 1
        v = 0
        for _ in range(zeros + 1):
            v = 2 * v + bits[pos]
            pos += 1
        return v

    table = {}
    sym = -1
    for _ in range(gamma()):
        sym += gamma()
        table[sym] = gamma()
    k = (n - 1).bit_length()
    M = 1 << k
    assert sum(table.values()) == M and max(table) < (1 << b)
    cum, run = {}, 0
    for s in sorted(table):
        cum[s] = run
        run += table[s]
    at = 10 + (pos + 7) // 8
    lanes = min(32, max(1, n // 512))
    x = []
    for j in range(lanes):
        x.append(int.from_bytes(bytes(buf[at:at + 4]), "little"))
        at += 4
    codes = []
    for i in range(n):
        j = i % lanes
        slot = x[j] % M
        s = next(s for s in table if cum[s] <= slot < cum[s] + table[s])
        codes.append(s)
        x[j] = table[s] * (x[j] // M) + slot - cum[s]
        while x[j] < RANS_L:
            x[j] = x[j] * 256 + buf[at]
            at += 1
    assert all(v == RANS_L for v in x), "final states are not L"
    return codes, b, mn, mx, at, table


def gamma_len(x: int) -> int:
    return 2 * (int(x).bit_length() - 1) + 1


def coder_cases(seed: int):
    """Blocks with the codes of real quantised groups (Laplacian, Gaussian and
    two-level data), a uniform block that must fall back to raw, and sizes
    around the lane and precision boundaries."""
    rng = np.random.default_rng(seed)
    for n in (2, 3, 100, 511, 512, 1000, 1024, 1537, 2048):
        for b in (1, 2, 3, 5, 8, 12, 16):
            kind = (n + b) % 3
            if kind == 0:
                v = rng.laplace(0.0, 0.05, n)
            elif kind == 1:
                v = rng.normal(-4.0, 1.0, n)
            else:
                v = rng.choice([-1.0, 0.25, 3.0], n, p=[0.7, 0.2, 0.1]) + rng.normal(0, 1e-3, n)
            out = oracle.group_cost(v.astype(np.float32), [b], want_codes=True)
            yield out["codes"][0], b, out["vmin"], out["vmax"]
    yield rng.integers(0, 1 << 16, 600).astype(np.uint16), 16, -1.0, 1.0


def check_coder_roundtrip(L, seed: int = 11):
    """Every block decodes, by the independent reader and by the oracle's own
    decoder, to the codes it was made from, and uses exactly its bytes."""
    saw_raw = saw_rans = False
    for codes, b, mn, mx in coder_cases(seed):
        n = codes.shape[0]
        blk = oracle.encode_block(codes, b, mn, mx, L=L)
        got, gb, gmn, gmx, used, table = read_block_py(blk, n)
        assert used == len(blk) and gb == b and np.float32(gmn) == np.float32(mn)
        assert np.array_equal(np.asarray(got, dtype=np.uint16), codes), (n, b)
        got2, _, _, _, used2 = oracle.decode_block(blk, n, L=L)
        assert used2 == len(blk) and np.array_equal(got2, codes)
        raw = 10 + (n * b + 7) // 8
        assert len(blk) <= raw
        if table is None:
            assert len(blk) == raw
            saw_raw = True
        else:
            saw_rans = True
    assert saw_raw and saw_rans
    const = oracle.encode_block(np.zeros(37, np.uint16), 7, 2.5, 2.5, L=L)
    assert len(const) == 9 and read_block_py(const, 37)[0] == [0] * 37


def check_coder_entropy(L, seed: int = 12):
    """With n a power of two the normalised frequencies are the counts, so the
    ideal code length of the static model is the entropy bound H of the cost
    table (n * -sum p log2 p).  rANS with states in [2^23, 2^31) and byte
    renormalisation then spends, over its lanes' states and bytes, between
    24 and 32 bits per lane above H, up to a rounding loss of at most
    -log2(1 - M / 2^23) bits per symbol; the table costs exactly the gamma
    code lengths of D, the gaps and the frequencies."""
    rng = np.random.default_rng(seed)
    for n in (1024, 4096, 16384):
        for b in (2, 4, 8, 12):
            v = rng.laplace(0.0, 0.05, n).astype(np.float32)
            out = oracle.group_cost(v, [b], want_codes=True)
            codes = out["codes"][0]
            blk = oracle.encode_block(codes, b, out["vmin"], out["vmax"], L=L)
            if blk[9] == 0:          # the table of a wide, short block outweighs its gain
                assert b >= 12 and n <= 4096, (n, b)
                continue
            counts = np.bincount(codes.astype(np.int64), minlength=1 << b)
            used = np.nonzero(counts)[0]
            tbits = gamma_len(len(used))
            prev = -1
            for s in used:
                tbits += gamma_len(int(s) - prev) + gamma_len(int(counts[s]))
                prev = int(s)
            lanes = min(32, max(1, n // 512))
            payload = 8 * (len(blk) - 10 - (tbits + 7) // 8)
            k = (n - 1).bit_length()
            eps = n * -math.log2(1.0 - 2.0 ** (k - 23)) + 1e-6
            over = payload - out["hbits"][0]
            assert 24 * lanes - eps < over <= 32 * lanes + eps, (n, b, over, lanes)


def check_coder_normalisation(L):
    """n not a power of two: f = floor(count M / n), the shortfall going to the
    most frequent code, the lowest one on ties; the table read back agrees."""
    rng = np.random.default_rng(13)
    for n in (600, 1000, 3000, 5000):
        codes = np.minimum(rng.geometric(0.05, n) - 1, 255).astype(np.uint16)
        codes[:2] = [0, 255]
        blk = oracle.encode_block(codes, 8, -1.0, 1.0, L=L)
        assert blk[9] == 1
        table = read_block_py(blk, n)[5]
        counts = np.bincount(codes.astype(np.int64), minlength=256)
        M = 1 << (n - 1).bit_length()
        expect = {int(s): int(counts[s]) * M // n for s in np.nonzero(counts)[0]}
        top = int(np.argmax(counts))
        expect[top] += M - sum(expect.values())
        assert table == expect, n
    # n = 707, M = 1024, counts 300, 300, 100, 7: floors 434, 434, 144, 10 sum to
    # 1022; codes 0 and 1 tie for the most frequent and the lower one takes the 2
    codes = np.array([0] * 300 + [1] * 300 + [2] * 100 + [3] * 7, dtype=np.uint16)
    blk = oracle.encode_block(codes, 2, 0.0, 1.0, L=L)
    assert blk[9] == 1
    assert read_block_py(blk, 707)[5] == {0: 436, 1: 434, 2: 144, 3: 10}


# ---- vector quantisation of the 1+D SH coefficients -------------------------

def vq_data(seed: int, n: int, K: int, D: int = 45, spread: float = 1.0, noise: float = 0.02):
    """K well-separated centres in [-spread, spread]^D and n vectors drawn
    around them (the source centre of each is returned too)."""
    rng = np.random.default_rng(seed)
    cent = rng.uniform(-spread, spread, size=(K, D)).astype(np.float32)
    src = rng.integers(0, K, size=n)
    x = (cent[src] + rng.normal(0, noise, size=(n, D))).astype(np.float32)
    return x, cent, src


def exact_argmin(x, cb):
    """FP64 squared distances: argmin and the gap to the runner-up."""
    d = ((x.astype(np.float64)[:, None, :] - cb.astype(np.float64)[None, :, :]) ** 2).sum(-1)
    order = np.argsort(d, axis=1, kind="stable")
    best = order[:, 0]
    rows = np.arange(x.shape[0])
    gap = d[rows, order[:, 1]] - d[rows, best] if cb.shape[0] > 1 else np.full(x.shape[0], np.inf)
    return best, gap, d


def check_vq_assign(L, seed: int = 14):
    """Vectors near well-separated centres go to their source centre; on
    random data the choice is the FP64 nearest centre wherever the FP64 gap to
    the runner-up exceeds the FP32 rounding of the scores; a duplicated centre
    never wins over its lower-index copy."""
    x, cent, src = vq_data(seed, 600, 64)
    idx, _ = oracle.vq_assign(x, cent, L=L)
    assert np.array_equal(idx, src)
    rng = np.random.default_rng(seed + 1)
    for K, D, scale in ((37, 45, 0.05), (200, 8, 1.0), (5, 3, 100.0)):
        x = rng.laplace(0, scale, size=(500, D)).astype(np.float32)
        cb = rng.laplace(0, scale, size=(K, D)).astype(np.float32)
        idx, score = oracle.vq_assign(x, cb, L=L)
        best, gap, d = exact_argmin(x, cb)
        xx = (x.astype(np.float64) ** 2).sum(1)
        cc = (cb.astype(np.float64) ** 2).sum(1)
        tol = 4 * D * 2.0 ** -24 * (xx[:, None] + cc[None, :]).max(1)
        ok = gap > 2 * tol
        assert np.array_equal(idx[ok], best[ok]), (K, D)
        rows = np.arange(x.shape[0])
        assert np.all(d[rows, idx] - d[rows, best] <= 2 * tol)          # near-ties: still near-optimal
        assert np.allclose(score.astype(np.float64) + xx, d[rows, idx], rtol=0, atol=tol.max())
    cb = cent[:10].copy()
    cb[7] = cb[3]                                                      # a duplicated centre
    xs = (cb[3] + 1e-3).reshape(1, -1).astype(np.float32)
    assert oracle.vq_assign(xs, cb, L=L)[0][0] == 3


def check_vq_update(L, seed: int = 15):
    """From zero counts one batch moves each centre to the mean of its batch
    vectors (centres with none stay); a second batch gives the running mean of
    both (the per-vector update with rate 1/count, carried out in FP64); a
    whole-data batch from zero counts is one Lloyd step (scipy's kmeans2)."""
    from scipy.cluster.vq import kmeans2
    x, cent, _ = vq_data(seed, 3000, 40, D=12, noise=0.3)
    rng = np.random.default_rng(seed)
    init = cent + rng.normal(0, 0.1, cent.shape).astype(np.float32)
    init[39] = 50.0                                                    # never the nearest: stays
    b1 = rng.choice(x.shape[0], 700, replace=False).astype(np.int32)
    b2 = rng.choice(x.shape[0], 900, replace=False).astype(np.int32)
    cb1, cnt1, a1 = oracle.vq_train(x, init, b1[None, :], L=L)
    assert cnt1.sum() == 700 and np.array_equal(cnt1, np.bincount(a1[0], minlength=40))
    assert np.array_equal(cb1[39], init[39]) and cnt1[39] == 0
    for k in np.nonzero(cnt1)[0]:
        mean = x[b1[a1[0] == k]].astype(np.float64).mean(0)
        assert np.allclose(cb1[k], mean, rtol=2.5e-7, atol=1e-7), k
    cb2, cnt2, a2 = oracle.vq_train(x, cb1, b2[None, :], counts=cnt1, L=L)
    # the literal per-vector update (Sculley): v += 1, eta = 1 / v, c += eta (x - c), in FP64
    c = cb1.astype(np.float64)
    v = cnt1.astype(np.float64)
    for j, row in enumerate(b2):
        k = a2[0][j]
        v[k] += 1
        c[k] += (x[row].astype(np.float64) - c[k]) / v[k]
    assert np.array_equal(cnt2, v.astype(np.int64))
    assert np.allclose(cb2, c, rtol=1e-6, atol=1e-7)
    # Lloyd: batch = every vector, counts zero
    allr = np.arange(x.shape[0], dtype=np.int32)[None, :]
    cbl, _, al = oracle.vq_train(x, init, allr, L=L)
    import warnings
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        ref_cb, ref_lab = kmeans2(x.astype(np.float64), init.astype(np.float64), iter=1, minit="matrix",
                                  missing="warn")
    assert np.array_equal(al[0], ref_lab)
    assert np.allclose(cbl, ref_cb, rtol=1e-6, atol=1e-7)
