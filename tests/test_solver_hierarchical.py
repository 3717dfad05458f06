"""The hierarchical solve of Sec. III-F (channel widths first, then each
channel's groups within S_c = A Q_c / sum Q_c) on host tables: the same
answer as a step-by-step restatement built from the flat solver; equal to the
flat solve when there is one channel; feasible and never below the exact
optimum (brute force) or the flat LP bound; tau by the flat rule."""
import ctypes

import numpy as np
import pytest

from oracle import mckp
from paper_2604_26799_gb300 import mgs
from tests.test_abi_cpu import synthetic_table


@pytest.fixture(scope="module")
def L():
    from paper_2604_26799_gb300 import build
    build.build()
    return mgs.lib()


def norm_dist(v, it, k, norm):
    if norm == mgs.MGS_NORM_L2:
        return float(np.sqrt(v["sse"][it, k]))
    if norm == mgs.MGS_NORM_L1:
        return float(v["l1"][it, k])
    if norm == mgs.MGS_NORM_LINF:
        return float(v["linf"][it, k])
    return float(v["sse"][it, k])


def channel_view(lay, base, ng):
    lv = mgs.mgs_table_layout()
    ctypes.memmove(ctypes.addressof(lv), ctypes.addressof(lay), ctypes.sizeof(lay))
    nb = lay.n_bits
    lv.n_ratios, lv.n_channels, lv.n_items = 1, 1, ng
    lv.item_begin[0], lv.item_begin[1] = 0, ng
    lv.n_groups[0] = ng
    lv.off_sse += 8 * base * nb
    lv.off_l1 += 8 * base * nb
    lv.off_hbits += 8 * base * nb
    lv.off_linf += 4 * base * nb
    lv.off_count += 4 * base
    lv.off_vmin += 4 * base
    lv.off_vmax += 4 * base
    return lv


def restated(buf, lay, grid_bits, keep, G, budget, opts, r):
    """Steps (1)-(3) for ratio r with the flat solver on hand-built sub-tables."""
    v = mgs.table_views(buf, lay)
    C, nb = lay.n_channels, lay.n_bits
    ng, ib = int(lay.n_groups[r]), int(lay.item_begin[r])
    g1 = mgs.Grid(np.array([1], np.int64), grid_bits, 1)
    l1 = mgs.mgs_table_layout_for(1, C, g1)
    b1 = np.zeros(l1.total_bytes, np.uint8)
    v1 = mgs.table_views(b1, l1)
    for c in range(C):
        n_c = 0
        for g in range(ng):
            it = ib + c * ng + g
            n_c += int(v["cnt"][it])
            for k in range(nb):
                v1["sse"][c, k] += norm_dist(v, it, k, opts.norm)
                v1["hbits"][c, k] += v["hbits"][it, k]
        v1["cnt"][c] = n_c
    o1 = mgs.solve_opts(rate_model=opts.rate_model, norm=mgs.MGS_NORM_SSE, const_bytes=opts.const_bytes,
                        meta_bytes_per_group=opts.meta_bytes_per_group * ng, delta_bytes=opts.delta_bytes)
    s1 = mgs.mgs_solve_budgets(b1, l1, g1, [budget], o1)[0]
    if s1["r_index"] < 0:
        return None
    qc = [grid_bits[k] for k in s1["choice"]]
    A = budget - opts.const_bytes - opts.delta_bytes
    qsum = float(sum(qc))
    choice, obj, byt = [], 0.0, 0.0
    gv = mgs.Grid(np.array([keep[r]], np.int64), grid_bits, G)
    for c in range(C):
        lv = channel_view(lay, ib + c * ng, ng)
        o2 = mgs.solve_opts(rate_model=opts.rate_model, norm=opts.norm, const_bytes=0.0,
                            meta_bytes_per_group=opts.meta_bytes_per_group, delta_bytes=0.0)
        s2 = mgs.mgs_solve_budgets(buf, lv, gv, [A * qc[c] / qsum], o2)[0]
        if s2["r_index"] < 0:
            return None
        choice.append(s2["choice"])
        obj += s2["objective"]
        byt += s2["est_bytes"]
    return dict(choice=np.concatenate(choice), objective=obj, bytes=byt + opts.const_bytes + opts.delta_bytes)


@pytest.mark.parametrize("rate_model,norm", [(0, 0), (1, 0), (0, 1), (1, 3), (0, 2)])
def test_hierarchical_matches_restatement(L, rate_model, norm):
    rng = np.random.default_rng(10 + rate_model + 2 * norm)
    keep = np.array([900, 2000, 3100], dtype=np.int64)
    bits = [1, 2, 4, 6, 8, 12]
    G, C = 128, 5
    buf, lay, grid, _ = synthetic_table(rng, keep, bits, G, C)
    opts = mgs.solve_opts(rate_model=rate_model, norm=norm, const_bytes=300.0)
    top = mgs.mgs_solve_budgets(buf, lay, grid, [1e15], opts)[0]["ratio_bytes"].max()
    for frac in (0.15, 0.3, 0.6):
        budget = float(top * frac)
        got = mgs.mgs_solve_hierarchical(buf, lay, grid, budget, opts)
        for r in range(len(keep)):
            ref = restated(buf, lay, bits, keep, G, budget, opts, r)
            if ref is None:
                assert got["ratio_status"][r] == -1
                continue
            assert got["ratio_status"][r] in (0, 1)
            assert got["ratio_objective"][r] == ref["objective"]
            assert got["ratio_bytes"][r] == ref["bytes"]
            assert ref["bytes"] <= budget * (1 + 1e-12)
            if got["r_index"] == r:
                assert np.array_equal(got["choice"], ref["choice"])
        flat = mgs.mgs_solve_budgets(buf, lay, grid, [budget], opts)[0]
        for r in range(len(keep)):
            if got["ratio_status"][r] >= 0:
                assert got["ratio_objective"][r] >= flat["ratio_lp_bound"][r] * (1 - 1e-12)


def test_hierarchical_one_channel_is_flat(L):
    """C = 1: S_c = A, so step (3) is the flat problem itself."""
    rng = np.random.default_rng(2)
    keep = np.array([500, 1500], dtype=np.int64)
    bits = [2, 3, 5, 8]
    buf, lay, grid, _ = synthetic_table(rng, keep, bits, 64, 1)
    opts = mgs.solve_opts(const_bytes=50.0)
    top = mgs.mgs_solve_budgets(buf, lay, grid, [1e15], opts)[0]["ratio_bytes"].max()
    for frac in (0.2, 0.5, 0.9):
        h = mgs.mgs_solve_hierarchical(buf, lay, grid, float(top * frac), opts)
        f = mgs.mgs_solve_budgets(buf, lay, grid, [float(top * frac)], opts)[0]
        assert h["r_index"] == f["r_index"]
        assert np.array_equal(h["ratio_objective"], f["ratio_objective"])
        assert np.array_equal(h["choice"], f["choice"])


def test_hierarchical_not_below_exact(L):
    """Tiny tables: the hierarchical answer is a feasible assignment, so its
    loss is at least the brute-force optimum of the same ratio."""
    rng = np.random.default_rng(7)
    checked = 0
    for trial in range(60):
        C = int(rng.integers(2, 4))
        G = int(rng.integers(2, 5))
        bits = sorted(rng.choice(np.arange(1, 10), size=3, replace=False).tolist())
        keep = np.array([int(rng.integers(2, 2 * G + 1))], dtype=np.int64)
        buf, lay, grid, v = synthetic_table(rng, keep, bits, G, C)
        if int(lay.n_items) > 7:
            continue
        opts = mgs.solve_opts(rate_model=mgs.MGS_RATE_FIXED)           # 9 B of metadata per item
        rates = mckp.item_rates(v, bits, "fixed")
        dist = mckp.item_dist(v, "sse")
        items = int(lay.n_items)
        lo = rates.min(axis=1).sum() / 8 + 9 * items
        hi = rates.max(axis=1).sum() / 8 + 9 * items
        budget = float(lo + (hi - lo) * rng.uniform(0.2, 0.9))
        h = mgs.mgs_solve_hierarchical(buf, lay, grid, budget, opts)
        best = mckp.solve_bruteforce(dist, rates, budget)
        if h["r_index"] < 0:
            continue
        ch = h["choice"]
        assert mckp.assignment_bytes(rates, ch, 0.0) <= budget + 1e-9
        assert h["objective"] >= best[0] - 1e-9 * max(1.0, abs(best[0]))
        checked += 1
    assert checked >= 10


def test_hierarchical_errors(L):
    rng = np.random.default_rng(1)
    buf, lay, grid, _ = synthetic_table(rng, np.array([100], np.int64), [2, 4], 16, 2)
    with pytest.raises(mgs.MgsError):
        mgs.mgs_solve_hierarchical(buf, lay, grid, -1.0, mgs.solve_opts())
    res = mgs.mgs_solve_hierarchical(buf, lay, grid, 1.0, mgs.solve_opts())
    assert res["r_index"] == -1
