"""C-ABI checks that need no GPU: the library loads and exports every entry
point of include/mgs.h; table layouts; the host budget solver against the
exact references in oracle/mckp.py."""
import os
import re

import numpy as np
import pytest

from oracle import mckp
from paper_2604_26799_gb300 import mgs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2604_26799_gb300 import build
    build.build()
    return mgs.lib()


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "mgs.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(mgs_[a-z_0-9]+)\s*\(", hdr)))


def test_exports_every_declared_symbol(L):
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), f"{name} declared in mgs.h but not exported"
    assert mgs.mgs_version().startswith("mgs")


def test_layout_matches_definition(L):
    keep = np.array([10, 4096, 5000, 8193], dtype=np.int64)
    g = mgs.Grid(keep, [2, 8, 16], 4096)
    lay = mgs.mgs_table_layout_for(10_000, 59, g)
    ng = [(k + 4095) // 4096 for k in keep]
    assert list(lay.n_groups[:4]) == ng
    assert lay.item_begin[0] == 0
    for r in range(4):
        assert lay.item_begin[r + 1] - lay.item_begin[r] == 59 * ng[r]
    assert lay.n_items == 59 * sum(ng)
    offs = [lay.off_sse, lay.off_l1, lay.off_hbits, lay.off_linf, lay.off_count, lay.off_vmin,
            lay.off_vmax, lay.total_bytes]
    assert all(o % 256 == 0 for o in offs) and offs == sorted(offs)
    assert lay.off_l1 - lay.off_sse >= 8 * lay.n_items * 3


@pytest.mark.parametrize("keep,bits,G", [
    ([0, 5], [4], 16),          # K = 0
    ([5, 5], [4], 16),          # not increasing
    ([5, 20], [4], 16),         # K > n
    ([5], [4, 4], 16),          # bits not increasing
    ([5], [0], 16),             # b = 0
    ([5], [17], 16),            # b > 16
    ([5], [4], 0),              # G = 0
    ([5], [4], 16385),          # G too large
])
def test_layout_rejects_bad_grids(L, keep, bits, G):
    with pytest.raises(mgs.MgsError) as e:
        mgs.mgs_table_layout_for(10, 59, mgs.Grid(keep, bits, G))
    assert e.value.status == -1


def synthetic_table(rng, keep, bits, G, C):
    """A host table with plausible values: SSE falls and entropy rises with b."""
    grid = mgs.Grid(keep, bits, G)
    n = int(max(keep))
    lay = mgs.mgs_table_layout_for(n, C, grid)
    buf = np.zeros(lay.total_bytes, dtype=np.uint8)
    v = mgs.table_views(buf, lay)
    ni, nb = int(lay.n_items), len(bits)
    for r in range(len(keep)):
        for c in range(C):
            for g in range(int(lay.n_groups[r])):
                it = int(lay.item_begin[r] + c * lay.n_groups[r] + g)
                v["cnt"][it] = min(G, int(keep[r]) - g * G)
    b = np.asarray(bits, dtype=np.float64)
    scale = rng.uniform(0.1, 10.0, size=(ni, 1))
    v["sse"][:] = scale * 4.0 ** (-b[None, :]) * v["cnt"][:, None] * rng.uniform(0.8, 1.2, (ni, nb))
    v["l1"][:] = np.sqrt(v["sse"])
    v["linf"][:] = np.sqrt(v["sse"]).astype(np.float32)
    ent = np.minimum(b[None, :], np.log2(np.maximum(v["cnt"][:, None], 2))) * v["cnt"][:, None]
    # entropy rates of a cost table are multiples of 2^-22 bits; the solver
    # works in those units
    v["hbits"][:] = np.round(ent * rng.uniform(0.5, 1.0, (ni, 1)) * 2.0 ** 22) / 2.0 ** 22
    return buf, lay, grid, v


def test_solver_against_exact_small(L):
    rng = np.random.default_rng(5)
    for trial in range(40):
        C = int(rng.integers(1, 3))
        G = int(rng.integers(3, 9))
        n_b = int(rng.integers(1, 4))
        bits = np.sort(rng.choice(np.arange(1, 12), size=n_b, replace=False))
        keep = np.array([int(rng.integers(1, 3 * G))], dtype=np.int64)
        buf, lay, grid, v = synthetic_table(rng, keep, bits, G, C)
        items = int(lay.n_items)
        if items > 6:
            continue
        for rate_model in (mgs.MGS_RATE_FIXED, mgs.MGS_RATE_ENTROPY):
            rates = mckp.item_rates(v, bits, "fixed" if rate_model else "entropy")
            dist = mckp.item_dist(v, "sse")
            lo = rates.min(axis=1).sum() / 8 + 9 * items
            hi = rates.max(axis=1).sum() / 8 + 9 * items
            budget = float(rng.uniform(lo - 2, hi + 2))
            sol = mgs.mgs_solve_budget(buf, lay, grid, budget, mgs.solve_opts(rate_model=rate_model))
            exact = mckp.solve_bruteforce(dist, rates, budget)
            if exact is None:
                assert sol["r_index"] == -1
                continue
            assert sol["r_index"] == 0
            ch = sol["choice"].astype(np.int64)
            est = mckp.assignment_bytes(rates, ch, 0.0)
            assert est <= budget + 1e-9
            assert abs(est - sol["est_bytes"]) <= 1e-9 * max(1.0, est)
            got = float(dist[np.arange(items), ch].sum())
            assert abs(got - sol["objective"]) <= 1e-9 * max(1.0, got)
            assert got >= exact[0] - 1e-9 * max(1.0, exact[0])
            assert sol["lp_bound"] <= exact[0] + 1e-9 * max(1.0, exact[0])
            step = np.max(dist.max(axis=1) - dist.min(axis=1))
            assert got <= sol["lp_bound"] + step + 1e-9
            assert mgs.mgs_estimate_size(buf, lay, grid, 0, ch, mgs.solve_opts(rate_model=rate_model)) \
                == pytest.approx(est, rel=1e-12)


def test_solver_tau_rule_and_scale(L):
    rng = np.random.default_rng(9)
    keep = np.array([200, 400, 800, 1600], dtype=np.int64)
    bits = [2, 4, 8, 12, 16]
    buf, lay, grid, v = synthetic_table(rng, keep, bits, 64, 7)
    for budget in (4e3, 1e4, 3e4, 1e5, 1e7):
        for rate_model in (0, 1):
            sol = mgs.mgs_solve_budget(buf, lay, grid, budget, mgs.solve_opts(rate_model=rate_model))
            per_r = []
            rates_all = mckp.item_rates(v, bits, "fixed" if rate_model else "entropy")
            for r in range(len(keep)):
                b0, b1 = int(lay.item_begin[r]), int(lay.item_begin[r + 1])
                rr = rates_all[b0:b1]
                bmin = rr.min(axis=1).sum() / 8 + 9 * (b1 - b0)
                btop = rr[:, -1].sum() / 8 + 9 * (b1 - b0)
                feas = bmin <= budget
                assert (sol["ratio_status"][r] == -1) == (not feas)
                per_r.append(dict(feasible=feas, objective=float(sol["ratio_objective"][r]),
                                  bytes_min=bmin, bytes_top=btop))
                if feas:
                    assert sol["ratio_bytes"][r] <= budget * (1 + 1e-12)
                    assert sol["ratio_lp_bound"][r] <= sol["ratio_objective"][r] * (1 + 1e-12) + 1e-12
            expect = mckp.choose_tau(per_r, budget)
            assert sol["r_index"] == (-1 if expect is None else expect)


def test_solve_budgets_equals_one_at_a_time(L):
    rng = np.random.default_rng(21)
    keep = np.array([300, 700, 1500], dtype=np.int64)
    bits = [2, 4, 6, 8, 12, 16]
    buf, lay, grid, v = synthetic_table(rng, keep, bits, 128, 5)
    budgets = [2e3, 5e3, 1.2e4, 3e4, 1e9]
    many = mgs.mgs_solve_budgets(buf, lay, grid, budgets, mgs.solve_opts())
    for b, m in zip(budgets, many):
        one = mgs.mgs_solve_budget(buf, lay, grid, b, mgs.solve_opts())
        assert one["r_index"] == m["r_index"]
        assert one["est_bytes"] == m["est_bytes"] and one["objective"] == m["objective"]
        assert np.array_equal(one["choice"], m["choice"])
