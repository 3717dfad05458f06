"""The device budget solve (Eq. (eq:ilp), Sec. III-F "Binary ILP for Q")
against the exact references of oracle/mckp.py, not against the host solver:

* tiny instances (at most 8 items) against brute-force enumeration, for both
  rate models: the device answer is feasible, never better than the optimum,
  its LP bound is below the optimum, and it is within one distortion step of
  the bound;
* fixed-rate instances of 50-300 items (integer bit counts) against the exact
  dynamic programme, on synthetic tables and on the oracle's own cost tables of
  small scenes: feasibility, the one-step gap, and the measured gap, which is
  printed (largest relative gap over the instances) and kept below 1e-2.

Needs a GB300."""
import numpy as np
import pytest

import oracle
from oracle import mckp
from paper_2604_26799_gb300 import mgs, synth
from tests.test_abi_cpu import synthetic_table

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2604_26799_gb300 import build
    build.build()
    c = mgs.mgs_create(0)
    yield c
    mgs.mgs_destroy(c)


def device_solve(ctx, buf, lay, grid, budgets, opts):
    return mgs.mgs_solve_budgets_device(ctx, torch.from_numpy(buf).cuda(), lay, grid, budgets, opts)


def check_against_exact(sol, dist, rates, budget, exact, tol=1e-9):
    """Feasible, no better than the optimum, LP bound below it, gap <= one step."""
    if exact is None:
        assert sol["r_index"] == -1
        return 0.0
    assert sol["r_index"] == 0
    items = dist.shape[0]
    ch = sol["choice"].astype(np.int64)
    est = mckp.assignment_bytes(rates, ch, 0.0)
    assert est <= budget * (1 + tol) + tol, (est, budget)
    assert abs(est - sol["est_bytes"]) <= tol * max(1.0, est)
    got = float(dist[np.arange(items), ch].sum())
    assert abs(got - sol["objective"]) <= tol * max(1.0, abs(got))
    opt = exact[0]
    assert got >= opt - tol * max(1.0, opt)
    assert sol["lp_bound"] <= opt + tol * max(1.0, opt)
    step = float(np.max(dist.max(axis=1) - dist.min(axis=1)))
    assert got <= sol["lp_bound"] + step + tol * max(1.0, got)
    return (got - opt) / opt if opt > 0 else 0.0


def test_device_solve_against_bruteforce(ctx):
    rng = np.random.default_rng(51)
    checked = 0
    for trial in range(60):
        C = int(rng.integers(1, 3))
        G = int(rng.integers(2, 9))
        n_b = int(rng.integers(1, 5))
        bits = np.sort(rng.choice(np.arange(1, 14), size=n_b, replace=False))
        keep = np.array([int(rng.integers(1, 4 * G))], dtype=np.int64)
        buf, lay, grid, v = synthetic_table(rng, keep, bits, G, C)
        items = int(lay.n_items)
        if items > 8 or n_b ** items > 70_000:
            continue
        for rate_model in (mgs.MGS_RATE_FIXED, mgs.MGS_RATE_ENTROPY):
            rates = mckp.item_rates(v, bits, "fixed" if rate_model == mgs.MGS_RATE_FIXED else "entropy")
            dist = mckp.item_dist(v, "sse")
            lo = rates.min(axis=1).sum() / 8 + 9 * items
            hi = rates.max(axis=1).sum() / 8 + 9 * items
            budgets = [float(x) for x in rng.uniform(lo - 2, hi + 2, size=3)]
            sols = device_solve(ctx, buf, lay, grid, budgets, mgs.solve_opts(rate_model=rate_model))
            for b, sol in zip(budgets, sols):
                check_against_exact(sol, dist, rates, b, mckp.solve_bruteforce(dist, rates, b))
                checked += 1
    assert checked >= 100


def fixed_rate_instances(rng):
    """Synthetic tables of 50-300 items with small integer bit counts."""
    for trial in range(6):
        C = int(rng.integers(2, 6))
        G = int(rng.integers(4, 12))
        n_b = int(rng.integers(2, 6))
        bits = np.sort(rng.choice(np.arange(1, 13), size=n_b, replace=False))
        target = int(rng.integers(60, 301))
        keep = np.array([max(1, (target // C) * G - int(rng.integers(0, G)))], dtype=np.int64)
        buf, lay, grid, v = synthetic_table(rng, keep, bits, G, C)
        yield buf, lay, grid, v, bits


def oracle_table_instances():
    """The oracle's cost tables of small scenes (4 channels), as a library table."""
    for seed, (n, G, bits) in enumerate([(1200, 16, [2, 4, 8]), (900, 8, [1, 3, 5, 7]),
                                         (2000, 40, [2, 6, 10])]):
        attrs, imp = synth.make_scene(n, seed=300 + seed)
        attrs = np.ascontiguousarray(attrs[:, [0, 7, 51, 55]])
        keep = np.array([n // 2], dtype=np.int64)
        grid = mgs.Grid(keep, bits, G)
        lay = mgs.mgs_table_layout_for(n, attrs.shape[1], grid)
        buf = np.zeros(lay.total_bytes, dtype=np.uint8)
        v = mgs.table_views(buf, lay)
        ref = oracle.cost_table(attrs, imp, keep, bits, G)
        for k in ("sse", "l1", "linf", "hbits", "cnt", "vmin", "vmax"):
            v[k][...] = ref[k]
        yield buf, lay, grid, v, np.asarray(bits)


@pytest.mark.parametrize("source", ["synthetic", "oracle_tables"])
def test_device_solve_against_exact_dp(ctx, source):
    rng = np.random.default_rng(52)
    inst = fixed_rate_instances(rng) if source == "synthetic" else oracle_table_instances()
    worst, n_checked = 0.0, 0
    for buf, lay, grid, v, bits in inst:
        items = int(lay.n_items)
        assert 50 <= items <= 300, items
        rates = mckp.item_rates(v, bits, "fixed")
        weights = np.rint(rates).astype(np.int64)
        assert np.array_equal(weights, rates)
        dist = mckp.item_dist(v, "sse")
        lo = rates.min(axis=1).sum() / 8 + 9 * items
        hi = rates.max(axis=1).sum() / 8 + 9 * items
        budgets = [float(lo + f * (hi - lo)) for f in (0.05, 0.3, 0.6, 0.9)]
        sols = device_solve(ctx, buf, lay, grid, budgets, mgs.solve_opts(rate_model=mgs.MGS_RATE_FIXED))
        for b, sol in zip(budgets, sols):
            exact = mckp.solve_dp_integer(dist, weights, b)
            gap = check_against_exact(sol, dist, rates, b, exact, tol=1e-9)
            worst = max(worst, gap)
            n_checked += 1
    print(f"\n[{source}] device solve vs exact DP: {n_checked} instances, largest relative gap {worst:.3e}")
    assert n_checked >= 12
    assert worst <= 1e-2
