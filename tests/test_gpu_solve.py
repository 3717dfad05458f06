"""The device budget solve gives the host solver's answers bit for bit: on
cost tables built on the GPU, on synthetic tables with many equal increment
keys, for every rate model and norm, at infeasible and all-fitting budgets,
from device and host table memory, and when the greedy completion takes
hundreds of increments (needs a GB300)."""
import numpy as np
import pytest

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


def assert_same(dev, host):
    assert len(dev) == len(host)
    for d, h in zip(dev, host):
        assert d["r_index"] == h["r_index"]
        assert d["est_bytes"] == h["est_bytes"]
        assert d["objective"] == h["objective"]
        assert d["lp_bound"] == h["lp_bound"]
        assert np.array_equal(d["choice"], h["choice"])
        for k in ("ratio_status", "ratio_objective", "ratio_bytes", "ratio_lp_bound"):
            assert np.array_equal(d[k], h[k]), k


def both(ctx, buf_host, lay, grid, budgets, opts, on_device=True):
    table = torch.from_numpy(buf_host).cuda() if on_device else buf_host
    dev = mgs.mgs_solve_budgets_device(ctx, table, lay, grid, budgets, opts)
    host = mgs.mgs_solve_budgets(buf_host, lay, grid, budgets, opts)
    return dev, host


def gpu_table(ctx, n, keep, bits, G, seed):
    attrs, imp = synth.make_scene(n, seed=seed)
    dev = torch.device("cuda:0")
    scene = mgs.mgs_scene_create(ctx, torch.from_numpy(attrs).to(dev), torch.from_numpy(imp).to(dev))
    try:
        grid = mgs.Grid(keep, bits, G)
        lay = mgs.mgs_table_layout_for(n, attrs.shape[1], grid)
        tab = torch.empty(lay.total_bytes, dtype=torch.uint8, device=dev)
        mgs.mgs_build_cost_table(ctx, scene, grid, tab)
        torch.cuda.synchronize()
    finally:
        mgs.mgs_scene_destroy(scene)
    return tab, lay, grid


def budget_range(host_buf, lay, grid, opts):
    """Budgets from below the smallest feasible size to above the largest."""
    sols = mgs.mgs_solve_budgets(host_buf, lay, grid, [1e15], opts)
    top = float(sols[0]["ratio_bytes"].max())
    return [1.0, top * 0.002, top * 0.01, top * 0.05, top * 0.2, top * 0.5, top * 1.5]


@pytest.mark.parametrize("rate_model,norm", [(0, 0), (1, 0), (0, 1), (0, 2), (0, 3), (1, 3)])
def test_device_solver_on_gpu_tables(ctx, rate_model, norm):
    n = 150_000
    keep = synth.keep_counts(n, list(synth.tenths()))
    tab, lay, grid = gpu_table(ctx, n, keep, [2, 3, 4, 6, 8, 10, 12, 16], 1024, seed=11)
    host = tab.cpu().numpy()
    opts = mgs.solve_opts(rate_model=rate_model, norm=norm)
    budgets = budget_range(host, lay, grid, opts)
    dev = mgs.mgs_solve_budgets_device(ctx, tab, lay, grid, budgets, opts)
    ref = mgs.mgs_solve_budgets(host, lay, grid, budgets, opts)
    assert_same(dev, ref)
    assert dev[0]["r_index"] == -1 and dev[-1]["r_index"] >= 0


def test_device_solver_synthetic_and_host_memory(ctx):
    rng = np.random.default_rng(3)
    for trial in range(6):
        keep = np.sort(rng.choice(np.arange(50, 3000), size=4, replace=False)).astype(np.int64)
        bits = sorted(rng.choice(np.arange(1, 17), size=int(rng.integers(1, 9)), replace=False).tolist())
        buf, lay, grid, _ = synthetic_table(rng, keep, bits, int(rng.integers(8, 200)), int(rng.integers(1, 9)))
        opts = mgs.solve_opts(rate_model=int(trial % 2))
        budgets = budget_range(buf, lay, grid, opts)
        for on_device in (True, False):
            dev, host = both(ctx, buf, lay, grid, budgets, opts, on_device=on_device)
            assert_same(dev, host)


def test_device_solver_equal_keys(ctx):
    """Every item identical: all increments of a level share one key, so the
    split falls inside a run of equal keys ordered by item."""
    rng = np.random.default_rng(4)
    keep = np.array([4000], dtype=np.int64)
    bits = [2, 4, 8, 12]
    buf, lay, grid, v = synthetic_table(rng, keep, bits, 8, 3)
    for k in ("sse", "l1", "hbits", "linf"):
        v[k][:] = v[k][0]
    v["cnt"][:] = v["cnt"][0]
    opts = mgs.solve_opts()
    budgets = budget_range(buf, lay, grid, opts) + [float(x) for x in np.linspace(1e3, 2e5, 23)]
    dev, host = both(ctx, buf, lay, grid, budgets, opts)
    assert_same(dev, host)


def test_device_solver_many_greedy_takes(ctx):
    """A split on a large increment leaves room for hundreds of small ones,
    taken one block-wide selection at a time."""
    n_big, n_small = 10, 6000
    n = n_big + n_small
    grid = mgs.Grid(np.array([n], dtype=np.int64), [1, 2, 3], 1)
    lay = mgs.mgs_table_layout_for(n, 1, grid)
    buf = np.zeros(lay.total_bytes, dtype=np.uint8)
    v = mgs.table_views(buf, lay)
    v["cnt"][:] = 1
    v["hbits"][:n_big] = [0.0, 1000.0, 1000.0]
    v["sse"][:n_big] = [100.0, 0.0, 0.0]
    v["hbits"][n_big:] = [0.0, 1.0, 2.0]
    v["sse"][n_big:] = [0.01, 0.005, 0.0049]
    v["l1"][:] = v["sse"]
    v["linf"][:] = v["sse"].astype(np.float32)
    opts = mgs.solve_opts(meta_bytes_per_group=0.0)
    budget = (5 * 1000 + 500) / 8.0
    dev, host = both(ctx, buf, lay, grid, [budget, 2 * budget], opts)
    assert_same(dev, host)
    # LP: five large increments, split on the sixth; the greedy step fills 500 bits
    # with the small items' first increments, in item order
    ch = dev[0]["choice"]
    assert (ch[:n_big] == 1).sum() == 5
    assert (ch[n_big:] == 1).sum() == 500 and (ch[n_big:n_big + 500] == 1).all()
